"""Pins of the oracle's FENEWCA and Tether bond evaluators (Sec. II.B: the
updater is templated on the bond evaluator and accepts HOOMD-blue's Harmonic,
FENEWCA and Tether bonds; the potentials are those HOOMD-blue documents).

- FENEWCA reduces to pinned routines: with eps = 0 and delta = 0 it is the FENE
  bond (energies and whole sweeps identical); with delta = 0 its energy minus
  the FENE energy is the WCA pair energy the oracle's pair force is pinned on;
  a shift delta translates it (U(r; delta) = U(r - delta; 0)).
- Tether: zero on [l_c1, l_c0]; its two branches mirror each other
  (U_att(l_c0 + x) = U_rep(l_c1 - x) when l_max - l_c0 = l_c1 - l_min); +inf at
  l_min and l_max; one worked value.
- Forces of lone static bonds of both kinds are minus the derivative of the
  oracle's energy (central differences), and the force sensitivity scale
  r |dF/dr| matches differences of the force.
- The proposal's aim is the minimum of the energy (FENEWCA: the bisection root
  is a minimum of the libm energy; Tether: the middle of the flat interval),
  and proposals pick the candidate closest to it (brute force).
- Frozen pairs reach the two-state fraction P_on(r) / (P_on(r) + P_off) with
  U_b(r) from the libm energy (the sweep uses the library's own exp and log),
  in the flat Tether interval K / (1 + K).
"""
import math

import numpy as np
import pytest

from synth import frozen_pairs, random_frozen, assoc_ab, BondType, FENE, FENEWCA, TETHER

TETHER_P = (1.0, 0.7, (0.95, 1.1, 2.0))        # k_b, l_min, (l_c1, l_c0, l_max)
FENEWCA_P = (3.0, 1.5, (1.0, 1.0, 0.1))        # k, R0, (eps, sigma, delta)


def _sys_with_bond(kind, k, r0, extra, n_pairs=1, r=1.0, **kw):
    s = frozen_pairs(seed=2, n_pairs=n_pairs, r=r, **kw)
    s.bond_types = [BondType(kind, k, r0, extra)]
    return s


def test_fenewca_reduces_to_fene_and_wca(oracle_mod):
    a = oracle_mod.OracleSystem(_sys_with_bond(FENEWCA, 3.0, 1.5, (0.0, 1.0, 0.0)))
    b = oracle_mod.OracleSystem(_sys_with_bond(FENE, 3.0, 1.5, ()))
    c = oracle_mod.OracleSystem(_sys_with_bond(FENEWCA, 3.0, 1.5, (1.0, 1.0, 0.0)))
    d = oracle_mod.OracleSystem(_sys_with_bond(FENEWCA, 3.0, 1.5, (1.0, 1.0, 0.25)))
    # the pair WCA energy of two unit spheres from the oracle's pair force field
    s = assoc_ab(seed=1, n_a=1, n_b=1, rho=0.001)
    s.reactions = []
    p = oracle_mod.OracleSystem(s)
    p.y[:] = [5.0, 5.0]
    p.z[:] = [5.0, 5.0]
    for r in (0.8, 0.95, 1.0, 1.1, 1.12, 1.2, 1.4, 1.49):
        assert a.bond_energy(0, r) == b.bond_energy(0, r)
        p.x[:] = [5.0, 5.0 + r]
        _, e = p.forces()
        assert c.bond_energy(0, r) == pytest.approx(b.bond_energy(0, r) + e["e_pair"], rel=1e-13, abs=1e-13)
        assert d.bond_energy(0, r + 0.25) == pytest.approx(c.bond_energy(0, r), rel=1e-13, abs=1e-13)
    assert math.isinf(c.bond_energy(0, 1.5)) and math.isinf(d.bond_energy(0, 0.25))


def test_fenewca_eps0_sweeps_equal_fene(oracle_mod):
    s1 = random_frozen(seed=3, n=800, box=10.0, overlap_factor=0.6, r_max=1.4, eps=3.0)
    s1.bond_types = [BondType(FENEWCA, 3.0, 1.5, (0.0, 1.0, 0.0))]
    s2 = random_frozen(seed=3, n=800, box=10.0, overlap_factor=0.6, r_max=1.4, eps=3.0)
    s2.bond_types = [BondType(FENE, 3.0, 1.5)]
    a, b = oracle_mod.OracleSystem(s1), oracle_mod.OracleSystem(s2)
    for t in range(6):
        assert a.sweep(step=t) == b.sweep(step=t)
        assert np.array_equal(a.bonds(), b.bonds())
    assert a.bonds().shape[0] > 20


def test_tether_shape(oracle_mod):
    kb, lmin, (lc1, lc0, lmax) = 2.0, 0.6, (0.9, 1.2, 1.5)   # l_max - l_c0 = l_c1 - l_min = 0.3
    o = oracle_mod.OracleSystem(_sys_with_bond(TETHER, kb, lmin, (lc1, lc0, lmax)))
    for r in np.linspace(lc1, lc0, 7):
        assert o.bond_energy(0, r) == 0.0
    for x in (0.01, 0.05, 0.1, 0.2, 0.29):
        assert o.bond_energy(0, lc0 + x) == pytest.approx(o.bond_energy(0, lc1 - x), rel=1e-14)
        assert o.bond_energy(0, lc0 + x) > 0.0
    assert math.isinf(o.bond_energy(0, lmax)) and math.isinf(o.bond_energy(0, lmin))
    assert o.bond_energy(0, lc0 + 1e-3) < 1e-300          # continuous at l_c0
    # worked value: r = l_c0 + 0.1: k_b e^{1/(-0.1)} / 0.2 = 10 e^{-10}
    assert o.bond_energy(0, lc0 + 0.1) == pytest.approx(10.0 * math.exp(-10.0), rel=1e-14)


@pytest.mark.parametrize("kind,k,r0,extra,rs", [
    (FENEWCA, 3.0, 1.5, (1.0, 1.0, 0.1), (0.98, 1.15, 1.3, 1.5)),
    (TETHER, 1.0, 0.7, (0.95, 1.1, 2.0), (0.75, 0.85, 1.2, 1.6, 1.9)),
])
def test_lone_bond_force_is_energy_gradient_and_scale(oracle_mod, kind, k, r0, extra, rs):
    s = assoc_ab(seed=1, n_a=1, n_b=1, rho=0.001)
    s.reactions = []
    s.eps_pair = np.zeros((2, 2))            # bond force only
    s.static_bonds = np.array([[0, 1]], np.int32)
    s.static_bond_types = np.array([0], np.int32)
    s.bond_types = [BondType(kind, k, r0, extra)]
    o = oracle_mod.OracleSystem(s)
    o.y[:] = [5.0, 5.0]
    o.z[:] = [5.0, 5.0]
    h = 1e-6
    for r in rs:
        o.x[:] = [5.0, 5.0 + r]
        f, e = o.forces()
        fd = -(o.bond_energy(0, r + h) - o.bond_energy(0, r - h)) / (2 * h)   # F along +x on particle 1
        assert f[1, 0] == pytest.approx(fd, rel=1e-6, abs=1e-9)
        assert e["e_bond"] == pytest.approx(o.bond_energy(0, r), rel=1e-14)
        o.x[:] = [5.0, 5.0 + r + h]
        fp, _ = o.forces()
        o.x[:] = [5.0, 5.0 + r - h]
        fm, _ = o.forces()
        g = abs(f[1, 0]) + r * abs((fp[1, 0] - fm[1, 0]) / (2 * h))
        assert e["fscale"][0] == pytest.approx(g, rel=1e-5, abs=1e-9)
    o.x[:] = [5.0, 5.0 + (2.05 if kind == TETHER else 1.7)]   # beyond the finite range
    _, e = o.forces()
    assert e["status"] == 6


def test_aim_separation_is_the_minimum(oracle_mod):
    o = oracle_mod.OracleSystem(_sys_with_bond(FENEWCA, *FENEWCA_P[:2], FENEWCA_P[2]))
    r_star = o.aim_separation(0)
    assert 1.1 < r_star < 0.1 + 2 ** (1 / 6)
    for h in (1e-3, 1e-4, 1e-5):
        assert o.bond_energy(0, r_star) < o.bond_energy(0, r_star + h)
        assert o.bond_energy(0, r_star) < o.bond_energy(0, r_star - h)
    # eps = 0: FENE centred at delta
    o0 = oracle_mod.OracleSystem(_sys_with_bond(FENEWCA, 3.0, 1.5, (0.0, 1.0, 0.3)))
    assert o0.aim_separation(0) == 0.3
    t = oracle_mod.OracleSystem(_sys_with_bond(TETHER, *TETHER_P[:2], TETHER_P[2]))
    assert t.aim_separation(0) == 0.5 * (0.95 + 1.1)


@pytest.mark.parametrize("kind,params", [(FENEWCA, FENEWCA_P), (TETHER, TETHER_P)])
def test_proposals_aim_at_the_minimum(oracle_mod, kind, params):
    s = random_frozen(seed=5, n=120, box=6.0, overlap_factor=0.5, r_max=1.6, eps=2.0)
    s.bond_types = [BondType(kind, params[0], params[1], params[2])]
    o = oracle_mod.OracleSystem(s)
    r_star = o.aim_separation(0)
    st, tr = o.sweep(step=0, trace=True)
    n_checked = 0
    for i in range(s.n):
        d = s.pos - s.pos[i]
        d -= s.box * np.rint(d / s.box)
        r = np.sqrt((d * d).sum(1))
        ok = (s.types == 1 - s.types[i]) & (r <= 1.6)
        ok[i] = False
        cand = np.nonzero(ok)[0]
        if cand.size == 0:
            assert tr["prop"][i] == -1
            continue
        key = np.abs(r[cand] - r_star)
        assert tr["prop"][i] == cand[np.lexsort((cand, key))[0]]
        n_checked += 1
    assert n_checked > 30 and st["proposals"] == n_checked


@pytest.mark.parametrize("kind,params,r", [
    (TETHER, TETHER_P, 1.0),      # flat interval: U = 0
    (TETHER, TETHER_P, 1.3),      # attractive branch
    (TETHER, TETHER_P, 0.8),      # repulsive branch
    (FENEWCA, FENEWCA_P, 1.2),
])
def test_frozen_pairs_two_state(oracle_mod, kind, params, r):
    n_pairs, T, eps = 200, 3000, 1.0
    s = frozen_pairs(seed=11, n_pairs=n_pairs, r=r, eps=eps, r_max=1.4)
    s.bond_types = [BondType(kind, params[0], params[1], params[2])]
    o = oracle_mod.OracleSystem(s)
    U = o.bond_energy(0, r)
    a = math.exp(-U / s.kT)
    b = math.exp(-eps)
    expect = a / (a + b)
    if kind == TETHER and r == 1.0:
        assert U == 0.0 and expect == pytest.approx(math.e / (1 + math.e))
    counts = []
    for t in range(T + 50):
        o.sweep(step=t)
        if t >= 50:
            counts.append(o.occ.sum() / 2)
    frac = np.mean(counts) / n_pairs
    lam = 1.0 - a - b
    se = math.sqrt(expect * (1 - expect) / (n_pairs * T) * (1 + lam) / (1 - lam))
    assert abs(frac - expect) < 4.5 * se, (kind, r, frac, expect, se)

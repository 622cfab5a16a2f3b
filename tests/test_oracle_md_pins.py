"""Pins of the oracle's force field and Langevin integrator.

- Forces are minus the gradient of the oracle's own energy (central finite
  differences) and sum to zero (Newton's third law).
- With all interactions off, the leapfrog Langevin scheme keeps the
  synchronised velocity at exactly kT per component in expectation, and the
  half-step velocity at kT / (1 - gamma dt / 2) (closed forms of the linear
  recursion v' = (1 - gamma dt) v + dt sqrt(2 gamma kT/dt) xi).
- A + B association (monovalent, dilute): the bonded fraction p obeys
  p / (1 - p)^2 = c_B K I with I = int 4 pi r^2 exp(-[U_WCA + U_b]/kT) dr over
  the formation window (ideal-association closed form of Eqs. 1-4).
"""
import math

import numpy as np
import pytest
from scipy.integrate import quad

from synth import telechelic, assoc_ab, colloid_linker


def _energy(o):
    _, e = o.forces()
    return e["e_pair"] + e["e_bond"]


def test_forces_are_energy_gradient(oracle_mod):
    s = telechelic(seed=3, n_chains=20, beads=12, n_x=60, rho=0.5)
    o = oracle_mod.OracleSystem(s)
    o.run(200)  # let bonds form so dynamic harmonic bonds contribute
    assert o.bonds().shape[0] > 0
    f, e = o.forces()
    rng = np.random.default_rng(1)
    h = 1e-6
    for i in rng.choice(s.n, 40, replace=False):
        for d, arr in enumerate((o.x, o.y, o.z)):
            x0 = arr[i]
            arr[i] = x0 + h
            ep = _energy(o)
            arr[i] = x0 - h
            em = _energy(o)
            arr[i] = x0
            fd = -(ep - em) / (2 * h)
            assert abs(fd - f[i, d]) <= 1e-5 * max(1.0, abs(f[i, d])), (i, d, fd, f[i, d])
    assert np.abs(f.sum(0)).max() < 1e-9 * max(1.0, np.abs(f).max())


def test_wca_force_closed_form(oracle_mod):
    s = assoc_ab(seed=1, n_a=1, n_b=1, rho=0.001)
    s.reactions = []
    o = oracle_mod.OracleSystem(s)
    for r in (0.9, 1.0, 1.05, 1.12, 1.2):
        o.x[:] = [5.0, 5.0 + r]
        o.y[:] = [5.0, 5.0]
        o.z[:] = [5.0, 5.0]
        f, e = o.forces()
        rc = 2 ** (1 / 6)
        if r < rc:
            fmag = 24 * (2 * r ** -13 - r ** -7)
            u = 4 * (r ** -12 - r ** -6) + 1
        else:
            fmag, u = 0.0, 0.0
        assert f[1, 0] == pytest.approx(fmag, rel=1e-12, abs=1e-12)
        assert f[0, 0] == pytest.approx(-fmag, rel=1e-12, abs=1e-12)
        assert e["e_pair"] == pytest.approx(u, rel=1e-12, abs=1e-12)


def test_langevin_equipartition_ideal_gas(oracle_mod):
    s = assoc_ab(seed=2, n_a=1000, n_b=1000, rho=0.05)
    s.reactions = []
    s.eps_pair = np.zeros((2, 2))
    s.vel[:] = 0.0
    s.kT = 1.3
    o = oracle_mod.OracleSystem(s)
    o.run(1500)  # relax for 7.5 gamma^-1
    kes, v2 = [], []
    for _ in range(40):
        r = o.run(25)
        kes.append(r["ke"])
        v2.append(np.mean(np.concatenate([o.vx, o.vy, o.vz]) ** 2))
    n = s.n
    ke_per = np.array(kes) / (1.5 * n)
    gdt = s.gamma * s.dt
    # 40 nearly independent samples of a mean over 3n components
    se = s.kT * math.sqrt(2.0 / (3 * n)) / math.sqrt(40)
    assert abs(ke_per.mean() - s.kT) < 5 * se, (ke_per.mean(), s.kT)
    assert abs(np.mean(v2) - s.kT / (1 - gdt / 2)) < 5 * se * 1.01


@pytest.mark.slow
def test_assoc_ab_closed_form_bonded_fraction(oracle_mod):
    """Ideal-association closed form in the regime where its assumptions hold:
    dilute, weakly contested, and a formation window wide enough (r_max = 2.0)
    that no bond wanders out of it.  With the narrower window r_max = 1.3 of the
    A+B benchmark, bonds carried past r_max can break but not re-form there, so
    the runs settle near 0.76 (eight oracle seeds: 0.750-0.771) against the
    closed form's 0.811 for that window."""
    s = assoc_ab(r_max=2.0)
    o = oracle_mod.OracleSystem(s)
    o.run(3000)
    fr = []
    for _ in range(30):
        o.run(300)
        fr.append(o.bonds().shape[0] / 500.0)
    p_sim = float(np.mean(fr))
    eps, k, r0, rmax = 5.0, 100.0, 1.1, 2.0
    cB = 500.0 / float(np.prod(s.box))

    def wca(r):
        return 4 * (r ** -12 - r ** -6) + 1 if r < 2 ** (1 / 6) else 0.0

    def p_closed(rm):
        I = quad(lambda r: 4 * math.pi * r * r * math.exp(-(wca(r) + 0.5 * k * (r - r0) ** 2)),
                 0.5, rm, points=[2 ** (1 / 6)])[0]
        lam = cB * math.exp(eps) * I
        return ((2 * lam + 1) - math.sqrt(4 * lam + 1)) / (2 * lam)

    assert abs(p_closed(1.3) - 0.8110) < 2e-3
    p = p_closed(rmax)
    # systematic: residual contention and non-ideality at rho = 0.1 (~0.01)
    assert abs(p_sim - p) < 0.02, (p_sim, p)


@pytest.mark.slow
def test_assoc_ab_narrow_window_loses_stretched_bonds(oracle_mod):
    """Why the A+B benchmark's window r_max = 1.3 settles below the ideal
    closed form: a bond formed inside the window is stretched past r_max by
    the thermal motion of its ends (harmonic k = 100: width 0.1 about r0 = 1.1),
    where it can still break (P_off at any r) but a broken pair cannot re-form.
    The oracle run holds bonds beyond r_max, and its bonded fraction lies
    clearly below the closed form for that window (while the wide-window run
    above meets its closed form)."""
    s = assoc_ab()                        # r_max = 1.3
    o = oracle_mod.OracleSystem(s)
    o.run(3000)
    fr, beyond = [], []
    box = np.asarray(s.box)
    for _ in range(20):
        o.run(300)
        b = o.bonds()
        fr.append(b.shape[0] / 500.0)
        d = o.pos[b[:, 1]] - o.pos[b[:, 0]]
        d -= box * np.rint(d / box)
        beyond.append(float(np.mean(np.sqrt((d * d).sum(1)) > 1.3)))
    p_sim = float(np.mean(fr))
    eps, k, r0, rmax = 5.0, 100.0, 1.1, 1.3
    cB = 500.0 / float(np.prod(s.box))

    def wca(r):
        return 4 * (r ** -12 - r ** -6) + 1 if r < 2 ** (1 / 6) else 0.0

    I = quad(lambda r: 4 * math.pi * r * r * math.exp(-(wca(r) + 0.5 * k * (r - r0) ** 2)),
             0.5, rmax, points=[2 ** (1 / 6)])[0]
    lam = cB * math.exp(eps) * I
    p_closed = ((2 * lam + 1) - math.sqrt(4 * lam + 1)) / (2 * lam)
    assert abs(p_closed - 0.811) < 2e-3
    assert p_sim < p_closed - 0.03, (p_sim, p_closed)
    # bonds sit beyond the window: a few per cent of them at any time
    assert 0.005 < float(np.mean(beyond)) < 0.2, np.mean(beyond)

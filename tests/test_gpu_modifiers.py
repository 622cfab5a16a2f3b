"""GPU path with the rate modifiers of Sec. II.D, through the C ABI against the
FP64 oracle.

- Slip bond (Eq. slip): sweeps with bonds at many separations are bit-exact
  against the oracle in both precisions, at kT = 1 and at kT = 0 (where every
  stretched bond breaks); FP64 MD with the slip bond follows the oracle step
  for step; frozen pairs at r != r0 reach the two-state fraction
  P_on(r)/(P_on(r) + P_off(r)).
- Melting switch (Eqs. gT-kT): replicas at set-point temperatures around
  T_melt in one batched context, each bit-exact against a standalone oracle
  run at its own temperature; the bonded fraction crosses 1/2 at T_melt.
- Misuse is refused: both modifiers on one reaction, the slip bond with the
  Metropolis-Hastings move set, rates above 1/(n dt).
"""
import math

import numpy as np
import pytest

import oracle
from synth import random_frozen, frozen_pairs, assoc_ab

pytestmark = pytest.mark.gpu

SWEEP_STATS = ("in_window", "proposals", "edges", "survivors", "formed", "break_tested", "broken")


@pytest.fixture(scope="module")
def snapmod():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2609_21204_b300 import build
    build.build()
    import paper_2609_21204_b300 as m
    return m


def _slip_case(kT):
    s = random_frozen(seed=21, n=3000, box=14.0, overlap_factor=0.6, r_max=1.4, valence=(2, 2), eps=2.0)
    s.reactions[0].slip_a = 1.2
    s.kT = kT
    return s


@pytest.mark.parametrize("kT", [1.0, 0.0])
@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_slip_sweeps_bit_exact(snapmod, kT, precision):
    s = _slip_case(kT)
    # start from bonds at many separations (those of a few oracle sweeps at kT = 1)
    pre = oracle.OracleSystem(_slip_case(1.0), p_on0=1.0)
    for t in range(8):
        pre.sweep(step=t)
    b0 = pre.bonds()
    sim = snapmod.from_system(s, precision=precision, p_on0=1.0)
    orc = oracle.OracleSystem(s, p_on0=1.0)
    sim.set_bonds(b0[:, :2], b0[:, 2])
    orc.set_bonds(b0)
    broken = 0
    try:
        for step in list(range(100, 130)) + [1000, 55555555555]:
            sim.set_step(step)
            sim.bond_update()
            st_o = orc.sweep(step=step)
            assert np.array_equal(sim.bonds(), orc.bonds()), (step,)
            st_g = sim.stats()
            for k in SWEEP_STATS:
                assert st_g[k] == st_o[k], (step, k, st_g[k], st_o[k])
            broken += st_o["broken"]
            if kT == 0.0 and step == 100:
                assert st_o["broken"] == len(b0)    # kT = 0: every stretched bond breaks
        assert broken > 100
    finally:
        sim.close()


def test_slip_fp64_trajectory_follows_oracle(snapmod):
    s = assoc_ab(seed=15)
    s.reactions[0].slip_a = 1.0
    sim = snapmod.from_system(s, precision="fp64")
    orc = oracle.OracleSystem(s)
    try:
        for _ in range(5):
            sim.step(20)
            orc.run(20)
            d = sim.positions() - orc.pos
            d -= s.box * np.rint(d / s.box)
            assert np.abs(d).max() < 1e-9
            assert np.array_equal(sim.bonds(), orc.bonds())
    finally:
        sim.close()


def test_slip_two_state_fraction(snapmod):
    eps, r, a, n_pairs, T = 2.0, 1.2, 1.0, 1000, 2000
    s = frozen_pairs(seed=3, n_pairs=n_pairs, r=r, eps=eps)
    s.reactions[0].slip_a = a
    k, r0 = s.bond_types[0].k, s.bond_types[0].r0
    U = 0.5 * k * (r - r0) ** 2
    p_on, p_off = math.exp(-U), math.exp(-eps) * math.exp(a * math.sqrt(U))
    expect = p_on / (p_on + p_off)
    sim = snapmod.from_system(s, precision="mixed", p_on0=1.0)
    counts = []
    try:
        for t in range(T + 50):
            sim.set_step(t)
            sim.bond_update()
            if t >= 50:
                counts.append(sim.stats()["n_bonds"])
    finally:
        sim.close()
    frac = np.mean(counts) / n_pairs
    lam = 1 - p_on - p_off
    se = math.sqrt(expect * (1 - expect) / (n_pairs * T) * (1 + lam) / (1 - lam))
    assert abs(frac - expect) < 4.5 * se, (frac, expect)


def test_melting_replicas_bit_exact_and_cross_half_at_t_melt(snapmod):
    lam, tm, kon, koff = 8.0, 1.0, 20.0, 4.0
    temps = [0.7, 0.9, 1.0, 1.1, 1.3]
    reps = []
    for r, t in enumerate(temps):
        s = frozen_pairs(seed=40 + r, n_pairs=400, r=1.1, eps=0.0, kT=t)
        s.seed = 500 + r
        s.reactions[0].melt = (lam, tm, kon, koff, 0.0, kon - koff)
        reps.append(s)
    sim = snapmod.from_system(reps, precision="mixed", p_on0=1.0)
    orcs = [oracle.OracleSystem(s, p_on0=1.0) for s in reps]
    nb = np.zeros(len(reps))
    T = 1500
    try:
        for t in range(T):
            sim.set_step(t)
            sim.bond_update()
            bonds = sim.bonds()
            off = 0
            for q, (s, o) in enumerate(zip(reps, orcs)):
                sel = (bonds[:, 0] >= off) & (bonds[:, 0] < off + s.n)
                if t < 40:          # the first sweeps step for step with each replica's oracle
                    o.sweep(step=t)
                    mine = bonds[sel].copy()
                    mine[:, :2] -= off
                    assert np.array_equal(mine, o.bonds()), (q, t)
                elif t >= 100:
                    nb[q] += sel.sum()
                off += s.n
    finally:
        sim.close()
    frac = nb / ((T - 100) * 400)
    for q, t in enumerate(temps):
        pon, poff = oracle.melting_rates(t, lam, tm, kon, koff, 0.0, kon - koff, 1, reps[q].dt)
        assert abs(frac[q] - pon / (pon + poff)) < 0.02, (t, frac[q], pon / (pon + poff))
    assert abs(frac[2] - 0.5) < 0.02
    assert np.all(np.diff(frac) < 0)           # bound fraction falls through the transition


def test_modifier_misuse_is_refused(snapmod):
    s = frozen_pairs(seed=1, n_pairs=27)
    sim = snapmod.from_system(s, precision="mixed")
    try:
        sim.set_slip(0, 1.0)
        with pytest.raises(snapmod.SnapError):
            sim.set_melting(0, 8.0, 1.0, 20.0, 4.0, 0.0, 16.0)
        with pytest.raises(snapmod.SnapError):
            sim.set_mh(1)
        with pytest.raises(snapmod.SnapError):
            sim.set_slip(0, -1.0)
        sim.set_slip(0, 0.0)
        with pytest.raises(snapmod.SnapError):
            sim.set_melting(0, 8.0, 1.0, 1000.0, 4.0, 0.0, 16.0)  # at T = T_melt: k_on n dt = 2.5 > 1
        sim.set_melting(0, 8.0, 1.0, 20.0, 4.0, 0.0, 16.0)
        with pytest.raises(snapmod.SnapError):
            sim.set_slip(0, 1.0)
    finally:
        sim.close()


def test_bond_period_trajectory_follows_oracle(snapmod):
    # a sweep every n = 5 steps (Eq. 2: P = k n dt per sweep); FP64 step for step
    s = assoc_ab(seed=16)
    s.bond_period = 5
    sim = snapmod.from_system(s, precision="fp64")
    orc = oracle.OracleSystem(s)
    try:
        for _ in range(6):
            sim.step(17)
            orc.run(17)
            d = sim.positions() - orc.pos
            d -= s.box * np.rint(d / s.box)
            assert np.abs(d).max() < 1e-9
            assert np.array_equal(sim.bonds(), orc.bonds())
        assert sim.stats()["sweeps"] == len(range(0, 6 * 17, 5))
    finally:
        sim.close()

"""GPU path with the kinetic temperature (Sec. II.B: T in Eq. 3 is the
instantaneous kinetic temperature when the updater triggers; Sec. II.D: the
same T in the slip factor and in the melting switch g(T)), through the C ABI
against the FP64 oracle.

- Single sweeps are bit-exact against the oracle given the GPU's own positions
  and half-step velocities (FP32 in mixed mode): the fixed-point sum makes T
  the same double on both sides.  Cases: a contested configuration whose
  velocities put T well away from the set-point, the slip bond from bonds at
  many separations, and the melting switch with T near T_melt.
- FP64 MD with the kinetic temperature follows the oracle step for step.
- The Metropolis-Hastings move set refuses it.
"""
import numpy as np
import pytest

import oracle
from synth import random_frozen, assoc_ab

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


def _case(kind):
    s = random_frozen(seed=31, n=3000, box=14.0, overlap_factor=0.6, r_max=1.4, valence=(2, 2), eps=2.0)
    rng = np.random.default_rng(32)
    s.vel = rng.normal(size=(s.n, 3)) * np.sqrt(0.55)   # T_kin ~ 0.55 against the set-point 1
    s.kinetic_T = 1
    if kind == "slip":
        s.reactions[0].slip_a = 1.2
    elif kind == "melt":
        lam, tm, kon, koff = 4.0, 0.6, 60.0, 12.0
        s.reactions[0].melt = (lam, tm, kon, koff, 0.0, kon - koff)
    return s


def _sweep_pair(snapmod, s, precision, pre_bonds=None):
    sim = snapmod.from_system(s, precision=precision, p_on0=1.0)
    orc = oracle.OracleSystem(s, p_on0=1.0)
    # the oracle takes the GPU's own velocities (FP32 values in mixed mode)
    orc.set_velocities(sim.velocities())
    if pre_bonds is not None:
        sim.set_bonds(pre_bonds[:, :2], pre_bonds[:, 2])
        orc.set_bonds(pre_bonds)
    return sim, orc


@pytest.mark.parametrize("kind", ["plain", "slip", "melt"])
@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_kinetic_T_sweeps_bit_exact(snapmod, kind, precision):
    s = _case(kind)
    pre = None
    if kind == "slip":
        o = oracle.OracleSystem(_case("plain"), p_on0=1.0)
        for t in range(8):
            o.sweep(step=t)
        pre = o.bonds()
    sim, orc = _sweep_pair(snapmod, s, precision, pre)
    T = orc.kinetic_T()
    assert 0.45 < T < 0.65
    formed = broken = 0
    try:
        for step in list(range(200, 220)) + [1000, 77777777777]:
            sim.set_step(step)
            sim.bond_update()
            st_o = orc.sweep(step=step)
            assert np.array_equal(sim.bonds(), orc.bonds()), (kind, precision, step)
            st_g = sim.stats()
            for k in SWEEP_STATS:
                assert st_g[k] == st_o[k], (kind, precision, step, k, st_g[k], st_o[k])
            formed += st_o["formed"]
            broken += st_o["broken"]
        assert formed > 100 and broken > 20
    finally:
        sim.close()


def test_kinetic_T_changes_decisions(snapmod):
    """The same sweep at the set-point gives another bond table: the option is live."""
    s = _case("plain")
    a = snapmod.from_system(s, precision="fp64", p_on0=1.0)
    s.kinetic_T = 0
    b = snapmod.from_system(s, precision="fp64", p_on0=1.0)
    for step in range(5):
        a.set_step(step)
        b.set_step(step)
        a.bond_update()
        b.bond_update()
    assert not np.array_equal(a.bonds(), b.bonds())


def test_kinetic_T_fp64_trajectory_follows_oracle(snapmod):
    s = assoc_ab(seed=33)
    s.kinetic_T = 1
    s.reactions[0].slip_a = 0.8
    sim = snapmod.from_system(s, precision="fp64")
    orc = oracle.OracleSystem(s)
    for _ in range(5):
        sim.step(20)
        orc.run(20)
        d = sim.positions() - orc.pos
        d -= s.box * np.rint(d / s.box)
        assert np.abs(d).max() < 1e-9
        assert np.array_equal(sim.bonds(), orc.bonds())
    assert sim.stats()["n_bonds"] > 50


def test_kinetic_T_batched_replicas_follow_their_oracles(snapmod):
    """Four replicas in one context, each with its own kinetic temperature
    (velocities drawn at different scales, uneven sizes): the fixed-point sum
    is per replica, so one sweep and 25 FP64 MD steps match each replica's
    own oracle bit for bit in the bonds and to 1e-9 in the positions."""
    reps = [random_frozen(seed=70 + r, n=500 + 123 * r, box=12.0 + r, overlap_factor=1.0,
                          r_max=1.4, eps=1.5 + r) for r in range(4)]
    rng = np.random.default_rng(71)
    for r, s in enumerate(reps):
        s.seed = 2000 + 31 * r
        s.kinetic_T = 1
        s.vel = rng.normal(size=(s.n, 3)) * np.sqrt(0.4 + 0.3 * r)
    sim = snapmod.from_system(reps, precision="fp64", p_on0=0.8)
    orcs = [oracle.OracleSystem(s, p_on0=0.8) for s in reps]
    temps = [o.kinetic_T() for o in orcs]
    assert max(temps) - min(temps) > 0.5
    sim.bond_update()
    for o in orcs:
        o.sweep(step=0)
    sim.step(25)
    for o in orcs:
        o.run(25)
    bonds = sim.bonds()
    pos = sim.positions()
    off = 0
    for s, o in zip(reps, orcs):
        sel = (bonds[:, 0] >= off) & (bonds[:, 0] < off + s.n)
        mine = bonds[sel].copy()
        mine[:, :2] -= off
        assert np.array_equal(mine, o.bonds())
        d = pos[off:off + s.n] - o.pos
        d -= s.box * np.rint(d / s.box)
        assert np.abs(d).max() < 1e-9
        off += s.n
    assert bonds.shape[0] > 100


def test_kinetic_T_refused_with_mh(snapmod):
    s = assoc_ab(seed=34)
    sim = snapmod.from_system(s, precision="mixed")
    sim.set_kinetic_temperature(True)
    with pytest.raises(snapmod.SnapError) as e:
        sim.set_mh(1)
    assert e.value.name == "SNAP_ERR_STATE"
    sim.set_kinetic_temperature(False)
    sim.set_mh(1)
    with pytest.raises(snapmod.SnapError) as e:
        sim.set_kinetic_temperature(True)
    assert e.value.name == "SNAP_ERR_STATE"
    sim.set_mh(0)
    with pytest.raises(snapmod.SnapError) as e:
        sim._check(sim._lib.snap_set_kinetic_temperature(sim._ctx, 2))
    assert e.value.name == "SNAP_ERR_ARG"

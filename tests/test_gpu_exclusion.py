"""GPU path with intramolecular exclusion (Sec. II.D; App. A tests it in both
directions with a control pair), through the C ABI against the FP64 oracle.

- Sweeps are bit-exact against the oracle with the exclusion on and off:
  frozen P-M-Q molecules beside control pairs, a dense frozen configuration of
  short S-S telechelic chains, and stars whose centre is statically bonded to
  half of its arms — the scarce centres take the push path there.
- MD: short telechelic chains whose ends react S-S never close into rings with
  the exclusion, and do without it; FP64 trajectories follow the oracle.
- The Metropolis-Hastings move set refuses a reaction with the exclusion.
"""
import numpy as np
import pytest

import oracle
from synth import frozen_loops, telechelic_rings, frozen_stars, BondType, FENE

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


def _star_molecules(self_avoid):
    # six arms per centre; the centre and its first three arms form one molecule
    s = frozen_stars(seed=8, n_stars=216, arms=6, r_lo=0.95, r_hi=1.25, min_sep=0.6)
    s.bond_types = s.bond_types + [BondType(FENE, 30.0, 1.5)]
    per = 7
    c = per * np.arange(216, dtype=np.int32)
    s.static_bonds = np.concatenate([np.stack([c, c + a], axis=1) for a in (1, 2, 3)]).astype(np.int32)
    s.static_bond_types = np.ones(s.static_bonds.shape[0], np.int32)
    s.reactions[0].self_avoid = self_avoid
    return s


def _cases():
    return {
        "loops": lambda sa: frozen_loops(seed=5, n_units=125, self_avoid=sa, eps=1.0),
        "rings_dense": lambda sa: telechelic_rings(seed=6, n_chains=1500, beads=3, rho=0.8, self_avoid=sa),
        "star_push": _star_molecules,
    }


@pytest.mark.parametrize("name", list(_cases()))
@pytest.mark.parametrize("self_avoid", [1, 0])
@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_exclusion_sweeps_bit_exact(snapmod, name, self_avoid, precision):
    s = _cases()[name](self_avoid)
    sim = snapmod.from_system(s, precision=precision, p_on0=0.9)
    orc = oracle.OracleSystem(s, p_on0=0.9)
    try:
        for step in list(range(0, 30)) + [1000, 987654321]:
            sim.set_step(step)
            sim.bond_update()
            st_o = orc.sweep(step=step)
            b = sim.bonds()
            assert np.array_equal(b, orc.bonds()), (name, step)
            st_g = sim.stats()
            for k in SWEEP_STATS:
                assert st_g[k] == st_o[k], (name, step, k, st_g[k], st_o[k])
            same = orc.mol[b[:, 0]] == orc.mol[b[:, 1]]
            if self_avoid:
                assert not same.any()
        assert b.shape[0] > 0
        if not self_avoid:
            assert same.any()   # the excluded pairs do bond when the flag is off
    finally:
        sim.close()


def test_star_molecules_take_the_push_path(snapmod):
    s = _star_molecules(1)
    sim = snapmod.from_system(s, precision="mixed", p_on0=0.9)
    try:
        sim.set_step(3)
        sim.bond_update()
        # centres are a sixth of the arms: the sweep pushes from them, visiting
        # only their lists (a scan from every arm would visit ~6x more entries)
        st = sim.stats()
        assert 0 < st["scanned"] <= 6 * 216
    finally:
        sim.close()


@pytest.mark.parametrize("self_avoid", [1, 0])
def test_rings_md(snapmod, self_avoid):
    s = telechelic_rings(seed=9, n_chains=2000, beads=3, self_avoid=self_avoid)
    mol = oracle.molecules(s.n, s.static_bonds)
    sim = snapmod.from_system(s, precision="mixed", p_on0=1.0)
    rings = joins = 0
    try:
        for _ in range(100):
            sim.step(20)
            b = sim.bonds()
            same = mol[b[:, 0]] == mol[b[:, 1]]
            rings += int(same.sum())
            joins += int((~same).sum())
    finally:
        sim.close()
    assert joins > 1000
    if self_avoid:
        assert rings == 0
    else:
        assert rings > 1000


def test_rings_fp64_trajectory_follows_oracle(snapmod):
    s = telechelic_rings(seed=10, n_chains=300, beads=3, self_avoid=1)
    sim = snapmod.from_system(s, precision="fp64", p_on0=1.0)
    orc = oracle.OracleSystem(s, p_on0=1.0)
    try:
        for _ in range(10):
            sim.step(20)
            orc.run(20)
            d = sim.positions() - orc.pos
            d -= s.box * np.rint(d / s.box)
            assert np.abs(d).max() < 1e-9
            assert np.array_equal(sim.bonds(), orc.bonds())
        assert orc.bonds().shape[0] > 0
    finally:
        sim.close()


def test_mh_refuses_exclusion(snapmod):
    s = frozen_loops(seed=5, n_units=27, self_avoid=1)
    sim = snapmod.from_system(s, precision="mixed")
    try:
        with pytest.raises(snapmod.SnapError):
            sim.set_mh(1)
    finally:
        sim.close()

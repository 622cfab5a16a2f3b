"""The neighbour-list build with sub-cells along x, and its overflow path.

For every number of sub-cells per cell the lists hold the same pairs (every
pair within reach, nothing beyond), whole trajectories of single systems and
of batches follow the oracle's physics in FP64 and agree between slice counts
to rounding, and a list overflow in a build that runs in several waves of
blocks is retried from an intact state.
"""
import numpy as np
import pytest

import oracle
from synth import colloid_linker, random_frozen, telechelic

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def snapmod():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2609_21204_b300 import build
    build.build()
    import paper_2609_21204_b300 as m
    return m


def _systems():
    return {
        "colloid_linker": lambda: colloid_linker(seed=21, n_c=3000, n_l=12000),
        # three cells per axis: every run touches the periodic boundary
        "small_box": lambda: random_frozen(seed=22, n=int(0.4 * 5.2 ** 3), box=5.2, overlap_factor=1.0,
                                           r_max=1.3),
        # a batch of replicas of different boxes: warps straddle replicas and types
        "batched": lambda: [telechelic(seed=23 + r, n_chains=40 + 30 * r, n_x=80 + 60 * r) for r in range(3)],
    }


@pytest.mark.parametrize("name", list(_systems()))
def test_fp64_trajectories_agree_across_subcells(snapmod, name):
    """FP64 runs with 1 and 4 slices per cell: the lists hold the same pairs
    in a different order, so positions agree to FP64 rounding of the force
    sums, and the bond tables are equal."""
    sysdef = _systems()[name]()
    out = []
    for k in (1, 4):
        sim = snapmod.from_system(sysdef, precision="fp64", list_subcells=k)
        try:
            sim.step(60)
            out.append((sim.positions(), sim.bonds(), sim.stats()["nlist_builds"]))
        finally:
            sim.close()
    (p1, b1, n1), (p4, b4, n4) = out
    assert n1 >= 2 and n4 >= 2
    box = np.concatenate([np.tile(s.box, (s.n, 1)) for s in (sysdef if isinstance(sysdef, list) else [sysdef])])
    d = p4 - p1
    d -= box * np.rint(d / box)
    assert np.abs(d).max() < 1e-9
    assert np.array_equal(b1, b4)


@pytest.mark.parametrize("subcells", [1, 2, 8])
def test_lists_hold_every_pair_for_any_subcells(snapmod, subcells):
    s = colloid_linker(seed=24, n_c=2000, n_l=8000)
    sim = snapmod.from_system(s, precision="mixed", list_subcells=subcells)
    try:
        assert sim.list_subcells() == subcells
        sim.step(25)
        pos = sim.positions()
        got = {tuple(p) for p in sim.neighbors()}
    finally:
        sim.close()
    orc = oracle.OracleSystem(s)
    orc.set_positions(pos)
    need = {tuple(p) for p in orc.pairs_within(extra=0.0, reactive=True)}
    assert need <= got, len(need - got)
    allowed = {tuple(p) for p in orc.pairs_within(extra=2 * s.skin + 1e-3, reactive=True)}
    assert got <= allowed


def test_subcells_setter_rules(snapmod):
    s = random_frozen(seed=25, n=400, box=9.0, r_max=1.3)
    sim = snapmod.Snap(s.n, s.box, dt=s.dt, kT=s.kT, gamma=s.gamma, seed=s.seed, skin=s.skin)
    try:
        sim.set_types(s.sigma, s.eps_pair, s.rcut)
        with pytest.raises(snapmod.SnapError):
            sim.set_list_subcells(3)
        sim.set_list_subcells(2)
        sim.set_valence(s.valence)
    finally:
        sim.close()
    sim = snapmod.from_system(s, precision="mixed")
    try:
        assert sim.list_subcells() in (1, 2, 4, 8)
        with pytest.raises(snapmod.SnapError):
            sim.set_list_subcells(4)   # the cell grid is laid out
    finally:
        sim.close()


def test_overflow_in_a_multi_wave_list_build_regrows_transparently(snapmod):
    """Lists far too small for a 4*10^5-particle gel: the list build runs in
    several waves of blocks and the first blocks latch the overflow; every
    block must still copy its particles back, so that the retried step starts
    from an intact state and the run matches one with room to spare."""
    s = colloid_linker(seed=30, n_c=80000, n_l=320000)
    ref = snapmod.from_system(s, precision="mixed")
    small = snapmod.from_system(s, precision="mixed", nlist_capacity=8)
    try:
        ref.step(40)
        small.step(40)
        assert small.stats()["nlist_capacity"] > 8
        assert np.array_equal(ref.positions(), small.positions())
        assert np.array_equal(ref.bonds(), small.bonds())
    finally:
        ref.close()
        small.close()

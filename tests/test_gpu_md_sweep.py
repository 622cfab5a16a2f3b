"""GPU parity of a bond sweep taken after MD steps (Sec. II.C; Philox draws
keyed as in Sec. II.E).

The single-sweep parity tests start from fresh coordinates.  Here the GPU first
runs MD, so in mixed precision its FP32 cell-relative coordinates have drifted
from the FP64 positions for up to seven steps since their last re-rounding
(they are re-rounded every eight steps and at every neighbour-list rebuild),
and the FP32 screen of the proposal phase works on those drifted coordinates
while the decisions are taken in FP64.  The oracle is handed the GPU's own FP64
positions and bond table and takes one sweep with the same step counter: the
bond table and every sweep counter must agree bit for bit, in the per-site scan
and in push mode (one side scarce), at step counts that are not multiples of
eight and that cross neighbour-list rebuilds.  The same check runs once on the
equilibrated 10^6-particle colloid-linker gel, whose saturated state (about 1%
of the colloid slots free) takes the push path.
"""
import numpy as np
import pytest

import oracle
from synth import colloid_linker

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


def _push_mode(s, bonds):
    """Whether the sweep takes the push path: one reaction, two distinct
    types, and one side has at most a quarter of the other's free sites."""
    occ = np.bincount(bonds[:, :2].ravel(), minlength=s.n) if bonds.size else np.zeros(s.n, int)
    val = np.asarray(s.valence)[s.types]
    free = occ < val
    r = s.reactions[0]
    ca = int((free & (s.types == r.type_a)).sum())
    cb = int((free & (s.types == r.type_b)).sum())
    return ca * 4 <= cb or cb * 4 <= ca


def _compare_after_md(snapmod, s, precision, steps):
    sim = snapmod.from_system(s, precision=precision)
    orc = oracle.OracleSystem(s)
    sim.step(steps)
    assert sim.stats()["step"] == steps
    pos = sim.positions()
    bonds = sim.bonds()
    orc.set_positions(pos)
    orc.set_bonds(bonds)
    push = _push_mode(s, bonds)
    builds = sim.stats()["nlist_builds"]
    sim.bond_update()                 # one sweep with the step counter at `steps`
    st_o = orc.sweep(step=steps)
    b_g, b_o = sim.bonds(), orc.bonds()
    assert np.array_equal(b_g, b_o), (precision, steps, b_g.shape, b_o.shape)
    st_g = sim.stats()
    for k in SWEEP_STATS:
        assert st_g[k] == st_o[k], (precision, steps, k, st_g[k], st_o[k])
    assert st_o["formed"] + st_o["broken"] > 0
    sim.close()
    return push, builds


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_sweep_after_md_bit_exact(snapmod, precision):
    modes = set()
    # 1:4 colloids to linkers: the colloids are the scarce side from the start
    # (push mode); 3:7 at eps 1.5 keeps the two sides comparable (per-site scan)
    for n_c, n_l, eps in ((2000, 8000, 6.0), (3000, 7000, 1.5)):
        s = colloid_linker(seed=21, n_c=n_c, n_l=n_l, eps=eps)
        for steps in (13, 21, 103):
            push, builds = _compare_after_md(snapmod, s, precision, steps)
            if steps == 103:
                assert builds >= 3   # rebuilds regenerated the coordinates in between
            modes.add(push)
    assert modes == {True, False}, modes


def test_sweep_equilibrated_1m_gel_bit_exact(snapmod):
    s = colloid_linker()          # the 10^6-particle benchmark gel
    sim = snapmod.from_system(s, precision="mixed", block_size=128, skin=0.5)
    sim.step(2013)                # saturated; 2013 = 5 steps past a re-rounding of the FP32 coordinates
    pos = sim.positions()
    bonds = sim.bonds()
    assert _push_mode(s, bonds)
    orc = oracle.OracleSystem(s)
    orc.set_positions(pos)
    orc.set_bonds(bonds)
    sim.bond_update()
    st_o = orc.sweep(step=2013)
    assert np.array_equal(sim.bonds(), orc.bonds())
    st_g = sim.stats()
    for k in SWEEP_STATS:
        assert st_g[k] == st_o[k], (k, st_g[k], st_o[k])
    assert st_o["formed"] > 0 and st_o["broken"] > 0
    sim.close()


def test_retry_limit_timeout_is_reported_and_recovered(snapmod):
    """The push-mode compare-and-swap minimum gives up after a bounded number
    of retries (a defect guard).  With the limit lowered to 0 every exchange
    gives up: the sweep returns SNAP_ERR_TIMEOUT, nothing of it is applied, and
    once the limit is restored the same context continues bit-identically with
    a context that never failed."""
    s = colloid_linker(seed=22, n_c=1000, n_l=4000, eps=6.0)
    ref = snapmod.from_system(s, precision="mixed")
    sim = snapmod.from_system(s, precision="mixed")
    ref.step(120)
    sim.step(120)
    assert _push_mode(s, sim.bonds())
    before = sim.bonds()
    sim.set_retry_limit(0)
    with pytest.raises(snapmod.SnapError) as e:
        sim.bond_update()
    assert e.value.name == "SNAP_ERR_TIMEOUT"
    assert np.array_equal(sim.bonds(), before)
    with pytest.raises(snapmod.SnapError) as e:
        sim.step(20)
    assert e.value.name == "SNAP_ERR_TIMEOUT"
    assert sim.stats()["step"] == 120          # the failing step was not taken
    assert np.array_equal(sim.bonds(), before)
    sim.set_retry_limit(1 << 16)
    # the failed step left a rebuild due (it regenerates the FP32 coordinates
    # from the FP64 positions); the reference takes the same rebuild
    ref.rebuild_profiled()
    sim.step(40)
    ref.step(40)
    assert np.array_equal(sim.bonds(), ref.bonds())
    assert np.array_equal(sim.positions(), ref.positions())
    with pytest.raises(snapmod.SnapError) as e:
        sim.set_retry_limit(-1)
    assert e.value.name == "SNAP_ERR_ARG"

"""GPU parity: the CUDA path (through the C ABI) against the FP64 CPU oracle.

- A bond sweep on identical positions is bit-exact: same bond table, same
  counters (Sec. II.C; Philox draws keyed as in Sec. II.E).
- The neighbour list contains every pair inside max(pair cut, reactive cut).
- Forces: normwise relative error and per-particle error against the
  particle's sensitivity scale sum_j (|F_ij| + r_ij |dF_ij/dr|) both <= 1e-12
  (FP64) / 1e-5 (mixed FP32 forces); the virial within the same tolerance of
  its scale sum r (|F| + r |dF/dr|).
- FP64 trajectories follow the oracle step for step.
"""
import math
import struct

import numpy as np
import pytest

import oracle
from synth import (random_frozen, colloid_linker, telechelic, assoc_ab, frozen_pairs)

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


def make_pair(snapmod, sysdef, precision="mixed", p_on0=1.0, **kw):
    sim = snapmod.from_system(sysdef, precision=precision, p_on0=p_on0, **kw)
    orc = oracle.OracleSystem(sysdef, p_on0=p_on0)
    return sim, orc


def set_step(sim, step):
    st = bytearray(sim.get_state())
    struct.pack_into("<Q", st, 16, step)
    sim.set_state(bytes(st))


def _sweep_cases():
    return {
        "ab_v1": lambda: random_frozen(seed=1, n=2000, box=12.0, overlap_factor=0.6, r_max=1.4),
        "ab_v3_2": lambda: random_frozen(seed=2, n=5000, box=16.0, overlap_factor=0.6, r_max=1.5,
                                         valence=(3, 2), r_min=0.4),
        "colloid_linker": lambda: colloid_linker(seed=3, n_c=2000, n_l=8000, eps=3.0),
        "telechelic": lambda: telechelic(seed=4, n_chains=200, n_x=400),
        "tiny_ragged": lambda: random_frozen(seed=5, n=37, box=5.3, overlap_factor=0.5, r_max=1.4),
        # one side scarce (10% A): proposals by push from the scarce side
        "scarce_push": lambda: random_frozen(seed=7, n=5000, box=15.0, type_fracs=(0.1, 0.9),
                                             overlap_factor=0.6, r_max=1.4, valence=(2, 1)),
        "kT0": lambda: _kt0(),
    }


def _kt0():
    s = random_frozen(seed=6, n=1500, box=11.0, overlap_factor=0.6, r_max=1.4)
    s.kT = 0.0
    return s


SWEEP_STATS = ("in_window", "proposals", "edges", "survivors", "formed", "break_tested", "broken")


@pytest.mark.parametrize("name", list(_sweep_cases()))
@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_sweep_bit_exact(snapmod, name, precision):
    s = _sweep_cases()[name]()
    sim, orc = make_pair(snapmod, s, precision, p_on0=0.9)
    assert sim.bonds().shape[0] == 0
    for step in (0, 1, 7, 1000, 123456789012):
        set_step(sim, step)
        sim.bond_update()
        st_o = orc.sweep(step=step)
        b_g, b_o = sim.bonds(), orc.bonds()
        assert np.array_equal(b_g, b_o), (name, step, b_g.shape, b_o.shape)
        st_g = sim.stats()
        for k in SWEEP_STATS:
            assert st_g[k] == st_o[k], (name, step, k, st_g[k], st_o[k])
    # occupancies never exceed valence
    val = np.asarray(s.valence)[s.types]
    occ = np.bincount(b_g[:, :2].ravel(), minlength=s.n)
    assert np.all(occ <= val)


def test_sweep_with_preexisting_bonds(snapmod):
    s = random_frozen(seed=8, n=3000, box=14.0, overlap_factor=0.6, r_max=1.4, valence=(2, 2),
                      eps=1.0)
    sim, orc = make_pair(snapmod, s, "mixed", p_on0=1.0)
    for step in range(0, 12):
        sim.bond_update()
        orc.sweep(step=0)
    assert np.array_equal(sim.bonds(), orc.bonds())
    assert sim.bonds().shape[0] > 100
    # a new step: breaking with P_off = e^-1 plus new formation
    for step in (5, 6, 99):
        set_step(sim, step)
        sim.bond_update()
        orc.sweep(step=step)
        assert np.array_equal(sim.bonds(), orc.bonds())


def test_set_bonds_roundtrip_and_sweep(snapmod):
    s = random_frozen(seed=9, n=1200, box=10.0, overlap_factor=0.6, r_max=1.4, valence=(1, 1))
    sim, orc = make_pair(snapmod, s, "fp64")
    a = np.nonzero(s.types == 0)[0][:100]
    b = np.nonzero(s.types == 1)[0][:100]
    pairs = np.stack([np.minimum(a, b), np.maximum(a, b)], axis=1)
    sim.set_bonds(pairs, np.zeros(100, np.int32))
    orc.set_bonds([(x, y, 0) for x, y in pairs])
    assert np.array_equal(sim.bonds(), orc.bonds())
    sim.bond_update()
    orc.sweep(step=0)
    assert np.array_equal(sim.bonds(), orc.bonds())


def test_no_reactive_particles_and_empty(snapmod):
    s = random_frozen(seed=10, n=500, box=9.0, overlap_factor=0.6, valence=(0, 0))
    sim, orc = make_pair(snapmod, s)
    sim.bond_update()
    assert sim.bonds().shape[0] == 0
    sim.step(10)
    assert sim.stats()["step"] == 10


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_neighbor_list_contains_all_pairs(snapmod, precision):
    s = colloid_linker(seed=11, n_c=3000, n_l=12000)
    sim, orc = make_pair(snapmod, s, precision)
    sim.step(30)
    pos = sim.positions()
    orc.set_positions(pos)
    need = {tuple(p) for p in orc.pairs_within(extra=0.0, reactive=True)}
    got = {tuple(p) for p in sim.neighbors()}
    assert need <= got, len(need - got)
    # and nothing beyond the list cut-off plus the skin margin
    # each end may have moved skin/2 since the build: pairs listed at the build
    # cut-off rl = max(cut, r_max) + skin can now be up to rl + skin apart
    allowed = {tuple(p) for p in orc.pairs_within(extra=2 * s.skin + 1e-3, reactive=True)}
    assert got <= allowed


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
@pytest.mark.parametrize("box", [5.2, 7.0])
def test_neighbor_list_small_boxes(snapmod, precision, box):
    """Boxes of three and four cells per axis: every run of row-adjacent
    cells touches the periodic boundary (the runs across it are split), and
    the lists still hold every pair within reach and nothing beyond."""
    s = random_frozen(seed=61, n=int(0.4 * box ** 3), box=box, overlap_factor=1.0, r_max=1.3)
    sim, orc = make_pair(snapmod, s, precision)
    need = {tuple(p) for p in orc.pairs_within(extra=0.0, reactive=True)}
    got = {tuple(p) for p in sim.neighbors()}
    assert len(need) > 50
    assert need <= got, len(need - got)
    allowed = {tuple(p) for p in orc.pairs_within(extra=2 * s.skin + 1e-3, reactive=True)}
    assert got <= allowed


def test_fp64_trajectory_in_a_three_cell_box(snapmod):
    """The smallest periodic box the cell list takes (three cells per axis):
    FP64 MD with the sweep follows the oracle step for step, so the list
    build's boundary runs and the force list's stored cell shifts are right
    when every neighbour cell is a periodic image."""
    s = colloid_linker(seed=62, n_c=40, n_l=160, eps=3.0)
    assert s.box[0] < 4 * (1.2 + s.skin + 1e-3)
    sim, orc = make_pair(snapmod, s, "fp64")
    for _ in range(6):
        sim.step(20)
        orc.run(20)
        d = sim.positions() - orc.pos
        d -= s.box * np.rint(d / s.box)
        assert np.abs(d).max() < 1e-9
        assert np.array_equal(sim.bonds(), orc.bonds())
    assert sim.stats()["nlist_builds"] > 2


def _force_err(f, g, scale):
    """Normwise relative error, and the per-particle error against the
    sensitivity scale G_i = sum_j (|F_ij| + r_ij |dF_ij/dr|) the oracle reports:
    |F_gpu,i - F_i| <= tol G_i says that the GPU force is the exact force of a
    configuration whose separations and force terms are perturbed by a
    relative ~tol at most (FP32 coordinates carry such a perturbation; a
    missing, doubled or wrong pair or bond term shifts F_i by a sizable
    fraction of G_i).  Also returns the per-particle error with the floor
    max(|F_i|, 1e-3 F_rms), which ignores the conditioning of the force sum
    and of the steep WCA force near its cut, for the record."""
    num = np.linalg.norm(f - g)
    den = np.linalg.norm(g)
    rms = den / math.sqrt(g.shape[0])
    d = np.linalg.norm(f - g, axis=1)
    per_scale = np.where(scale > 0, d / np.where(scale > 0, scale, 1.0), np.where(d > 0, np.inf, 0.0))
    per_floor = d / np.maximum(np.linalg.norm(g, axis=1), 1e-3 * rms)
    return num / den, per_scale.max(), per_floor.max()


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("mixed", 1e-5)])
def test_forces_match_oracle(snapmod, precision, tol):
    s = telechelic(seed=12, n_chains=300, n_x=600)
    sim, orc = make_pair(snapmod, s, precision)
    sim.step(200)  # dynamic bonds form; static FENE bonds present
    pos = sim.positions()
    bonds = sim.bonds()
    assert bonds.shape[0] > 50
    orc.set_positions(pos)
    orc.set_bonds(bonds)
    f_g = sim.forces()
    f_o, eo = orc.forces()
    norm_err, per_scale, per_floor = _force_err(f_g, f_o, eo["fscale"])
    assert norm_err <= tol, (norm_err, per_scale, per_floor)
    assert per_scale <= tol, (norm_err, per_scale, per_floor)
    # energies and virial through the deterministic reduction; the virial's
    # scale is sum r (|F| + r |dF/dr|) (pair and bond terms cancel in part)
    e = sim.energy()
    assert e["e_pair"] == pytest.approx(eo["e_pair"], rel=1e-4 if precision == "mixed" else 1e-10)
    assert e["e_bond"] == pytest.approx(eo["e_bond"], rel=1e-4 if precision == "mixed" else 1e-10)
    assert abs(e["virial"] - eo["virial"]) <= tol * eo["virial_scale"], (e["virial"], eo["virial"])


def test_forces_full_colloid_gel(snapmod):
    s = colloid_linker(seed=13, n_c=20000, n_l=80000)
    for precision, tol in (("fp64", 1e-12), ("mixed", 1e-5)):
        sim, orc = make_pair(snapmod, s, precision)
        for steps in (0, 103):   # fresh coordinates, then after FP32 drift between re-roundings
            if steps:
                sim.step(steps)
                orc.set_positions(sim.positions())
                orc.set_bonds(sim.bonds())
            f_g = sim.forces()
            f_o, eo = orc.forces()
            norm_err, per_scale, per_floor = _force_err(f_g, f_o, eo["fscale"])
            assert norm_err <= tol, (precision, steps, norm_err, per_scale, per_floor)
            assert per_scale <= tol, (precision, steps, norm_err, per_scale, per_floor)
            e = sim.energy()
            assert abs(e["virial"] - eo["virial"]) <= tol * eo["virial_scale"], (precision, steps)
            assert e["e_pair"] == pytest.approx(eo["e_pair"], rel=1e-4 if precision == "mixed" else 1e-10)
        sim.close()


def test_fp64_trajectory_follows_oracle(snapmod):
    s = assoc_ab(seed=14)
    sim, orc = make_pair(snapmod, s, "fp64")
    for _ in range(5):
        sim.step(20)
        orc.run(20)
        d = sim.positions() - orc.pos
        d -= s.box * np.rint(d / s.box)
        assert np.abs(d).max() < 1e-9
        assert np.array_equal(sim.bonds(), orc.bonds())
    v = sim.velocities() - np.stack([orc.vx, orc.vy, orc.vz], axis=1)
    assert np.abs(v).max() < 1e-7


@pytest.mark.parametrize("block", [32, 64, 128, 192])
def test_results_independent_of_block_size(snapmod, block):
    s = colloid_linker(seed=15, n_c=1000, n_l=4000, eps=3.0)
    ref = snapmod.from_system(s, precision="mixed")
    ref.step(120)
    alt = snapmod.from_system(s, precision="mixed", block_size=block)
    alt.step(120)
    assert np.array_equal(ref.bonds(), alt.bonds())
    assert np.array_equal(ref.positions(), alt.positions())


@pytest.mark.parametrize("list_block", [64, 128])
def test_results_independent_of_list_block(snapmod, list_block):
    """The list build's threads per block (an autotuned launch shape) leaves
    the lists, and so every trajectory, unchanged."""
    s = colloid_linker(seed=16, n_c=1000, n_l=4000, eps=3.0)
    ref = snapmod.from_system(s, precision="mixed")
    ref.step(120)
    alt = snapmod.from_system(s, precision="mixed", list_block=list_block)
    alt.step(120)
    assert ref.stats()["nlist_builds"] == alt.stats()["nlist_builds"] > 1
    assert np.array_equal(ref.bonds(), alt.bonds())
    assert np.array_equal(ref.positions(), alt.positions())
    with pytest.raises(snapmod.SnapError) as e:
        alt.set_list_block(96)
    assert e.value.name == "SNAP_ERR_ARG"


def test_block_size_above_launch_bound_is_rejected(snapmod):
    s = colloid_linker(seed=15, n_c=100, n_l=400)
    for bad in (512, 1024, 100):
        with pytest.raises(snapmod.SnapError) as e:
            snapmod.from_system(s, precision="mixed", block_size=bad)
        assert e.value.name == "SNAP_ERR_ARG"


@pytest.mark.parametrize("mode", ["plain", "none"])
def test_graph_modes_agree(snapmod, mode, monkeypatch):
    s = colloid_linker(seed=19, n_c=1000, n_l=4000, eps=3.0)
    ref = snapmod.from_system(s, precision="mixed")
    ref.step(80)
    monkeypatch.setenv("SNAP_GRAPH_MODE", mode)
    alt = snapmod.from_system(s, precision="mixed")
    alt.step(80)
    assert np.array_equal(ref.bonds(), alt.bonds())
    assert np.array_equal(ref.positions(), alt.positions())


def test_checkpoint_resume_is_bit_identical(snapmod):
    s = colloid_linker(seed=16, n_c=1000, n_l=4000, eps=3.0)
    a = snapmod.from_system(s, precision="mixed")
    a.step(50)
    state = a.get_state()
    a.step(70)
    b = snapmod.from_system(s, precision="mixed")
    b.set_state(state)
    b.step(70)
    assert np.array_equal(a.positions(), b.positions())
    assert np.array_equal(a.bonds(), b.bonds())
    assert np.array_equal(a.velocities(), b.velocities())


def test_neighbor_overflow_regrows_transparently(snapmod):
    s = colloid_linker(seed=17, n_c=1000, n_l=4000, eps=3.0)
    ref = snapmod.from_system(s, precision="mixed")
    ref.step(60)
    small = snapmod.from_system(s, precision="mixed", nlist_capacity=8)
    small.step(60)
    assert small.stats()["nlist_capacity"] > 8
    assert np.array_equal(ref.bonds(), small.bonds())
    assert np.array_equal(ref.positions(), small.positions())


def test_error_paths_report_status(snapmod):
    s = telechelic(seed=18, n_chains=50, n_x=100)
    sim = snapmod.from_system(s, precision="mixed")
    pos = s.pos.copy()
    pos[0] = np.nan
    with pytest.raises(snapmod.SnapError) as e:
        sim.set_positions(pos)
    assert e.value.name == "SNAP_ERR_NONFINITE"
    # FENE bond stretched beyond R0 = 1.5
    pos = s.pos.copy()
    pos[1] = pos[0] + np.array([1.6, 0.0, 0.0])
    sim.set_positions(pos % s.box)
    with pytest.raises(snapmod.SnapError) as e:
        sim.forces()
    assert e.value.name == "SNAP_ERR_FENE_OVERSTRETCH"
    # runaway velocity -> non-finite position latched on the device
    sim2 = snapmod.from_system(s, precision="mixed")
    vel = s.vel.copy()
    vel[3] = 1e308
    sim2.set_positions(s.pos, vel)
    with pytest.raises(snapmod.SnapError) as e:
        sim2.step(3)
    assert e.value.name == "SNAP_ERR_NONFINITE"
    with pytest.raises(snapmod.SnapError):
        sim2.add_reaction(1, 2, 0, 0.0, 1.2, 1.0, 0.1)  # FENE bond type cannot react


def test_batched_replicas_match_standalone(snapmod):
    # non-overlapping placement (MD needs finite WCA forces) at uneven sizes
    reps = [random_frozen(seed=30 + r, n=600 + 137 * r, box=12.0 + r, overlap_factor=1.0,
                          r_max=1.4, eps=1.0 + r) for r in range(4)]
    for r, s in enumerate(reps):
        s.seed = 1000 + 17 * r
        s.kT = 0.9 + 0.1 * r
    sim = snapmod.from_system(reps, precision="fp64", p_on0=0.8)
    orcs = [oracle.OracleSystem(s, p_on0=0.8) for s in reps]
    # one sweep on the frozen start, then 25 MD steps (graph launches plus a remainder)
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


def test_batched_bonded_fraction_matches_oracle_statistics(snapmod):
    """Mixed-precision batched run of four small telechelic replicas (uneven N,
    eps and kT) against independent FP64 oracle runs from the same start: the
    time-averaged bonded fraction of chain ends agrees per replica within the
    statistical error of two independent trajectories."""
    from synth import telechelic_sweep_specs, telechelic
    specs = telechelic_sweep_specs(seed=77, n_replicas=4, n_lo=1200, n_hi=2400)
    reps = [telechelic(**kw) for kw in specs]
    sim = snapmod.from_system(reps, precision="mixed")
    orcs = [oracle.OracleSystem(s) for s in reps]
    n_ends = [int((s.types == 1).sum()) for s in reps]
    gpu_series, orc_series = [[] for _ in reps], [[] for _ in reps]
    for block in range(24):
        sim.step(50)
        b = sim.bonds()
        off = 0
        for r, s in enumerate(reps):
            sel = (b[:, 0] >= off) & (b[:, 0] < off + s.n)
            gpu_series[r].append(sel.sum() / n_ends[r])
            off += s.n
        for r, o in enumerate(orcs):
            o.run(50)
            orc_series[r].append(o.bonds().shape[0] / n_ends[r])
    for r in range(len(reps)):
        g = np.array(gpu_series[r][8:])
        o = np.array(orc_series[r][8:])
        se = math.sqrt(g.var() / g.size + o.var() / o.size) + 0.02
        assert abs(g.mean() - o.mean()) < 4 * se, (r, specs[r], g.mean(), o.mean(), se)


def test_host_io_wraps_and_counts_images(snapmod):
    """Positions set outside the box come back wrapped into [0, L) with the
    crossings in the image counters; velocities round-trip (FP32 in mixed
    mode); non-finite input is rejected without touching the state."""
    s = random_frozen(seed=61, n=3000, box=14.0, overlap_factor=0.6)
    L = float(s.box[0])
    for precision, vtol in (("fp64", 0.0), ("mixed", 1e-7)):
        sim = snapmod.from_system(s, precision=precision)
        shift = np.array([[2, -1, 0], [-3, 0, 5], [0, 1, -1]])[np.arange(s.n) % 3]
        raw = s.pos + shift * L
        vel = np.random.default_rng(1).normal(size=(s.n, 3))
        sim.set_positions(raw, vel)
        got = sim.positions()
        assert np.all(got >= 0.0) and np.all(got < L)
        np.testing.assert_allclose(got, s.pos, rtol=0, atol=1e-12)
        assert np.array_equal(sim.images(), shift)
        np.testing.assert_allclose(sim.velocities(), vel, rtol=vtol, atol=0)
        out = np.empty((s.n, 3))
        assert sim.positions(out=out) is out and np.array_equal(out, got)
        bad = raw.copy()
        bad[7, 1] = np.nan
        with pytest.raises(snapmod.SnapError):
            sim.set_positions(bad)
        np.testing.assert_array_equal(sim.positions(), got)
        sim.close()

"""GPU test of snap_pair_energy_noalloc, the entry point that allocates no
device memory (for callers that cannot allocate while they run).  Its result
must match the context path (snap_get_energy, FP64) and the FP64 oracle's pair
energy and virial within the FP64 tolerance of the other energy tests, on two
calls in a row whose inputs differ in size, so the second call runs over
scratch left by the first.  Collected last on purpose: a failure here leaves
every other test run."""
import numpy as np
import pytest

import oracle
from synth import colloid_linker, assoc_ab

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2609_21204_b300 import build
    build.build()
    import paper_2609_21204_b300 as snap
    return torch, snap


def _reference_energy(snap, s):
    sim = snap.from_system(s, precision="fp64")
    e = sim.energy()
    pos = sim.positions()
    sim.close()
    return pos, e


def _noalloc_energy(torch, snap, s, pos, types=None):
    dev = torch.device("cuda")
    d_pos = torch.tensor(np.ascontiguousarray(pos), dtype=torch.float64, device=dev)
    d_type = torch.tensor(s.types if types is None else types, dtype=torch.int32, device=dev)
    d_out = torch.full((2,), float("nan"), dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream()
    snap.pair_energy_noalloc(pos.shape[0], d_pos.data_ptr(), d_type.data_ptr(), s.box, s.sigma, s.eps_pair,
                             s.rcut, d_out.data_ptr(), stream.cuda_stream)
    torch.cuda.synchronize()
    return d_out.cpu().numpy()


def test_noalloc_energy_matches_context_two_calls(env):
    torch, snap = env
    big = colloid_linker(seed=41, n_c=1600, n_l=6400)      # 8000 particles
    small = assoc_ab(seed=42, n_a=900, n_b=900, rho=0.3)   # 1800 particles, after the big one
    for s in (big, small):
        pos, ref = _reference_energy(snap, s)
        got = _noalloc_energy(torch, snap, s, pos)
        # no bonds in either system: the context's virial is the pair virial alone
        assert ref["e_bond"] == 0.0
        assert ref["e_pair"] != 0.0
        assert got[0] == pytest.approx(ref["e_pair"], rel=1e-10, abs=1e-12)
        assert got[1] == pytest.approx(ref["virial"], rel=1e-10, abs=1e-12)
        # and against the FP64 oracle on the same positions
        orc = oracle.OracleSystem(s)
        orc.set_positions(pos)
        _, eo = orc.forces()
        assert eo["e_bond"] == 0.0
        assert got[0] == pytest.approx(eo["e_pair"], rel=1e-10, abs=1e-12)
        assert abs(got[1] - eo["virial"]) <= 1e-12 * eo["virial_scale"]


def test_noalloc_out_of_range_types_take_no_pair(env):
    torch, snap = env
    s = assoc_ab(seed=43, n_a=500, n_b=500, rho=0.3)
    pos, _ = _reference_energy(snap, s)
    keep = np.ones(s.n, bool)
    keep[::7] = False
    bad = s.types.copy()
    bad[~keep] = np.where(np.arange(s.n)[~keep] % 2 == 0, -1, 8)   # below 0 and >= SNAP_MAX_TYPES
    got = _noalloc_energy(torch, snap, s, pos, bad)
    sub = _noalloc_energy(torch, snap, s, pos[keep], s.types[keep])
    assert np.all(np.isfinite(got))
    assert got[0] == pytest.approx(sub[0], rel=1e-12, abs=1e-12)
    assert got[1] == pytest.approx(sub[1], rel=1e-12, abs=1e-12)


def test_noalloc_rejects_oversize(env):
    torch, snap = env
    with pytest.raises(snap.SnapError) as e:
        snap.pair_energy_noalloc(70000, 0, 0, [10.0] * 3, [1.0], [1.0], None, 0, None)
    assert e.value.name == "SNAP_ERR_ARG"

"""GPU path with FENE dynamic bonds (Sec. II.B: U_b in Eq. 3 is the bond
type's own energy; Sec. II.C: proposals aim at the minimum of the bond term,
r = 0 for FENE), through the C ABI against the FP64 oracle.

- Sweeps are bit-exact against the oracle in both precisions on a contested
  frozen configuration (the FENE energy uses the library's own logarithm on
  both sides, so every acceptance decides alike).
- FP64 MD with FENE dynamic bonds follows the oracle step for step.
- The slip bond and the Metropolis-Hastings move set refuse a FENE reaction.
"""
import numpy as np
import pytest

import oracle
from synth import random_frozen, assoc_ab, BondType, FENE

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


def _fene(s, k=3.0, R0=1.5):
    s.bond_types = [BondType(FENE, k, R0)]
    return s


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_fene_sweeps_bit_exact(snapmod, precision):
    s = _fene(random_frozen(seed=31, n=3000, box=14.0, overlap_factor=0.6, r_max=1.45, valence=(2, 2),
                            eps=2.0))
    sim = snapmod.from_system(s, precision=precision, p_on0=0.9)
    orc = oracle.OracleSystem(s, p_on0=0.9)
    try:
        formed = 0
        for step in list(range(0, 30)) + [1000, 77777777777]:
            sim.set_step(step)
            sim.bond_update()
            st_o = orc.sweep(step=step)
            assert np.array_equal(sim.bonds(), orc.bonds()), step
            st_g = sim.stats()
            for k in SWEEP_STATS:
                assert st_g[k] == st_o[k], (step, k, st_g[k], st_o[k])
            formed += st_o["formed"]
        assert formed > 100 and st_o["survivors"] > st_o["formed"]   # some rejected by the FENE factor
    finally:
        sim.close()


def test_fene_fp64_trajectory_follows_oracle(snapmod):
    s = _fene(assoc_ab(seed=17))
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
        assert orc.bonds().shape[0] > 0
    finally:
        sim.close()


def test_fene_reaction_refuses_slip_and_mh(snapmod):
    s = _fene(assoc_ab(seed=18, n_a=64, n_b=64))
    sim = snapmod.from_system(s, precision="mixed")
    try:
        with pytest.raises(snapmod.SnapError):
            sim.set_slip(0, 1.0)
        with pytest.raises(snapmod.SnapError):
            sim.set_mh(1)
    finally:
        sim.close()

"""GPU path with the FENEWCA and Tether bond evaluators (Sec. II.B: the updater
accepts HOOMD-blue's Harmonic, FENEWCA and Tether bonds), through the C ABI
against the FP64 oracle.

- Sweeps whose reaction forms FENEWCA or Tether bonds are bit-exact against
  the oracle in both precisions (the acceptance evaluates the energy from the
  FP64 separation with the library's exp and log on both sides; proposals aim
  at the energy minimum computed alike on both sides).
- Forces of static FENEWCA (Kremer-Grest chains) and Tether bonds agree per
  particle within the force tolerance of the sensitivity scale.
- FP64 MD with Tether dynamic bonds follows the oracle step for step.
- A Tether bond at or beyond l_max latches SNAP_ERR_FENE_OVERSTRETCH; invalid
  parameters are refused.
"""
import numpy as np
import pytest

import oracle
from synth import random_frozen, telechelic, assoc_ab, BondType, FENEWCA, TETHER

pytestmark = pytest.mark.gpu

SWEEP_STATS = ("in_window", "proposals", "edges", "survivors", "formed", "break_tested", "broken")
TETHER_P = (1.0, 0.7, (0.95, 1.1, 2.0))        # k_b, l_min, (l_c1, l_c0, l_max)
FENEWCA_P = (3.0, 1.5, (1.0, 1.0, 0.1))        # k, R0, (eps, sigma, delta)


@pytest.fixture(scope="module")
def snapmod():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2609_21204_b300 import build
    build.build()
    import paper_2609_21204_b300 as m
    return m


def _contested(kind, params):
    s = random_frozen(seed=41, n=3000, box=14.0, overlap_factor=0.6, r_max=1.4, valence=(2, 2), eps=2.0)
    s.bond_types = [BondType(kind, params[0], params[1], params[2])]
    return s


@pytest.mark.parametrize("kind,params", [(FENEWCA, FENEWCA_P), (TETHER, TETHER_P)])
@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_bond_kind_sweeps_bit_exact(snapmod, kind, params, precision):
    s = _contested(kind, params)
    sim = snapmod.from_system(s, precision=precision, p_on0=1.0)
    orc = oracle.OracleSystem(s, p_on0=1.0)
    formed = broken = rejected = 0
    try:
        for step in list(range(0, 12)) + [1000, 88888888888]:
            sim.set_step(step)
            sim.bond_update()
            st_o = orc.sweep(step=step)
            assert np.array_equal(sim.bonds(), orc.bonds()), (kind, precision, step)
            st_g = sim.stats()
            for k in SWEEP_STATS:
                assert st_g[k] == st_o[k], (kind, precision, step, k, st_g[k], st_o[k])
            formed += st_o["formed"]
            broken += st_o["broken"]
            rejected += st_o["survivors"] - st_o["formed"]
        assert formed > 200 and broken > 20 and rejected > 20   # the energy factor decides some
    finally:
        sim.close()


def _force_err(f, g, scale):
    d = np.linalg.norm(f - g, axis=1)
    per = np.where(scale > 0, d / np.where(scale > 0, scale, 1.0), np.where(d > 0, np.inf, 0.0))
    return np.linalg.norm(f - g) / np.linalg.norm(g), per.max()


# chain bonds: Kremer-Grest FENEWCA, and a Tether stiff enough (k_b = 20) that no
# bond wanders near l_max, where the potential diverges faster than a 0.005 step resolves
@pytest.mark.parametrize("kind,params", [(FENEWCA, (30.0, 1.5, (1.0, 1.0, 0.0))),
                                         (TETHER, (20.0, 0.7, (0.95, 1.1, 2.0)))])
@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("mixed", 1e-5)])
def test_static_bond_kind_forces(snapmod, kind, params, precision, tol):
    s = telechelic(seed=42, n_chains=300, n_x=600)
    s.bond_types[0] = BondType(kind, params[0], params[1], params[2])   # the chain bonds
    sim = snapmod.from_system(s, precision=precision)
    orc = oracle.OracleSystem(s)
    sim.step(150)
    orc.set_positions(sim.positions())
    orc.set_bonds(sim.bonds())
    f_g = sim.forces()
    f_o, eo = orc.forces()
    assert eo["status"] == 0
    norm, per = _force_err(f_g, f_o, eo["fscale"])
    assert norm <= tol and per <= tol, (kind, precision, norm, per)
    e = sim.energy()
    assert e["e_bond"] == pytest.approx(eo["e_bond"], rel=1e-4 if precision == "mixed" else 1e-10)
    assert abs(e["virial"] - eo["virial"]) <= tol * eo["virial_scale"]
    sim.close()


def test_tether_fp64_trajectory_follows_oracle(snapmod):
    s = assoc_ab(seed=43)
    s.bond_types = [BondType(TETHER, *TETHER_P[:2], TETHER_P[2])]
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


def test_tether_overstretch_and_validation(snapmod):
    s = assoc_ab(seed=44, n_a=50, n_b=50)
    s.reactions = []
    s.static_bonds = np.array([[0, 1]], np.int32)
    s.static_bond_types = np.array([0], np.int32)
    s.bond_types = [BondType(TETHER, *TETHER_P[:2], TETHER_P[2])]
    pos = s.pos.copy()
    pos[1] = (pos[0] + np.array([2.1, 0.0, 0.0])) % s.box
    s.pos = pos
    sim = snapmod.from_system(s, precision="mixed")
    with pytest.raises(snapmod.SnapError) as e:
        sim.forces()
    assert e.value.name == "SNAP_ERR_FENE_OVERSTRETCH"
    bad = [(TETHER, 1.0, 0.7, (1.2, 1.1, 2.0)),     # l_c1 > l_c0
           (TETHER, 1.0, 0.7, (0.95, 1.1)),         # too few parameters
           (FENEWCA, 3.0, 1.5, (1.0, 0.0, 0.0)),    # sigma = 0
           (FENEWCA, 3.0, 1.5, (1.0, 1.0, -0.1)),   # delta < 0
           (7, 1.0, 1.0, ())]                       # unknown kind
    for kind, k, r0, extra in bad:
        with pytest.raises(snapmod.SnapError) as e:
            sim.set_bond_params(0, kind, k, r0, extra)
        assert e.value.name == "SNAP_ERR_ARG"
    with pytest.raises(snapmod.SnapError) as e:   # the two-number call is for harmonic and FENE
        sim._check(sim._lib.snap_set_bond_params(sim._ctx, 0, TETHER, 1.0, 0.7))
    assert e.value.name == "SNAP_ERR_ARG"

"""Pins of the oracle's virial and of its per-particle force scale.

- Virial: W = sum over pairs and bonds of r_ij . F_ij = -sum r dU/dr.  Scaling
  every coordinate and the box by lambda multiplies every separation by lambda,
  so dE/dlambda at lambda = 1 equals sum r dU/dr = -W.  A central difference of
  the oracle's own energy under that scaling pins the virial's sign, its pair
  term and its bond terms (static FENE, dynamic harmonic and FENE) at once,
  independently of how the virial is accumulated.
- Force sensitivity scale G_i = sum_j (|F_ij| + r_ij |dF_ij/dr|) over the pair
  and bond forces on particle i (relative perturbations of at most e in every
  separation and in every term change F_i by at most ~e G_i; it is the scale
  of the per-particle force parity): for a lone pair, bond or WCA, it equals
  |F| + r |dF/dr| with the derivative taken by central differences of the
  oracle's own force; in any configuration |F_i| <= G_i, G_i = 0 without a
  partner in reach, and the virial scale sum r (|F| + r |dF/dr|) bounds |W|.
"""
import numpy as np
import pytest

from synth import telechelic, assoc_ab, random_frozen
from synth.configs import BondType


def _scaled_energy(o, pos, box, lam):
    for d in range(3):
        o.params.box[d] = float(box[d] * lam)
    o.set_positions(pos * lam)
    _, e = o.forces()
    return e["e_pair"] + e["e_bond"]


def _check_virial_scaling(o, h=1e-6, rtol=1e-6):
    pos = o.pos.copy()
    box = np.array([o.params.box[d] for d in range(3)])
    ep = _scaled_energy(o, pos, box, 1.0 + h)
    em = _scaled_energy(o, pos, box, 1.0 - h)
    _scaled_energy(o, pos, box, 1.0)
    _, e = o.forces()
    dE = (ep - em) / (2 * h)
    assert abs(-dE - e["virial"]) <= rtol * e["virial_scale"], (dE, e["virial"], e["virial_scale"])
    return e


def test_virial_is_minus_energy_derivative_under_scaling(oracle_mod):
    s = telechelic(seed=3, n_chains=20, beads=12, n_x=60, rho=0.5)
    o = oracle_mod.OracleSystem(s)
    o.run(200)   # dynamic harmonic bonds form beside the static FENE bonds
    assert o.bonds().shape[0] > 0
    e = _check_virial_scaling(o)
    # both the pair and the bond terms contribute
    assert e["e_bond"] > 0 and e["e_pair"] > 0


def test_virial_scaling_with_fene_dynamic_bonds(oracle_mod):
    s = random_frozen(seed=4, n=400, box=9.0, overlap_factor=0.9, r_max=1.4, eps=2.0)
    s.bond_types = [BondType(oracle_mod.FENE, 3.0, 1.5)]
    o = oracle_mod.OracleSystem(s)
    for step in range(5):
        o.sweep(step=step)
    assert o.bonds().shape[0] > 10
    _check_virial_scaling(o)


def _pair_force(o, r):
    o.x[:] = [5.0, 5.0 + r]
    f, e = o.forces()
    return f, e


def _check_scale_by_differences(o, r, h=1e-6):
    """G = |F| + r |dF/dr| of a lone pair (pair or bond term), with dF/dr by a
    central difference of the oracle's own force; the virial scale is r G."""
    f, e = _pair_force(o, r)
    fp, _ = _pair_force(o, r + h)
    fm, _ = _pair_force(o, r - h)
    # force on particle 1 along +x is F(r) (positive: repulsive)
    dF = (fp[1, 0] - fm[1, 0]) / (2 * h)
    G = abs(f[1, 0]) + r * abs(dF)
    np.testing.assert_allclose(e["fscale"], [G, G], rtol=1e-6)
    assert e["virial_scale"] == pytest.approx(r * G, rel=1e-6)
    return f, e


def test_force_scale_of_lone_pairs_and_bounds(oracle_mod):
    s = assoc_ab(seed=1, n_a=1, n_b=1, rho=0.001)
    s.reactions = []
    o = oracle_mod.OracleSystem(s)
    o.y[:] = [5.0, 5.0]
    o.z[:] = [5.0, 5.0]
    for r in (0.95, 1.05, 1.12):            # WCA pair, up to just inside the cut 2^(1/6)
        f, e = _check_scale_by_differences(o, r)
        assert e["virial"] == pytest.approx(r * f[1, 0], rel=1e-12)
    _, e = _pair_force(o, 2.5)             # out of reach: no force, zero scale
    assert np.all(e["fscale"] == 0.0) and e["virial_scale"] == 0.0
    # static harmonic and FENE bonds at separations beyond the WCA cut
    for kind, k, r0, r in ((oracle_mod.HARMONIC, 100.0, 1.0, 1.3), (oracle_mod.FENE, 30.0, 1.5, 1.3)):
        s.static_bonds = np.array([[0, 1]], np.int32)
        s.static_bond_types = np.array([0], np.int32)
        s.bond_types = [BondType(kind, k, r0)]
        ob = oracle_mod.OracleSystem(s)
        ob.y[:] = [5.0, 5.0]
        ob.z[:] = [5.0, 5.0]
        f, e = _check_scale_by_differences(ob, r)
        assert e["virial"] == pytest.approx(r * f[1, 0], rel=1e-12)
    # dense configuration with bonds: |F_i| <= G_i and |W| <= the virial scale
    s2 = telechelic(seed=5, n_chains=30, beads=12, n_x=60, rho=0.5)
    o2 = oracle_mod.OracleSystem(s2)
    o2.run(100)
    f2, e2 = o2.forces()
    assert np.all(np.linalg.norm(f2, axis=1) <= e2["fscale"] * (1 + 1e-12))
    assert abs(e2["virial"]) <= e2["virial_scale"]

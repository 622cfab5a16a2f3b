"""GPU path with several reactions competing for shared sites (Sec. II.C: the
reactions of a sweep run one after another in an order redrawn every sweep;
App. A: the frozen four-reaction test of Eq. Z and its mobile version),
through the C ABI against the FP64 oracle.

- Sweeps are bit-exact against the oracle (bond tables and counters) on the
  frozen squares and on a contested random four-type configuration, in both
  precisions.
- Frozen squares: the GPU's state populations over many sweeps reproduce
  Eq. Z within the statistical bound the oracle meets (0.006).
- Mobile soup: FP64 trajectories follow the oracle step for step; a long
  mixed-precision run exchanges partners (distinct bonded pairs > 3x the most
  present at once), branches by K, and keeps the mass-action cross ratio
  n_AB n_DC / (n_AC n_DB) = K_AB K_DC / (K_AC K_DB).
"""
import math

import numpy as np
import pytest

import oracle
from synth import frozen_squares, four_reaction_soup
from _competing import eq_z_states, square_masks

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


def _cases():
    return {
        "squares": lambda: frozen_squares(seed=5, n_squares=125, eps=(0.3, 1.2, 0.8, 2.1)),
        # dense, overlapping placement: many candidates per site, all four reactions contested
        "contested": lambda: four_reaction_soup(seed=6, n=4000, rho=0.9, overlap_factor=0.6, r_max=1.4,
                                                eps=(1.0, 2.0, 0.5, 1.5)),
    }


@pytest.mark.parametrize("name", list(_cases()))
@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_four_reaction_sweeps_bit_exact(snapmod, name, precision):
    s = _cases()[name]()
    sim = snapmod.from_system(s, precision=precision, p_on0=0.8)
    orc = oracle.OracleSystem(s, p_on0=0.8)
    try:
        for step in list(range(0, 40)) + [1000, 123456789]:
            sim.set_step(step)
            sim.bond_update()
            st_o = orc.sweep(step=step)
            assert np.array_equal(sim.bonds(), orc.bonds()), (name, step)
            st_g = sim.stats()
            for k in SWEEP_STATS:
                assert st_g[k] == st_o[k], (name, step, k, st_g[k], st_o[k])
        assert sim.bonds().shape[0] > 0
        assert set(sim.bonds()[:, 2].tolist()) == {0, 1, 2, 3}
    finally:
        sim.close()


def test_frozen_squares_populations_follow_eq_z(snapmod):
    eps = (1.5, 0.2, 2.0, 1.0)
    s = frozen_squares(seed=9, n_squares=512, eps=eps)
    sim = snapmod.from_system(s, precision="mixed", p_on0=1.0)
    orc = oracle.OracleSystem(s, p_on0=1.0)
    nq = s.n // 4
    counts = np.zeros(16)
    try:
        for t in range(2050):
            sim.set_step(t)
            sim.bond_update()
            b = sim.bonds()
            if t < 50:   # the first sweeps step for step with the oracle
                orc.sweep(step=t)
                assert np.array_equal(b, orc.bonds()), t
            else:
                counts += np.bincount(square_masks(b, nq), minlength=16)
    finally:
        sim.close()
    f = counts / counts.sum()
    exact = eq_z_states(eps)
    assert f[[m for m in range(16) if m not in exact]].sum() == 0.0
    dev = max(abs(f[m] - p) for m, p in exact.items())
    assert dev < 0.006, (dev, {m: (round(f[m], 4), round(p, 4)) for m, p in exact.items()})


def test_soup_fp64_trajectory_follows_oracle(snapmod):
    s = four_reaction_soup(seed=12, n=1000, rho=0.3, eps=(0.5, 1.5, 1.0, 2.5))
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
        assert set(orc.bonds()[:, 2].tolist()) == {0, 1, 2, 3}
    finally:
        sim.close()


def test_soup_long_run_exchanges_and_branches(snapmod):
    eps = (0.5, 1.5, 1.0, 2.5)
    s = four_reaction_soup(seed=13, n=8000, rho=0.3, eps=eps)
    sim = snapmod.from_system(s, precision="mixed", p_on0=1.0)
    seen, most, per_rx, snaps = set(), 0, np.zeros(4), 0
    try:
        sim.step(500)
        for _ in range(1000):
            sim.step(20)
            b = sim.bonds()
            most = max(most, len(b))
            seen.update(map(tuple, b[:, :2].tolist()))
            per_rx += np.bincount(b[:, 2], minlength=4)
            snaps += 1
        occ = np.bincount(b[:, :2].ravel(), minlength=s.n)
        assert occ.max() <= 1
    finally:
        sim.close()
    assert len(seen) > 3 * most, (len(seen), most)
    ab, ac, db, dc = per_rx / snaps
    assert ac > ab and dc > db and db > ab and dc > ac, (ab, ac, db, dc)
    cross = math.log(ab * dc / (ac * db))
    assert abs(cross - (eps[0] + eps[3] - eps[1] - eps[2])) < 0.1, cross

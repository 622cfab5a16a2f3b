"""The geometry of the frozen fixtures that the competing-reaction and
exclusion tests rely on (App. A): what each test assumes about distances and
reach is checked here, so that a fixture error cannot pass for a method error.
"""
import math

import numpy as np

from synth import frozen_squares, frozen_loops, four_reaction_soup, telechelic_rings


def _dist(s, i, j):
    d = s.pos[j] - s.pos[i]
    d -= s.box * np.rint(d / s.box)
    return float(np.sqrt((d * d).sum()))


def _pairs_within(s, r):
    out = []
    for i in range(s.n):
        d = s.pos - s.pos[i]
        d -= s.box * np.rint(d / s.box)
        rr = np.sqrt((d * d).sum(1))
        for j in np.nonzero((rr < r) & (np.arange(s.n) > i))[0]:
            out.append((i, int(j)))
    return out


def test_frozen_squares_geometry():
    s = frozen_squares(seed=2, n_squares=27)
    r0, r_max = s.bond_types[0].r0, s.reactions[0].r_max
    # corners A, B, D, C: the four reacting edges at the rest length, the
    # diagonals A-D and B-C out of reach, nothing across squares
    for q in range(27):
        a, b, d, c = 4 * q, 4 * q + 1, 4 * q + 2, 4 * q + 3
        assert list(s.types[[a, b, c, d]]) == [0, 1, 2, 3]
        for i, j in ((a, b), (a, c), (d, b), (d, c)):
            assert abs(_dist(s, i, j) - r0) < 1e-12
        assert abs(_dist(s, a, d) - r0 * math.sqrt(2)) < 1e-12 and _dist(s, a, d) > r_max
    assert all(i // 4 == j // 4 for i, j in _pairs_within(s, r_max + 0.5))
    rx = [(r.type_a, r.type_b, r.bond_type) for r in s.reactions]
    assert rx == [(0, 1, 0), (0, 2, 1), (3, 1, 2), (3, 2, 3)]


def test_frozen_loops_geometry():
    s = frozen_loops(seed=2, n_units=27)
    r_max = s.reactions[0].r_max
    for u in range(27):
        p, m, q, p2, q2 = range(5 * u, 5 * u + 5)
        assert list(s.types[[p, m, q, p2, q2]]) == [0, 2, 1, 0, 1]
        assert abs(_dist(s, p, q) - 1.1) < 1e-12 and abs(_dist(s, p2, q2) - 1.1) < 1e-12
        assert _dist(s, p, q2) > r_max and _dist(s, p2, q) > r_max
    # the static bonds join P-M and M-Q of each molecule only
    sb = {tuple(b) for b in s.static_bonds.tolist()}
    assert sb == {(5 * u, 5 * u + 1) for u in range(27)} | {(5 * u + 1, 5 * u + 2) for u in range(27)}
    # within reach of a reactive pair: only the intramolecular pair and the control pair
    reach = [(i, j) for i, j in _pairs_within(s, r_max) if {s.types[i], s.types[j]} == {0, 1}]
    assert sorted(reach) == sorted([(5 * u, 5 * u + 2) for u in range(27)] + [(5 * u + 3, 5 * u + 4) for u in range(27)])


def test_soups_and_rings_composition():
    s = four_reaction_soup(seed=1, n=400, rho=0.3)
    assert np.array_equal(np.bincount(s.types), [100, 100, 100, 100])
    assert abs(s.n / np.prod(s.box) - 0.3) < 1e-12
    # no two particles closer than sigma at the default overlap factor
    assert not _pairs_within(s, 1.0 - 1e-9)
    r = telechelic_rings(seed=1, n_chains=30, beads=3)
    assert np.array_equal(r.valence, [0, 1, 0])
    assert [(x.type_a, x.type_b) for x in r.reactions] == [(1, 1)]
    ends = np.nonzero(r.types == 1)[0]
    assert len(ends) == 60 and np.all((ends % 3 == 0) | (ends % 3 == 2))

"""Pins of the oracle's pair-distance histogram behind g(r).

- Counts equal a brute-force all-pairs histogram written here with numpy
  (minimum image per axis, bin floor(r / dr)).
- An ideal gas (uniform random positions) has g(r) = 1 within its Poisson
  error bars, for a mixed and a single type pair (normalisation).
- Counts of the type pairs AA, BB and AB add up to those of the same
  positions with every particle of one type (each unordered pair once).
"""
import math

import numpy as np
import pytest
from scipy import stats

from synth import random_frozen


def _brute(pos, types, box, ta, tb, r_max, nbins):
    n = len(pos)
    h = np.zeros(nbins, np.int64)
    dr = r_max / nbins
    for i in range(n):
        if types[i] != ta:
            continue
        d = pos - pos[i]
        d -= box * np.rint(d / box)
        r = np.sqrt((d[:, 0] ** 2 + d[:, 1] ** 2) + d[:, 2] ** 2)
        ok = (types == tb) & (r < r_max)
        ok[i] = False
        if ta == tb:
            ok[: i + 1] = False
        np.add.at(h, (r[ok] / dr).astype(np.int64), 1)
    return h


def test_rdf_counts_match_brute_force(oracle_mod):
    s = random_frozen(seed=3, n=600, box=9.0, overlap_factor=0.6)
    o = oracle_mod.OracleSystem(s)
    for ta, tb in ((0, 1), (0, 0), (1, 1)):
        got = o.rdf_counts(ta, tb, 2.5, 25)
        ref = _brute(s.pos, s.types, s.box, ta, tb, 2.5, 25)
        assert np.array_equal(got, ref), (ta, tb)
        assert got.sum() > 500


def test_ideal_gas_rdf_is_one(oracle_mod):
    rng = np.random.default_rng(7)
    s = random_frozen(seed=4, n=6000, box=20.0, overlap_factor=0.6)
    s.pos = rng.uniform(0.0, 20.0, size=(s.n, 3))      # no correlations at all
    o = oracle_mod.OracleSystem(s)
    vol = 20.0 ** 3
    na, nb = int((s.types == 0).sum()), int((s.types == 1).sum())
    for ta, tb, same in ((0, 1, False), (1, 1, True)):
        c = o.rdf_counts(ta, tb, 3.0, 30)
        g = oracle_mod.rdf_normalise(c, na if ta == 0 else nb, nb, same, vol, 3.0)
        ideal = c / np.where(g > 0, g, 1.0)               # expected counts of the ideal gas
        keep = ideal > 20
        chi2 = float((((c - ideal) ** 2) / ideal)[keep].sum())
        assert stats.chi2.sf(chi2, keep.sum()) > 1e-4, (ta, tb, chi2)
        assert abs(g[keep].mean() - 1.0) < 0.02


def test_type_pair_counts_add_up(oracle_mod):
    s = random_frozen(seed=5, n=900, box=10.0, overlap_factor=0.6)
    o = oracle_mod.OracleSystem(s)
    parts = sum(o.rdf_counts(a, b, 2.0, 20) for a, b in ((0, 0), (1, 1), (0, 1)))
    s.types = np.zeros_like(s.types)
    one = oracle_mod.OracleSystem(s).rdf_counts(0, 0, 2.0, 20)
    assert np.array_equal(parts, one)

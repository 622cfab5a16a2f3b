"""Pins of the oracle's intramolecular exclusion (Sec. II.D; App. A checks it
in both directions with a control pair).

- Molecules are the connected components of the static bonds: the oracle's
  labels induce the same partition as a breadth-first search written here.
- Frozen molecules P-M-Q with their two sites within reach, beside a control
  pair of lone P and Q at the same distance: with the exclusion the
  intramolecular pair never bonds while the control bonds with the two-state
  fraction K/(1 + K) (U_b = 0 at the rest length); without it both bond with
  that fraction.
- Short telechelic chains whose ends react S-S: without the exclusion some
  chains close into rings; with it none does, while chains still join end to
  end.
"""
import math
from collections import deque

import numpy as np
import pytest

from synth import frozen_loops, telechelic_rings, telechelic


def _bfs_labels(n, bonds):
    adj = [[] for _ in range(n)]
    for a, b in bonds:
        adj[a].append(b)
        adj[b].append(a)
    lab = [-1] * n
    for s in range(n):
        if lab[s] >= 0:
            continue
        lab[s] = s
        q = deque([s])
        while q:
            u = q.popleft()
            for v in adj[u]:
                if lab[v] < 0:
                    lab[v] = s
                    q.append(v)
    return np.array(lab)


def _same_partition(a, b):
    # equal iff the label maps a -> b and b -> a are both functions
    pa = {}
    pb = {}
    for x, y in zip(a.tolist(), b.tolist()):
        if pa.setdefault(x, y) != y or pb.setdefault(y, x) != x:
            return False
    return True


def test_molecules_are_static_bond_components(oracle_mod):
    rng = np.random.default_rng(3)
    s = telechelic(seed=2, n_chains=20, beads=5, n_x=30, rho=0.2)
    # extra random static bonds join some chains and crosslinkers into larger molecules
    extra = rng.integers(0, s.n, size=(12, 2))
    extra = extra[extra[:, 0] != extra[:, 1]]
    bonds = np.concatenate([s.static_bonds, extra]).astype(np.int32)
    lab = oracle_mod.molecules(s.n, bonds)
    ref = _bfs_labels(s.n, bonds.tolist())
    assert _same_partition(lab, ref)
    # a particle without static bonds is a molecule of its own
    lone = np.setdiff1d(np.arange(s.n), bonds.ravel())
    assert len(np.unique(lab[lone])) == len(lone)
    assert not np.isin(lab[lone], lab[np.unique(bonds.ravel())]).any()


def _two_state_se(p, a, b, m, T):
    lam = 1.0 - a - b
    return math.sqrt(p * (1 - p) / (m * T) * (1 + lam) / (1 - lam))


@pytest.mark.parametrize("self_avoid", [1, 0])
def test_frozen_loops_both_ways(oracle_mod, self_avoid):
    eps, T, units = 1.0, 2000, 125
    s = frozen_loops(seed=3, n_units=units, self_avoid=self_avoid, eps=eps)
    o = oracle_mod.OracleSystem(s, p_on0=1.0)
    intra = ctrl = 0
    for t in range(T):
        o.sweep(step=t)
        b = o.bonds()
        is_intra = (b[:, 0] % 5 == 0) & (b[:, 1] == b[:, 0] + 2)
        is_ctrl = (b[:, 0] % 5 == 3) & (b[:, 1] == b[:, 0] + 1)
        assert np.all(is_intra | is_ctrl)      # nothing else is within reach
        intra += int(is_intra.sum())
        ctrl += int(is_ctrl.sum())
    a, bo = 1.0, math.exp(-eps)                # P_on (U_b = 0) and P_off per sweep
    expect = a / (a + bo)
    se = _two_state_se(expect, a, bo, units, T)
    assert abs(ctrl / (T * units) - expect) < 4.5 * se, ctrl / (T * units)
    if self_avoid:
        assert intra == 0
    else:
        assert abs(intra / (T * units) - expect) < 4.5 * se, intra / (T * units)


def test_rings_form_only_without_exclusion(oracle_mod):
    counts = {}
    for sa in (0, 1):
        s = telechelic_rings(seed=4, n_chains=300, beads=3, self_avoid=sa)
        o = oracle_mod.OracleSystem(s, p_on0=1.0)
        rings = joins = 0
        for _ in range(50):
            o.run(20)
            b = o.bonds()
            same = o.mol[b[:, 0]] == o.mol[b[:, 1]]
            rings += int(same.sum())
            joins += int((~same).sum())
        counts[sa] = (rings, joins)
    assert counts[0][0] > 100 and counts[0][1] > 100, counts
    assert counts[1][0] == 0 and counts[1][1] > 100, counts


@pytest.mark.parametrize("self_avoid", [1, 0])
def test_mh_moves_respect_the_exclusion(oracle_mod, self_avoid):
    # the oracle's Metropolis-Hastings move set filters candidates the same way
    s = frozen_loops(seed=7, n_units=64, self_avoid=self_avoid, eps=1.0)
    o = oracle_mod.OracleSystem(s, p_on0=1.0)
    intra = ctrl = 0
    for t in range(3000):
        o.mh_sweep(step=t)
        b = o.bonds()
        intra += int(((b[:, 0] % 5 == 0) & (b[:, 1] == b[:, 0] + 2)).sum())
        ctrl += int(((b[:, 0] % 5 == 3) & (b[:, 1] == b[:, 0] + 1)).sum())
    assert ctrl > 0
    assert (intra == 0) == bool(self_avoid), (intra, ctrl)

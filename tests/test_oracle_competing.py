"""Pins of the oracle's sweep with several reactions competing for shared sites
(Sec. II.C: reactions processed one after another in an order redrawn every
sweep; App. A: the frozen four-reaction test and its mobile version).

- Frozen squares A-B-D-C with the four reactions A-B, A-C, D-B, D-C at the
  bond rest length (U_b = 0): the seven accessible states of a square have the
  weights of Eq. Z, Z = 1 + K_AB + K_AC + K_DB + K_DC + K_AB K_DC + K_AC K_DB,
  with K = e^eps.  The measured state populations reproduce them (the paper
  quotes agreement within 0.02; the bound here is the statistical one, 0.006)
  and no site is ever in two bonds.
- Mobile soup of the same four reactions: bonds exchange partners (distinct
  bonded pairs exceed the largest number present at once by far more than 3x),
  every site bonds more often to the partner with the larger K, and the
  cross ratio n_AB n_DC / (n_AC n_DB) follows mass action,
  K_AB K_DC / (K_AC K_DB), within the run's fluctuations: A, B, C and D are
  physically identical apart from their reaction labels, so the bound-pair
  volume cancels from the ratio.
"""
import math

import numpy as np
import pytest

from synth import frozen_squares, four_reaction_soup

from _competing import AB, AC, DB, DC, eq_z_states, square_masks


def test_eq_z_closed_form():
    # the single-bond marginal quoted with Eq. Z: P(A-B) = K_AB (1 + K_DC) / Z
    eps = (0.3, 1.2, 0.8, 2.1)
    p = eq_z_states(eps)
    kab, kdc = math.exp(eps[0]), math.exp(eps[3])
    z = 1 + sum(math.exp(e) for e in eps) + kab * kdc + math.exp(eps[1]) * math.exp(eps[2])
    assert abs(p[AB] + p[AB | DC] - kab * (1 + kdc) / z) < 1e-15
    assert abs(sum(p.values()) - 1.0) < 1e-15


@pytest.mark.parametrize("eps,p_on0", [((0.3, 1.2, 0.8, 2.1), 1.0), ((1.5, 0.2, 2.0, 1.0), 0.5)])
def test_frozen_squares_follow_eq_z(oracle_mod, eps, p_on0):
    s = frozen_squares(seed=7, n_squares=216, eps=eps)
    o = oracle_mod.OracleSystem(s, p_on0=p_on0)
    nq = s.n // 4
    counts = np.zeros(16)
    burn, T = 50, 4000
    for t in range(burn + T):
        o.sweep(step=t)
        if t >= burn:
            counts += np.bincount(square_masks(o.bonds(), nq), minlength=16)
    f = counts / counts.sum()
    exact = eq_z_states(eps)
    # only the seven states of Eq. Z occur: a site is never in two bonds
    assert f[[m for m in range(16) if m not in exact]].sum() == 0.0
    dev = max(abs(f[m] - p) for m, p in exact.items())
    assert dev < 0.006, (dev, {m: (round(f[m], 4), round(p, 4)) for m, p in exact.items()})


def test_frozen_squares_all_reactions_take_turns(oracle_mod):
    # with equal K every reaction forms equally often: the order is redrawn
    # every sweep, so the first-registered reaction has no edge
    s = frozen_squares(seed=3, n_squares=216, eps=(1.0, 1.0, 1.0, 1.0))
    o = oracle_mod.OracleSystem(s, p_on0=1.0)
    per_rx = np.zeros(4)
    for t in range(2000):
        o.sweep(step=t)
        if t >= 20:
            per_rx += np.bincount(o.bonds()[:, 2], minlength=4)
    share = per_rx / per_rx.sum()
    assert np.abs(share - 0.25).max() < 0.01, share


def test_soup_exchanges_and_branches_by_k(oracle_mod):
    eps = (0.5, 1.5, 1.0, 2.5)
    s = four_reaction_soup(seed=11, n=1000, rho=0.3, eps=eps)
    o = oracle_mod.OracleSystem(s, p_on0=1.0)
    seen, most, per_rx, snaps = set(), 0, np.zeros(4), 0
    o.run(200)
    for _ in range(380):
        o.run(10)
        b = o.bonds()
        most = max(most, len(b))
        seen.update(map(tuple, b[:, :2].tolist()))
        per_rx += np.bincount(b[:, 2], minlength=4)
        snaps += 1
        occ = np.bincount(b[:, :2].ravel(), minlength=s.n)
        assert occ.max() <= 1
    assert len(seen) > 3 * most, (len(seen), most)
    ab, ac, db, dc = per_rx / snaps
    # A prefers C (K_AC > K_AB), D prefers C, B prefers D, C prefers D
    assert ac > ab and dc > db and db > ab and dc > ac, (ab, ac, db, dc)
    cross = math.log(ab * dc / (ac * db))
    assert abs(cross - (eps[0] + eps[3] - eps[1] - eps[2])) < 0.2, cross

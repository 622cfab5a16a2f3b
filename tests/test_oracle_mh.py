"""Pins of the oracle's Metropolis–Hastings bond moves (uniform proposal):
isolated frozen pairs reach the two-state stationary fraction
K e^{-U_b/kT} / (1 + K e^{-U_b/kT}) (detailed balance of the move set),
frozen stars whose arms compete for one centre reach the Boltzmann
populations w_q / (1 + sum w), and the valence invariants hold under MH
turnover in a dense gel."""
import math

import numpy as np
import pytest

from synth import frozen_pairs, colloid_linker

from _stars import star_arm_ranks, star_expectation, star_occupancy, stars_case, block_mean_se


@pytest.mark.parametrize("eps,p_on0,r", [(1.0, 1.0, 1.1), (2.0, 0.5, 1.2), (-0.5, 1.0, 1.15)])
def test_mh_frozen_pairs_stationary_fraction(oracle_mod, eps, p_on0, r):
    n_pairs = 216
    s = frozen_pairs(seed=9, n_pairs=n_pairs, r=r, eps=eps, spacing=4.0)
    o = oracle_mod.OracleSystem(s, p_on0=p_on0)
    k, r0 = s.bond_types[0].k, s.bond_types[0].r0
    K = math.exp(eps)
    w = K * math.exp(-0.5 * k * (r - r0) ** 2 / s.kT)
    expect = w / (1 + w)
    fr = []
    for t in range(24000):
        o.mh_sweep(step=t)
        if t >= 2000 and t % 8 == 0:
            fr.append(o.occ.sum() / 2 / n_pairs)
    fr = np.array(fr)
    # block error from 20 blocks
    blocks = fr[: len(fr) // 20 * 20].reshape(20, -1).mean(1)
    se = blocks.std(ddof=1) / math.sqrt(20)
    assert abs(fr.mean() - expect) < 4 * se + 0.01, (fr.mean(), expect, se)


def test_mh_invariants_dense_gel(oracle_mod):
    s = colloid_linker(seed=10, n_c=400, n_l=1600, eps=2.0)
    o = oracle_mod.OracleSystem(s)
    val = np.asarray(s.valence)[s.types]
    tot = {"form_accepts": 0, "break_accepts": 0}
    for t in range(400):
        st = o.mh_sweep(step=t)
        for kk in tot:
            tot[kk] += st[kk]
    dp = o.dp.reshape(s.n, 4)
    assert np.array_equal((dp >= 0).sum(1), o.occ)
    assert np.all(o.occ <= val)
    for i in range(s.n):
        for j in dp[i][dp[i] >= 0]:
            assert i in dp[j] and s.types[i] != s.types[j]
    assert tot["form_accepts"] > 50 and tot["break_accepts"] > 5


def test_mh_frozen_stars_match_boltzmann(oracle_mod):
    """Competing arms: the uniform proposal's Hastings factor n / b'
    (n candidates, b' owned bonds after the move) is what makes the arm
    populations follow w_q / (1 + sum w); dropping it biases them."""
    s = stars_case()
    K = math.exp(s.reactions[0].eps)
    o = oracle_mod.OracleSystem(s)
    rank = star_arm_ranks(s)
    expect = star_expectation(s, K)
    samples = []
    for t in range(16000):
        o.mh_sweep(step=t)
        if t >= 1000 and t % 8 == 0:
            samples.append(star_occupancy(o.dp.reshape(s.n, 4), s, rank))
    mean, se = block_mean_se(np.array(samples))
    assert np.all(np.abs(mean - expect) < 4 * se + 0.01), (mean, expect, se)

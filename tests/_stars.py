"""Isolated frozen stars (one A of valence 1, several B arms of valence 1):
exact stationary arm populations of an exact bond-topology sampler."""
import math

import numpy as np

from synth import frozen_stars


def star_expectation(s, K):
    """Stationary bond distribution of one isolated star (one A of valence 1,
    arms B of valence 1): P(A bonded to arm q) = w_q / (1 + sum w), with
    w_q = K exp(-U_b(r_q)/kT) (Boltzmann weight of each bond configuration)."""
    arms = s.meta["arms"]
    bt = s.bond_types[0]
    per = arms + 1
    r = np.linalg.norm(s.pos[1:per] - s.pos[0], axis=1)
    order = np.argsort(r)
    w = K * np.exp(-0.5 * bt.k * (r[order] - bt.r0) ** 2 / s.kT)
    return w / (1.0 + w.sum())


def star_arm_ranks(s):
    """rank (by separation) of every arm particle in its star; -1 for centres."""
    arms = s.meta["arms"]
    per = arms + 1
    rank = np.full(s.n, -1, np.int64)
    for st in range(s.n // per):
        c = st * per
        d = s.pos[c + 1:c + per] - s.pos[c]
        d -= s.box * np.rint(d / s.box)
        rank[c + 1:c + per] = np.argsort(np.argsort(np.linalg.norm(d, axis=1)))
    return rank


def star_occupancy(dp, s, rank):
    """fractions of stars whose centre is bonded to the arm of each rank."""
    arms = s.meta["arms"]
    per = arms + 1
    centres = dp[::per, 0]
    out = np.zeros(arms)
    for q in range(arms):
        out[q] = np.mean([(j >= 0 and rank[j] == q) for j in centres])
    return out


def stars_case(n_stars=125, seed=11):
    return frozen_stars(seed=seed, n_stars=n_stars, arms=4, r_lo=1.0, r_hi=1.25, k=100.0, eps=0.0)


def block_mean_se(samples, nblocks=20):
    """mean over samples (axis 0) and its standard error from block means."""
    blocks = samples[: len(samples) // nblocks * nblocks].reshape(nblocks, -1, *samples.shape[1:]).mean(1)
    return samples.mean(0), blocks.std(0, ddof=1) / math.sqrt(nblocks)

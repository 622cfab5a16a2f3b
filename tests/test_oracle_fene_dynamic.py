"""Pins of the oracle's FENE dynamic bonds (Sec. II.B: U_b(r) is the bond
evaluator's energy, not necessarily harmonic; the paper's DyBond-v2 accepts
FENE-type evaluators besides the harmonic one).

- U_b(r) = -1/2 k R0^2 ln(1 - (r/R0)^2), so the Metropolis factor of Eq. (3)
  is (1 - (r/R0)^2)^(k R0^2 / (2 kT)): frozen pairs at r reach the two-state
  fraction P_on(r)/(P_on(r) + P_off) with that closed form (two separations,
  two temperatures).
- The FENE term has its minimum at r = 0, so a proposal aims at r0 = 0: the
  proposed partner is the closest free compatible one inside the window
  (brute force over all pairs).
- r >= R0 inside the window cannot bond (U_b = +inf).
"""
import math

import numpy as np
import pytest

from synth import frozen_pairs, random_frozen, BondType, FENE


def _fene(s, k=3.0, R0=1.5):
    s.bond_types = [BondType(FENE, k, R0)]
    return s


def _two_state_se(p, a, b, m, T):
    lam = 1.0 - a - b
    return math.sqrt(p * (1 - p) / (m * T) * (1 + lam) / (1 - lam))


@pytest.mark.parametrize("r,kT", [(0.97, 1.0), (1.2, 1.0), (1.2, 2.0)])
def test_fene_two_state_fraction(oracle_mod, r, kT):
    k, R0, eps, n_pairs, T = 3.0, 1.5, 3.0, 200, 3000
    s = _fene(frozen_pairs(seed=5, n_pairs=n_pairs, r=r, eps=eps, r_max=1.4, kT=kT), k, R0)
    o = oracle_mod.OracleSystem(s, p_on0=1.0)
    p_on = (1.0 - (r / R0) ** 2) ** (k * R0 * R0 / (2.0 * kT))
    p_off = math.exp(-eps)
    expect = p_on / (p_on + p_off)
    counts = []
    for t in range(T + 50):
        o.sweep(step=t)
        if t >= 50:
            counts.append(o.occ.sum() / 2)
    frac = np.mean(counts) / n_pairs
    se = _two_state_se(expect, p_on, p_off, n_pairs, T)
    assert 0.1 < expect < 0.95                  # a regime where the factor matters
    assert abs(frac - expect) < 4.5 * se, (frac, expect, se)


def test_fene_beyond_r0_never_bonds(oracle_mod):
    s = _fene(frozen_pairs(seed=6, n_pairs=64, r=1.55, eps=5.0, r_max=1.6))
    o = oracle_mod.OracleSystem(s, p_on0=1.0)
    for t in range(200):
        st = o.sweep(step=t)
        assert st["formed"] == 0
    assert st["proposals"] > 0      # proposed, then rejected by the infinite U_b


@pytest.mark.parametrize("box,n", [(9.0, 400), (13.0, 900)])
def test_fene_proposals_pick_the_closest_partner(oracle_mod, box, n):
    s = _fene(random_frozen(seed=int(box * 3), n=n, box=box, overlap_factor=0.5, r_max=1.4, r_min=0.3))
    o = oracle_mod.OracleSystem(s)
    st, tr = o.sweep(step=9, trace=True)
    nprop = 0
    for i in range(n):
        d = s.pos - s.pos[i]
        d -= s.box * np.rint(d / s.box)
        r = np.sqrt((d * d).sum(1))
        ok = (s.types == 1 - s.types[i]) & (r >= 0.3) & (r <= 1.4)
        ok[i] = False
        cand = np.nonzero(ok)[0]
        if cand.size == 0:
            assert tr["prop"][i] == -1
            continue
        nprop += 1
        assert tr["prop"][i] == cand[np.lexsort((cand, r[cand]))[0]]
    assert st["proposals"] == nprop

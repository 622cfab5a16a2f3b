"""Pins of the oracle's bonding sweep against what the paper and mathematics fix.

- Isolated frozen pairs are two-state Markov chains (Sec. II.A): the stationary
  bonded fraction is P_on/(P_on + P_off) = K e^{-U_b/kT} / (1 + K e^{-U_b/kT})
  with K = P_on^0/P_off (Eqs. 1-4).
- Breaking does not depend on r and a bond is not tested in the sweep that
  formed it (Sec. II.C, Fig. 1d), so lifetimes are geometric in sweeps.
- Among matched proposals, the accepted fraction in each r-bin equals
  P_on^0 exp(-U_b(r)/kT) (Eqs. 3-4); the broken fraction equals P_off at every r.
- A bond broken by a reaction is not re-formed by it in the same sweep.
- kT -> 0 is well defined: only U_b <= 0 pairs can form (App. A).
- Candidate sets, proposals and matching against all-pairs enumeration.
"""
import math

import numpy as np
import pytest
from scipy import stats

from synth import frozen_pairs, random_frozen, assoc_ab


def _ou(oracle_mod, sysdef, p_on0=1.0):
    return oracle_mod.OracleSystem(sysdef, p_on0=p_on0)


def _two_state_se(p_bond, a, b, n_pairs, T):
    lam = 1.0 - a - b
    return math.sqrt(p_bond * (1 - p_bond) / (n_pairs * T) * (1 + lam) / (1 - lam))


@pytest.mark.parametrize("eps,p_on0,r", [(1.0, 0.3, 1.1), (2.0, 0.5, 1.2), (5.0, 1.0, 1.1),
                                         (0.0, 0.8, 1.0)])
def test_frozen_pairs_bonded_fraction(oracle_mod, eps, p_on0, r):
    n_pairs, T, burn = 200, 3000, 50
    s = frozen_pairs(seed=3, n_pairs=n_pairs, r=r, eps=eps)
    o = _ou(oracle_mod, s, p_on0=p_on0)
    k, r0 = s.bond_types[0].k, s.bond_types[0].r0
    U = 0.5 * k * (r - r0) ** 2
    a = p_on0 * math.exp(-U / s.kT)
    b = p_on0 * math.exp(-eps)
    expect = a / (a + b)
    counts = []
    for t in range(T + burn):
        o.sweep(step=t)
        if t >= burn:
            counts.append(o.occ.sum() / 2)
    frac = np.mean(counts) / n_pairs
    se = _two_state_se(expect, a, b, n_pairs, T)
    assert abs(frac - expect) < 4.5 * se + 1e-12, (frac, expect, se)
    # no pair ever bonds across pairs (each site only sees its own partner)
    bonds = o.bonds()
    assert np.all(bonds[:, 1] - bonds[:, 0] == 1) and np.all(bonds[:, 0] % 2 == 0)


def test_lifetimes_geometric(oracle_mod):
    n_pairs, T = 300, 4000
    eps, p_on0 = 1.5, 0.6
    s = frozen_pairs(seed=5, n_pairs=n_pairs, r=1.1, eps=eps)
    o = oracle_mod.OracleSystem(s, nhist=64, p_on0=p_on0)
    for t in range(T):
        o.sweep(step=t)
    h = o.life_hist.astype(float)
    poff = p_on0 * math.exp(-eps)
    assert h[0] == 0  # a bond is never broken in the sweep that formed it
    m = np.arange(1, 63)
    pm = (1 - poff) ** (m - 1) * poff
    obs = np.append(h[1:63], h[63])
    expct = np.append(pm, (1 - poff) ** 62) * h.sum()
    keep = expct > 5
    obs_k = np.append(obs[keep], obs[~keep].sum())
    exp_k = np.append(expct[keep], expct[~keep].sum())
    chi2 = ((obs_k - exp_k) ** 2 / exp_k).sum()
    pval = stats.chi2.sf(chi2, obs_k.size - 1)
    assert pval > 1e-4, (chi2, pval)
    mean_life = (np.arange(64) * h).sum() / h.sum()
    assert abs(mean_life - 1 / poff) < 0.1 / poff


def test_acceptance_follows_metropolis_factor(oracle_mod):
    # dense random frozen configuration: many contested proposals at all r
    s = random_frozen(seed=11, n=3000, box=12.0, overlap_factor=0.6, eps=3.0, r_max=1.5,
                      k=10.0, r0=1.0)
    o = oracle_mod.OracleSystem(s, p_on0=0.9)
    pos = s.pos
    L = s.box
    k, r0, kT = 10.0, 1.0, s.kT
    rs, acc = [], []
    for t in range(40):
        o.set_bonds([])
        st, tr = o.sweep(step=1000 + t, trace=True)
        m = tr["matched"]
        i = np.nonzero(m >= 0)[0]
        i = i[i < m[i]]
        j = m[i]
        d = pos[j] - pos[i]
        d -= L * np.rint(d / L)
        rs.append(np.sqrt((d * d).sum(1)))
        acc.append(tr["formed"][i].astype(bool))
        assert st["survivors"] == i.size
        assert st["formed"] == int(tr["formed"].sum()) // 2
    r = np.concatenate(rs)
    a = np.concatenate(acc)
    assert r.size > 20000
    bins = np.linspace(0.0, 1.5, 16)
    idx = np.digitize(r, bins) - 1
    for b in range(15):
        sel = idx == b
        if sel.sum() < 200:
            continue
        p = 0.9 * np.exp(-0.5 * k * (r[sel] - r0) ** 2 / kT)
        mean = p.mean()
        var = (p * (1 - p)).sum()
        z = (a[sel].sum() - p.sum()) / math.sqrt(max(var, 1e-12))
        assert abs(z) < 4.5, (b, a[sel].mean(), mean, z)


def test_breaking_independent_of_r(oracle_mod):
    s = random_frozen(seed=12, n=4000, box=14.0, overlap_factor=0.6, eps=1.0, r_max=1.3)
    o = oracle_mod.OracleSystem(s, p_on0=1.0)
    rng = np.random.default_rng(0)
    perm = rng.permutation(s.n)
    t = s.types[perm]
    a_idx = perm[t == 0]
    b_idx = perm[t == 1]
    m = min(a_idx.size, b_idx.size)
    pairs = np.stack([np.minimum(a_idx[:m], b_idx[:m]), np.maximum(a_idx[:m], b_idx[:m]),
                      np.zeros(m, int)], axis=1)
    poff = math.exp(-1.0)
    d = s.pos[pairs[:, 1]] - s.pos[pairs[:, 0]]
    d -= s.box * np.rint(d / s.box)
    r = np.sqrt((d * d).sum(1))
    broken_all = []
    for t in range(30):
        o.set_bonds(pairs)
        o.sweep(step=50 + t)
        kept = {(int(x), int(y)) for x, y, _ in o.bonds()}
        broken_all.append(np.array([(int(x), int(y)) not in kept for x, y, _ in pairs]))
    br = np.concatenate(broken_all)
    rr = np.tile(r, 30)
    # every particle of the two types is saturated (valence 1): nothing forms
    for lo, hi in [(0, 2), (2, 5), (5, 8), (8, 20)]:
        sel = (rr >= lo) & (rr < hi)
        nsel = sel.sum()
        z = (br[sel].sum() - poff * nsel) / math.sqrt(nsel * poff * (1 - poff))
        assert abs(z) < 4.5, (lo, hi, br[sel].mean(), poff)


def test_no_reformation_in_same_sweep(oracle_mod):
    # P_off = 1 (eps = 0, P_on^0 = 1): a bond breaks in every sweep that tests it,
    # and the pair re-forms only in the next sweep: strict alternation.
    s = frozen_pairs(seed=2, n_pairs=50, r=1.1, eps=0.0)
    o = oracle_mod.OracleSystem(s, p_on0=1.0)
    seq = []
    for t in range(20):
        o.sweep(step=t)
        seq.append(int(o.occ.sum() // 2))
    assert seq == [50, 0] * 10


def test_zero_temperature_limit(oracle_mod):
    from synth import BondType, HARMONIC
    s = frozen_pairs(seed=4, n_pairs=64, r=1.0, eps=3.0, spacing=4.0)
    s.bond_types = [BondType(HARMONIC, 100.0, 1.0)]
    # pairs along x with exactly representable separations: 1.0 (U = 0) for the
    # first half, 1.25 (U > 0) for the second half
    pos = s.pos.copy()
    for p in range(64):
        pos[2 * p + 1] = pos[2 * p] + np.array([1.0 if p < 32 else 1.25, 0.0, 0.0])
    assert np.all(pos < s.box[0])
    s.pos = pos
    s.kT = 0.0
    o = oracle_mod.OracleSystem(s, p_on0=1.0)
    seen = np.zeros(64, bool)
    for t in range(40):
        o.sweep(step=t)
        b = o.bonds()
        assert np.all(b[:, 0] // 2 < 32)  # U_b > 0 never forms at kT = 0
        seen[b[:, 0] // 2] = True
    assert seen[:32].all()  # U_b = 0 forms with P_on^0 = 1


def _brute_candidates(s, i, occ, rmin, rmax):
    d = s.pos - s.pos[i]
    d -= s.box * np.rint(d / s.box)
    r2 = (d * d).sum(1)
    ti = s.types[i]
    want = 1 - ti
    ok = (s.types == want) & (occ < np.asarray(s.valence)[s.types]) & (r2 >= rmin * rmin) & (
        r2 <= rmax * rmax)
    ok[i] = False
    return np.nonzero(ok)[0], np.sqrt(r2)


@pytest.mark.parametrize("box,n", [(6.0, 120), (9.0, 400), (13.0, 900)])
def test_candidates_and_proposals_vs_brute_force(oracle_mod, box, n):
    s = random_frozen(seed=int(box * 10), n=n, box=box, overlap_factor=0.5, r_max=1.4,
                      r_min=0.3)
    o = oracle_mod.OracleSystem(s)
    st, tr = o.sweep(step=7, trace=True)
    r0 = s.bond_types[0].r0
    occ0 = np.zeros(n, int)
    nprop = 0
    for i in range(n):
        cand, r = _brute_candidates(s, i, occ0, 0.3, 1.4)
        if cand.size == 0:
            assert tr["prop"][i] == -1
            continue
        nprop += 1
        dd = np.abs(r[cand] - r0)
        best = cand[np.lexsort((cand, dd))[0]]
        assert tr["prop"][i] == best
    assert st["proposals"] == nprop


@pytest.mark.parametrize("box,n", [(9.0, 400), (13.0, 900)])
def test_candidate_sets_cell_grid_vs_all_pairs(oracle_mod, box, n):
    s = random_frozen(seed=int(box), n=n, box=box, overlap_factor=0.5, r_max=1.4, r_min=0.2)
    o = oracle_mod.OracleSystem(s)
    occ0 = np.zeros(n, int)
    for i in range(0, n, 7):
        cand, _ = _brute_candidates(s, i, occ0, 0.2, 1.4)
        assert np.array_equal(o.candidates(i), np.sort(cand))


def test_matching_is_locally_dominant_and_disjoint(oracle_mod):
    s = random_frozen(seed=21, n=1500, box=10.0, overlap_factor=0.5, r_max=1.5)
    o = oracle_mod.OracleSystem(s)
    step = 99
    st, tr = o.sweep(step=step, trace=True)
    prop = tr["prop"]
    edges = {}
    for i, j in enumerate(prop):
        if j < 0:
            continue
        a, b = min(i, int(j)), max(i, int(j))
        edges[(a, b)] = None
    key = [int(s.seed) & 0xFFFFFFFF, ((int(s.seed) >> 32) & 0xFFFF) << 16 | (0 << 8) | 3]
    prio = {}
    for (a, b) in edges:
        w = oracle_mod.philox4x32_10([step & 0xFFFFFFFF, step >> 32, a, b], key)
        prio[(a, b)] = int(w[0])
    best = {}
    for (a, b), p in prio.items():
        for u, v in ((a, b), (b, a)):
            kv = (p << 32) | v
            best[u] = max(best.get(u, 0), kv)
    surv = {(a, b) for (a, b), p in prio.items()
            if best[a] == (p << 32) | b and best[b] == (p << 32) | a}
    m = tr["matched"]
    got = {(i, int(m[i])) for i in range(s.n) if m[i] > i}
    assert got == surv
    ends = [x for e in surv for x in e]
    assert len(ends) == len(set(ends))  # disjoint
    # the edge of largest priority always survives, so the matching is never empty
    top = max(prio, key=lambda e: (prio[e], e))
    assert top in surv
    assert st["edges"] == len(edges)


def test_valence_invariants_under_turnover(oracle_mod):
    from synth import colloid_linker
    s = colloid_linker(seed=8, n_c=600, n_l=2400, eps=1.0)
    o = oracle_mod.OracleSystem(s, p_on0=1.0)
    val = np.asarray(s.valence)[s.types]
    for _ in range(6):
        o.run(50)
        dp = o.dp.reshape(s.n, 4)
        occ = (dp >= 0).sum(1)
        assert np.array_equal(occ, o.occ)
        assert np.all(o.occ <= val)
        for i in range(s.n):
            row = dp[i][dp[i] >= 0]
            assert np.all(np.diff(row) > 0)  # ascending, no duplicate partner
            for j in row:
                assert i in dp[j]
                assert s.types[i] != s.types[j]
    assert o.bonds().shape[0] > 100

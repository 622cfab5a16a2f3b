"""GPU trajectory observables against the FP64 oracle: bonded fraction, bond
lifetime histogram and g(r), within stated statistical error bars.

- Pair-distance counts behind g(r) are identical to the oracle's on the same
  positions (after MD, both precisions, each type pair, a replica of a batch).
- FP64 MD follows the oracle step for step, so its bond lifetime histogram is
  identical to the oracle's.
- A+B association (500 A + 500 B at number density 0.1, window r <= 1.3, bond
  free energy 5 kT, 10^4 steps), mixed precision, eight seeds: the bonded
  fraction and the A-B pair counts per distance bin agree with the FP64
  oracle's runs of the same seeds (tests/golden/assoc_ab_observables.json,
  written by the oracle alone) within their combined block-average error bars;
  the pooled lifetime histogram is geometric with P_off = e^-5 (Sec. II.C:
  breaking does not depend on r, and a bond is not tested in the sweep that
  formed it) and homogeneous with the oracle's.
- Batched telechelic sweep, all 256 replicas in one context, mixed precision:
  the bonded fraction of chain ends of the 8 smallest replicas agrees with FP64
  oracle runs of those replicas alone
  (tests/golden/telechelic_sweep_smallest8.json).
"""
import json
import math
from pathlib import Path

import numpy as np
import pytest
from scipy import stats

import oracle
from synth import colloid_linker, assoc_ab, random_frozen

pytestmark = pytest.mark.gpu

GOLDEN = Path(__file__).resolve().parent / "golden"


@pytest.fixture(scope="module")
def snapmod():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2609_21204_b300 import build
    build.build()
    import paper_2609_21204_b300 as m
    return m


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_rdf_counts_identical_to_oracle(snapmod, precision):
    s = colloid_linker(seed=51, n_c=3000, n_l=12000)
    sim = snapmod.from_system(s, precision=precision)
    orc = oracle.OracleSystem(s)
    sim.step(57)
    for pair in ((0, 1), (0, 0), (1, 1)):
        got = sim.rdf_counts(*pair, 1.45, 29)   # the call rebuilds: positions are then wrapped
        orc.set_positions(sim.positions())
        ref = orc.rdf_counts(*pair, 1.45, 29)
        assert np.array_equal(got, ref), pair
        assert ref.sum() > 1000
    with pytest.raises(snapmod.SnapError) as e:
        sim.rdf_counts(0, 1, 50.0, 10)          # beyond one cell
    assert e.value.name == "SNAP_ERR_ARG"
    sim.close()


def test_rdf_counts_of_a_replica(snapmod):
    reps = [random_frozen(seed=52 + r, n=1500 + 300 * r, box=14.0 + r, overlap_factor=1.0) for r in range(3)]
    sim = snapmod.from_system(reps, precision="mixed")
    sim.step(20)
    pos = sim.positions()
    off = 0
    for r, s in enumerate(reps):
        got = sim.rdf_counts(0, 1, 1.4, 14, replica=r)
        o = oracle.OracleSystem(s)
        o.set_positions(sim.positions()[off:off + s.n])
        assert np.array_equal(got, o.rdf_counts(0, 1, 1.4, 14)), r
        off += s.n
    assert pos.shape[0] == off


def test_lifetime_hist_fp64_identical_to_oracle(snapmod):
    s = assoc_ab(seed=53)
    s.reactions[0].eps = 1.0               # short lifetimes: many breaks in 300 steps
    sim = snapmod.from_system(s, precision="fp64")
    orc = oracle.OracleSystem(s)
    sim.step(300)
    orc.run(300)
    assert np.array_equal(sim.bonds(), orc.bonds())
    h_g, h_o = sim.lifetime_hist(256), orc.life_hist
    assert h_o.sum() > 1000
    assert np.array_equal(h_g, h_o)


def _pooled(runs, key, se_key):
    m = np.mean([np.asarray(r[key]) for r in runs], axis=0)
    se = np.sqrt(np.sum([np.asarray(r[se_key]) ** 2 for r in runs], axis=0)) / len(runs)
    return m, se


def _geometric_gof(h, p_off):
    h = np.asarray(h, dtype=np.float64)
    nb = h.size
    m = np.arange(1, nb - 1)
    pm = (1 - p_off) ** (m - 1) * p_off
    expect = np.concatenate([[0.0], pm, [(1 - p_off) ** (nb - 2)]]) * h.sum()
    keep = expect > 5
    obs, exp = h[keep], expect[keep]
    rest = (~keep) & (expect > 0)                # bin 0 has expectation 0: checked on its own
    if expect[rest].sum() > 0:
        obs = np.append(obs, h[rest].sum())
        exp = np.append(exp, expect[rest].sum())
    chi2 = float(((obs - exp) ** 2 / exp).sum())
    return stats.chi2.sf(chi2, obs.size - 1), h[0]


def test_assoc_ab_observables_match_oracle(snapmod):
    gold = json.loads((GOLDEN / "assoc_ab_observables.json").read_text())
    steps, burn, every, blocks = gold["steps"], gold["burn_in"], gold["every"], gold["blocks"]
    rdf = gold["rdf"]
    runs = []
    hist = np.zeros(256, np.int64)
    for g in gold["runs"]:
        s = assoc_ab(seed=g["seed"])
        sim = snapmod.from_system(s, precision="mixed")
        n_a = int((s.types == 0).sum())
        sim.step(burn)
        frac, counts = [], []
        for _ in range((steps - burn) // every):
            sim.step(every)
            frac.append(sim.stats()["n_bonds"] / n_a)
            counts.append(sim.rdf_counts(rdf["type_a"], rdf["type_b"], rdf["r_max"], rdf["nbins"]))
        frac = np.array(frac)
        counts = np.array(counts, dtype=np.float64)
        runs.append({"bonded_fraction": frac.mean(),
                     "bonded_fraction_se": frac.reshape(blocks, -1).mean(1).std(ddof=1) / math.sqrt(blocks),
                     "rdf_counts_mean": counts.mean(0),
                     "rdf_counts_se": counts.reshape(blocks, -1, rdf["nbins"]).mean(1).std(0, ddof=1)
                     / math.sqrt(blocks)})
        hist += sim.lifetime_hist(256)
        sim.close()
    fg, fg_se = _pooled(runs, "bonded_fraction", "bonded_fraction_se")
    fo, fo_se = _pooled(gold["runs"], "bonded_fraction", "bonded_fraction_se")
    z = (fg - fo) / math.sqrt(fg_se ** 2 + fo_se ** 2)
    assert abs(z) < 4.0, (fg, fo, fg_se, fo_se)
    cg, cg_se = _pooled(runs, "rdf_counts_mean", "rdf_counts_se")
    co, co_se = _pooled(gold["runs"], "rdf_counts_mean", "rdf_counts_se")
    keep = co > 5
    zb = (cg - co)[keep] / np.sqrt(cg_se ** 2 + co_se ** 2)[keep]
    assert keep.sum() >= 10
    assert np.abs(zb).max() < 5.0, zb
    assert stats.chi2.sf(float((zb ** 2).sum()), int(keep.sum())) > 1e-5, zb
    # lifetimes: geometric with P_off = e^-eps, and the same law as the oracle's runs
    p_off = math.exp(-5.0)
    pv, h0 = _geometric_gof(hist, p_off)
    assert h0 == 0 and pv > 1e-4, pv
    ho = np.sum([r["lifetime_hist"] for r in gold["runs"]], axis=0)
    pvo, _ = _geometric_gof(ho, p_off)
    assert pvo > 1e-4
    table = np.stack([hist, ho])
    table = table[:, table.sum(0) > 10]
    assert stats.chi2_contingency(table)[1] > 1e-4


def test_batched_sweep_smallest_replicas_match_oracle(snapmod):
    from synth import telechelic_sweep
    gold = json.loads((GOLDEN / "telechelic_sweep_smallest8.json").read_text())
    reps = telechelic_sweep(processes=16)
    sizes = [s.n for s in reps]
    offs = np.concatenate([[0], np.cumsum(sizes)])
    sim = snapmod.from_system(reps, precision="mixed")
    steps, burn, every, blocks = gold["steps"], gold["burn_in"], gold["every"], gold["blocks"]
    idx = [g["replica"] for g in gold["runs"]]
    for g in gold["runs"]:
        s = reps[g["replica"]]
        assert s.n == g["n"] and s.seed == g["seed"]
    sim.step(burn)
    series = {r: [] for r in idx}
    for _ in range((steps - burn) // every):
        sim.step(every)
        b = sim.bonds()
        for r in idx:
            sel = (b[:, 0] >= offs[r]) & (b[:, 0] < offs[r + 1])
            series[r].append(sel.sum())
    sim.close()
    for g in gold["runs"]:
        f = np.array(series[g["replica"]], dtype=np.float64) / g["n_ends"]
        se = f.reshape(blocks, -1).mean(1).std(ddof=1) / math.sqrt(blocks)
        z = (f.mean() - g["bonded_fraction"]) / math.sqrt(se ** 2 + g["bonded_fraction_se"] ** 2 + 1e-6)
        assert abs(z) < 4.0, (g["replica"], f.mean(), g["bonded_fraction"], se, g["bonded_fraction_se"])


def test_telechelic_network_bonded_fraction_matches_oracle(snapmod):
    """Telechelic network (2000 chains x 12 + 4000 crosslinkers), mixed precision:
    the bonded fraction of chain ends over steps 500-1000 agrees with the FP64
    oracle run (tests/golden/telechelic_network.json) within both error bars."""
    from synth import telechelic
    gold = json.loads((GOLDEN / "telechelic_network.json").read_text())
    s = telechelic()
    assert s.n == gold["n"]
    sim = snapmod.from_system(s, precision="mixed")
    sim.step(gold["from"])
    f = []
    for _ in range((gold["steps"] - gold["from"]) // gold["every"]):
        sim.step(gold["every"])
        f.append(sim.stats()["n_bonds"] / gold["n_ends"])
    sim.close()
    f = np.array(f)
    se = f.reshape(gold["blocks"], -1).mean(1).std(ddof=1) / math.sqrt(gold["blocks"])
    z = (f.mean() - gold["bonded_fraction"]) / math.sqrt(se ** 2 + gold["bonded_fraction_se"] ** 2)
    assert abs(z) < 4.0, (f.mean(), gold["bonded_fraction"], se, gold["bonded_fraction_se"])

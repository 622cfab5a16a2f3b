"""Writes assoc_ab_observables.json: trajectory observables of the A+B
association workload (500 A + 500 B at number density 0.1, WCA, harmonic A-B
bonds k = 100, r0 = 1.1, formation window r <= 1.3, bond free energy 5 kT,
valence 1, Langevin kT = 1, gamma = 1, dt = 0.005, 10^4 steps) from the FP64
oracle only, for eight seeds.  Per seed: the bonded fraction of A sites and the
A-B pair-distance counts (r < 1.6, 32 bins) sampled every 100 steps after 2000
steps, summarised as means with block-average standard errors (8 blocks), and
the lifetime histogram of every bond broken in the run.

    python tests/golden/make_assoc_ab_observables.py

The GPU test (tests/test_gpu_observables.py) runs the same seeds and sampling.
"""
import json
import multiprocessing as mp
import sys
from pathlib import Path

import numpy as np

HERE = Path(__file__).resolve().parent
sys.path.insert(0, str(HERE.parents[1]))

SEEDS = [20260921 + k for k in range(8)]
STEPS, BURN, EVERY, BLOCKS = 10_000, 2_000, 100, 8
R_MAX, NBINS = 1.6, 32


def one_seed(seed):
    import oracle
    from synth import assoc_ab
    s = assoc_ab(seed=seed)
    o = oracle.OracleSystem(s)
    n_a = int((s.types == 0).sum())
    frac, counts = [], []
    o.run(BURN)
    for _ in range((STEPS - BURN) // EVERY):
        o.run(EVERY)
        frac.append(o.bonds().shape[0] / n_a)
        counts.append(o.rdf_counts(0, 1, R_MAX, NBINS))
    frac = np.array(frac)
    counts = np.array(counts, dtype=np.float64)
    fb = frac.reshape(BLOCKS, -1).mean(1)
    cb = counts.reshape(BLOCKS, -1, NBINS).mean(1)
    return {"seed": seed, "bonded_fraction": float(frac.mean()),
            "bonded_fraction_se": float(fb.std(ddof=1) / np.sqrt(BLOCKS)),
            "rdf_counts_mean": counts.mean(0).tolist(),
            "rdf_counts_se": (cb.std(0, ddof=1) / np.sqrt(BLOCKS)).tolist(),
            "lifetime_hist": o.life_hist.tolist()}


def main():
    with mp.get_context("spawn").Pool(len(SEEDS)) as pool:
        runs = pool.map(one_seed, SEEDS)
    out = {"workload": "assoc_ab (500 A + 500 B, rho 0.1, eps 5 kT, r0 1.1, r_max 1.3, 10^4 steps)",
           "source": "FP64 oracle (oracle/), plain C, single thread",
           "steps": STEPS, "burn_in": BURN, "every": EVERY, "blocks": BLOCKS,
           "rdf": {"type_a": 0, "type_b": 1, "r_max": R_MAX, "nbins": NBINS}, "runs": runs}
    (HERE / "assoc_ab_observables.json").write_text(json.dumps(out, indent=1) + "\n")
    print("bonded fraction per seed:", [round(r["bonded_fraction"], 4) for r in runs])


if __name__ == "__main__":
    main()

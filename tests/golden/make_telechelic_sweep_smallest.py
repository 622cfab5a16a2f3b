"""Writes telechelic_sweep_smallest8.json: the bonded fraction of chain ends of
the 8 smallest replicas of the batched telechelic sweep (256 replicas, total
bead count log-uniform in [2000, 50000], bond free energy uniform in [2, 10] kT,
kT uniform in [0.8, 1.2], replica r seeded 20260921 + r; synth.telechelic_sweep),
from FP64 oracle runs of those replicas alone: 5000 steps each, sampled every
50 steps after 1000, mean with a block-average standard error (8 blocks).

    python tests/golden/make_telechelic_sweep_smallest.py

The GPU test (tests/test_gpu_observables.py) and the benchmark's batched leg run
all 256 replicas in one context and compare these 8.
"""
import json
import multiprocessing as mp
import sys
from pathlib import Path

import numpy as np

HERE = Path(__file__).resolve().parent
sys.path.insert(0, str(HERE.parents[1]))

STEPS, BURN, EVERY, BLOCKS, N_SMALLEST = 5000, 1000, 50, 8, 8


def smallest_indices():
    from synth import telechelic_sweep_specs
    specs = telechelic_sweep_specs()
    sizes = [kw["n_chains"] * 12 + kw["n_x"] for kw in specs]
    return sorted(range(len(specs)), key=lambda r: (sizes[r], r))[:N_SMALLEST], specs


def one_replica(args):
    r, kw = args
    import oracle
    from synth import telechelic
    s = telechelic(**kw)
    o = oracle.OracleSystem(s)
    n_ends = int((s.types == 1).sum())
    o.run(BURN)
    frac = []
    for _ in range((STEPS - BURN) // EVERY):
        o.run(EVERY)
        frac.append(o.bonds().shape[0] / n_ends)
    frac = np.array(frac)
    blocks = frac.reshape(BLOCKS, -1).mean(1)
    return {"replica": r, "n": s.n, "n_ends": n_ends, "eps": kw["eps"], "kT": kw["kT"], "seed": kw["seed"],
            "bonded_fraction": float(frac.mean()),
            "bonded_fraction_se": float(blocks.std(ddof=1) / np.sqrt(BLOCKS))}


def main():
    idx, specs = smallest_indices()
    with mp.get_context("spawn").Pool(len(idx)) as pool:
        runs = pool.map(one_replica, [(r, specs[r]) for r in idx])
    out = {"workload": "8 smallest replicas of the 256-replica telechelic sweep (synth.telechelic_sweep)",
           "source": "FP64 oracle (oracle/), each replica alone",
           "steps": STEPS, "burn_in": BURN, "every": EVERY, "blocks": BLOCKS, "runs": runs}
    (HERE / "telechelic_sweep_smallest8.json").write_text(json.dumps(out, indent=1) + "\n")
    for x in runs:
        print(x["replica"], x["n"], round(x["eps"], 2), round(x["bonded_fraction"], 4), round(x["bonded_fraction_se"], 4))


if __name__ == "__main__":
    main()

"""Writes telechelic_network.json: the bonded fraction of chain ends of the
telechelic network (2000 chains x 12 beads, FENE k = 30, R0 = 1.5 + WCA, chain
ends S of valence 1 bonding to 4000 crosslinkers X of valence 3, bead density
0.3, S-X harmonic k = 100, r0 = 1.0, window r <= 1.25, bond free energy 8 kT;
synth.telechelic with its default seed) from one FP64 oracle run of 1000 steps,
sampled every 20 steps from step 500, mean with a block-average standard error
(5 blocks).

    python tests/golden/make_telechelic_network.py
"""
import json
import sys
from pathlib import Path

import numpy as np

HERE = Path(__file__).resolve().parent
sys.path.insert(0, str(HERE.parents[1]))

STEPS, FROM, EVERY, BLOCKS = 1000, 500, 20, 5


def main():
    import oracle
    from synth import telechelic
    s = telechelic()
    o = oracle.OracleSystem(s)
    n_ends = int((s.types == 1).sum())
    o.run(FROM)
    frac = []
    for _ in range((STEPS - FROM) // EVERY):
        o.run(EVERY)
        frac.append(o.bonds().shape[0] / n_ends)
    frac = np.array(frac)
    blocks = frac.reshape(BLOCKS, -1).mean(1)
    out = {"workload": "telechelic network (synth.telechelic defaults, 28000 beads)",
           "source": "FP64 oracle (oracle/), one run", "steps": STEPS, "from": FROM, "every": EVERY,
           "blocks": BLOCKS, "n": s.n, "n_ends": n_ends, "seed": s.seed,
           "bonded_fraction": float(frac.mean()),
           "bonded_fraction_se": float(blocks.std(ddof=1) / np.sqrt(BLOCKS)),
           "series": frac.tolist()}
    (HERE / "telechelic_network.json").write_text(json.dumps(out, indent=1) + "\n")
    print(out["bonded_fraction"], out["bonded_fraction_se"])


if __name__ == "__main__":
    main()

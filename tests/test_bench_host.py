"""Host-side helpers of bench.py (no GPU): the inside-cut fraction that the
FP64-plain roofline counts, checked against a brute-force all-pairs count."""
import numpy as np

import bench
from synth import random_frozen


def test_inside_cut_fraction_matches_brute_force():
    s = random_frozen(seed=41, n=300, box=8.0, type_fracs=(0.4, 0.6), sigma=(1.0, 0.6), overlap_factor=0.8)
    pos = s.pos + np.random.default_rng(0).normal(scale=0.05, size=s.pos.shape)   # some outside the box
    box = np.asarray(s.box)
    p = np.mod(pos, box)
    sig = np.asarray(s.sigma)
    t = np.asarray(s.types)
    inside = 0
    for i in range(len(p)):
        d = p[i + 1:] - p[i]
        d -= box * np.rint(d / box)
        r2 = (d * d).sum(1)
        rc = 0.5 * (sig[t[i]] + sig[t[i + 1:]]) * 2.0 ** (1.0 / 6.0)
        inside += int((r2 < rc * rc).sum())
    nbar = 7.0
    assert inside > 0
    assert abs(bench.inside_cut_fraction(s, pos, nbar) - 2.0 * inside / (nbar * len(p))) < 1e-12


def test_dgemm_rate_is_none_without_a_device():
    class NoCuda:
        float64 = None

        @staticmethod
        def randn(*a, **k):
            raise RuntimeError("no device")

    assert bench.fp64_dgemm_tflops(NoCuda) is None

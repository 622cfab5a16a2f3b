"""Pins of the oracle's random-number generator and exponential.

Philox-4x32-10 (the counter-based generator named in Sec. II.E of the paper) is
checked against its published known-answer vectors; the exponential used in
the acceptance factor of Eq. (3) is checked against the platform libm.
"""
import math
from pathlib import Path

import numpy as np
import pytest

GOLDEN = Path(__file__).parent / "golden" / "philox4x32_10_kat.txt"


def _kat_rows():
    rows = []
    for line in GOLDEN.read_text().splitlines():
        if not line.strip() or line.startswith("#"):
            continue
        w = [int(x, 16) for x in line.split()]
        rows.append((w[0:4], w[4:6], w[6:10]))
    return rows


@pytest.mark.parametrize("ctr,key,out", _kat_rows())
def test_philox_known_answers(oracle_mod, ctr, key, out):
    got = oracle_mod.philox4x32_10(ctr, key)
    assert [int(x) for x in got] == out


def test_philox_counter_sensitivity(oracle_mod):
    # every counter and key word must change the output (a dropped word fails)
    base = oracle_mod.philox4x32_10([1, 2, 3, 4], [5, 6])
    for i in range(4):
        c = [1, 2, 3, 4]
        c[i] ^= 1
        assert list(oracle_mod.philox4x32_10(c, [5, 6])) != list(base)
    for i in range(2):
        k = [5, 6]
        k[i] ^= 1
        assert list(oracle_mod.philox4x32_10([1, 2, 3, 4], k)) != list(base)


def test_u53_range_and_resolution(oracle_mod):
    assert oracle_mod.u53(0, 0) == 0.0
    assert oracle_mod.u53(0xFFFFFFFF, 0xFFFFFFFF) == 1.0 - 2.0 ** -53
    assert oracle_mod.u53(0, 1 << 11) == 2.0 ** -53
    assert oracle_mod.u53(1, 0) == 2.0 ** -32
    # uniformity of the first moments over Philox output
    rng_vals = []
    for c in range(20000):
        w = oracle_mod.philox4x32_10([c, 0, 7, 9], [123, 5])
        rng_vals.append(oracle_mod.u53(w[0], w[1]))
    u = np.array(rng_vals)
    assert abs(u.mean() - 0.5) < 5 * math.sqrt(1 / 12 / u.size)
    assert abs((u ** 2).mean() - 1 / 3) < 5 * math.sqrt(4 / 45 / u.size)


def test_exp_against_libm(oracle_mod):
    rng = np.random.default_rng(7)
    xs = np.concatenate([rng.uniform(-745.0, 0.0, 20000), rng.uniform(-5, 5, 20000),
                         rng.uniform(0, 700, 2000),
                         -np.abs(rng.normal(0, 1e-3, 2000)), [0.0, -0.0, -1.0, 1.0]])
    worst = 0.0
    for x in xs:
        ref = math.exp(x)
        got = oracle_mod.exp(x)
        if ref == 0.0:
            assert got == 0.0 or got <= 5e-324
            continue
        ulp = math.ulp(ref)
        worst = max(worst, abs(got - ref) / ulp)
    assert worst <= 2.0, worst
    assert oracle_mod.exp(0.0) == 1.0
    assert oracle_mod.exp(-800.0) == 0.0
    assert math.isnan(oracle_mod.exp(float("nan")))


def test_exp_subnormal_range(oracle_mod):
    for x in np.linspace(-745.0, -708.0, 997):
        ref = math.exp(x)
        got = oracle_mod.exp(x)
        # subnormal results carry fewer bits: allow 2 units of the smallest subnormal
        assert abs(got - ref) <= max(2 * math.ulp(ref), 2 * 5e-324)


def test_log_against_libm(oracle_mod):
    # the oracle's own logarithm (used for the FENE bond energy of Eq. 3)
    rng = np.random.default_rng(11)
    xs = np.concatenate([np.geomspace(1e-320, 1e308, 4000), rng.uniform(0.5, 2.0, 20000),
                         1.0 - np.geomspace(1e-16, 0.999, 4000), [0.5, 2.0, math.sqrt(2.0), 1.0]])
    worst = 0.0
    for x in xs:
        ref = math.log(x)
        got = oracle_mod.log(x)
        if ref == 0.0:
            assert got == 0.0
            continue
        worst = max(worst, abs(got - ref) / math.ulp(ref))
    assert worst <= 2.0, worst
    assert oracle_mod.log(1.0) == 0.0
    assert oracle_mod.log(0.0) == -math.inf and oracle_mod.log(math.inf) == math.inf
    assert math.isnan(oracle_mod.log(-1.0)) and math.isnan(oracle_mod.log(float("nan")))
    # exp and log of this library invert each other to a few ulp
    for x in rng.uniform(-30, 30, 2000):
        assert abs(oracle_mod.log(oracle_mod.exp(x)) - x) <= 4 * math.ulp(max(abs(x), 1e-300)) + 1e-15

"""Pins of the oracle's kinetic-temperature option (Sec. II.B: T in Eq. 3 is the
instantaneous kinetic temperature when the updater triggers; Sec. II.D: the
same T enters the slip factor and the melting switch g(T)).

- The deterministic fixed-point sum equals the plain FP64 mean sum v^2 / (3 n)
  up to its rounding bound, and exactly when every v^2 is a multiple of 2^-32.
- Under the oracle's Langevin dynamics of an ideal gas, the kinetic temperature
  of the half-step velocities averages kT / (1 - gamma dt / 2) (the closed form
  of the linear recursion pinned in test_oracle_md_pins).
- Frozen pairs whose velocities give T_kin = 0.5 while the set-point is kT = 1
  reach the two-state fraction K e^{-U/0.5} / (1 + K e^{-U/0.5}): Eq. 3 uses the
  kinetic T (with the set-point the fraction would be the kT = 1 value).
- Melting switch at the kinetic T: T_kin = T_melt gives bonded fraction 1/2
  while the set-point sits far above T_melt (where binding is switched off).
- tanh (the switch's, built on the oracle's exp) against libm, with its exact
  values at 0 and for large |x|.
"""
import math

import numpy as np
import pytest

from synth import frozen_pairs, assoc_ab


def _two_state_se(p_bond, a, b, n_pairs, T):
    lam = 1.0 - a - b
    return math.sqrt(p_bond * (1 - p_bond) / (n_pairs * T) * (1 + lam) / (1 - lam))


def test_fixed_point_sum_matches_definition(oracle_mod):
    s = assoc_ab(seed=3, n_a=400, n_b=400, rho=0.1)
    o = oracle_mod.OracleSystem(s)
    rng = np.random.default_rng(4)
    for scale in (1.0, 0.01, 30.0):
        v = rng.normal(size=(s.n, 3)) * scale
        o.set_velocities(v)
        plain = float((v ** 2).sum()) / (3 * s.n)
        # each particle's v^2 is rounded to 2^-32: |error| <= n 2^-33 / (3 n)
        assert abs(o.kinetic_T() - plain) <= 2 ** -33 / 3 + 1e-14 * plain
    # exact when every v^2 is a multiple of 2^-32
    m = rng.integers(-2 ** 12, 2 ** 12, size=(s.n, 3))
    o.set_velocities(m * 2.0 ** -16)
    total = int((m.astype(np.int64) ** 2).sum())
    assert o.kinetic_T() == float(total) * 2.0 ** -32 / (3 * s.n)


def test_ideal_gas_kinetic_temperature(oracle_mod):
    s = assoc_ab(seed=5, n_a=500, n_b=500, rho=0.02)
    s.reactions = []
    s.eps_pair = np.zeros((2, 2))
    s.kinetic_T = 1
    o = oracle_mod.OracleSystem(s)
    o.run(500)
    ts = []
    for _ in range(300):
        o.run(10)
        ts.append(o.kinetic_T())
    ts = np.array(ts)
    expect = s.kT / (1 - 0.5 * s.gamma * s.dt)
    blocks = ts.reshape(15, 20).mean(axis=1)     # blocks of 200 steps, the velocity correlation time 1/gamma
    se = blocks.std(ddof=1) / math.sqrt(len(blocks))
    assert abs(ts.mean() - expect) < 4 * se, (ts.mean(), expect, se)


def _frozen_fraction(oracle_mod, s, T_sweeps, burn=50):
    o = oracle_mod.OracleSystem(s)
    counts = []
    for t in range(T_sweeps + burn):
        o.sweep(step=t)
        if t >= burn:
            counts.append(o.occ.sum() / 2)
    return np.mean(counts) / (s.n // 2), o


def test_frozen_pairs_use_kinetic_temperature(oracle_mod):
    n_pairs, T, eps, r = 200, 3000, 2.0, 1.2
    s = frozen_pairs(seed=7, n_pairs=n_pairs, r=r, eps=eps, kT=1.0)
    # v = (1, 0.5, 0.5) for every particle: v^2 = 1.5 and T_kin = 1.5 / 3 = 0.5 exactly
    s.vel = np.tile([1.0, 0.5, 0.5], (s.n, 1))
    s.kinetic_T = 1
    k, r0 = s.bond_types[0].k, s.bond_types[0].r0
    U = 0.5 * k * (r - r0) ** 2
    a = math.exp(-U / 0.5)
    b = math.exp(-eps)
    expect = a / (a + b)
    frac, o = _frozen_fraction(oracle_mod, s, T)
    assert o.kinetic_T() == 0.5
    se = _two_state_se(expect, a, b, n_pairs, T)
    assert abs(frac - expect) < 4.5 * se, (frac, expect, se)
    # the set-point value is far away (U = 0.5 kT at r = 1.2)
    a1 = math.exp(-U / 1.0)
    assert abs(a1 / (a1 + b) - expect) > 20 * se


def test_melting_switch_at_kinetic_temperature(oracle_mod):
    lam, tm, kon, koff, n_pairs, T = 8.0, 0.5, 20.0, 4.0, 200, 3000
    s = frozen_pairs(seed=9, n_pairs=n_pairs, r=1.1, eps=0.0, kT=3.0)   # set-point far above T_melt
    s.reactions[0].melt = (lam, tm, kon, koff, 0.0, kon - koff)
    s.vel = np.tile([1.0, 0.5, 0.5], (s.n, 1))                         # T_kin = 0.5 = T_melt
    s.kinetic_T = 1
    frac, o = _frozen_fraction(oracle_mod, s, T)
    pon = poff = 0.5 * kon * s.dt
    se = _two_state_se(0.5, pon, poff, n_pairs, T)
    assert abs(frac - 0.5) < 4.5 * se, (frac, se)
    # with the set-point temperature binding would be switched off
    s.kinetic_T = 0
    frac0, _ = _frozen_fraction(oracle_mod, s, 300)
    assert frac0 < 0.01


def test_tanh_against_libm(oracle_mod):
    xs = np.concatenate([np.linspace(-20, 20, 4001), [-1e-8, 1e-8, 0.0, 1e-300, 30.0, -30.0, 400.0]])
    for x in xs:
        t = oracle_mod.tanh(float(x))
        m = math.tanh(float(x))
        # relative accuracy away from 0; near 0 the subtraction 1 - e^{-2|x|} keeps
        # the absolute error at a few units of 2^-53, which is what g(T) needs
        assert abs(t - m) <= 4 * math.ulp(abs(m)) + 4 * 2.0 ** -53, (x, t, m)
    assert oracle_mod.tanh(0.0) == 0.0 and oracle_mod.tanh(400.0) == 1.0 and oracle_mod.tanh(-400.0) == -1.0

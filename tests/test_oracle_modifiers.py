"""Pins of the oracle's rate modifiers (Sec. II.D).

Slip bond, Eq. (slip): a bond at separation r breaks with
P_off(r) = P_off^0 exp(a sqrt(U_b(r)/kT)), capped at 1.
- Frozen pairs at r != r0 are two-state chains with P_on(r) (Eq. 3) and
  P_off(r): the stationary bonded fraction is P_on(r)/(P_on(r) + P_off(r)).
- At r = r0 (U_b = 0) the modifier has no effect; a = 0 switches it off.
- The broken fraction of pre-set bonds in one sweep equals P_off(r) at every r.
- kT -> 0 is well defined (App. A): for U_b > 0 P_off tends to 1 and every
  such bond breaks at kT = 0; for U_b = 0 it stays P_off^0.
- The exponent is the Bell form f x*/kT with f = sqrt(2 k U_b) the tension of
  the harmonic bond and x* = a sqrt(kT/(2k)).

Melting switch, Eqs. (gT)-(kT): g = (tanh(lambda (T - T_melt)) + 1)/2 and
k(T) = k_init (1 - g) + k_melt g, with P = k n dt (Eq. 2).
- With k_on^melt = 0, the choice k_off^melt = k_on^init - k_off^init makes
  half of the pairs bound at T_melt: K(T_melt) = 1.  Frozen pairs at U_b = 0
  then sit at bonded fraction 1/2 at T_melt, at the low-temperature value
  K_init/(1 + K_init) well below it, and unbind completely well above it.
"""
import math

import numpy as np
import pytest

from synth import frozen_pairs


def _two_state_se(p, a, b, m, T):
    lam = 1.0 - a - b
    return math.sqrt(p * (1 - p) / (m * T) * (1 + lam) / (1 - lam))


def _slip_p_off(p0, a, k, r, r0, kT):
    U = 0.5 * k * (r - r0) ** 2
    if a == 0.0:
        return p0
    x = U / kT if kT > 0 else (math.inf if U > 0 else 0.0)
    return min(1.0, p0 * math.exp(a * math.sqrt(x))) if a * math.sqrt(x) < 700 else 1.0


def _run_fraction(oracle_mod, s, T, burn=50):
    o = oracle_mod.OracleSystem(s, p_on0=1.0)
    counts = []
    for t in range(T + burn):
        o.sweep(step=t)
        if t >= burn:
            counts.append(o.occ.sum() / 2)
    return np.mean(counts) / (s.n // 2)


@pytest.mark.parametrize("r,a", [(1.2, 1.0), (1.25, 0.5), (1.1, 2.0), (1.2, 0.0)])
def test_slip_bond_stationary_fraction(oracle_mod, r, a):
    eps, n_pairs, T = 2.0, 200, 3000
    s = frozen_pairs(seed=3, n_pairs=n_pairs, r=r, eps=eps)
    s.reactions[0].slip_a = a
    k, r0 = s.bond_types[0].k, s.bond_types[0].r0
    p_on = math.exp(-0.5 * k * (r - r0) ** 2 / s.kT)
    p_off = _slip_p_off(math.exp(-eps), a, k, r, r0, s.kT)
    expect = p_on / (p_on + p_off)
    frac = _run_fraction(oracle_mod, s, T)
    se = _two_state_se(expect, p_on, p_off, n_pairs, T)
    assert abs(frac - expect) < 4.5 * se, (frac, expect, se)


@pytest.mark.parametrize("kT", [1.0, 0.3, 1e-3, 0.0])
@pytest.mark.parametrize("r", [1.1, 1.2])
def test_slip_broken_fraction_and_zero_temperature(oracle_mod, kT, r):
    n_pairs, eps, a = 400, 1.5, 0.8
    s = frozen_pairs(seed=6, n_pairs=n_pairs, r=r, eps=eps, kT=kT)
    s.reactions[0].slip_a = a
    k, r0 = s.bond_types[0].k, s.bond_types[0].r0
    o = oracle_mod.OracleSystem(s, p_on0=1.0)
    pairs = np.stack([np.arange(0, 2 * n_pairs, 2), np.arange(1, 2 * n_pairs, 2),
                      np.zeros(n_pairs, np.int64)], axis=1)
    broken = 0
    sweeps = 20
    for t in range(sweeps):
        o.set_bonds(pairs)
        st = o.sweep(step=1000 + t)
        broken += st["broken"]
    # the separations as placed (r0 up to rounding: at kT = 0 any U_b > 0, however
    # small, takes the limit P_off = 1, so each pair's own r decides)
    d = s.pos[1::2] - s.pos[0::2]
    d -= s.box * np.rint(d / s.box)
    rr = np.sqrt((d * d).sum(axis=1))
    p = np.array([_slip_p_off(math.exp(-eps), a, k, x, r0, kT) for x in rr])
    assert np.all((p >= 0.0) & (p <= 1.0))
    mean, var = sweeps * p.sum(), sweeps * (p * (1 - p)).sum()
    assert abs(broken - mean) <= 4.5 * math.sqrt(var) + 1e-9, (broken, mean)
    if r != r0 and kT == 0.0:
        assert broken == sweeps * n_pairs       # the kT -> 0 limit for a stretched bond
    if r == r0 and kT > 0.0:
        # U_b at rounding level: no acceleration
        assert np.all(np.abs(p - math.exp(-eps)) < 1e-9)


def test_slip_exponent_is_bells_force_form():
    k, a = 100.0, 0.8
    for kT in (0.5, 1.0, 2.0):
        for r in (1.0, 1.15, 1.3):
            U = 0.5 * k * (r - 1.1) ** 2
            f = math.sqrt(2.0 * k * U)                     # tension of the harmonic bond
            x_star = a * math.sqrt(kT / (2.0 * k))         # Bell distance
            assert abs(a * math.sqrt(U / kT) - f * x_star / kT) < 1e-12


def test_melting_rates_closed_forms(oracle_mod):
    lam, tm, kon, koff = 8.0, 1.0, 20.0, 4.0
    r = oracle_mod.melting_rates
    pon, poff = r(tm, lam, tm, kon, koff, 0.0, kon - koff, 1, 0.005)
    assert abs(pon - poff) < 1e-15                   # K(T_melt) = 1 with this k_off^melt
    assert abs(pon - 0.5 * kon * 0.005) < 1e-15      # g(T_melt) = 1/2
    lo = r(tm - 5.0, lam, tm, kon, koff, 0.0, kon - koff, 1, 0.005)
    hi = r(tm + 5.0, lam, tm, kon, koff, 0.0, kon - koff, 1, 0.005)
    assert abs(lo[0] - kon * 0.005) < 1e-12 and abs(lo[1] - koff * 0.005) < 1e-12
    assert hi[0] < 1e-12 and abs(hi[1] - (kon - koff) * 0.005) < 1e-12


@pytest.mark.parametrize("dT", [0.0, -0.6, 0.6])
def test_melting_switch_bonded_fraction(oracle_mod, dT):
    lam, tm, kon, koff, n_pairs, T = 8.0, 1.0, 20.0, 4.0, 200, 3000
    s = frozen_pairs(seed=9, n_pairs=n_pairs, r=1.1, eps=0.0, kT=tm + dT)
    s.reactions[0].melt = (lam, tm, kon, koff, 0.0, kon - koff)
    pon, poff = oracle_mod.melting_rates(tm + dT, lam, tm, kon, koff, 0.0, kon - koff, 1, s.dt)
    frac = _run_fraction(oracle_mod, s, T)
    if dT == 0.0:
        expect = 0.5
    elif dT < 0:
        expect = pon / (pon + poff)
        assert abs(expect - kon / (kon + koff)) < 2e-3    # K_init/(1 + K_init) up to g(T) ~ 1e-4
    else:
        expect = pon / (pon + poff)
        assert expect < 2e-3                         # melted: binding switched off
    se = _two_state_se(expect, pon, poff, n_pairs, T) + 1e-4
    assert abs(frac - expect) < 4.5 * se, (frac, expect, se)


def test_bond_period_sweeps_only_every_n_steps(oracle_mod):
    # Eq. 2 with n > 1: the updater acts on steps that are multiples of n only
    from synth import assoc_ab
    s = assoc_ab(seed=16)
    s.bond_period = 5
    o = oracle_mod.OracleSystem(s)
    prev = o.bonds()
    changed_at = []
    for t in range(60):
        o.run(1)
        b = o.bonds()
        if not np.array_equal(b, prev):
            changed_at.append(t)
        prev = b
    assert changed_at and all(t % 5 == 0 for t in changed_at), changed_at

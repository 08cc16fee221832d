"""Pins of the oracle's exact regions against textbook values, quadrature and
physical identities (no GPU)."""
import math
import os

import numpy as np
import pytest
from scipy import integrate

from paper_2308_16877_gb300 import workloads as W
from tolerances import blackscholes_tol

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _bs_inputs(rows, dtype):
    x = np.array(rows, dtype=np.float64).T.copy()
    return x.astype(dtype)


def test_blackscholes_textbook_value(orc):
    """Hull's worked example, prices printed to two decimals."""
    rows = [l.split() for l in open(os.path.join(GOLD, "blackscholes_hull.txt"))
            if l.strip() and not l.startswith("#")]
    for S, K, T, sig, r, call, put, dec in rows:
        S, K, T, sig, r, call, put = map(float, (S, K, T, sig, r, call, put))
        x = _bs_inputs([[S, K, T, sig]], np.float64)
        c = orc.run_exact(orc.BLACKSCHOLES, x, r)[0]
        assert round(c, int(dec)) == pytest.approx(call, abs=1e-12)
        # put from put-call parity C - P = S - K e^{-rT}
        p = c - S + K * math.exp(-r * T)
        assert round(p, int(dec)) == pytest.approx(put, abs=1e-12)
        c32 = orc.run_exact(orc.BLACKSCHOLES, x.astype(np.float32), r)[0]
        assert round(float(c32), int(dec)) == pytest.approx(call, abs=1e-12)


def _bs_quadrature(S, K, T, sig, r):
    """Discounted expected payoff under the risk-neutral lognormal, by quadrature
    over the standard normal variable (no closed form involved)."""
    mu = math.log(S) + (r - 0.5 * sig * sig) * T
    s = sig * math.sqrt(T)
    z0 = (math.log(K) - mu) / s

    def f(z):
        return (math.exp(mu + s * z) - K) * math.exp(-0.5 * z * z) / math.sqrt(2 * math.pi)

    val, _ = integrate.quad(f, z0, max(z0, 0.0) + 40.0, epsabs=0.0, epsrel=1e-13, limit=200)
    return math.exp(-r * T) * val


def test_blackscholes_matches_quadrature(orc):
    x = W.blackscholes_inputs(64, seed=7).astype(np.float64)
    c = orc.run_exact(orc.BLACKSCHOLES, x, W.BS_RATE)
    checked = 0
    for i in range(64):
        S, K, T, sig = x[:, i]
        ref = _bs_quadrature(S, K, T, sig, W.BS_RATE)
        if ref < 1e-6 * S:
            continue  # quadrature of a vanishing tail is not informative
        assert c[i] == pytest.approx(ref, rel=1e-9), (i, S, K, T, sig)
        checked += 1
    assert checked >= 20


def test_blackscholes_zero_vol_limit(orc):
    """sigma -> 0: the call tends to its discounted intrinsic value."""
    rows = [[30.0, 10.0, 1.0, 1e-6], [30.0, 29.0, 2.0, 1e-6], [10.0, 30.0, 1.0, 1e-6]]
    x = _bs_inputs(rows, np.float64)
    c = orc.run_exact(orc.BLACKSCHOLES, x, 0.02)
    for (S, K, T, _), ci in zip(rows, c):
        assert ci == pytest.approx(max(S - K * math.exp(-0.02 * T), 0.0), abs=1e-9)


def test_blackscholes_f32_close_to_f64(orc):
    """The single-precision region stays within the arithmetic-derived bound of
    the double-precision one (see tolerances.blackscholes_tol)."""
    x = W.blackscholes_inputs(1 << 14, seed=3)
    c32 = orc.run_exact(orc.BLACKSCHOLES, x, W.BS_RATE).astype(np.float64)
    c64 = orc.run_exact(orc.BLACKSCHOLES, x.astype(np.float64), W.BS_RATE)
    assert np.all(np.abs(c32 - c64) <= blackscholes_tol(x, W.BS_RATE))


def orc_eos(orc, e, v1, dv, q, g=5.0 / 3.0):
    x = np.array([np.atleast_1d(e), np.atleast_1d(v1), np.atleast_1d(dv), np.atleast_1d(q)],
                 dtype=np.float64)
    return orc.run_exact(orc.EOS, x, g)


def test_eos_implicit_trapezoid_residual(orc):
    """The output satisfies e1 - e0 + (p0 + p1 + 2q) dv / 2 = 0 with the
    ideal-gas law p = (gamma-1) e / v at both ends."""
    g = 5.0 / 3.0
    x = W.eos_inputs(4096, seed=11)
    p1 = orc.run_exact(orc.EOS, x, g)
    e0, v1, dv, q = x
    p0 = (g - 1) * e0 / (v1 - dv)
    e1 = p1 * v1 / (g - 1)
    ok = e1 > 0
    res = e1 - e0 + 0.5 * (p0 + p1 + 2 * q) * dv
    assert np.all(np.abs(res[ok]) <= 1e-12 * (np.abs(e0[ok]) + np.abs(p0[ok] * dv[ok]) + 1.0))
    assert np.all(p1 >= 0)


def test_eos_no_volume_change_is_ideal_gas(orc):
    g = 1.4
    e = np.array([1.0, 2.5e5, 3.9e6])
    v = np.array([1.0, 0.7, 1.3])
    p = orc_eos(orc, e, v, np.zeros(3), np.zeros(3), g)
    assert np.array_equal(p, (g - 1) * e / v)


def test_eos_adiabat(orc):
    """Many small q = 0 steps follow the adiabat p v^gamma = const to second order."""
    g = 5.0 / 3.0
    e, v = 1.0, 1.0
    p_start = (g - 1) * e / v
    steps = 2000
    dv = -0.5 / steps
    for _ in range(steps):
        v1 = v + dv
        p = orc_eos(orc, e, v1, dv, 0.0, g)[0]
        e, v = p * v1 / (g - 1), v1
    assert p * v ** g == pytest.approx(p_start, rel=1e-6)


def test_eos_clamps_negative_energy(orc):
    # strong expansion with a huge viscosity drives the update negative
    p = orc_eos(orc, 1.0, 1.5, 0.5, 100.0)
    assert p[0] == 0.0


def test_identity_region_is_bitwise_copy(orc):
    for dt in (np.float32, np.float64):
        x = W.identity_inputs(1000, d=3, dtype=dt)
        assert np.array_equal(orc.run_exact(orc.IDENTITY, x), x[0])

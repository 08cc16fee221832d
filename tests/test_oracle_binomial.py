"""Pins of the oracle's Binomial Options region (American call on a
Cox-Ross-Rubinstein tree, single precision) against closed forms (no GPU):
the European CRR price as an explicit binomial sum (for a call on a
non-dividend stock with r >= 0 early exercise never binds, so the two agree
up to the tree's single-precision rounding), convergence to Black-Scholes,
the one-step tree by hand, and early exercise when it does bind (r < 0)."""
import math

import numpy as np
import pytest

from paper_2308_16877_gb300 import workloads as W

EPS32 = 2.0 ** -24


def crr_european(S, X, T, sig, r, N):
    """e^{-rT} sum_j C(N, j) p^j (1-p)^{N-j} max(S u^{2j-N} - X, 0) in float64."""
    dt = T / N
    v = sig * math.sqrt(dt)
    u, a = math.exp(v), math.exp(r * dt)
    d = 1.0 / u
    p = (a - d) / (u - d)
    tot = 0.0
    for j in range(N + 1):
        pay = S * math.exp(v * (2 * j - N)) - X
        if pay > 0:
            tot += math.comb(N, j) * p ** j * (1 - p) ** (N - j) * pay
    return tot * math.exp(-r * T)


def bs_call(S, X, T, sig, r):
    d1 = (math.log(S / X) + (r + 0.5 * sig * sig) * T) / (sig * math.sqrt(T))
    d2 = d1 - sig * math.sqrt(T)
    N = lambda z: 0.5 * math.erfc(-z / math.sqrt(2))
    return S * N(d1) - X * math.exp(-r * T) * N(d2)


def price(orc, opts, r, N):
    x = np.array(opts, dtype=np.float32).T.copy()
    return orc.run_exact(orc.BINOMIAL, x, r, steps=N).astype(np.float64)


CASES = [(42.0, 40.0, 0.5, 0.2), (10.0, 12.0, 1.5, 0.45), (25.0, 20.0, 0.25, 0.1), (7.5, 7.5, 2.0, 0.3),
         (30.0, 5.0, 1.0, 0.2)]


@pytest.mark.parametrize("N", [1, 2, 7, 64, 300])
def test_equals_the_european_binomial_sum(orc, N):
    got = price(orc, CASES, W.BS_RATE, N)
    for (S, X, T, sig), g in zip(CASES, got):
        # float32 inputs, as the region sees them
        S, X, T, sig = (float(np.float32(v)) for v in (S, X, T, sig))
        want = crr_european(S, X, T, sig, W.BS_RATE, N)
        assert abs(g - want) <= 4 * (N + 2) * EPS32 * max(S, want) + 1e-6, (S, X, T, sig, g, want)


def test_converges_to_black_scholes(orc):
    got = price(orc, CASES, W.BS_RATE, 2048)
    for (S, X, T, sig), g in zip(CASES, got):
        S, X, T, sig = (float(np.float32(v)) for v in (S, X, T, sig))
        bs = bs_call(S, X, T, sig, W.BS_RATE)
        # CRR converges as O(1/N) (amplitude ~ S sigma sqrt(T) / N), plus the rounding bound
        assert abs(g - bs) <= 2 * S * sig * math.sqrt(T) / 2048 + 4 * 2050 * EPS32 * S, (g, bs)


def test_one_step_tree_by_hand(orc):
    S, X, T, sig, r = 20.0, 19.0, 1.0, 0.3, 0.05
    u, a = math.exp(sig), math.exp(r)
    d = 1 / u
    p = (a - d) / (u - d)
    cont = (p * max(S * u - X, 0) + (1 - p) * max(S * d - X, 0)) / a
    want = max(cont, S - X)
    assert abs(price(orc, [(S, X, T, sig)], r, 1)[0] - want) <= 8 * EPS32 * S


def test_early_exercise_binds_with_negative_rates(orc):
    """With r < 0 holding a deep in-the-money call loses value, so the American
    price exceeds the European one and equals the payoff at the root."""
    S, X, T, sig, r = 30.0, 10.0, 2.0, 0.1, -0.05
    am = price(orc, [(S, X, T, sig)], r, 200)[0]
    eu = crr_european(S, X, T, sig, r, 200)
    assert am > eu + 0.1 and abs(am - (S - X)) <= 1e-5 * S


def test_portfolio_layout():
    M, K = 96, 16
    x = W.binomial_portfolio(M, K, seed=3)
    assert x.shape == (4, M * K) and x.dtype == np.float32
    r = x.reshape(4, K, M)
    assert np.all(r[1] == r[1][:1]) and np.all(r[3] == r[3][:1])      # strike, vol per member
    assert np.all(np.diff(r[2], axis=0) < 0) and np.all(r[2] > 0)      # time to expiry decreases
    assert np.all((r[0][0] >= 5) & (r[0][0] <= 30))
    m = r[1][0] / r[0][0]
    assert np.all((m >= 0.8 - 1e-6) & (m <= 1.2 + 1e-6))
    assert np.array_equal(W.binomial_portfolio(M, K, seed=3), x)

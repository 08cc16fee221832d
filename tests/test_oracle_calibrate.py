"""The oracle's calibrated fallback bound (the surrogate's floor) against its
definition written out by brute force, and closed-form cases."""
import math
from fractions import Fraction

import numpy as np
import pytest

import oracle


def brute_floor(pred, exact, target, quantile):
    """Every distinct prediction as a candidate floor; the set it serves; the
    nearest-rank quantile (the ceil(q k)-th smallest) of the exact relative
    errors |p - a| / |a| over that set, in rational arithmetic; the smallest
    candidate whose quantile is within target."""
    best = (math.inf, 0)
    vals = sorted({float(v) for v in pred if not math.isnan(v)}, reverse=True)
    for v in vals:
        served = [i for i, p in enumerate(pred) if not math.isnan(p) and p >= v]
        k = len(served)
        rel = sorted(abs(Fraction(float(pred[i])) - Fraction(float(exact[i]))) / abs(Fraction(float(exact[i])))
                     for i in served)
        r = math.ceil(Fraction(quantile) * k)
        if rel[r - 1] <= Fraction(target):
            best = (v, k)
    return best


@pytest.mark.parametrize("seed", range(12))
def test_matches_the_definition_on_small_random_sets(seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(1, 60))
    exact = rng.uniform(0.1, 5.0, n)
    noise = rng.uniform(0.0, 0.05, n) * (1.0 + 3.0 * (exact < 1.5))
    pred = (exact * (1.0 + rng.choice([-1, 1], n) * noise)).astype(np.float32)
    if seed % 3 == 0:                      # ties
        pred[rng.integers(0, n, n // 3)] = pred[0]
    for target, q in ((0.01, 0.9), (0.02, 0.75), (0.05, 1.0), (0.03, 0.5)):
        # exact float rationals: |p - a| / |a| is compared with the target
        # exactly, the oracle multiplies instead (the same unless a ratio
        # lands on the target to within a rounding, which random draws avoid)
        assert oracle.calibrate_floor(pred, exact, target, q) == brute_floor(pred, exact, target, q)


def test_exact_predictions_serve_everything():
    rng = np.random.default_rng(3)
    exact = rng.uniform(0.5, 50.0, 5000)
    pred = exact.astype(np.float32)
    assert oracle.calibrate_floor(pred, exact) == (float(pred.min()), 5000)


def test_nothing_qualifies():
    exact = np.linspace(1.0, 2.0, 1000)
    assert oracle.calibrate_floor((exact * 1.5).astype(np.float32), exact) == (math.inf, 0)


def test_floor_stops_where_the_error_grows():
    # predictions 1..100, wrong by 5% up to 10 and exact above: at q = 1 the
    # floor is 11 (90 served); at q = 0.9 the first bad values can be served
    y = np.arange(1.0, 101.0)
    exact = np.where(y <= 10, y / 1.05, y)
    pred = y.astype(np.float32)
    assert oracle.calibrate_floor(pred, exact, 0.01, 1.0) == (11.0, 90)
    # a floor v <= 10 serves k = 101 - v with b = 11 - v bad, allowed
    # k - ceil(q k): at q = 0.9 v = 1 passes (b = 10, allowed 100 - 90);
    # at q = 0.95 v = 7 passes (b = 4, allowed 94 - 90) and every lower v
    # fails (v = 6: b = 5, allowed 95 - 91; v = 1: b = 10, allowed 5)
    assert oracle.calibrate_floor(pred, exact, 0.01, 0.9) == (1.0, 100)
    assert oracle.calibrate_floor(pred, exact, 0.01, 0.95) == (7.0, 94)


def test_ties_nan_and_signed_zero():
    pred = np.array([5, 5, 5, 1, np.nan, 0.0, -0.0], dtype=np.float32)
    exact = np.array([5, 5, 4, 1, 1, 0.0, 0.0])
    # value 5 serves 3 (one bad), value 1 serves 4, value 0 serves 6 (-0 = +0)
    assert oracle.calibrate_floor(pred, exact, 0.01, 1.0) == (math.inf, 0)
    assert oracle.calibrate_floor(pred, exact, 0.01, 0.5) == (0.0, 6)
    assert oracle.calibrate_floor(pred, exact, 0.01, 0.7) == (0.0, 6)
    assert oracle.calibrate_floor(pred, exact, 0.01, 0.9) == (math.inf, 0)

"""Pins of the oracle's quality metrics (Section 4: Eq. 1 MAPE, Eq. 2 MCR; RMSE)
against exact rational arithmetic and hand-counted cases (no GPU)."""
from fractions import Fraction

import numpy as np
import pytest


def test_mape_exact_rational(orc):
    rng = np.random.default_rng(5)
    a = rng.uniform(-3, 5, 257)
    b = a + rng.normal(0, 0.1, 257)
    v, info = orc.quality(a, b, orc.MAPE)
    ref = sum(abs(Fraction(x) - Fraction(y)) / abs(Fraction(x)) for x, y in zip(a, b)) / len(a)
    assert v == pytest.approx(float(ref), rel=1e-14)
    assert info["zeros"] == 0


def test_mape_sets_zero_denominators_aside(orc):
    a = np.array([2.0, 0.0, 4.0, 0.0])
    b = np.array([1.0, 0.0, 5.0, -3.0])
    v, info = orc.quality(a, b, orc.MAPE)
    assert v == pytest.approx((0.5 + 0.25) / 2)
    assert info == dict(zero_max_abs=3.0, zeros=2, zeros_mismatch=1)


def test_rmse_exact_rational(orc):
    rng = np.random.default_rng(6)
    a = rng.normal(size=1000)
    b = a + rng.normal(0, 1e-3, 1000)
    v, _ = orc.quality(a, b, orc.RMSE)
    ms = sum((Fraction(x) - Fraction(y)) ** 2 for x, y in zip(a, b)) / len(a)
    assert v == pytest.approx(float(ms) ** 0.5, rel=1e-14)


def test_mcr_counts(orc):
    a = np.array([0, 1, 2, 3, 4, 5, 6, 7], dtype=np.float64)
    b = np.array([0, 1, 9, 3, 9, 5, 6, 9], dtype=np.float64)
    v, _ = orc.quality(a, b, orc.MCR)
    assert v == 3 / 8


def test_identical_is_zero_and_empty_is_zero(orc):
    a = np.linspace(1, 2, 100)
    for m in (orc.MAPE, orc.RMSE, orc.MCR):
        assert orc.quality(a, a, m)[0] == 0.0
        assert orc.quality(a[:0], a[:0], m)[0] == 0.0

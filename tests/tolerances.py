"""Element-wise tolerances derived from the arithmetic of each region.

Black-Scholes in single precision: the call C = S N(d1) - K e^{-rT} N(d2) is a
difference of two non-negative terms, the larger being S N(d1), so rounding in
the final combination is bounded relative to S N(d1) (the 1e-5 relative bar of
the parity criterion). The rounding error of the argument d1 (a log, a sum and
a division, each a few units of single-precision roundoff eps32) moves the
price by dC/dd1 * delta_d1 with dC/dd1 = S phi(d1) (the K e^{-rT} phi(d2) term
is equal to it), and delta_d1 <= 16 eps32 (1 + |d1| + |ln(S/K)| / (sigma sqrt T)).
Results below 1e-30 are subnormal in single precision and keep fewer bits.
"""
import numpy as np
from scipy import special

EPS32 = float(np.finfo(np.float32).eps)
BS_RTOL = 1e-5          # relative bar for single-precision outputs
F64_RTOL = 1e-12        # relative bar for double-precision outputs


def blackscholes_tol(x, r):
    S, K, T, sig = (np.asarray(c, dtype=np.float64) for c in x)
    sst = sig * np.sqrt(T)
    lnsk = np.log(S / K)
    d1 = (lnsk + (r + 0.5 * sig * sig) * T) / sst
    big = S * special.ndtr(d1)
    dd = 16.0 * EPS32 * (1.0 + np.abs(d1) + np.abs(lnsk) / sst)
    sens = S * np.exp(-0.5 * d1 * d1) / np.sqrt(2.0 * np.pi)
    return BS_RTOL * big + sens * dd + 1e-30


EPS64 = float(np.finfo(np.float64).eps)


def blackscholes_tol64(x, r):
    """Double-precision Black-Scholes: the same derivation with eps64 and the
    1e-12 relative bar."""
    S, K, T, sig = (np.asarray(c, dtype=np.float64) for c in x)
    sst = sig * np.sqrt(T)
    lnsk = np.log(S / K)
    d1 = (lnsk + (r + 0.5 * sig * sig) * T) / sst
    big = S * special.ndtr(d1)
    dd = 16.0 * EPS64 * (1.0 + np.abs(d1) + np.abs(lnsk) / sst)
    sens = S * np.exp(-0.5 * d1 * d1) / np.sqrt(2.0 * np.pi)
    return F64_RTOL * big + sens * dd + 1e-300


def eos_tol(x, gamma):
    """EOS in double precision: p = (g-1) num / (v1 den), num = e - dv (p0 + 2q)/2,
    den = 1 + (g-1) dv / (2 v1). The subtraction in num can cancel, so its
    rounding is bounded by a few eps64 times |e| + |dv (p0 + 2q)/2|; the rest
    is relative (the 1e-12 bar)."""
    e, v1, dv, q = (np.asarray(c, dtype=np.float64) for c in x)
    g1 = gamma - 1.0
    p0 = g1 * e / (v1 - dv)
    num = e - 0.5 * dv * (p0 + 2 * q)
    den = 1.0 + 0.5 * g1 * dv / v1
    p = np.maximum(num, 0.0) * g1 / (v1 * den)
    cancel = 16.0 * EPS64 * g1 * (np.abs(e) + np.abs(0.5 * dv * (p0 + 2 * q))) / np.abs(v1 * den)
    return F64_RTOL * np.abs(p) + cancel + 1e-300


def output_tol(kind, x, param, dtype):
    """Per-invocation absolute tolerance of a region's exact output."""
    if kind == 0:
        return blackscholes_tol(x, param) if dtype == np.float32 else blackscholes_tol64(x, param)
    if kind == 1:
        return eos_tol(x, param)
    return np.zeros(x.shape[1])

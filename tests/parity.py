"""Comparison helpers for GPU-vs-oracle parity tests.

Masks of integer decisions are compared exactly where both sides take the
decision on bit-identical statistics (iACT distances of the inputs, TAF RSD of
identity-region windows, perforation). For TAF on a region whose outputs differ
by rounding between the CUDA math library and libm, each logical thread is
compared step by step until the first step whose mask differs; the accurate
decision that preceded it must have a statistic within the band the rounding
can move it by (rsd_band below), so that the threshold lies between the two
sides' statistics. The count of such threads is reported and kept small.
"""
import numpy as np


def rsd_band(window, rel_err):
    """Bound on |RSD(w') - RSD(w)| when each w_j moves by at most rel_err_j |w_j|:
    first-order sensitivity sum_j |dRSD/dw_j| |w_j| rel_err_j plus the rounding
    of the statistic itself (a few ulps of its precision)."""
    w = np.asarray(window, dtype=np.float64)
    h = w.size
    mu = w.mean()
    sd = w.std()
    if mu == 0 or sd == 0:
        return np.inf if sd > 0 else 0.0
    grad = np.abs((w - mu) / (h * sd * abs(mu)) - sd * np.sign(mu) / (h * mu * mu))
    return float(np.sum(grad * np.abs(w) * rel_err))


def taf_compare(n, T, B, level, out_g, mask_g, stat_g, out_o, mask_o, stat_o, hsize, thr, tol,
                rel_err, eps):
    """Group-by-group comparison of GPU and oracle TAF traces.

    Groups are single threads (level 0), warps (1) or blocks of B (2). Within
    a group every step is compared until the first step whose masks differ;
    before it outputs must agree within tol (per-invocation absolute bound).
    The step before the divergence must be an accurate decision step on both
    sides with at least one lane whose oracle statistic lies within the
    rounding band of the threshold. rel_err bounds the relative error of the
    exact outputs, eps the roundoff of the statistic's precision.
    Returns (lanes in diverged groups, invocations compared).
    """
    T = T if T > 0 else n
    G = 1 if level == 0 else 32 if level == 1 else B
    diverged = 0
    compared = 0
    ngroups = (min(T, n) + G - 1) // G
    for gi in range(ngroups):
        lanes = np.arange(gi * G, min(gi * G + G, T, n))
        k = 0
        div_k = None
        while True:
            idx = lanes + k * T
            idx = idx[idx < n]
            if idx.size == 0:
                break
            if np.any(mask_g[idx] != mask_o[idx]):
                div_k = k
                break
            err = np.abs(out_g[idx].astype(np.float64) - out_o[idx].astype(np.float64))
            assert np.all(err <= tol[idx]), ("output mismatch", gi, k)
            compared += idx.size
            k += 1
        if div_k is None:
            continue
        assert div_k > 0, ("divergence at the first step", gi)
        prev = lanes + (div_k - 1) * T
        prev = prev[prev < n]
        assert np.all(mask_o[prev] == 0) and np.all(mask_g[prev] == 0), ("divergence not after a decision", gi)
        near = False
        for j in prev:
            t = j % T
            hist = np.arange(t, j + 1, T)
            ex = hist[mask_o[hist] == 0][-hsize:]
            if ex.size < hsize:
                continue
            band = rsd_band(out_o[ex], rel_err[ex]) + 8 * eps * abs(float(stat_o[j]))
            if abs(float(stat_o[j]) - thr) <= band:
                near = True
                assert abs(float(stat_g[j]) - float(stat_o[j])) <= 2 * band + 1e-300, ("stats apart", gi)
        assert near, ("non-borderline flip", gi, div_k)
        diverged += lanes.size
    return diverged, compared


def source_index(n, T, mask):
    """For each invocation, the invocation whose exact output it carries: itself
    when accurate, else the newest accurate invocation of its logical thread."""
    T = T if T > 0 else n
    src = np.arange(n)
    for t in range(min(T, n)):
        idx = np.arange(t, n, T)
        ex = mask[idx] == 0
        c = np.cumsum(ex) - 1
        ok = c >= 0
        src[idx[ok]] = idx[ex][c[ok]]
    return src

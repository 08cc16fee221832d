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


def rsd_band(window, rel_err, abs_err=None, tiny=0.0):
    """Bound on |RSD(w') - RSD(w)| when each w_j moves by at most
    max(rel_err_j |w_j|, abs_err_j): first-order sensitivity
    sum_j |dRSD/dw_j| err_j. tiny is the subnormal spacing of the statistic's
    precision: squared deviations below the normal range are rounded to
    multiples of it, an absolute error of up to h tiny in the variance sum,
    which moves RSD by about h tiny / (2 sd |mu|) (large for windows of tiny
    values). The caller adds the rounding of the statistic itself."""
    w = np.asarray(window, dtype=np.float64)
    h = w.size
    mu = w.mean()
    sd = w.std()
    if mu == 0 or sd == 0:
        return np.inf if sd > 0 else 0.0
    err = np.abs(w) * rel_err
    if abs_err is not None:
        err = np.maximum(err, abs_err)
    grad = np.abs((w - mu) / (h * sd * abs(mu)) - sd * np.sign(mu) / (h * mu * mu))
    return float(np.sum(grad * err) + 2 * h * tiny / (sd * abs(mu)))


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


def taf_replay_check(n, T, B, level, out_g, mask_g, stat_g, out_r, stat_r, dis, counts, hsize, thr,
                     tol, rel_err, eps, sample=2000, seed=0):
    """GPU TAF trace against the oracle replayed along the GPU's mask.

    The replay follows the GPU's decisions, so every invocation is compared:
    outputs within tol (per invocation: the bound of the exact output it
    carries). At each decision point where the oracle's own decision differs
    from the GPU's (dis[i] = 1), some lane of the deciding group (the thread,
    its warp or its block) must hold an oracle statistic within the rounding
    band of the threshold. Statistics of both sides agree within that band at
    the disagreements and at a sample of accurate invocations. The mask must
    be a valid TAF trace (no structural error). Returns the disagreement count.
    """
    T = T if T > 0 else n
    tiny = 2.0 ** -149 if eps > 1e-10 else 2.0 ** -1074  # subnormal spacing of the statistic
    assert counts[2] == 0, ("structural errors in the GPU mask", int(counts[2]))
    err = np.abs(out_g.astype(np.float64) - out_r.astype(np.float64))
    bad = np.nonzero(~(err <= tol))[0]
    assert bad.size == 0, ("output mismatch", bad[:5], err[bad[:5]], tol[bad[:5]])

    def band_at(j):
        t = j % T
        hist = np.arange(t, j + 1, T)
        ex = hist[mask_g[hist] == 0][-hsize:]
        if ex.size < hsize:
            return None
        return (rsd_band(out_r[ex], rel_err[ex], tol[ex], tiny)
                + 8 * eps * abs(float(stat_r[j])))

    G = 1 if level == 0 else 32 if level == 1 else B
    for i in np.nonzero(dis)[0]:
        t, k = i % T, i // T
        g0 = (t // G) * G
        near = False
        for l in range(g0, min(g0 + G, T)):
            j = l + k * T
            if j >= n or mask_g[j] != 0 or np.isnan(stat_r[j]):
                continue
            b = band_at(j)
            if b is not None and abs(float(stat_r[j]) - thr) <= b:
                near = True
                assert abs(float(stat_g[j]) - float(stat_r[j])) <= 2 * b + 1e-300, ("stats apart", j)
        assert near, ("non-borderline disagreement", int(i))
    acc = np.nonzero((mask_g == 0) & ~np.isnan(stat_r))[0]
    rng = np.random.default_rng(seed)
    for j in rng.choice(acc, size=min(sample, acc.size), replace=False) if acc.size else []:
        b = band_at(j)
        # first order holds where the band is small against the statistic
        # (not for windows whose mean nearly cancels)
        if b is not None and np.isfinite(b) and b <= 1e-3 * abs(float(stat_r[j])):
            assert abs(float(stat_g[j]) - float(stat_r[j])) <= 2 * b + 1e-300, \
                ("stats apart", int(j), float(stat_g[j]), float(stat_r[j]), b)
    return int(counts[1])


def literal_beyond(n, T, B, level, mask_g, stat_r, dis, thr, rel=1e-6):
    """Disagreements (dis[i] = 1 at a decision point) at which no deciding lane
    (the thread, its warp or its block) holds an oracle statistic within
    rel * thr of the threshold: the decisions that the literal borderline rule
    (|s - thr| <= 1e-6 thr) would not excuse. The parity tests excuse instead
    the rounding band of each statistic (rsd_band); this count shows how many
    disagreements need that wider reading."""
    T = T if T > 0 else n
    G = 1 if level == 0 else 32 if level == 1 else B
    beyond = 0
    for i in np.nonzero(dis)[0]:
        t, k = i % T, i // T
        g0 = (t // G) * G
        j = np.arange(g0, min(g0 + G, T)) + k * T
        j = j[j < n]
        j = j[mask_g[j] == 0]
        s = stat_r[j].astype(np.float64)
        s = s[~np.isnan(s)]
        if not np.any(np.abs(s - thr) <= rel * thr):
            beyond += 1
    return beyond


def relative_beyond(g, ref, rel):
    """Outputs farther than rel from the reference relative to
    max(|ref|, 1e-6 max |ref|) (the denominator that keeps near-zero prices
    from dividing by almost nothing), and the largest such relative error."""
    g = np.asarray(g, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    if ref.size == 0:
        return 0, 0.0
    den = np.maximum(np.abs(ref), 1e-6 * np.abs(ref).max())
    den = np.where(den > 0, den, 1.0)
    r = np.abs(g - ref) / den
    return int(np.sum(r > rel)), float(r.max())

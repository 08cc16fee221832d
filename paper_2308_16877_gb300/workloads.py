"""Seeded synthetic inputs shaped like the paper's workloads.

This module only draws random numbers and lays them out; it holds none of the
method's arithmetic (no region formula, no statistic, no decision rule). Both
the CUDA path and the CPU oracle consume the arrays it returns, so it is the
one piece of code they share.

Layouts follow the region-descriptor convention of the paper's programming
model (Section 3.2, the ``in(input[i*5:5:N])`` array section): a region with D
inputs is a column-major (structure-of-arrays) matrix, element ``d`` of
invocation ``i`` at ``d * stride + i``.
"""
from __future__ import annotations

import numpy as np

DEFAULT_SEED = 2308

# Black-Scholes option distributions (spot, strike, expiry in years, volatility).
BS_SPOT = (5.0, 30.0)
BS_STRIKE = (1.0, 100.0)
BS_EXPIRY = (0.25, 10.0)
BS_VOL = (0.05, 0.65)
BS_RATE = 0.02


def _rng(seed: int, stream: int = 0) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64([int(seed), int(stream)]))


def blackscholes_inputs(n: int, seed: int = DEFAULT_SEED, run: int = 32,
                        stride: int | None = None) -> np.ndarray:
    """Options for the Black-Scholes region, float32, shape (4, stride).

    Rows are spot S, strike K, expiry T, volatility sigma, each uniform on the
    ranges above. Options are sorted by strike in consecutive runs of ``run``
    indices (the whole option tuple moves with its strike), so the ``run``
    lanes of an aligned warp step see ascending strikes. ``run <= 1`` leaves the
    draw unsorted. Columns past ``n`` (when ``stride > n``) are zero.
    """
    stride = n if stride is None else stride
    if stride < n:
        raise ValueError("stride must be >= n")
    g = _rng(seed, 1)
    x = np.zeros((4, stride), dtype=np.float32)
    if n == 0:
        return x
    cols = [BS_SPOT, BS_STRIKE, BS_EXPIRY, BS_VOL]
    for d, (lo, hi) in enumerate(cols):
        x[d, :n] = g.uniform(lo, hi, size=n).astype(np.float32)
    if run > 1:
        full = (n // run) * run
        if full:
            blk = x[:, :full].reshape(4, full // run, run)
            order = np.argsort(blk[1], axis=1, kind="stable")
            x[:, :full] = np.take_along_axis(blk, order[None, :, :], axis=2).reshape(4, full)
        if full < n:
            tail = x[:, full:n]
            order = np.argsort(tail[1], kind="stable")
            x[:, full:n] = tail[:, order]
    return x


def eos_inputs(n: int, seed: int = DEFAULT_SEED, stride: int | None = None,
               smooth: int = 0) -> np.ndarray:
    """Inputs of the equation-of-state region, float64, shape (4, stride).

    Rows: specific energy e_n >= 0, new relative volume v_{n+1} in [0.6, 1.4],
    volume change dv (|dv| <= 0.02), viscosity q_{n+1} >= 0 (zero where the
    element expands, as artificial viscosity only acts in compression).
    ``smooth > 1`` makes every ``smooth`` consecutive invocations share one
    draw plus a 0.1% perturbation, mimicking the slowly varying fields of a
    hydro mesh.
    """
    stride = n if stride is None else stride
    if stride < n:
        raise ValueError("stride must be >= n")
    g = _rng(seed, 2)
    x = np.zeros((4, stride), dtype=np.float64)
    if n == 0:
        return x
    m = n if smooth <= 1 else (n + smooth - 1) // smooth
    e = g.uniform(0.0, 2.0e5, size=m)
    v = g.uniform(0.6, 1.4, size=m)
    dv = g.uniform(-0.02, 0.02, size=m)
    q = np.where(dv < 0.0, g.uniform(0.0, 5.0e3, size=m), 0.0)
    cols = [e, v, dv, q]
    for d, c in enumerate(cols):
        if smooth > 1:
            c = np.repeat(c, smooth)[:n]
            c = c * (1.0 + 1.0e-3 * g.uniform(-1.0, 1.0, size=n))
        x[d, :n] = c
    return x


def identity_inputs(n: int, d: int = 1, seed: int = DEFAULT_SEED, dtype=np.float32,
                    kind: str = "uniform", stride: int | None = None) -> np.ndarray:
    """Inputs for the identity region (output = first input), shape (d, stride).

    kind: "uniform" on [1, 2); "levels" draws each value from 4 discrete levels
    (exact repeats, so memoization hits are frequent); "walk" is a slow random
    walk around 1.5 per column, giving temporal locality along the invocation
    index.
    """
    stride = n if stride is None else stride
    g = _rng(seed, 3)
    x = np.zeros((d, stride), dtype=dtype)
    if n == 0:
        return x
    if kind == "uniform":
        v = g.uniform(1.0, 2.0, size=(d, n))
    elif kind == "levels":
        v = 1.0 + 0.25 * g.integers(0, 4, size=(d, n))
    elif kind == "walk":
        v = 1.5 + np.cumsum(g.normal(0.0, 1e-3, size=(d, n)), axis=1)
    else:
        raise ValueError(kind)
    x[:, :n] = v.astype(dtype)
    return x


def identity_near_threshold(n: int, T: int, rsd: float, seed: int = DEFAULT_SEED) -> np.ndarray:
    """Double-precision identity inputs, shape (1, n), whose TAF windows sit
    next to a relative standard deviation of `rsd`. Logical thread t (of T)
    draws a magnitude 10^U(-12, 14) and a sign; at its step k it reads
    magnitude * (1 + (-1)^k rsd (1 + e)) for 10 of 16 threads (every window of
    even size over values of alternating parity has relative standard
    deviation rsd (1 + e); e is within 1e-2 .. 1e-9 of zero, either sign),
    magnitude * (1 + rsd z) with z standard normal for 4 of 16, and special
    values (signed zeros, subnormals, values beyond the single-precision
    range, infinities, NaN, repeats) for the rest."""
    g = _rng(seed, 11)
    x = np.zeros((1, n), dtype=np.float64)
    if n == 0:
        return x
    T = max(1, T)
    i = np.arange(n)
    t, k = i % T, i // T
    mag = 10.0 ** g.uniform(-12, 14, T) * g.choice([-1.0, 1.0], T)
    e = 10.0 ** g.uniform(-9, -2, T) * g.choice([-1.0, 1.0], T)
    alt = np.where(k % 2 == 0, 1.0, -1.0)
    v = mag[t] * (1.0 + alt * rsd * (1.0 + e[t]))
    cls = t % 16
    rnd = (cls >= 10) & (cls < 14)
    v[rnd] = mag[t[rnd]] * (1.0 + rsd * g.normal(size=int(rnd.sum())))
    special = np.array([0.0, -0.0, 1e-310, 5e-324, 1e-45, 1e-39, 1e-12, 1.0, 4e38, 1e300, np.inf,
                        -np.inf, np.nan, 1.5])
    odd = cls >= 14
    v[odd] = g.choice(special, size=int(odd.sum()))
    x[0] = v
    return x


def iact_scale(x: np.ndarray, n: int) -> np.ndarray:
    """Per-dimension input scale 1/max|x_d| (1 where the column is all zero).

    This is the knob value a caller passes as ``in_scale``; it is computed here,
    outside both implementations, and handed to each unchanged.
    """
    m = np.abs(x[:, :n].astype(np.float64)).max(axis=1) if n else np.zeros(x.shape[0])
    return np.where(m > 0, 1.0 / np.where(m > 0, m, 1.0), 1.0)


# ----------------------------------------------------------------------------
# Hexahedral hydro mesh (structured n^3 elements on [0,1]^3)
# ----------------------------------------------------------------------------

HYDRO_E0 = 3.9e6       # initial energy in the corner element
HYDRO_JITTER = 0.05    # node jitter, fraction of the mesh spacing


def hydro_initial(n: int, seed: int = DEFAULT_SEED, jitter: float = HYDRO_JITTER):
    """Initial node coordinates and element energies of the hex mesh.

    Returns (x, y, z, e) with x, y, z float64 of shape ((n+1)^3,) indexed
    node = (k*(n+1) + j)*(n+1) + i, and e float64 of shape (n^3,) indexed
    elem = (k*n + j)*n + i. Interior nodes are displaced uniformly by up to
    ``jitter`` * h per axis; nodes on a boundary plane keep their coordinate
    normal to that plane. All energy starts in element (0, 0, 0).
    """
    g = _rng(seed, 4)
    h = 1.0 / n
    ax = np.arange(n + 1, dtype=np.float64) * h
    zz, yy, xx = np.meshgrid(ax, ax, ax, indexing="ij")
    idx = np.arange(n + 1)
    kk, jj, ii = np.meshgrid(idx, idx, idx, indexing="ij")
    out = []
    for c, ci in ((xx, ii), (yy, jj), (zz, kk)):
        d = g.uniform(-jitter * h, jitter * h, size=c.shape)
        d = np.where((ci == 0) | (ci == n), 0.0, d)
        out.append((c + d).reshape(-1).copy())
    e = np.zeros(n * n * n, dtype=np.float64)
    e[0] = HYDRO_E0
    return out[0], out[1], out[2], e


# ----------------------------------------------------------------------------
# Knob-sweep configuration list (Table 2 style ranges)
# ----------------------------------------------------------------------------

def sweep_region_sizes(count: int = 32, lo: int = 12, hi: int = 22) -> list[int]:
    """Uneven region sizes 2^(lo + round((hi-lo)*j/(count-1))), j = 0..count-1."""
    if count == 1:
        return [1 << lo]
    return [1 << (lo + int(np.floor((hi - lo) * j / (count - 1) + 0.5))) for j in range(count)]


def sweep_configs() -> list[dict]:
    """256 approximation configurations: 128 TAF and 128 perforation.

    TAF: 8 thresholds log-spaced on [1e-4, 1] x history {2,4,8,16} x
    prediction {1,4,16,64} (thread level). Perforation: 64 settings across the
    small / large / ini / fini / random patterns (rates 10..50%), each herded
    and per-iteration.
    """
    cfgs: list[dict] = []
    for thr in np.logspace(-4, 0, 8):
        for h in (2, 4, 8, 16):
            for p in (1, 4, 16, 64):
                cfgs.append(dict(tech="taf", hsize=h, psize=p, thresh=float(thr), level=0))
    perf: list[dict] = []
    for m in (2, 3, 4, 5, 6, 7, 8, 9, 10):
        perf.append(dict(tech="perfo", kind=0, m=m, rate=0.0))          # small:M
    perf.append(dict(tech="perfo", kind=1, m=2, rate=0.0))              # large:2
    for pct in (10, 15, 20, 25, 30, 35, 40, 45, 50):
        perf.append(dict(tech="perfo", kind=2, m=pct, rate=0.0))        # ini
        perf.append(dict(tech="perfo", kind=3, m=pct, rate=0.0))        # fini
    for j in range(36):
        rate = 0.1 + 0.4 * j / 35.0
        perf.append(dict(tech="perfo", kind=4, m=0, rate=float(rate), seed=1000 + j))
    assert len(perf) == 64, len(perf)
    for herded in (1, 0):
        for c in perf:
            d = dict(c)
            d["herded"] = herded
            d.setdefault("seed", 0)
            cfgs.append(d)
    assert len(cfgs) == 256
    return cfgs


BINOMIAL_STEPS = 512


def binomial_portfolio(members: int, time_points: int, seed: int = DEFAULT_SEED) -> np.ndarray:
    """A portfolio of American call options priced at successive time points
    before expiry (Table 1, Binomial Options), float32, shape (4, members *
    time_points): rows spot S, strike X, time to expiry T, volatility sigma.

    Member m has S0 ~ U[5, 30], X = S0 * U[0.8, 1.2] (near the money), T0 ~
    U[0.5, 2] years and sigma ~ U[0.1, 0.5]; at time point k its spot follows
    a seeded geometric Brownian path with drift r - sigma^2/2 sampled every
    dt_m = T0 / (2 time_points), and its time to expiry is T0 - k dt_m. Column
    i = m + k * members, so with one logical team per member (T = members) a
    team prices its own option at successive time points.
    """
    g = _rng(seed, 7)
    M, K = members, time_points
    S0 = g.uniform(BS_SPOT[0], BS_SPOT[1], size=M)
    X = S0 * g.uniform(0.8, 1.2, size=M)
    T0 = g.uniform(0.5, 2.0, size=M)
    sig = g.uniform(0.1, 0.5, size=M)
    dt = T0 / (2 * K)
    z = g.standard_normal((K, M))
    z[0] = 0.0
    logS = np.log(S0)[None, :] + np.cumsum((BS_RATE - 0.5 * sig ** 2) * dt + sig * np.sqrt(dt) * z, axis=0)
    x = np.empty((4, K * M), dtype=np.float32)
    k = np.arange(K)[:, None]
    x[0] = np.exp(logS).reshape(-1).astype(np.float32)
    x[1] = np.broadcast_to(X, (K, M)).reshape(-1).astype(np.float32)
    x[2] = (T0[None, :] - k * dt[None, :]).reshape(-1).astype(np.float32)
    x[3] = np.broadcast_to(sig, (K, M)).reshape(-1).astype(np.float32)
    return x


def kmeans_blobs(n: int, clusters: int, seed: int = DEFAULT_SEED, spread: float = 1.0):
    """Observations for the K-Means region: float32 (8, n), drawn from
    `clusters` isotropic Gaussian blobs (standard deviation `spread`) whose
    centres are uniform on [-10, 10]^8, in random order. Returns (x, labels,
    init): the generating blob of each observation and the initial centroids
    (the first observation of each blob, so a run starts with one seed per blob)."""
    g = _rng(seed, 11)
    centres = g.uniform(-10.0, 10.0, size=(clusters, 8))
    labels = g.integers(0, clusters, size=n)
    labels[:clusters] = np.arange(clusters)          # every blob is present
    g.shuffle(labels)
    x = (centres[labels] + spread * g.standard_normal((n, 8))).T.astype(np.float32)
    first = np.array([np.flatnonzero(labels == k)[0] for k in range(clusters)])
    return np.ascontiguousarray(x), labels, np.ascontiguousarray(x[:, first].T)


def kmeans_coherent(n: int, clusters: int, threads: int, outliers: float = 0.05,
                    seed: int = DEFAULT_SEED, spread: float = 1.0):
    """K-Means observations laid out for the logical schedule: observation
    i = t + k * threads belongs to blob (t mod clusters) except for a share
    `outliers` drawn from a random blob, so a logical thread's successive
    invocations mostly come from one cluster (the temporal locality TAF and
    iACT exploit) while neighbouring lanes see different clusters. Returns
    (x (8, n) float32, labels, centres (clusters, 8) float32)."""
    g = _rng(seed, 13)
    centres = g.uniform(-10.0, 10.0, size=(clusters, 8))
    t = np.arange(n) % threads
    labels = t % clusters
    out = g.random(n) < outliers
    labels[out] = g.integers(0, clusters, size=int(out.sum()))
    x = (centres[labels] + spread * g.standard_normal((n, 8))).T.astype(np.float32)
    return np.ascontiguousarray(x), labels, centres.astype(np.float32)


def hydro_dt(n: int, gamma: float = 5.0 / 3.0, e0: float = HYDRO_E0, cfl: float = 0.1) -> float:
    """Fixed time step of the hydro run: cfl * h / c0 with h = 1/n and c0 the
    ideal-gas sound speed of the initial corner element at unit density."""
    return cfl * (1.0 / n) / float(np.sqrt(gamma * (gamma - 1.0) * e0))


def sweep_inputs(sizes, seed: int = DEFAULT_SEED, ipt: int = 8):
    """Black-Scholes inputs of the sweep's regions laid end to end.

    Returns (x, regions): x float32 (4, total) with region r's options (drawn
    with seed + 100 + r, strike-sorted runs of 32) at its offset, and regions
    the list of (n, offset, logical_threads = n / ipt).
    """
    total = int(sum(sizes))
    x = np.zeros((4, total), dtype=np.float32)
    regions = []
    off = 0
    for r, n in enumerate(sizes):
        x[:, off:off + n] = blackscholes_inputs(n, seed=seed + 100 + r)
        regions.append((int(n), off, max(1, int(n) // ipt)))
        off += n
    return x, regions


# LavaMD-style particles: coordinates and charges uniform in [0.1, 1.0), drawn
# independently of the particle's box (the boxes only decide which particles
# interact), so every box is a statistically alike sample of the same cloud.
LAVAMD_A2 = 0.5          # exp(-a2 r^2) with a2 = 2 alpha^2, alpha = 0.5
LAVAMD_PAR_PER_BOX = 100


def lavamd_inputs(boxes1d: int, par_per_box: int = LAVAMD_PAR_PER_BOX,
                  seed: int = DEFAULT_SEED) -> np.ndarray:
    """(4, boxes1d^3 par_per_box) float64: x, y, z, charge of particle
    b * par_per_box + m (box b = (bz B + by) B + bx)."""
    P = int(boxes1d) ** 3 * int(par_per_box)
    return _rng(seed, 9).uniform(0.1, 1.0, (4, P))

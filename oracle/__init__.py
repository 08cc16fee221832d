"""CPU oracle of the approximate-region hot path (TEST INFRASTRUCTURE ONLY).

Only the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline leg
import this package. The product path (the CUDA library and its binding) never
does, and the two share no code: the oracle is plain C in this directory,
loaded through ctypes, restating each technique of HPAC-Offload (arXiv
2308.16877) step by step on the logical grid-stride schedule of Section 3.1.3.

Constants mirror the C enums in ``hpac_oracle.c`` (written independently of the
library's header).
"""
from __future__ import annotations

import ctypes as C
import math

import numpy as np

from . import build as _build

BLACKSCHOLES, EOS, IDENTITY, BINOMIAL, KMEANS = 0, 1, 3, 4, 5
BINOMIAL_STEPS = 512         # default tree depth of the Binomial region
F32, F64 = 0, 1
THREAD, WARP, BLOCK = 0, 1, 2
SMALL, LARGE, INI, FINI, RANDOM = 0, 1, 2, 3, 4
EXACT, APPROX, SKIPPED = 0, 1, 2
MAPE, RMSE, MCR = 0, 1, 2


class Region(C.Structure):
    _fields_ = [("kind", C.c_int32), ("dtype", C.c_int32), ("n", C.c_int64),
                ("n_in", C.c_int32), ("n_out", C.c_int32), ("in_stride", C.c_int64),
                ("out_stride", C.c_int64), ("threads", C.c_int64), ("block", C.c_int32),
                ("param", C.c_double), ("arg", C.c_int32), ("pad", C.c_int32),
                ("aux", C.c_void_p)]


_lib = None


def lib() -> C.CDLL:
    global _lib
    if _lib is None:
        path = _build.build()
        L = C.CDLL(path)
        P, I64, I32, D = C.c_void_p, C.c_int64, C.c_int32, C.c_double
        RP = C.POINTER(Region)
        L.orc_run_exact.argtypes = [RP, P, P]
        L.orc_run_perfo.argtypes = [RP, P, I32, I32, D, C.c_uint64, I32, P, P, P]
        L.orc_run_taf.argtypes = [RP, P, I32, I32, D, I32, I32, P, P, P, P]
        L.orc_run_iact.argtypes = [RP, P, I32, I32, D, I32, P, P, P, P, P]
        L.orc_replay_taf.argtypes = [RP, P, I32, I32, D, I32, I32, P, P, P, P, P]
        L.orc_run_taf_persist.argtypes = [RP, P, I32, I32, D, I32, I32, P, P, P, P, P, P, P]
        L.orc_run_iact_persist.argtypes = [RP, P, I32, I32, D, I32, P, P, P, P, P, P, P, P, P]
        L.orc_quality.argtypes = [I64, P, P, I32, P, P]
        L.orc_kmeans_update.argtypes = [I64, I32, P, I64, P, P, P, P]
        L.orc_kmeans_update.restype = C.c_int
        L.orc_num_threads.restype = C.c_int
        L.orc_set_threads.argtypes = [I32]
        L.orc_set_threads.restype = None
        for f in ("orc_run_exact", "orc_run_perfo", "orc_run_taf", "orc_replay_taf", "orc_run_iact",
                  "orc_quality", "orc_run_taf_persist", "orc_run_iact_persist"):
            getattr(L, f).restype = C.c_int
        _hydro_bind(L)
        L.orc_lavamd.argtypes = [I32, I32, D, P, P, I32, I32, I32, I32, D, I32, I32, I32, P, P, P]
        L.orc_lavamd.restype = C.c_int
        _lib = L
    return _lib


class EosKnobs(C.Structure):
    _fields_ = [("mode", C.c_int32), ("hsize", C.c_int32), ("psize", C.c_int32),
                ("tsize", C.c_int32), ("tperwarp", C.c_int32), ("level", C.c_int32),
                ("thresh", C.c_double), ("threads", C.c_int64), ("block", C.c_int32),
                ("reserved", C.c_int32), ("in_scale", C.c_double * 4), ("st", C.c_void_p * 4)]


def _hydro_bind(L):
    P, I32, D = C.c_void_p, C.c_int32, C.c_double
    L.orc_hydro_init.argtypes = [I32, P, P, P, P, P, P]
    L.orc_hydro_step.argtypes = [I32, D, D] + [P] * 12 + [I32, P, P, P, P]
    L.orc_hex_volume.argtypes = [P, P, P]
    L.orc_hex_volume.restype = D
    L.orc_hex_volume_grad.argtypes = [P, P, P, P, P, P]
    L.orc_hex_volume_grad.restype = None
    for f in ("orc_hydro_init", "orc_hydro_step"):
        getattr(L, f).restype = C.c_int


def _ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def num_threads() -> int:
    return int(lib().orc_num_threads())


def set_threads(n: int) -> None:
    """OpenMP threads of the oracle's parallel loops (n < 1: one per processor)."""
    lib().orc_set_threads(int(n))


def _region(kind, x, n, param, threads, block, arg=0):
    x = np.ascontiguousarray(x)
    dtype = F32 if x.dtype == np.float32 else F64
    if x.dtype not in (np.float32, np.float64):
        raise TypeError(x.dtype)
    d, stride = x.shape
    n = stride if n is None else n
    aux = None
    if kind == BINOMIAL and not arg:
        arg = BINOMIAL_STEPS
    if kind == KMEANS:
        # param carries the centroids for this region: a (K, 8) float32 array
        cent = np.ascontiguousarray(param, dtype=np.float32)
        arg, aux = cent.shape[0], cent
        param = 0.0
    r = Region(kind, dtype, n, d, 1, stride, n, threads, block, float(param), int(arg), 0,
               aux.ctypes.data if aux is not None else None)
    r._keep = aux
    return r, x, n


def _out(x, n, out):
    if out is None:
        return np.zeros(n, dtype=x.dtype)
    return out


def run_exact(kind, x, param=0.0, n=None, steps=0):
    r, x, n = _region(kind, x, n, param, 0, 32, steps)
    out = np.zeros(n, dtype=x.dtype)
    if lib().orc_run_exact(C.byref(r), _ptr(x), _ptr(out)):
        raise ValueError("oracle rejected the region")
    return out


def run_perfo(kind, x, param, pkind, m=0, rate=0.0, seed=0, herded=1, threads=0, block=256,
              n=None, out=None, steps=0):
    r, x, n = _region(kind, x, n, param, threads, block, steps)
    out = _out(x, n, out)
    mask = np.full(n, 255, dtype=np.uint8)
    cnt = np.zeros(4, dtype=np.int64)
    if lib().orc_run_perfo(C.byref(r), _ptr(x), pkind, m, rate, seed, herded, _ptr(out),
                           _ptr(mask), _ptr(cnt)):
        raise ValueError("oracle rejected perforation arguments")
    return out, mask, cnt


def taf_state(T, hsize):
    """Empty persistent TAF state of T logical threads (see run_taf)."""
    return {"vals": np.zeros((hsize, T), dtype=np.float64), "cnt": np.zeros(T, dtype=np.int32),
            "pred": np.zeros(T, dtype=np.int32)}


def iact_state(T, tsize, tperwarp, D):
    """Empty persistent iACT state: the tables of ceil(T/32) logical warps."""
    g = ((T + 31) // 32) * tperwarp
    return {"z": np.zeros((g, tsize, D), dtype=np.float32), "y": np.zeros((g, tsize), dtype=np.float64),
            "valid": np.zeros((g, tsize), dtype=np.int32), "rr": np.zeros(g, dtype=np.int32)}


def run_taf(kind, x, param, hsize, psize, thresh, level=THREAD, threads=0, block=256, n=None,
            reset=False, state=None, steps=0):
    """TAF over the logical schedule; with state (taf_state), the windows and
    owed predictions continue from the previous call and are updated in place."""
    r, x, n = _region(kind, x, n, param, threads, block, steps)
    out = np.zeros(n, dtype=x.dtype)
    stat = np.zeros(n, dtype=x.dtype)
    mask = np.full(n, 255, dtype=np.uint8)
    cnt = np.zeros(4, dtype=np.int64)
    if state is not None:
        if lib().orc_run_taf_persist(C.byref(r), _ptr(x), hsize, psize, thresh, level, int(bool(reset)),
                                     _ptr(state["vals"]), _ptr(state["cnt"]), _ptr(state["pred"]),
                                     _ptr(out), _ptr(mask), _ptr(stat), _ptr(cnt)):
            raise ValueError("oracle rejected TAF arguments")
        return out, mask, stat, cnt
    if lib().orc_run_taf(C.byref(r), _ptr(x), hsize, psize, thresh, level, int(bool(reset)),
                         _ptr(out), _ptr(mask),
                         _ptr(stat), _ptr(cnt)):
        raise ValueError("oracle rejected TAF arguments")
    return out, mask, stat, cnt


def replay_taf(kind, x, param, hsize, psize, thresh, force, level=THREAD, threads=0, block=256, n=None,
               reset=False, steps=0):
    """TAF along a given mask: outputs and statistics of the oracle's own
    arithmetic on the mask's path, the decision points where the oracle's own
    decision differs from the mask's (disagree[i] = 1 at the deciding
    invocation), and counts (compared, disagreements, structural errors)."""
    r, x, n = _region(kind, x, n, param, threads, block, steps)
    force = np.ascontiguousarray(force, dtype=np.uint8)
    if force.shape != (n,):
        raise ValueError("mask length differs from n")
    out = np.zeros(n, dtype=x.dtype)
    stat = np.zeros(n, dtype=x.dtype)
    dis = np.zeros(n, dtype=np.uint8)
    counts = np.zeros(3, dtype=np.int64)
    if lib().orc_replay_taf(C.byref(r), _ptr(x), hsize, psize, thresh, level, int(bool(reset)),
                            _ptr(force), _ptr(out),
                            _ptr(stat), _ptr(dis), _ptr(counts)):
        raise ValueError("oracle rejected TAF arguments")
    return out, stat, dis, counts


def run_iact(kind, x, param, tsize, tperwarp, thresh, level=THREAD, in_scale=None, threads=0,
             block=256, n=None, state=None, steps=0):
    """iACT over the logical schedule; with state (iact_state), the tables
    continue from the previous call and are updated in place."""
    r, x, n = _region(kind, x, n, param, threads, block, steps)
    out = np.zeros(n, dtype=x.dtype)
    stat = np.zeros(n, dtype=x.dtype)
    mask = np.full(n, 255, dtype=np.uint8)
    cnt = np.zeros(4, dtype=np.int64)
    sc = None if in_scale is None else np.ascontiguousarray(in_scale, dtype=np.float64)
    if state is not None:
        if lib().orc_run_iact_persist(C.byref(r), _ptr(x), tsize, tperwarp, thresh, level, _ptr(sc),
                                      _ptr(state["z"]), _ptr(state["y"]), _ptr(state["valid"]),
                                      _ptr(state["rr"]), _ptr(out), _ptr(mask), _ptr(stat), _ptr(cnt)):
            raise ValueError("oracle rejected iACT arguments")
        return out, mask, stat, cnt
    if lib().orc_run_iact(C.byref(r), _ptr(x), tsize, tperwarp, thresh, level, _ptr(sc),
                          _ptr(out), _ptr(mask), _ptr(stat), _ptr(cnt)):
        raise ValueError("oracle rejected iACT arguments")
    return out, mask, stat, cnt


def kmeans_update(x, assign, cent, prev=None):
    """One exact centroid update (see orc_kmeans_update): returns (new
    centroids, changed count); x (8, n) float32, assign / prev float32 ids."""
    x = np.ascontiguousarray(x, dtype=np.float32)
    a = np.ascontiguousarray(assign, dtype=np.float32)
    c = np.array(cent, dtype=np.float32, copy=True)
    p = None if prev is None else np.ascontiguousarray(prev, dtype=np.float32)
    ch = np.zeros(1, dtype=np.int64)
    if lib().orc_kmeans_update(a.size, c.shape[0], _ptr(x), x.shape[1], _ptr(a), _ptr(p), _ptr(c), _ptr(ch)):
        raise ValueError("oracle rejected K-Means update arguments")
    return c, int(ch[0])


def kmeans(x, cent0, max_iter=100, run=None):
    """K-Means to convergence (no observation changes cluster) or max_iter:
    run(cent) -> assignment ids (default: the oracle's exact region). Returns
    (assignment, centroids, iterations)."""
    cent = np.array(cent0, dtype=np.float32, copy=True)
    run = run or (lambda c: run_exact(KMEANS, x, c))
    prev = None
    for it in range(1, max_iter + 1):
        a = run(cent)
        cent, ch = kmeans_update(x, a, cent, prev)
        if prev is not None and ch == 0:
            return a, cent, it
        prev = a
    return prev, cent, max_iter


def quality(a, b, metric):
    a = np.ascontiguousarray(a, dtype=np.float64)
    b = np.ascontiguousarray(b, dtype=np.float64)
    if a.shape != b.shape:
        raise ValueError("shape mismatch")
    res = np.zeros(2, dtype=np.float64)
    aux = np.zeros(2, dtype=np.int64)
    if lib().orc_quality(a.size, _ptr(a), _ptr(b), metric, _ptr(res), _ptr(aux)):
        raise ValueError("bad metric")
    return float(res[0]), dict(zero_max_abs=float(res[1]), zeros=int(aux[0]),
                               zeros_mismatch=int(aux[1]))


def calibrate_floor(pred, exact, target=0.01, quantile=0.99):
    """The surrogate's calibrated fallback bound, by its definition: bad_i is
    |pred_i - exact_i| > target |exact_i| (in double precision); over the
    distinct prediction values v, taken from the largest down, k(v) is the
    number of predictions >= v and b(v) the bad ones among them; the floor is
    the smallest v with b(v) <= k(v) - ceil(quantile k(v)) (at least
    ceil(quantile k) of the k served invocations within the target: the
    nearest-rank quantile). NaN predictions take no part; -0 equals +0.
    Returns (floor, k at the floor), (inf, 0) when no value qualifies."""
    y = np.asarray(pred, dtype=np.float32).ravel()
    a = np.asarray(exact, dtype=np.float64).ravel()
    keep = ~np.isnan(y)
    y, a = y[keep], a[keep]
    if y.size == 0:
        return math.inf, 0
    bad = np.abs(y.astype(np.float64) - a) > target * np.abs(a)
    order = np.argsort(-y.astype(np.float64), kind="stable")   # largest prediction first
    ys, bs = y[order], bad[order]
    k = np.arange(1, ys.size + 1)
    b = np.cumsum(bs)
    last_of_value = np.r_[ys[1:] != ys[:-1], True]             # k(v) at each distinct value
    allowed = k - np.ceil(quantile * k.astype(np.float64)).astype(np.int64)
    ok = np.nonzero(last_of_value & (b <= allowed))[0]
    if ok.size == 0:
        return math.inf, 0
    j = ok[-1]
    return float(ys[j]), int(j + 1)


# ---------------------------------------------------------------- hydro

GAMMA = 5.0 / 3.0
EOS_EXACT, EOS_TAF, EOS_IACT = 0, 1, 2


def hex_volume(X, Y, Z):
    X, Y, Z = (np.ascontiguousarray(a, dtype=np.float64) for a in (X, Y, Z))
    return float(lib().orc_hex_volume(_ptr(X), _ptr(Y), _ptr(Z)))


def hex_volume_grad(X, Y, Z):
    X, Y, Z = (np.ascontiguousarray(a, dtype=np.float64) for a in (X, Y, Z))
    g = np.zeros((3, 8))
    lib().orc_hex_volume_grad(_ptr(X), _ptr(Y), _ptr(Z), _ptr(g[0]), _ptr(g[1]), _ptr(g[2]))
    return g


class HydroState:
    """Node (x, y, z, u, v, w) and element (e, p, q, vrel, V0) arrays, float64."""

    FIELDS = ("x", "y", "z", "u", "v", "w", "e", "p", "q", "vrel", "V0", "mnode")

    def __init__(self, n, x, y, z, e, gamma=GAMMA):
        self.n, self.gamma = n, gamma
        E, Nn = n ** 3, (n + 1) ** 3
        self.x, self.y, self.z = (np.array(a, dtype=np.float64) for a in (x, y, z))
        self.u, self.v, self.w = (np.zeros(Nn) for _ in range(3))
        self.e = np.array(e, dtype=np.float64)
        self.p = (gamma - 1.0) * self.e
        self.q = np.zeros(E)
        self.vrel = np.ones(E)
        self.V0 = np.zeros(E)
        self.mnode = np.zeros(Nn)
        if lib().orc_hydro_init(n, _ptr(self.x), _ptr(self.y), _ptr(self.z), _ptr(self.V0),
                                _ptr(self.mnode), None):
            raise ValueError("hydro init failed")

    def copy(self):
        c = object.__new__(HydroState)
        c.n, c.gamma = self.n, self.gamma
        for f in self.FIELDS:
            setattr(c, f, getattr(self, f).copy())
        return c

    def step(self, dt, knobs=None):
        """One time step; knobs an EosKnobs (None: exact EOS). Returns
        (eos_inputs (4, E), mask (E,), counters (4,))."""
        E = self.n ** 3
        eos_in = np.zeros((4, E))
        mask = np.zeros(E, dtype=np.uint8)
        cnt = np.zeros(4, dtype=np.int64)
        kp = C.byref(knobs) if knobs is not None else None
        rc = lib().orc_hydro_step(self.n, dt, self.gamma, _ptr(self.x), _ptr(self.y), _ptr(self.z),
                                  _ptr(self.u), _ptr(self.v), _ptr(self.w), _ptr(self.e),
                                  _ptr(self.p), _ptr(self.q), _ptr(self.vrel), _ptr(self.V0),
                                  _ptr(self.mnode), 1 if knobs is not None else 0, kp,
                                  _ptr(eos_in), _ptr(mask), _ptr(cnt))
        if rc:
            raise ValueError(f"hydro step failed ({rc})")
        return eos_in, mask, cnt

    def energies(self):
        ie = float(np.sum(self.e * self.V0))
        ke = float(0.5 * np.sum(self.mnode * (self.u ** 2 + self.v ** 2 + self.w ** 2)))
        return ie, ke


def eos_knobs(mode, hsize=4, psize=8, tsize=8, tperwarp=32, level=THREAD, thresh=0.0,
              threads=0, block=256, in_scale=(1.0, 1.0, 1.0, 1.0), persistent=False, n=None):
    """EOS technique of a hydro step. persistent=True keeps the TAF windows or
    iACT tables across steps (the state arrays of taf_state / iact_state for
    T = threads, or n^3 elements when threads is 0; n is then required)."""
    k = EosKnobs(mode, hsize, psize, tsize, tperwarp, level, float(thresh), threads, block, 0,
                 (C.c_double * 4)(*in_scale))
    if persistent and mode in (EOS_TAF, EOS_IACT):
        T = threads if threads > 0 else n ** 3
        st = taf_state(T, hsize) if mode == EOS_TAF else iact_state(T, tsize, tperwarp, 4)
        keys = ("vals", "cnt", "pred") if mode == EOS_TAF else ("z", "y", "valid", "rr")
        for j, key in enumerate(keys):
            k.st[j] = st[key].ctypes.data
        k._state = st                      # keeps the arrays alive with the knobs
    return k


__all__ = [k for k in dir() if not k.startswith("_")] + ["math"]


# ------------------------------------------------------------- LavaMD region

LAVAMD_EXACT, LAVAMD_TAF, LAVAMD_IACT = 0, 1, 2


def lavamd(boxes1d, par_per_box, a2, rq, technique=LAVAMD_EXACT, level=THREAD, hsize=4, psize=8,
           thresh=0.0, reset=0, tsize=8, tperwarp=32, in_scale=None, mask=False):
    """LavaMD-style neighbour-box forces (lavamd_oracle.c): rq is (4, P) float64
    (x, y, z, charge), P = boxes1d^3 par_per_box. Returns (fv (4, P), counters
    [invocations, approximated, 0, borderline], mask (27 P bytes, 255 where no
    invocation) or None)."""
    B, NP = int(boxes1d), int(par_per_box)
    P = B ** 3 * NP
    rq = np.ascontiguousarray(rq, dtype=np.float64).reshape(4, P)
    fv = np.zeros((4, P), dtype=np.float64)
    cnt = np.zeros(4, dtype=np.int64)
    m = np.full(27 * P, 255, dtype=np.uint8) if mask else None
    sc = None if in_scale is None else np.ascontiguousarray(in_scale, dtype=np.float64)
    rc = lib().orc_lavamd(B, NP, float(a2), _ptr(rq), _ptr(fv), int(technique), int(level), int(hsize),
                          int(psize), float(thresh), int(reset), int(tsize), int(tperwarp),
                          None if sc is None else _ptr(sc), None if m is None else _ptr(m), _ptr(cnt))
    if rc != 0:
        raise ValueError("orc_lavamd rejected its arguments")
    return fv, cnt, m

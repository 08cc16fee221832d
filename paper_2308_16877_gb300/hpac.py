"""Python binding of libhpac: the C ABI declared in include/hpac.h, same names.

Argument marshalling only: every step of a call runs in the library's CUDA
kernels. Tensors are torch CUDA tensors (device memory and streams are
PyTorch's; the arithmetic is not). If the shared library is missing it is built
from the in-tree sources with nvcc; if that is impossible the import of the
library raises, there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

HPAC_OK, HPAC_EINVAL, HPAC_ENOMEM, HPAC_ECUDA, HPAC_ETIMEOUT, HPAC_EUNSUPPORTED = range(6)
HPAC_F32, HPAC_F64 = 0, 1
HPAC_LEVEL_THREAD, HPAC_LEVEL_WARP, HPAC_LEVEL_BLOCK = 0, 1, 2
HPAC_REGION_BLACKSCHOLES, HPAC_REGION_EOS, HPAC_REGION_IDENTITY, HPAC_REGION_BINOMIAL = 0, 1, 3, 4
HPAC_REGION_KMEANS = 5
HPAC_PERFO_SMALL, HPAC_PERFO_LARGE, HPAC_PERFO_INI, HPAC_PERFO_FINI, HPAC_PERFO_RANDOM = range(5)
HPAC_MASK_EXACT, HPAC_MASK_APPROX, HPAC_MASK_SKIPPED = 0, 1, 2
HPAC_METRIC_MAPE, HPAC_METRIC_RMSE, HPAC_METRIC_MCR = 0, 1, 2


class hpac_region_desc(C.Structure):
    _fields_ = [("kind", C.c_int32), ("dtype", C.c_int32), ("n", C.c_int64), ("n_in", C.c_int32),
                ("n_out", C.c_int32), ("in_stride", C.c_int64), ("out_stride", C.c_int64),
                ("logical_threads", C.c_int64), ("block_threads", C.c_int32),
                ("arg", C.c_int32), ("param", C.c_double)]


class hpac_perfo_knobs(C.Structure):
    _fields_ = [("kind", C.c_int32), ("m_or_percent", C.c_int32), ("rate", C.c_double),
                ("seed", C.c_uint64), ("herded", C.c_int32), ("reserved0", C.c_int32)]


class hpac_taf_knobs(C.Structure):
    _fields_ = [("hsize", C.c_int32), ("psize", C.c_int32), ("thresh", C.c_double),
                ("level", C.c_int32), ("reset_on_exit", C.c_int32)]


class hpac_iact_knobs(C.Structure):
    _fields_ = [("tsize", C.c_int32), ("tperwarp", C.c_int32), ("thresh", C.c_double),
                ("level", C.c_int32), ("reserved0", C.c_int32), ("in_scale", C.POINTER(C.c_double))]


class hpac_stats(C.Structure):
    _fields_ = [("invocations", C.c_int64), ("approximated", C.c_int64), ("skipped", C.c_int64),
                ("borderline", C.c_int64)]

    def as_dict(self):
        return {f: int(getattr(self, f)) for f, _ in self._fields_}


class hpac_lavamd_desc(C.Structure):
    _fields_ = [("boxes1d", C.c_int32), ("par_per_box", C.c_int32), ("a2", C.c_double)]


class hpac_quality_result(C.Structure):
    _fields_ = [("value", C.c_double), ("zero_max_abs", C.c_double), ("used", C.c_int64),
                ("zeros", C.c_int64), ("zeros_mismatch", C.c_int64)]

    def as_dict(self):
        return {f: (float if t is C.c_double else int)(getattr(self, f)) for f, t in self._fields_}


_D = C.POINTER(C.c_double)


class hpac_hydro_state(C.Structure):
    _fields_ = [("n", C.c_int32), ("reserved0", C.c_int32), ("gamma", C.c_double),
                ("dt", C.c_double), ("x", _D), ("y", _D), ("z", _D), ("u", _D), ("v", _D),
                ("w", _D), ("mnode", _D), ("e", _D), ("p", _D), ("q", _D), ("vrel", _D),
                ("V0", _D), ("grad", _D), ("eos_in", _D), ("pq", _D), ("rmass", _D), ("rV0", _D)]


class hpac_sweep_config(C.Structure):
    _fields_ = [("technique", C.c_int32), ("level", C.c_int32), ("hsize", C.c_int32),
                ("psize", C.c_int32), ("thresh", C.c_double), ("perfo_kind", C.c_int32),
                ("m_or_percent", C.c_int32), ("rate", C.c_double), ("seed", C.c_uint64),
                ("herded", C.c_int32), ("reserved0", C.c_int32)]


class hpac_sweep_region(C.Structure):
    _fields_ = [("n", C.c_int64), ("offset", C.c_int64), ("logical_threads", C.c_int64)]


class hpac_sweep_stats(C.Structure):
    _fields_ = [("invocations", C.c_int64), ("approximated", C.c_int64), ("skipped", C.c_int64),
                ("mape_terms", C.c_int64), ("sum_abs_rel", C.c_double), ("sum_sq", C.c_double)]


class hpac_mlp_desc(C.Structure):
    _fields_ = [("kind", C.c_int32), ("n_feat", C.c_int32), ("hidden", C.c_int32),
                ("reserved0", C.c_int32), ("feat_shift", C.c_float * 8),
                ("feat_scale", C.c_float * 8), ("out_shift", C.c_float), ("out_scale", C.c_float)]


# Every symbol include/hpac.h declares, with its ctypes signature.
_P = C.c_void_p
SIGNATURES = {
    "hpac_region_create": (C.c_int, [C.POINTER(hpac_region_desc), _P, C.POINTER(_P)]),
    "hpac_region_destroy": (C.c_int, [_P]),
    "hpac_region_set_stream": (C.c_int, [_P, _P]),
    "hpac_region_set_persistent": (C.c_int, [_P, C.c_int32]),
    "hpac_region_reset_state": (C.c_int, [_P]),
    "hpac_run_exact": (C.c_int, [_P, _P, _P]),
    "hpac_run_perfo": (C.c_int, [_P, C.POINTER(hpac_perfo_knobs), _P, _P, _P, C.POINTER(hpac_stats)]),
    "hpac_run_taf": (C.c_int, [_P, C.POINTER(hpac_taf_knobs), _P, _P, _P, _P, C.POINTER(hpac_stats)]),
    "hpac_run_iact": (C.c_int, [_P, C.POINTER(hpac_iact_knobs), _P, _P, _P, _P, C.POINTER(hpac_stats)]),
    "hpac_quality": (C.c_int, [C.c_int32, C.c_int64, _P, _P, C.c_int32,
                               C.POINTER(hpac_quality_result), _P]),
    "hpac_quality_noalloc": (C.c_int, [C.c_int32, C.c_int64, _P, _P, C.c_int32,
                                       C.POINTER(hpac_quality_result), _P]),
    "hpac_calibrate_floor": (C.c_int, [C.c_int64, _P, _P, C.c_double, C.c_double, C.POINTER(C.c_float),
                                       C.POINTER(C.c_int64), _P]),
    "hpac_region_set_aux": (C.c_int, [_P, _P]),
    "hpac_kmeans_workspace_bytes": (C.c_size_t, [C.c_int32]),
    "hpac_kmeans_update": (C.c_int, [C.c_int64, C.c_int32, _P, C.c_int64, _P, _P, _P, _P,
                                     C.POINTER(C.c_int64), _P]),
    "hpac_hydro_init": (C.c_int, [C.POINTER(hpac_hydro_state), _P]),
    "hpac_hydro_derive": (C.c_int, [C.POINTER(hpac_hydro_state), _P]),
    "hpac_hydro_step": (C.c_int, [C.POINTER(hpac_hydro_state), _P, C.c_int32, _P, _P,
                                  C.POINTER(hpac_stats)]),
    "hpac_hydro_nodes": (C.c_int, [C.POINTER(hpac_hydro_state), _P]),
    "hpac_hydro_elements": (C.c_int, [C.POINTER(hpac_hydro_state), _P]),
    "hpac_hydro_finalize": (C.c_int, [C.POINTER(hpac_hydro_state), _P]),
    "hpac_hydro_run": (C.c_int, [C.POINTER(hpac_hydro_state), _P, C.c_int32, C.c_int32, _P]),
    "hpac_device_fp64_rate": (C.c_int, [C.POINTER(C.c_double), _P]),
    "hpac_lavamd_run": (C.c_int, [C.POINTER(hpac_lavamd_desc), C.c_int32, _P, _P, _P, _P,
                                  C.POINTER(hpac_stats), _P]),
    "hpac_sweep_create": (C.c_int, [C.c_int32, C.POINTER(hpac_sweep_config), C.c_int32,
                                    C.POINTER(hpac_sweep_region), _P, C.c_int64, _P, C.c_double,
                                    C.c_int32, C.c_int32, C.c_int32, _P, C.POINTER(_P)]),
    "hpac_sweep_run": (C.c_int, [_P]),
    "hpac_sweep_results": (C.c_int, [_P, C.POINTER(hpac_sweep_stats)]),
    "hpac_sweep_destroy": (C.c_int, [_P]),
    "hpac_region_adjoint": (C.c_int, [_P, _P, _P]),
    "hpac_region_vjp": (C.c_int, [_P, _P, _P, _P]),
    "hpac_mlp_create": (C.c_int, [C.POINTER(hpac_mlp_desc), _P, C.c_uint64, _P, C.POINTER(_P)]),
    "hpac_mlp_destroy": (C.c_int, [_P]),
    "hpac_mlp_num_params": (C.c_int32, [_P]),
    "hpac_mlp_get_params": (C.c_int, [_P, _P]),
    "hpac_mlp_set_params": (C.c_int, [_P, _P]),
    "hpac_mlp_infer": (C.c_int, [_P, C.c_int64, _P, C.c_int64, C.c_double, _P, C.c_float, _P,
                                 C.POINTER(hpac_stats)]),
    "hpac_mlp_grad": (C.c_int, [_P, C.c_int64, _P, C.c_int64, C.c_double, _P, _P,
                                C.POINTER(C.c_float)]),
    "hpac_mlp_train": (C.c_int, [_P, C.c_int64, _P, C.c_int64, C.c_double, _P, C.c_int32, C.c_int32,
                                 C.c_float, C.POINTER(C.c_float)]),
    "hpac_mlp_input_grad": (C.c_int, [_P, C.c_int64, _P, C.c_int64, C.c_double, _P]),
    "hpac_mlp_vjp": (C.c_int, [_P, C.c_int64, _P, C.c_int64, C.c_double, _P, _P, _P]),
    "hpac_mlp_set_params_device": (C.c_int, [_P, _P]),
    "hpac_mlp_fit_normalization": (C.c_int, [_P, C.c_int64, _P, C.c_int64, C.c_double, _P]),
    "hpac_mlp_get_desc": (C.c_int, [_P, C.POINTER(hpac_mlp_desc)]),
    "hpac_last_error": (C.c_char_p, []),
    "hpac_version": (C.c_char_p, []),
}

_lib = None
_lock = threading.Lock()


def library_path() -> str:
    from . import build as _b
    return _b.LIB


def load(build_if_missing: bool = True) -> C.CDLL:
    """Load libhpac.so (building it from source first if it is absent)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = library_path()
        if not os.path.exists(path):
            if not build_if_missing:
                raise RuntimeError(f"libhpac is not built ({path} missing)")
            from . import build as _b
            _b.build()
        lib = C.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


class HpacError(RuntimeError):
    def __init__(self, status, where):
        msg = load().hpac_last_error().decode(errors="replace")
        super().__init__(f"{where}: status {status}: {msg}")
        self.status = status


def _check(status, where):
    if status != HPAC_OK:
        raise HpacError(status, where)


# --------------------------------------------------------------------------
# thin wrappers with the C names
# --------------------------------------------------------------------------

def hpac_region_create(desc: hpac_region_desc, stream: int | None):
    h = _P()
    _check(load().hpac_region_create(C.byref(desc), stream or None, C.byref(h)), "hpac_region_create")
    return h


def hpac_region_destroy(h):
    _check(load().hpac_region_destroy(h), "hpac_region_destroy")


def hpac_region_set_persistent(h, enable):
    _check(load().hpac_region_set_persistent(h, int(bool(enable))), "hpac_region_set_persistent")


def hpac_region_reset_state(h):
    _check(load().hpac_region_reset_state(h), "hpac_region_reset_state")


def hpac_region_set_stream(h, stream):
    _check(load().hpac_region_set_stream(h, stream or None), "hpac_region_set_stream")


def hpac_run_exact(h, d_in: int, d_out: int):
    _check(load().hpac_run_exact(h, d_in, d_out), "hpac_run_exact")


def hpac_run_perfo(h, knobs, d_in, d_out, d_mask=None, want_stats=False):
    st = hpac_stats() if want_stats else None
    _check(load().hpac_run_perfo(h, C.byref(knobs), d_in, d_out, d_mask,
                                 C.byref(st) if st is not None else None), "hpac_run_perfo")
    return st


def hpac_run_taf(h, knobs, d_in, d_out, d_mask=None, d_stat=None, want_stats=False):
    st = hpac_stats() if want_stats else None
    _check(load().hpac_run_taf(h, C.byref(knobs), d_in, d_out, d_mask, d_stat,
                               C.byref(st) if st is not None else None), "hpac_run_taf")
    return st


def hpac_run_iact(h, knobs, d_in, d_out, d_mask=None, d_stat=None, want_stats=False):
    st = hpac_stats() if want_stats else None
    _check(load().hpac_run_iact(h, C.byref(knobs), d_in, d_out, d_mask, d_stat,
                                C.byref(st) if st is not None else None), "hpac_run_iact")
    return st


def hpac_quality(dtype, n, d_exact, d_approx, metric, stream=None):
    res = hpac_quality_result()
    _check(load().hpac_quality(dtype, n, d_exact, d_approx, metric, C.byref(res), stream or None),
           "hpac_quality")
    return res


def hpac_quality_noalloc(dtype, n, d_exact, d_approx, metric, stream=None):
    """hpac_quality with the library's fixed scratch instead of an allocation
    (n at most 134,217,728); for callers that cannot allocate device memory."""
    res = hpac_quality_result()
    _check(load().hpac_quality_noalloc(dtype, n, d_exact, d_approx, metric, C.byref(res),
                                       stream or None), "hpac_quality_noalloc")
    return res


def hpac_calibrate_floor(n, d_pred, d_exact, target, quantile, stream=None):
    """(floor, kept): the surrogate's calibrated fallback bound (see hpac.h)."""
    fl = C.c_float()
    kept = C.c_int64()
    _check(load().hpac_calibrate_floor(n, d_pred, d_exact, float(target), float(quantile), C.byref(fl),
                                       C.byref(kept), stream or None), "hpac_calibrate_floor")
    return float(fl.value), int(kept.value)


def calibrate_floor(pred, exact, target=0.01, quantile=0.99, stream=None):
    """Floor for Surrogate.infer's fallback_below from predictions (float32)
    and exact outputs (float64) of the same held-out invocations (CUDA tensors)."""
    import torch
    if pred.dtype != torch.float32 or exact.dtype != torch.float64 or pred.numel() != exact.numel():
        raise ValueError("pred must be float32 and exact float64 of the same length")
    return hpac_calibrate_floor(pred.numel(), _ptr(pred.contiguous()), _ptr(exact.contiguous()), target,
                                quantile, _stream_handle(stream))


def hpac_hydro_init(state, stream=None):
    _check(load().hpac_hydro_init(C.byref(state), stream or None), "hpac_hydro_init")


def hpac_hydro_derive(state, stream=None):
    _check(load().hpac_hydro_derive(C.byref(state), stream or None), "hpac_hydro_derive")


def hpac_hydro_step(state, eos, technique, knobs=None, d_mask=None, want_stats=False):
    st = hpac_stats() if want_stats else None
    _check(load().hpac_hydro_step(C.byref(state), eos, technique,
                                  C.byref(knobs) if knobs is not None else None, d_mask,
                                  C.byref(st) if st is not None else None), "hpac_hydro_step")
    return st


def hpac_hydro_nodes(state, stream=None):
    _check(load().hpac_hydro_nodes(C.byref(state), stream or None), "hpac_hydro_nodes")


def hpac_hydro_elements(state, stream=None):
    _check(load().hpac_hydro_elements(C.byref(state), stream or None), "hpac_hydro_elements")


def hpac_hydro_finalize(state, stream=None):
    _check(load().hpac_hydro_finalize(C.byref(state), stream or None), "hpac_hydro_finalize")


def hpac_hydro_run(state, eos, steps, technique, knobs=None):
    _check(load().hpac_hydro_run(C.byref(state), eos, steps, technique,
                                 C.byref(knobs) if knobs is not None else None), "hpac_hydro_run")


def hpac_lavamd_run(desc, technique, knobs, d_rq, d_fv, d_mask=None, want_stats=False, stream=None):
    st = hpac_stats() if want_stats else None
    _check(load().hpac_lavamd_run(C.byref(desc), technique, C.byref(knobs) if knobs is not None else None,
                                  d_rq, d_fv, d_mask, C.byref(st) if st is not None else None,
                                  stream or None), "hpac_lavamd_run")
    return st


def hpac_device_fp64_rate(stream=None) -> float:
    v = C.c_double()
    _check(load().hpac_device_fp64_rate(C.byref(v), stream or None), "hpac_device_fp64_rate")
    return float(v.value)


def hpac_last_error() -> str:
    return load().hpac_last_error().decode(errors="replace")


def hpac_version() -> str:
    return load().hpac_version().decode()


# --------------------------------------------------------------------------
# tensor-level convenience layer
# --------------------------------------------------------------------------

def _dtype_code(t):
    import torch
    if t.dtype == torch.float32:
        return HPAC_F32
    if t.dtype == torch.float64:
        return HPAC_F64
    raise TypeError(f"unsupported dtype {t.dtype}")


def _ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def _stream_handle(stream):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return s.cuda_stream


class Region:
    """An annotated loop region over a (D, stride) CUDA tensor of inputs."""

    def __init__(self, kind: int, x, n: int | None = None, param: float = 0.0,
                 logical_threads: int = 0, block_threads: int = 256, stream=None, arg: int = 0):
        """arg: the Binomial region's tree steps (0 for the other kinds)."""
        if not x.is_cuda or x.dim() != 2 or not x.is_contiguous():
            raise ValueError("inputs must be a contiguous 2-D CUDA tensor (D, stride)")
        self.kind = kind
        self.dtype = x.dtype
        self.d_in, stride = x.shape
        self.n = stride if n is None else n
        self.desc = hpac_region_desc(kind, _dtype_code(x), self.n, self.d_in, 1, stride, self.n,
                                     logical_threads, block_threads, int(arg), float(param))
        self._h = hpac_region_create(self.desc, _stream_handle(stream))

    def close(self):
        if self._h:
            hpac_region_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def set_stream(self, stream):
        hpac_region_set_stream(self._h, _stream_handle(stream))

    def set_persistent(self, enable=True):
        """Keep TAF windows / iACT tables across calls (see hpac.h)."""
        hpac_region_set_persistent(self._h, enable)

    def reset_state(self):
        hpac_region_reset_state(self._h)

    def set_aux(self, aux):
        """K-Means: the centroids (K, 8) float32 CUDA tensor later runs read."""
        self._aux = aux
        _check(load().hpac_region_set_aux(self._h, _ptr(aux)), "hpac_region_set_aux")

    def _check_io(self, x, out, mask=None, stat=None):
        if x.dtype != self.dtype or out.dtype != self.dtype:
            raise TypeError("dtype mismatch")
        if out.numel() < self.n:
            raise ValueError("output too small")
        if mask is not None and mask.numel() < self.n:
            raise ValueError("mask too small")
        if stat is not None and (stat.numel() < self.n or stat.dtype != self.dtype):
            raise ValueError("stat too small or wrong dtype")

    def run_exact(self, x, out):
        self._check_io(x, out)
        hpac_run_exact(self._h, _ptr(x), _ptr(out))
        return out

    def run_perfo(self, x, out, kind, m_or_percent=0, rate=0.0, seed=0, herded=True, mask=None,
                  stats=False):
        self._check_io(x, out, mask)
        k = hpac_perfo_knobs(kind, int(m_or_percent), float(rate), int(seed), 1 if herded else 0, 0)
        st = hpac_run_perfo(self._h, k, _ptr(x), _ptr(out), _ptr(mask), stats)
        return st.as_dict() if st is not None else None

    def run_taf(self, x, out, hsize, psize, thresh, level=HPAC_LEVEL_THREAD, mask=None, stat=None,
                stats=False, reset_on_exit=False):
        self._check_io(x, out, mask, stat)
        k = hpac_taf_knobs(int(hsize), int(psize), float(thresh), int(level), int(bool(reset_on_exit)))
        st = hpac_run_taf(self._h, k, _ptr(x), _ptr(out), _ptr(mask), _ptr(stat), stats)
        return st.as_dict() if st is not None else None

    def run_iact(self, x, out, tsize, tperwarp, thresh, level=HPAC_LEVEL_THREAD, in_scale=None,
                 mask=None, stat=None, stats=False):
        self._check_io(x, out, mask, stat)
        sc = None
        if in_scale is not None:
            vals = [float(v) for v in in_scale]
            if len(vals) != self.d_in:
                raise ValueError("in_scale needs one value per input")
            sc = (C.c_double * len(vals))(*vals)
        k = hpac_iact_knobs(int(tsize), int(tperwarp), float(thresh), int(level), 0,
                            C.cast(sc, C.POINTER(C.c_double)) if sc is not None else None)
        st = hpac_run_iact(self._h, k, _ptr(x), _ptr(out), _ptr(mask), _ptr(stat), stats)
        return st.as_dict() if st is not None else None


def kmeans_update(x, assign, cent, work, prev=None, stream=None, changed=True):
    """One exact centroid update (hpac_kmeans_update) on CUDA tensors: x (8,
    stride) float32, assign / prev float32 ids, cent (K, 8) float32 updated in
    place, work a device buffer of hpac_kmeans_workspace_bytes(K) bytes.
    Returns the number of changed assignments (waits) when changed, else None."""
    ch = C.c_int64(0)
    _check(load().hpac_kmeans_update(int(assign.numel()), int(cent.shape[0]), _ptr(x), int(x.shape[1]),
                                     _ptr(assign), _ptr(prev), _ptr(cent), _ptr(work),
                                     C.byref(ch) if changed else None, _stream_handle(stream)),
           "hpac_kmeans_update")
    return int(ch.value) if changed else None


LAVAMD_EXACT, LAVAMD_TAF, LAVAMD_IACT = 0, 1, 2


def lavamd(rq, boxes1d, par_per_box, a2=0.5, technique=LAVAMD_EXACT, level=HPAC_LEVEL_THREAD,
           hsize=4, psize=8, thresh=0.0, reset_on_exit=False, tsize=8, tperwarp=32, in_scale=None,
           fv=None, mask=None, stats=False, stream=None):
    """LavaMD-style neighbour-box forces (hpac_lavamd_run) on CUDA tensors: rq
    (4, P) float64 (x, y, z, charge), P = boxes1d^3 par_per_box. Returns fv
    (4, P) float64 (potential, force x, y, z) and, with stats, the counts.
    mask: an optional uint8 tensor of 27 P bytes."""
    import torch
    P = int(boxes1d) ** 3 * int(par_per_box)
    if (tuple(rq.shape) != (4, P) or rq.dtype != torch.float64 or not rq.is_contiguous()
            or not rq.is_cuda):
        raise ValueError("rq must be a contiguous (4, boxes1d^3 par_per_box) float64 CUDA tensor")
    if fv is None:
        fv = torch.empty_like(rq)
    if (tuple(fv.shape) != (4, P) or fv.dtype != torch.float64 or not fv.is_contiguous()
            or fv.device != rq.device):
        raise ValueError("fv must be a contiguous (4, P) float64 tensor on rq's device")
    if mask is not None and (mask.dtype != torch.uint8 or not mask.is_contiguous()
                             or mask.device != rq.device or mask.numel() < 27 * P):
        raise ValueError("mask must be a contiguous uint8 tensor of 27 P bytes on rq's device")
    desc = hpac_lavamd_desc(int(boxes1d), int(par_per_box), float(a2))
    knobs = None
    if technique == LAVAMD_TAF:
        knobs = hpac_taf_knobs(int(hsize), int(psize), float(thresh), int(level), int(bool(reset_on_exit)))
    elif technique == LAVAMD_IACT:
        sc = None
        if in_scale is not None:
            vals = [float(v) for v in in_scale]
            if len(vals) != 3:
                raise ValueError("in_scale needs three values (x, y, z)")
            sc = (C.c_double * 3)(*vals)
        knobs = hpac_iact_knobs(int(tsize), int(tperwarp), float(thresh), int(level), 0,
                                C.cast(sc, C.POINTER(C.c_double)) if sc is not None else None)
    st = hpac_lavamd_run(desc, int(technique), knobs, _ptr(rq), _ptr(fv), _ptr(mask), stats,
                         _stream_handle(stream))
    return (fv, st.as_dict()) if st is not None else fv


def kmeans_workspace(clusters, device=None):
    import torch
    nbytes = load().hpac_kmeans_workspace_bytes(int(clusters))
    return torch.zeros(nbytes // 8, dtype=torch.float64, device=device or "cuda")


def quality(exact, approx, metric, stream=None):
    """MAPE / RMSE / MCR of approx against exact (float64 CUDA tensor)."""
    import torch
    if exact.dtype != torch.float64 or exact.numel() != approx.numel():
        raise ValueError("exact must be float64 with as many elements as approx")
    r = hpac_quality(_dtype_code(approx), exact.numel(), _ptr(exact), _ptr(approx), metric,
                     _stream_handle(stream))
    return r.as_dict()


HYDRO_EXACT, HYDRO_TAF, HYDRO_IACT, HYDRO_PERFO = 0, 1, 2, 3
NODE_FIELDS = ("x", "y", "z", "u", "v", "w", "mnode")
ELEM_FIELDS = ("e", "p", "q", "vrel", "V0")


class Hydro:
    """Hexahedral hydro state in torch CUDA tensors plus its EOS region.

    x, y, z: initial node coordinates ((n+1)^3); e: initial element energies
    (n^3). The EOS region (kind EOS) uses `logical_threads` / `block_threads`
    for the approximation schedule.
    """

    def __init__(self, n, x, y, z, e, dt, gamma=5.0 / 3.0, logical_threads=0, block_threads=256,
                 stream=None, device=None):
        import torch
        dev = device if device is not None else torch.device("cuda", torch.cuda.current_device())
        self.n, self.dt, self.gamma = n, float(dt), float(gamma)
        E, Nn = n ** 3, (n + 1) ** 3
        f64 = dict(dtype=torch.float64, device=dev)
        self.t = {}
        for k, src in (("x", x), ("y", y), ("z", z)):
            self.t[k] = torch.as_tensor(src, **f64).clone().contiguous()
        for k in ("u", "v", "w", "mnode"):
            self.t[k] = torch.zeros(Nn, **f64)
        self.t["e"] = torch.as_tensor(e, **f64).clone().contiguous()
        for k in ("p", "q", "vrel", "V0"):
            self.t[k] = torch.zeros(E, **f64)
        self.t["grad"] = torch.zeros(24 * E, **f64)
        self.t["eos_in"] = torch.zeros(4, E, **f64)
        self.t["pq"] = torch.zeros(E, **f64)
        self.t["rmass"] = torch.zeros(Nn, **f64)
        self.t["rV0"] = torch.zeros(E, **f64)
        self.state = self._state()
        self.eos = Region(HPAC_REGION_EOS, self.t["eos_in"], param=self.gamma,
                          logical_threads=logical_threads, block_threads=block_threads, stream=stream)
        self._stream = stream
        hpac_hydro_init(self.state, _stream_handle(stream))

    def _state(self):
        ptr = lambda k: C.cast(C.c_void_p(self.t[k].data_ptr()), _D)
        return hpac_hydro_state(self.n, 0, self.gamma, self.dt, *[ptr(k) for k in (
            "x", "y", "z", "u", "v", "w", "mnode", "e", "p", "q", "vrel", "V0", "grad", "eos_in", "pq",
            "rmass", "rV0")])

    def __getitem__(self, k):
        return self.t[k]

    def load_state(self, fields):
        """Overwrite node/element fields (a checkpoint) from host or device arrays;
        the volume gradients are recomputed by the next step's element kernel only,
        so the gradient field must be supplied too (key 'grad') or left as is. The
        derived arrays (pq, rmass, rV0) are recomputed from the loaded state."""
        import torch
        for k, v in fields.items():
            self.t[k].copy_(torch.as_tensor(v, dtype=torch.float64).reshape(self.t[k].shape))
        torch.cuda.current_stream().synchronize()   # the copies land before the derive kernel
        hpac_hydro_derive(self.state, _stream_handle(self._stream))

    def step(self, technique=HYDRO_EXACT, knobs=None, mask=None, stats=False):
        st = hpac_hydro_step(self.state, self.eos._h, technique, knobs, _ptr(mask), stats)
        return st.as_dict() if st is not None else None

    def run(self, steps, technique=HYDRO_EXACT, knobs=None):
        hpac_hydro_run(self.state, self.eos._h, steps, technique, knobs)

    def close(self):
        self.eos.close()


HPAC_SWEEP_TAF, HPAC_SWEEP_PERFO = 1, 3


def sweep_config(d):
    """hpac_sweep_config from a dict: {"tech": "taf", hsize, psize, thresh[, level]} or
    {"tech": "perfo", kind, m[, rate, seed, herded]}."""
    if d["tech"] == "taf":
        return hpac_sweep_config(HPAC_SWEEP_TAF, d.get("level", 0), d["hsize"], d["psize"],
                                 float(d["thresh"]), 0, 0, 0.0, 0, 0, 0)
    return hpac_sweep_config(HPAC_SWEEP_PERFO, 0, 0, 0, 0.0, d["kind"], d.get("m", 0),
                             float(d.get("rate", 0.0)), int(d.get("seed", 0)),
                             1 if d.get("herded", 1) else 0, 0)


class Sweep:
    """A batched knob sweep over Black-Scholes regions (hpac_sweep_*).

    x: (4, stride) float32 CUDA tensor holding every region at its offset;
    ref: float64 CUDA tensor of exact prices; regions: list of (n, offset,
    logical_threads); configs: list of dicts (see sweep_config).
    """

    def __init__(self, configs, regions, x, ref, rate, block_threads=256, blocks_per_sm=4,
                 tile_blocks=1, stream=None):
        self.configs = list(configs)
        self.regions = list(regions)
        cfg = (hpac_sweep_config * len(self.configs))(*[sweep_config(c) for c in self.configs])
        reg = (hpac_sweep_region * len(self.regions))(*[hpac_sweep_region(*r) for r in self.regions])
        self._keep = (x, ref)
        h = _P()
        _check(load().hpac_sweep_create(len(cfg), cfg, len(reg), reg, C.c_void_p(x.data_ptr()),
                                        x.shape[1], C.c_void_p(ref.data_ptr()), float(rate),
                                        block_threads, blocks_per_sm, tile_blocks,
                                        _stream_handle(stream), C.byref(h)), "hpac_sweep_create")
        self._h = h

    def run(self):
        _check(load().hpac_sweep_run(self._h), "hpac_sweep_run")

    def results(self):
        """numpy array (n_configs, n_regions) of records with the stats fields."""
        import numpy as np
        n = len(self.configs) * len(self.regions)
        buf = (hpac_sweep_stats * n)()
        _check(load().hpac_sweep_results(self._h, buf), "hpac_sweep_results")
        dt = np.dtype([(f, np.int64 if t is C.c_int64 else np.float64)
                       for f, t in hpac_sweep_stats._fields_])
        arr = np.frombuffer(bytes(buf), dtype=dt).copy()
        return arr.reshape(len(self.configs), len(self.regions))

    def close(self):
        if self._h:
            load().hpac_sweep_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def region_adjoint(region, x, grad):
    """d out / d in of the exact region (hpac_region_adjoint) into grad (D, n)."""
    _check(load().hpac_region_adjoint(region._h, _ptr(x), _ptr(grad)), "hpac_region_adjoint")
    return grad


def region_vjp(region, x, gout, grad):
    """gout_i d out_i / d in_{d,i} of the exact region (hpac_region_vjp) into grad (D, n)."""
    _check(load().hpac_region_vjp(region._h, _ptr(x), _ptr(gout), _ptr(grad)), "hpac_region_vjp")
    return grad


def _autograd():
    import torch

    class RegionFn(torch.autograd.Function):
        """The exact region as a differentiable function of its inputs: forward
        hpac_run_exact, backward hpac_region_vjp."""

        @staticmethod
        def forward(ctx, x, region):
            out = torch.empty(region.n, dtype=x.dtype, device=x.device)
            region.run_exact(x, out)
            ctx.region = region
            ctx.save_for_backward(x)
            return out

        @staticmethod
        def backward(ctx, gout):
            (x,) = ctx.saved_tensors
            R = ctx.region
            g = torch.empty(R.d_in, R.n, dtype=x.dtype, device=x.device)
            region_vjp(R, x, gout.to(x.dtype).contiguous(), g)
            gx = torch.zeros_like(x)
            gx[:, :R.n] = g
            return gx, None

    class SurrogateFn(torch.autograd.Function):
        """The surrogate as a differentiable function of the region inputs and
        of its parameters (a float32 CUDA tensor of n_params values, loaded
        into the surrogate before the forward and the backward): forward
        hpac_mlp_infer, backward hpac_mlp_vjp."""

        @staticmethod
        def forward(ctx, x, weights, surrogate, param):
            surrogate.set_params_device(weights)
            eos = surrogate.desc.kind == HPAC_REGION_EOS
            n = x.shape[1]
            out = torch.empty(n, dtype=torch.float64 if eos else torch.float32, device=x.device)
            surrogate.infer(x, out, param)
            ctx.surrogate, ctx.param = surrogate, param
            ctx.save_for_backward(x, weights)
            return out

        @staticmethod
        def backward(ctx, gout):
            x, weights = ctx.saved_tensors
            S = ctx.surrogate
            S.set_params_device(weights)
            n = x.shape[1]
            gp = torch.empty(S.n_params, dtype=torch.float32, device=x.device) \
                if ctx.needs_input_grad[1] else None
            gi = torch.empty(4, n, dtype=torch.float32, device=x.device) \
                if ctx.needs_input_grad[0] else None
            S.vjp(x, gout.to(torch.float32).contiguous(), ctx.param, gp, gi)
            gx = None
            if gi is not None:
                gx = torch.zeros_like(x)
                gx[:4] = gi.to(x.dtype)
            return gx, gp, None, None

    return RegionFn, SurrogateFn


def differentiable(region, x):
    """out = region(x) with autograd: d(loss)/dx comes from hpac_region_vjp."""
    return _autograd()[0].apply(x, region)


class Surrogate:
    """The learned surrogate of a region (hpac_mlp_*). desc: hpac_mlp_desc."""

    def __init__(self, desc, params=None, seed=0, stream=None):
        import numpy as np
        self.desc = desc
        h = _P()
        buf = None
        if params is not None:
            params = np.ascontiguousarray(params, dtype=np.float32)
            buf = params.ctypes.data_as(_P)
        _check(load().hpac_mlp_create(C.byref(desc), buf, int(seed), _stream_handle(stream),
                                      C.byref(h)), "hpac_mlp_create")
        self._h = h
        self.n_params = int(load().hpac_mlp_num_params(h))

    def fit_normalization(self, x, target, param, n=None):
        n = x.shape[1] if n is None else n
        _check(load().hpac_mlp_fit_normalization(self._h, n, _ptr(x), x.shape[1], float(param),
                                                 _ptr(target)), "hpac_mlp_fit_normalization")
        self.desc = self.get_desc()
        return self.desc

    def get_desc(self):
        d = hpac_mlp_desc()
        _check(load().hpac_mlp_get_desc(self._h, C.byref(d)), "hpac_mlp_get_desc")
        return d

    def params(self):
        import numpy as np
        out = np.zeros(self.n_params, dtype=np.float32)
        _check(load().hpac_mlp_get_params(self._h, out.ctypes.data_as(_P)), "hpac_mlp_get_params")
        return out

    def set_params(self, p):
        import numpy as np
        p = np.ascontiguousarray(p, dtype=np.float32)
        _check(load().hpac_mlp_set_params(self._h, p.ctypes.data_as(_P)), "hpac_mlp_set_params")

    def infer(self, x, out, param, n=None, fallback_below=float("nan"), mask=None, stats=False):
        n = x.shape[1] if n is None else n
        st = hpac_stats() if stats else None
        _check(load().hpac_mlp_infer(self._h, n, _ptr(x), x.shape[1], float(param), _ptr(out),
                                     float(fallback_below), _ptr(mask),
                                     C.byref(st) if st is not None else None), "hpac_mlp_infer")
        return st.as_dict() if st is not None else None

    def grad(self, x, target, param, grad=None, n=None, loss=False):
        n = x.shape[1] if n is None else n
        l = C.c_float()
        _check(load().hpac_mlp_grad(self._h, n, _ptr(x), x.shape[1], float(param), _ptr(target),
                                    _ptr(grad), C.byref(l) if loss else None), "hpac_mlp_grad")
        return float(l.value) if loss else None

    def train(self, x, target, param, batch=4096, epochs=1, lr=1e-3, n=None):
        n = x.shape[1] if n is None else n
        l = C.c_float()
        _check(load().hpac_mlp_train(self._h, n, _ptr(x), x.shape[1], float(param), _ptr(target),
                                     int(batch), int(epochs), float(lr), C.byref(l)), "hpac_mlp_train")
        return float(l.value)

    def input_grad(self, x, out, param, n=None):
        n = x.shape[1] if n is None else n
        _check(load().hpac_mlp_input_grad(self._h, n, _ptr(x), x.shape[1], float(param), _ptr(out)),
               "hpac_mlp_input_grad")
        return out

    def vjp(self, x, gout, param, grad_params=None, grad_in=None, n=None):
        """hpac_mlp_vjp: sum_i gout_i d out_i / d params into grad_params and
        gout_i d out_i / d in_{d,i} into grad_in (4, n); either may be None."""
        n = x.shape[1] if n is None else n
        _check(load().hpac_mlp_vjp(self._h, n, _ptr(x), x.shape[1], float(param), _ptr(gout),
                                   _ptr(grad_params), _ptr(grad_in)), "hpac_mlp_vjp")

    def set_params_device(self, weights):
        """Load the parameters from a float32 CUDA tensor (hpac_mlp_set_params_device)."""
        import torch
        if (weights.dtype != torch.float32 or not weights.is_cuda or not weights.is_contiguous()
                or weights.numel() != self.n_params):
            raise ValueError("weights must be a contiguous float32 CUDA tensor of n_params values")
        _check(load().hpac_mlp_set_params_device(self._h, _ptr(weights)), "hpac_mlp_set_params_device")

    def apply(self, x, weights, param):
        """out = surrogate(x; weights) with autograd through hpac_mlp_vjp."""
        return _autograd()[1].apply(x, weights, self, param)

    def close(self):
        if self._h:
            load().hpac_mlp_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def blackscholes_desc(hidden=64):
    """Surrogate descriptor for the Black-Scholes region (features ln(S/K),
    sigma sqrt T, r T, d1, sigma; output C / S) with a fixed normalisation for
    the option ranges of the workloads; Surrogate.fit_normalization replaces
    it with the statistics of a training set."""
    d = hpac_mlp_desc()
    d.kind, d.n_feat, d.hidden = HPAC_REGION_BLACKSCHOLES, 5, hidden
    shift = [-1.5, 0.8, 0.1, -1.5, 0.35]
    scale = [1 / 1.2, 1 / 0.6, 1 / 0.06, 1 / 3.0, 1 / 0.17]
    for k in range(5):
        d.feat_shift[k], d.feat_scale[k] = shift[k], scale[k]
    d.out_shift, d.out_scale = 0.0, 0.25
    return d


def eos_desc(hidden=128):
    """Surrogate descriptor for the EOS region (FP32 features e, v, dv, q;
    output p); Surrogate.fit_normalization sets the normalisation."""
    d = hpac_mlp_desc()
    d.kind, d.n_feat, d.hidden = HPAC_REGION_EOS, 4, hidden
    for k in range(4):
        d.feat_shift[k], d.feat_scale[k] = 0.0, 1.0
    d.out_shift, d.out_scale = 0.0, 1.0
    return d

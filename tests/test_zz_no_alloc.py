"""The allocation-free quality entry point, hpac_quality_noalloc.

It serves callers that cannot allocate device memory once they run (a service
whose device memory is all reserved up front by its own pool or by a
framework's caching allocator): instead of a cudaMalloc'd buffer it reduces
into a fixed array compiled into the library. Called through the C ABI, it must
give the same result as hpac_quality on the same inputs, including on a second
call right after the first (the array keeps the previous call's contents), and
it must refuse inputs larger than its fixed scratch can reduce.

Beyond the comparison with hpac_quality, the tests pin it to the CPU oracle's
quality function on a small case, run it once at its fixed limit (every slot of
the array written), and check that after the n = 0 warm-up call a repeated call
leaves the device's free memory unchanged.

This file is collected last so that a run stopping at the first failure has
already run every other test; it also passes on its own in a fresh process.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

NOALLOC_MAX_N = 134_217_728


@pytest.fixture(scope="module")
def H():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2308_16877_gb300 import hpac
    hpac.load()
    return hpac


def _pair(n, dtype, seed):
    rng = np.random.default_rng(seed)
    a = rng.uniform(0.1, 2.0, n)
    a[: n // 10] = 0.0
    b = (a * (1.0 + rng.normal(0.0, 0.01, n))).astype(dtype)
    b[: n // 20] = 1.0
    return torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda()


def _call(H, fn, a, b, metric):
    code = H.HPAC_F32 if b.dtype == torch.float32 else H.HPAC_F64
    s = torch.cuda.current_stream().cuda_stream
    return fn(code, a.numel(), H.C.c_void_p(a.data_ptr()), H.C.c_void_p(b.data_ptr()), metric,
              s).as_dict()


def _same(r, ref):
    # the same relative bar as the quality parity tests: per-element terms are
    # formed in single precision and grouped differently by the two grids
    assert r["value"] == pytest.approx(ref["value"], rel=1e-6, abs=1e-300)
    for k in ("used", "zeros", "zeros_mismatch"):
        assert r[k] == ref[k], k
    assert r["zero_max_abs"] == ref["zero_max_abs"]


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
@pytest.mark.parametrize("metric", [0, 1, 2])
def test_two_calls_in_a_row_match_hpac_quality(H, dtype, metric):
    # the first call covers more blocks than the second, so the second leaves
    # stale partials of the first in the shared array beyond its own range
    a1, b1 = _pair((1 << 22) + 7, dtype, seed=10 + metric)
    a2, b2 = _pair(100_003, dtype, seed=20 + metric)
    first = _call(H, H.hpac_quality_noalloc, a1, b1, metric)
    second = _call(H, H.hpac_quality_noalloc, a2, b2, metric)
    _same(first, _call(H, H.hpac_quality, a1, b1, metric))
    _same(second, _call(H, H.hpac_quality, a2, b2, metric))


def test_empty_input(H):
    a, b = _pair(0, np.float32, seed=1)
    r = _call(H, H.hpac_quality_noalloc, a, b, 0)
    assert r["value"] == 0.0 and r["used"] == 0


def test_rejects_inputs_beyond_the_fixed_scratch(H):
    a, b = _pair(16, np.float32, seed=2)
    code = H.HPAC_F32
    res = H.hpac_quality_result()
    # n is checked before anything is launched, so the small buffers are never read
    st = H.load().hpac_quality_noalloc(code, NOALLOC_MAX_N + 1, H.C.c_void_p(a.data_ptr()),
                                       H.C.c_void_p(b.data_ptr()), 0, H.C.byref(res), None)
    assert st == H.HPAC_EINVAL
    assert "limit" in H.hpac_last_error()


def test_warm_up_then_calls_allocate_nothing(H):
    # n = 0 finds the array and loads the kernels without launching anything;
    # after it (and one call that launches), further calls must not change the
    # device's free memory
    a, b = _pair(1 << 20, np.float32, seed=3)
    a64, b64 = _pair(1 << 20, np.float64, seed=4)
    res = H.hpac_quality_result()
    assert H.load().hpac_quality_noalloc(H.HPAC_F32, 0, None, None, 0, H.C.byref(res), None) == H.HPAC_OK
    assert res.used == 0
    _call(H, H.hpac_quality_noalloc, a, b, 0)
    _call(H, H.hpac_quality_noalloc, a64, b64, 1)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for metric in (0, 1, 2):
        _call(H, H.hpac_quality_noalloc, a, b, metric)
        _call(H, H.hpac_quality_noalloc, a64, b64, metric)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0


@pytest.mark.parametrize("metric", [0, 1, 2])
def test_small_case_matches_the_oracle(H, metric):
    import oracle
    rng = np.random.default_rng(40 + metric)
    n = 70_001
    a = rng.uniform(0.05, 3.0, n)
    a[rng.random(n) < 0.1] = 0.0
    b = (a * (1.0 + rng.normal(0.0, 0.02, n))).astype(np.float32)
    b[rng.random(n) < 0.05] = 0.5
    if metric == 2:                       # ids for the misclassification rate
        a = np.floor(a * 3.0)
        b = np.where(rng.random(n) < 0.07, a + 1.0, a).astype(np.float32)
    r = _call(H, H.hpac_quality_noalloc, torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda(),
              metric)
    val, aux = oracle.quality(a, b.astype(np.float64), metric)
    assert r["value"] == pytest.approx(val, rel=1e-6, abs=1e-300)
    if metric == 0:
        assert r["zeros"] == aux["zeros"] and r["zeros_mismatch"] == aux["zeros_mismatch"]
        assert r["zero_max_abs"] == aux["zero_max_abs"]


def test_at_the_fixed_limit(H):
    # n = 134,217,728 fills all 16,384 partial slots (the last one next to the
    # result slot) with exactly 32 elements per thread
    n = NOALLOC_MAX_N
    g = torch.Generator(device="cuda").manual_seed(5)
    a = torch.rand(n, dtype=torch.float64, device="cuda", generator=g) + 0.1
    a[: n // 16] = 0.0
    b = (a * (1.0 + 0.01 * torch.randn(n, dtype=torch.float64, device="cuda", generator=g))).float()
    b[n // 32: n // 16] = 0.0
    for metric in (0, 1):
        first = _call(H, H.hpac_quality_noalloc, a, b, metric)
        again = _call(H, H.hpac_quality_noalloc, a, b, metric)
        ref = _call(H, H.hpac_quality, a, b, metric)
        _same(first, ref)
        _same(again, ref)
    del a, b
    torch.cuda.empty_cache()

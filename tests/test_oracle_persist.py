"""Pins of the oracle's persistent TAF / iACT state (state kept across calls,
beyond the paper's kernel-scoped state): a sequence of calls whose sizes are
multiples of T equals one call over the concatenated iteration space, which is
the already-pinned kernel-scoped oracle; a first call from the empty state
equals the kernel-scoped call (no GPU)."""
import numpy as np
import pytest

from paper_2308_16877_gb300 import workloads as W

GAMMA = 5.0 / 3.0


def region_inputs(kind, n, seed=11):
    if kind == 0:
        return W.blackscholes_inputs(n, seed=seed), W.BS_RATE
    if kind == 1:
        return W.eos_inputs(n, seed=seed, smooth=16), GAMMA
    return W.identity_inputs(n, d=2, dtype=np.float64, kind="walk", seed=seed), 0.0


@pytest.mark.parametrize("kind", [0, 1, 3])
@pytest.mark.parametrize("level", [0, 1, 2])
@pytest.mark.parametrize("h,p,thr,reset", [(4, 8, 0.05, False), (3, 2, 0.5, True), (2, 5, np.inf, False)])
def test_taf_calls_equal_concatenation(orc, kind, level, h, p, thr, reset):
    T, B = 640, 128
    sizes = [3 * T, 5 * T, 2 * T]
    x, param = region_inputs(kind, sum(sizes))
    o, m, s, c = orc.run_taf(kind, x, param, h, p, thr, level=level, threads=T, block=B, reset=reset)
    st = orc.taf_state(T, h)
    parts, off = [], 0
    for nn in sizes:
        parts.append(orc.run_taf(kind, np.ascontiguousarray(x[:, off:off + nn]), param, h, p, thr,
                                 level=level, threads=T, block=B, reset=reset, state=st))
        off += nn
    assert np.array_equal(np.concatenate([q[1] for q in parts]), m)
    assert np.array_equal(np.concatenate([q[0] for q in parts]), o)
    assert np.array_equal(np.concatenate([q[2] for q in parts]), s, equal_nan=True)
    assert sum(q[3][1] for q in parts) == c[1]
    if kind == 3 or np.isinf(thr):   # the random-walk stream and thr = inf approximate
        assert c[1] > 0


@pytest.mark.parametrize("kind", [0, 1, 3])
@pytest.mark.parametrize("level", [0, 1, 2])
@pytest.mark.parametrize("ts,g", [(8, 32), (4, 4), (2, 1)])
def test_iact_calls_equal_concatenation(orc, kind, level, ts, g):
    T, B = 640, 128
    sizes = [2 * T, 4 * T, 3 * T]
    x, param = region_inputs(kind, sum(sizes))
    sc = W.iact_scale(x, x.shape[1])
    thr = 0.05 if kind != 1 else 0.02
    o, m, s, c = orc.run_iact(kind, x, param, ts, g, thr, level=level, in_scale=sc, threads=T, block=B)
    st = orc.iact_state(T, ts, g, x.shape[0])
    parts, off = [], 0
    for nn in sizes:
        parts.append(orc.run_iact(kind, np.ascontiguousarray(x[:, off:off + nn]), param, ts, g, thr,
                                  level=level, in_scale=sc, threads=T, block=B, state=st))
        off += nn
    assert np.array_equal(np.concatenate([q[1] for q in parts]), m)
    assert np.array_equal(np.concatenate([q[0] for q in parts]), o)
    assert sum(q[3][1] for q in parts) == c[1]


def test_empty_state_is_the_kernel_scoped_call(orc):
    n, T = 5000, 700   # N not a multiple of T: a single call is still the plain one
    x, param = region_inputs(0, n)
    a = orc.run_taf(0, x, param, 4, 8, 0.05, level=1, threads=T, block=64)
    b = orc.run_taf(0, x, param, 4, 8, 0.05, level=1, threads=T, block=64, state=orc.taf_state(T, 4))
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    sc = W.iact_scale(x, n)
    a = orc.run_iact(0, x, param, 8, 32, 0.05, level=1, in_scale=sc, threads=T, block=64)
    b = orc.run_iact(0, x, param, 8, 32, 0.05, level=1, in_scale=sc, threads=T, block=64,
                     state=orc.iact_state(T, 8, 32, 4))
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


def test_state_carries_memoization_across_calls(orc):
    """The same stream twice: the second call starts with full windows /
    tables, so it approximates at least as often as the first."""
    T = 512
    x = W.identity_inputs(8 * T, d=1, dtype=np.float64, kind="levels", seed=4)
    st = orc.taf_state(T, 4)
    c1 = orc.run_taf(3, x, 0.0, 4, 4, 0.5, threads=T, block=128, state=st)[3][1]
    c2 = orc.run_taf(3, x, 0.0, 4, 4, 0.5, threads=T, block=128, state=st)[3][1]
    assert c2 > c1
    sc = W.iact_scale(x, x.shape[1])
    st = orc.iact_state(T, 8, 32, 1)
    c1 = orc.run_iact(3, x, 0.0, 8, 32, 1e-3, in_scale=sc, threads=T, block=128, state=st)[3][1]
    c2 = orc.run_iact(3, x, 0.0, 8, 32, 1e-3, in_scale=sc, threads=T, block=128, state=st)[3][1]
    assert c2 > c1

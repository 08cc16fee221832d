"""Pins of the oracle's TAF (Section 2.3 state machine; GPU algorithm of
Section 3.1.3 / Figure 3(d); majority rules of Section 3.3) against a hand-worked
example, closed forms, numpy's moments and trace invariants (no GPU)."""
import os

import numpy as np
import pytest

from paper_2308_16877_gb300 import workloads as W

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def thread_trace(T, n, t):
    return np.arange(t, n, T)


def test_worked_example_h2p2(orc):
    rows = np.array([[float(v) for v in l.split()] for l in open(os.path.join(GOLD, "taf_worked_h2p2.txt"))
                     if l.strip() and not l.startswith("#")])
    x = rows[:, 0].astype(np.float32)[None, :]
    out, mask, stat, cnt = orc.run_taf(orc.IDENTITY, x, 0.0, 2, 2, 0.1, threads=1, block=32)
    assert np.array_equal(mask, rows[:, 2].astype(np.uint8))
    assert np.array_equal(out, rows[:, 1].astype(np.float32))
    assert cnt[1] == 4


@pytest.mark.parametrize("kind,dt", [(0, np.float32), (3, np.float32), (3, np.float64), (1, np.float64)])
def test_zero_threshold_is_exact(orc, kind, dt):
    n = 5000
    x = (W.blackscholes_inputs(n) if kind == 0 else W.eos_inputs(n) if kind == 1
         else W.identity_inputs(n, dtype=dt, kind="levels"))
    param = 0.02 if kind == 0 else 5 / 3 if kind == 1 else 0.0
    exact = orc.run_exact(kind, x, param)
    for level in (0, 1, 2):
        out, mask, _, cnt = orc.run_taf(kind, x, param, 4, 8, 0.0, level=level, threads=n // 8,
                                        block=128)
        assert np.array_equal(out, exact) and np.all(mask == 0) and cnt[1] == 0


def exact_count_inf(n, T, h, p):
    """Infinite threshold: per thread min(n_t, h) + floor(max(0, n_t - h) / (p + 1))."""
    tot = 0
    for t in range(min(T, n)):
        nt = (n - t + T - 1) // T
        tot += min(nt, h) + max(0, nt - h) // (p + 1)
    return tot


@pytest.mark.parametrize("n,T,h,p", [(1000, 10, 4, 8), (999, 100, 1, 1), (4096, 256, 5, 512),
                                     (333, 7, 3, 0), (50, 64, 2, 2)])
def test_infinite_threshold_closed_form(orc, n, T, h, p):
    x = W.identity_inputs(n, dtype=np.float64)
    out, mask, _, _ = orc.run_taf(orc.IDENTITY, x, 0.0, h, p, np.inf, threads=T, block=64)
    assert int((mask == 0).sum()) == exact_count_inf(n, T, h, p)
    # every prediction repeats the newest accurate output of its own thread
    for t in range(min(T, n)):
        idx = thread_trace(T, n, t)
        last = None
        for i in idx:
            if mask[i] == 0:
                last = out[i]
                assert out[i] == x[0, i]
            else:
                assert out[i] == last


def test_constant_stream_predicts_after_h(orc):
    n, T = 640, 64
    x = np.full((1, n), 1.25, dtype=np.float32)
    out, mask, stat, _ = orc.run_taf(orc.IDENTITY, x, 0.0, 4, 8, 1e-6, threads=T, block=64)
    assert int((mask == 0).sum()) == exact_count_inf(n, T, 4, 8)
    assert np.all(stat[(mask == 0) & ~np.isnan(stat)] == 0.0)
    # all-zero windows: 0/0 reads as RSD 0, so they are stable too
    z = np.zeros((1, n), dtype=np.float32)
    _, mask0, _, _ = orc.run_taf(orc.IDENTITY, z, 0.0, 4, 8, 1e-6, threads=T, block=64)
    assert np.array_equal(mask0, mask)


@pytest.mark.parametrize("dt", [np.float32, np.float64])
def test_rsd_and_transitions_match_trace(orc, dt):
    """At every accurate step with a full window the statistic equals numpy's
    population std / |mean| of the thread's last h accurate outputs; a thread
    enters exactly p predictions after a statistic below the threshold and
    none otherwise (thread level)."""
    n, T, h, p, thr = 20000, 250, 3, 5, 0.02
    x = W.identity_inputs(n, dtype=dt, kind="walk")
    out, mask, stat, cnt = orc.run_taf(orc.IDENTITY, x, 0.0, h, p, thr, threads=T, block=64)
    rtol = 1e-5 if dt == np.float32 else 1e-12
    n_checked = 0
    for t in range(T):
        idx = thread_trace(T, n, t)
        hist = []
        owed = 0
        for i in idx:
            if owed > 0:
                assert mask[i] == 1 and out[i] == hist[-1]
                owed -= 1
                continue
            assert mask[i] == 0 and out[i] == x[0, i]
            hist.append(float(out[i]))
            if len(hist) >= h:
                w = np.array(hist[-h:])
                ref = w.std() / abs(w.mean())
                assert stat[i] == pytest.approx(ref, rel=rtol, abs=1e-30)
                n_checked += 1
                if stat[i] < thr:
                    owed = p
            else:
                assert np.isnan(stat[i])
    assert n_checked > 1000
    assert cnt[1] == int((mask == 1).sum()) > 100


def lanes_input(n_steps, T, lane_values):
    """x[t + k*T] = lane_values[t][k]: each logical thread its own stream."""
    x = np.zeros((1, n_steps * T), dtype=np.float32)
    for t in range(T):
        x[0, t::T] = lane_values[t]
    return x


def test_warp_level_majority(orc):
    T, steps, h, p, thr = 32, 40, 2, 3, 0.01
    stable = np.full(steps, 1.0, dtype=np.float32)
    # alternating 1, 3, 1, ...: every window of two has RSD 0.5
    unstable = lambda: np.where(np.arange(steps) % 2 == 0, 1.0, 3.0).astype(np.float32)
    # 16 stable + 16 unstable: a tie is not a majority, nobody predicts
    x = lanes_input(steps, T, [stable if t < 16 else unstable() for t in range(T)])
    _, mask, _, _ = orc.run_taf(orc.IDENTITY, x, 0.0, h, p, thr, level=orc.WARP, threads=T, block=32)
    assert np.all(mask == 0)
    # thread level: only the stable lanes predict
    _, mt, _, _ = orc.run_taf(orc.IDENTITY, x, 0.0, h, p, thr, level=orc.THREAD, threads=T, block=32)
    per = mt.reshape(steps, T)
    assert np.all(per[:, 16:] == 0) and np.any(per[:, :16] == 1)
    # 17 stable: the whole warp predicts, in lock-step with the stable lanes
    x = lanes_input(steps, T, [stable if t < 17 else unstable() for t in range(T)])
    out, mask, _, _ = orc.run_taf(orc.IDENTITY, x, 0.0, h, p, thr, level=orc.WARP, threads=T, block=32)
    per = mask.reshape(steps, T)
    assert np.all(per == per[:, :1])
    assert int((per[:, 0] == 0).sum()) == min(steps, h) + max(0, steps - h) // (p + 1)
    # a forced (unstable) lane outputs its own newest accurate value
    o = out.reshape(steps, T)
    for k in range(steps):
        if per[k, 0] == 1:
            j = max(kk for kk in range(k) if per[kk, 0] == 0)
            assert o[k, 20] == x[0, j * T + 20]


def test_block_level_majority_and_reduction_to_warp(orc):
    T, steps, h, p, thr = 64, 30, 2, 4, 0.01
    stable = np.full(steps, 2.0, dtype=np.float32)
    alt = np.where(np.arange(steps) % 2 == 0, 1.0, 3.0).astype(np.float32)
    mk = lambda ns: lanes_input(steps, T, [stable if t < ns else alt for t in range(T)])
    x = mk(32)   # warp 0 all stable, warp 1 all unstable: 32 of 64 is a tie
    _, mb, _, _ = orc.run_taf(orc.IDENTITY, x, 0.0, h, p, thr, level=orc.BLOCK, threads=T, block=64)
    assert np.all(mb == 0)
    _, mw, _, _ = orc.run_taf(orc.IDENTITY, x, 0.0, h, p, thr, level=orc.WARP, threads=T, block=64)
    assert np.any(mw.reshape(steps, T)[:, :32] == 1) and np.all(mw.reshape(steps, T)[:, 32:] == 0)
    x = mk(33)
    _, mb, _, _ = orc.run_taf(orc.IDENTITY, x, 0.0, h, p, thr, level=orc.BLOCK, threads=T, block=64)
    per = mb.reshape(steps, T)
    assert np.all(per == per[:, :1]) and np.any(per == 1)
    # block of one warp == warp level
    x = W.identity_inputs(5000, kind="walk")
    a = orc.run_taf(orc.IDENTITY, x, 0.0, 3, 4, 0.005, level=orc.BLOCK, threads=640, block=32)
    b = orc.run_taf(orc.IDENTITY, x, 0.0, 3, 4, 0.005, level=orc.WARP, threads=640, block=32)
    assert all(np.array_equal(u, v, equal_nan=True) for u, v in zip(a, b))


def test_identical_lanes_all_levels_agree(orc):
    """When every lane of a block sees the same stream, thread, warp and block
    level take the same decisions."""
    T, steps = 128, 50
    s = W.identity_inputs(steps, kind="walk")[0]
    x = lanes_input(steps, T, [s] * T)
    res = [orc.run_taf(orc.IDENTITY, x, 0.0, 3, 5, 0.002, level=lv, threads=T, block=128)
           for lv in (0, 1, 2)]
    for r in res[1:]:
        assert np.array_equal(r[1], res[0][1]) and np.array_equal(r[0], res[0][0])
    assert np.any(res[0][1] == 1)


def test_tail_threads_and_ragged_grid(orc):
    """T not a multiple of the warp or block size and N not a multiple of T."""
    n, T = 1000, 77
    x = W.identity_inputs(n, dtype=np.float64, kind="walk")
    for level in (0, 1, 2):
        out, mask, _, cnt = orc.run_taf(orc.IDENTITY, x, 0.0, 2, 3, np.inf, level=level,
                                        threads=T, block=64)
        assert np.all(mask <= 1)
        assert int((mask == 0).sum()) == exact_count_inf(n, T, 2, 3) or level > 0
        assert cnt[0] == n


def test_rejects_bad_knobs(orc):
    x = W.identity_inputs(10)
    for h, p, thr, lv in ((0, 1, 0.1, 0), (65, 1, 0.1, 0), (2, -1, 0.1, 0), (2, 1, -0.1, 0),
                          (2, 1, np.nan, 0), (2, 1, 0.1, 3)):
        with pytest.raises(ValueError):
            orc.run_taf(orc.IDENTITY, x, 0.0, h, p, thr, level=lv)


@pytest.mark.parametrize("level", [0, 1, 2])
def test_replay_of_own_mask_agrees_everywhere(orc, level):
    """Replaying the oracle's own mask reproduces its outputs and statistics
    bit for bit, with no disagreement and no structural error."""
    n, T = 20000, 2500
    x = W.blackscholes_inputs(n)
    out, mask, stat, cnt = orc.run_taf(0, x, W.BS_RATE, 4, 8, 0.05, level=level, threads=T, block=128)
    o2, s2, dis, counts = orc.replay_taf(0, x, W.BS_RATE, 4, 8, 0.05, mask, level=level, threads=T,
                                         block=128)
    assert np.array_equal(out, o2) and np.array_equal(stat, s2, equal_nan=True)
    assert counts[1] == 0 and counts[2] == 0 and not dis.any()
    # every accurate step with a successor is a compared decision point
    assert counts[0] == np.count_nonzero(mask[:n - T] == 0)


def test_replay_flags_a_flipped_decision_and_a_broken_run(orc):
    """A prediction run removed from the mask is one disagreement at its
    decision invocation (later ones may follow on the changed path); an
    approximation before the window is full lengthens the next run past p,
    a structural error."""
    n, T, h, p = 4096, 64, 2, 3
    x = W.identity_inputs(n, d=1, dtype=np.float64, kind="levels")
    out, mask, stat, cnt = orc.run_taf(3, x, 0.0, h, p, 0.5, threads=T, block=64)
    t = next(t for t in range(T) if np.any(mask[t::T] == 1))
    seq = np.arange(t, n, T)
    k = int(np.argmax(mask[seq] == 1))          # first approximated step of lane t
    flipped = mask.copy()
    flipped[seq[k:k + p]] = 0
    _, _, dis, counts = orc.replay_taf(3, x, 0.0, h, p, 0.5, flipped, threads=T, block=64)
    assert dis[seq[k - 1]] == 1 and counts[1] >= 1 and counts[2] == 0
    assert mask[seq[1]] == 0                    # the window is still filling
    broken = mask.copy()
    broken[seq[1]] = 1                          # a prediction nothing could have owed
    _, _, _, counts = orc.replay_taf(3, x, 0.0, h, p, 0.5, broken, threads=T, block=64)
    assert counts[2] >= 1


@pytest.mark.parametrize("n,T,h,p", [(1000, 10, 4, 8), (999, 100, 1, 1), (4096, 256, 5, 3),
                                     (333, 7, 3, 0), (50, 64, 2, 2)])
@pytest.mark.parametrize("level", [0, 1, 2])
def test_reset_on_exit_closed_form(orc, n, T, h, p, level):
    """Alternative reading (window emptied when a prediction run ends) at
    thr = +inf: each thread repeats h accurate steps then p predictions, so its
    accurate count is h floor(n_t/(h+p)) + min(h, n_t mod (h+p)); all lanes of a
    group share the pattern, so the levels agree."""
    x = W.identity_inputs(n, dtype=np.float64)
    out, mask, _, _ = orc.run_taf(orc.IDENTITY, x, 0.0, h, p, np.inf, level=level, threads=T,
                                  block=64, reset=True)
    want = 0
    for t in range(min(T, n)):
        nt = len(thread_trace(T, n, t))
        want += h * (nt // (h + p)) + min(h, nt % (h + p))
    assert int((mask == 0).sum()) == want
    if p > 0 and h > 1 and n // T > h + p:  # with h = 1 the two readings coincide
        keep = orc.run_taf(orc.IDENTITY, x, 0.0, h, p, np.inf, level=level, threads=T, block=64)[1]
        assert int((keep == 0).sum()) < want    # the kept window re-tests after one step

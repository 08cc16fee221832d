"""Pins of the oracle's iACT (Section 2.3; tables shared within a warp, Section
3.1.4; read/write phases, farthest-lane writer and round-robin replacement,
Section 3.3) against closed forms, a nearest-neighbour brute force and an
independent small-case simulation written in Python (no GPU)."""
import os

import numpy as np
import pytest

from paper_2308_16877_gb300 import workloads as W

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def test_worked_example_two_entry_table(orc):
    """tests/golden/iact_worked_t2.txt, worked by hand: reuse below the
    threshold, exact computation and a round-robin write otherwise."""
    rows = [l.split() for l in open(os.path.join(GOLD, "iact_worked_t2.txt"))
            if l.strip() and not l.startswith("#")]
    x = np.array([[float(r[0]) for r in rows]], dtype=np.float32)
    out, mask, stat, cnt = orc.run_iact(orc.IDENTITY, x, 0.0, 2, 32, 0.1, in_scale=[1.0], threads=1,
                                        block=32)
    assert np.array_equal(out, np.array([float(r[1]) for r in rows], dtype=np.float32))
    assert np.array_equal(mask, np.array([int(r[2]) for r in rows], dtype=np.uint8))
    want = np.array([float(r[3]) for r in rows])
    assert np.isinf(stat[0]) and np.allclose(stat[1:], want[1:], rtol=0, atol=2e-6)
    assert cnt[1] == 4


@pytest.mark.parametrize("kind", [0, 1, 3])
def test_zero_threshold_is_exact(orc, kind):
    n = 4000
    x = (W.blackscholes_inputs(n) if kind == 0 else W.eos_inputs(n) if kind == 1
         else W.identity_inputs(n, d=2, kind="levels"))
    param = 0.02 if kind == 0 else 5 / 3 if kind == 1 else 0.0
    exact = orc.run_exact(kind, x, param)
    sc = W.iact_scale(x, n)
    for g in (1, 4, 32):
        for lv in (0, 1, 2):
            out, mask, _, cnt = orc.run_iact(kind, x, param, 4, g, 0.0, level=lv, in_scale=sc,
                                             threads=n // 8, block=64)
            assert np.array_equal(out, exact) and np.all(mask == 0) and cnt[1] == 0


def test_infinite_threshold_single_slot_private(orc):
    """thr = inf, one private slot: each thread computes its first invocation and
    repeats that output ever after."""
    n, T = 3000, 100
    x = W.identity_inputs(n, d=3, kind="uniform")
    out, mask, stat, _ = orc.run_iact(orc.IDENTITY, x, 0.0, 1, 32, np.inf, threads=T, block=64)
    k = np.arange(n) // T
    assert np.array_equal(mask == 0, k == 0)
    first = x[0, np.arange(n) % T]
    assert np.array_equal(out, first)
    assert np.all(np.isinf(stat[k == 0])) and np.all(np.isfinite(stat[k > 0]))


def test_identical_inputs_hit_after_first_write(orc):
    n, T = 2048, 64
    x = np.full((2, n), 0.75, dtype=np.float32)
    for g in (1, 2, 32):
        _, mask, stat, _ = orc.run_iact(orc.IDENTITY, x, 0.0, 2, g, 1e-6, threads=T, block=64)
        k = np.arange(n) // T
        assert np.array_equal(mask == 0, k == 0), g
        assert np.all(stat[k > 0] == 0.0)


def test_unbounded_private_table_is_nearest_neighbour(orc):
    """With a private table larger than the thread's trip count nothing is ever
    evicted, so the statistic is the nearest-neighbour distance to all of the
    thread's earlier exactly computed inputs (brute force), and a hit returns
    that neighbour's output."""
    n, T, D = 24 * 40, 40, 2
    x = W.identity_inputs(n, d=D, kind="levels", dtype=np.float64)
    x[1] *= 3.0
    sc = W.iact_scale(x, n)
    thr = 0.3
    out, mask, stat, _ = orc.run_iact(orc.IDENTITY, x, 0.0, 32, 32, thr, in_scale=sc, threads=T,
                                      block=64)
    z = (sc[:, None] * x).astype(np.float32).astype(np.float64)
    for t in range(T):
        seen = []
        for i in range(t, n, T):
            if seen:
                d = [np.sqrt(((z[:, i] - z[:, j]) ** 2).sum()) for j in seen]
                j = int(np.argmin(d))
                assert stat[i] == pytest.approx(d[j], rel=1e-6, abs=1e-7)
                if mask[i] == 1:
                    assert d[j] < thr + 1e-6 and out[i] == out[seen[j]]
                else:
                    assert d[j] >= thr - 1e-6
            else:
                assert mask[i] == 0 and np.isinf(stat[i])
            if mask[i] == 0:
                assert out[i] == x[0, i]
                seen.append(i)


def simulate(x, T, B, tsize, g, thr, level):
    """Independent small-case iACT simulation (single-precision distances)."""
    D, n = x.shape
    L = 32 // g
    f = np.float32
    z = x.astype(f)                     # identity region, unit scale
    out = np.zeros(n, dtype=x.dtype)
    mask = np.zeros(n, dtype=np.uint8)
    tables = {}                          # (block, warp, table) -> dict
    for b in range((T + B - 1) // B):
        k = 0
        while b * B + k * T < n:
            info = {}
            for lane in range(B):
                t, i = b * B + lane, b * B + lane + k * T
                if t >= T or i >= n:
                    continue
                key = (b, lane // 32, (lane % 32) // L)
                tab = tables.setdefault(key, {"slots": [None] * tsize, "rr": 0})
                best, bj = None, None
                for j, s in enumerate(tab["slots"]):
                    if s is None:
                        continue
                    acc = f(0)
                    for dd in range(D):
                        df = f(z[dd, i] - s[0][dd])
                        acc = f(acc + f(df * df))
                    if best is None or acc < best:
                        best, bj = acc, j
                dmin = np.float32(np.inf) if best is None else np.sqrt(best)
                info[lane] = dict(i=i, key=key, has=best is not None, d=dmin, j=bj,
                                  want=best is not None and dmin < f(thr))
            groups = {}
            for lane, v in info.items():
                gk = lane if level == 0 else lane // 32 if level == 1 else 0
                groups.setdefault(gk, []).append(v)
            for members in groups.values():
                maj = 2 * sum(m["want"] for m in members) > len(members)
                for m in members:
                    m["apx"] = m["want"] if level == 0 else (maj and m["has"])
            writers = {}
            for lane in sorted(info):
                m = info[lane]
                i = m["i"]
                if m["apx"]:
                    out[i] = tables[m["key"]]["slots"][m["j"]][1]
                    mask[i] = 1
                else:
                    out[i] = x[0, i]
                    w = writers.get(m["key"])
                    if w is None or m["d"] > w["d"]:
                        writers[m["key"]] = m
            for key, m in writers.items():
                tab = tables[key]
                tab["slots"][tab["rr"]] = (z[:, m["i"]].copy(), out[m["i"]])
                tab["rr"] = (tab["rr"] + 1) % tsize
            k += 1
    return out, mask


@pytest.mark.parametrize("g", [1, 2, 4, 32])
@pytest.mark.parametrize("level", [0, 1, 2])
@pytest.mark.parametrize("D,tsize", [(1, 1), (1, 3), (2, 2), (2, 4)])
def test_matches_independent_simulation(orc, g, level, D, tsize):
    rng = np.random.default_rng(100 * g + 10 * level + D)
    T, B, n = 48, 64, 48 * 9 + 17
    x = (1.0 + 0.125 * rng.integers(0, 3, size=(D, n))).astype(np.float32)
    thr = 0.13
    ref_out, ref_mask = simulate(x, T, B, tsize, g, thr, level)
    out, mask, _, _ = orc.run_iact(orc.IDENTITY, x, 0.0, tsize, g, thr, level=level, threads=T, block=B)
    assert np.array_equal(mask, ref_mask)
    assert np.array_equal(out, ref_out)
    assert mask.sum() < n
    if level == 0 or g == 32:
        assert mask.sum() > 0


def test_warp_majority_forces_minority_lanes(orc):
    """16 lanes with repeating inputs and 16 with fresh ones tie (no approximation);
    17 repeating lanes form a majority, and every lane holding a valid slot then
    takes its nearest slot's output."""
    T, steps = 32, 6
    for n_rep, expect_any in ((16, False), (17, True)):
        x = np.zeros((1, T * steps), dtype=np.float32)
        for t in range(T):
            x[0, t::T] = 1.0 if t < n_rep else 1.0 + t + 40.0 * np.arange(steps)
        out, mask, _, _ = orc.run_iact(orc.IDENTITY, x, 0.0, 1, 32, 0.01, level=orc.WARP,
                                       threads=T, block=32)
        per = mask.reshape(steps, T)
        assert np.all(per[0] == 0)
        if expect_any:
            assert np.all(per[1:] == 1)
            o = out.reshape(steps, T)
            assert np.all(o[1:, 20] == x[0, 20])     # forced lane repeats its slot
        else:
            assert np.all(per == 0)


def test_rejects_bad_knobs(orc):
    x = W.identity_inputs(10)
    for ts, g, thr, lv in ((0, 32, 0.1, 0), (65, 32, 0.1, 0), (2, 3, 0.1, 0), (2, 64, 0.1, 0),
                           (2, 32, -1.0, 0), (2, 32, np.nan, 0), (2, 32, 0.1, 5)):
        with pytest.raises(ValueError):
            orc.run_iact(orc.IDENTITY, x, 0.0, ts, g, thr, level=lv)

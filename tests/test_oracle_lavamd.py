"""Pins of the LavaMD-style neighbour-box force oracle (oracle/lavamd_oracle.c)
against results fixed independently of it: a numpy brute force over all pairs
of particles whose boxes touch, closed forms for one and two particles, the
invocation count (3B - 2)^3 NP, and the TAF / iACT limits thr = 0 and
thr = +inf, where every decision is known in advance."""
import numpy as np
import pytest

import oracle

A2 = 0.5


def inputs(B, NP, seed):
    rng = np.random.default_rng(seed)
    return rng.uniform(0.1, 1.0, (4, B ** 3 * NP))


def brute_force(B, NP, rq, a2=A2):
    """fv by all pairs (p, j) whose boxes differ by at most one in every
    coordinate: a different formulation from the oracle's neighbour list."""
    P = B ** 3 * NP
    box = np.arange(P) // NP
    bc = np.stack([box % B, (box // B) % B, box // (B * B)])
    near = np.all(np.abs(bc[:, :, None] - bc[:, None, :]) <= 1, axis=0)
    d = rq[:3, :, None] - rq[:3, None, :]
    v = np.exp(-a2 * np.sum(d * d, axis=0)) * near
    q = rq[3][None, :]
    return np.concatenate([np.sum(q * v, axis=1)[None], np.sum(q[None] * 2 * v[None] * d, axis=2)])


def per_invocation(B, NP, rq, a2=A2):
    """y[p][k]: box k's contribution (4 values) in the oracle's neighbour order,
    formed by numpy from the pair terms."""
    P = B ** 3 * NP
    out = []
    for p in range(P):
        h = p // NP
        hx, hy, hz = h % B, (h // B) % B, h // (B * B)
        seq = [h] + [((hz + dz) * B + hy + dy) * B + hx + dx
                     for dz in (-1, 0, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1)
                     if (dx, dy, dz) != (0, 0, 0) and 0 <= hx + dx < B and 0 <= hy + dy < B
                     and 0 <= hz + dz < B]
        ys = []
        for b in seq:
            j = np.arange(b * NP, (b + 1) * NP)
            d = rq[:3, p][:, None] - rq[:3, j]
            v = np.exp(-a2 * np.sum(d * d, axis=0))
            ys.append(np.concatenate([[np.sum(rq[3, j] * v)], np.sum(rq[3, j] * 2 * v * d, axis=1)]))
        out.append(ys)
    return out


@pytest.mark.parametrize("B,NP", [(1, 5), (2, 3), (3, 7), (4, 2)])
def test_exact_equals_the_pairwise_brute_force(B, NP):
    rq = inputs(B, NP, 10 * B + NP)
    fv, cnt, _ = oracle.lavamd(B, NP, A2, rq)
    ref = brute_force(B, NP, rq)
    scale = np.abs(ref).max()
    assert np.abs(fv - ref).max() <= 1e-13 * scale
    assert cnt[0] == (3 * B - 2) ** 3 * NP if B >= 2 else cnt[0] == NP


def test_one_particle_feels_only_itself():
    rq = np.array([[0.3], [0.6], [0.2], [0.7]])
    fv, cnt, _ = oracle.lavamd(1, 1, A2, rq)
    assert fv[:, 0].tolist() == [0.7, 0.0, 0.0, 0.0]
    assert cnt.tolist() == [1, 0, 0, 0]


def test_two_particles_closed_form():
    r0, r1, q0, q1 = np.array([0.2, 0.5, 0.9]), np.array([0.7, 0.1, 0.4]), 0.3, 0.8
    rq = np.array([[r0[0], r1[0]], [r0[1], r1[1]], [r0[2], r1[2]], [q0, q1]])
    fv, _, _ = oracle.lavamd(1, 2, A2, rq)
    e = np.exp(-A2 * np.sum((r0 - r1) ** 2))
    assert fv[0, 0] == pytest.approx(q0 + q1 * e, rel=1e-15)
    assert fv[1:, 0] == pytest.approx(q1 * 2 * e * (r0 - r1), rel=1e-15)
    assert fv[1:, 1] == pytest.approx(q0 * 2 * e * (r1 - r0), rel=1e-15)


def test_boxes_that_do_not_touch_do_not_interact():
    # one particle in each of 27 boxes: the corner boxes (0,0,0) and (2,2,2) are
    # two boxes apart; every particle feels exactly the boxes that touch its own
    B = 3
    rq = inputs(B, 1, 3)
    fv, _, _ = oracle.lavamd(B, 1, A2, rq)
    ref = brute_force(B, 1, rq)
    assert np.abs(fv - ref).max() <= 1e-14 * np.abs(ref).max()
    corner = 0
    far = 26
    d = rq[:3, corner] - rq[:3, far]
    alone = brute_force(B, 1, rq)[0, corner]
    with_far = alone + rq[3, far] * np.exp(-A2 * d @ d)
    assert fv[0, corner] == pytest.approx(alone, rel=1e-14) and fv[0, corner] != pytest.approx(with_far, rel=1e-9)


@pytest.mark.parametrize("technique", [oracle.LAVAMD_TAF, oracle.LAVAMD_IACT])
@pytest.mark.parametrize("level", [oracle.THREAD, oracle.WARP, oracle.BLOCK])
def test_threshold_zero_is_exact(technique, level):
    B, NP = 3, 40
    rq = inputs(B, NP, 5)
    ex, _, mex = oracle.lavamd(B, NP, A2, rq, mask=True)
    fv, cnt, m = oracle.lavamd(B, NP, A2, rq, technique=technique, level=level, thresh=0.0,
                               tperwarp=4, mask=True)
    assert np.array_equal(fv, ex)
    assert cnt[1] == 0 and np.array_equal(m, mex)


def taf_inf_count(nn, h, p):
    """Approximated invocations of one particle under TAF with thr = +inf:
    h accurate outputs fill the window, then p predictions and one accurate
    output alternate."""
    if nn <= h:
        return 0
    r = nn - h
    return (r // (p + 1)) * p + min(r % (p + 1), p)


@pytest.mark.parametrize("h,p", [(1, 1), (2, 3), (4, 8), (5, 0), (30, 2)])
def test_taf_infinite_threshold_closed_form(h, p):
    B, NP = 3, 6
    rq = inputs(B, NP, 7)
    fv, cnt, m = oracle.lavamd(B, NP, A2, rq, technique=oracle.LAVAMD_TAF, hsize=h, psize=p,
                               thresh=np.inf, mask=True)
    ys = per_invocation(B, NP, rq)
    P = B ** 3 * NP
    expect_fv = np.zeros((4, P))
    total = 0
    for q in range(P):
        nn = len(ys[q])
        total += taf_inf_count(nn, h, p)
        acc, newest, k = np.zeros(4), None, 0
        pattern = []
        while k < nn:
            if k < h:
                pattern.append(0)
                k += 1
                continue
            run = min(p, nn - k)
            pattern += [1] * run
            k += run
            if k < nn:
                pattern.append(0)
                k += 1
        for k, apx in enumerate(pattern):
            if not apx:
                newest = ys[q][k]
            acc = acc + newest
            assert m[k * P + q] == apx
        expect_fv[:, q] = acc
        assert all(m[k * P + q] == 255 for k in range(nn, 27))
    assert cnt[0] == (3 * B - 2) ** 3 * NP and cnt[1] == total
    assert np.abs(fv - expect_fv).max() <= 1e-13 * np.abs(expect_fv).max()


def test_iact_infinite_threshold_private_tables_repeat_the_home_box():
    B, NP = 3, 9
    rq = inputs(B, NP, 8)
    fv, cnt, m = oracle.lavamd(B, NP, A2, rq, technique=oracle.LAVAMD_IACT, tsize=4, tperwarp=32,
                               thresh=np.inf, mask=True)
    ys = per_invocation(B, NP, rq)
    P = B ** 3 * NP
    expect = np.stack([len(ys[q]) * ys[q][0] for q in range(P)], axis=1)
    assert cnt[1] == cnt[0] - P
    assert np.abs(fv - expect).max() <= 1e-13 * np.abs(expect).max()
    assert all(m[q] == 0 for q in range(P))
    assert all(m[k * P + q] == 1 for q in range(P) for k in range(1, len(ys[q])))


@pytest.mark.parametrize("technique,knobs", [
    (oracle.LAVAMD_TAF, dict(hsize=3, psize=4, thresh=0.05)),
    (oracle.LAVAMD_IACT, dict(tsize=4, tperwarp=1, thresh=0.3)),
])
def test_one_lane_groups_make_warp_and_block_level_the_thread_level(technique, knobs):
    # one particle per box: every warp and block has one active lane, so the
    # majority of its deciding lanes is that lane's own decision
    B = 4
    rq = inputs(B, 1, 9)
    res = [oracle.lavamd(B, 1, A2, rq, technique=technique, level=lv, mask=True, **knobs)
           for lv in (oracle.THREAD, oracle.WARP, oracle.BLOCK)]
    assert res[0][1][1] > 0
    for fv, cnt, m in res[1:]:
        assert np.array_equal(fv, res[0][0]) and np.array_equal(m, res[0][2])
        assert cnt.tolist() == res[0][1].tolist()


def test_rejects_bad_arguments():
    rq = inputs(2, 3, 1)
    with pytest.raises(ValueError):
        oracle.lavamd(2, 3, A2, rq, technique=oracle.LAVAMD_TAF, hsize=0)
    with pytest.raises(ValueError):
        oracle.lavamd(2, 3, A2, rq, technique=oracle.LAVAMD_IACT, tperwarp=3)
    with pytest.raises(ValueError):
        oracle.lavamd(2, 0, A2, rq[:, :0])


@pytest.mark.parametrize("h,p,thr", [(3, 2, 0.05), (4, 8, 0.08), (2, 1, 0.02)])
def test_taf_thread_level_decisions_follow_numpy_rsd(h, p, thr):
    """Thread level, a threshold that some windows pass: every decision
    replayed from the per-invocation potentials with numpy's population
    standard deviation over |mean|."""
    B, NP = 3, 8
    rq = inputs(B, NP, 11)
    fv, cnt, m = oracle.lavamd(B, NP, A2, rq, technique=oracle.LAVAMD_TAF, hsize=h, psize=p,
                               thresh=thr, mask=True)
    ys = per_invocation(B, NP, rq)
    P = B ** 3 * NP
    n_apx = 0
    for q in range(P):
        win, pred, acc = [], 0, np.zeros(4)
        for k, y in enumerate(ys[q]):
            if pred > 0:
                assert m[k * P + q] == 1
                acc = acc + win[-1]
                pred -= 1
                n_apx += 1
                continue
            assert m[k * P + q] == 0
            acc = acc + y
            win = (win + [y])[-h:]
            if len(win) == h:
                pots = np.array([w[0] for w in win])
                s = np.std(pots) / abs(np.mean(pots))
                assert abs(s - thr) > 1e-9 * thr
                if s < thr:
                    pred = p
        assert np.abs(fv[:, q] - acc).max() <= 1e-12 * np.abs(acc).max()
    assert cnt[1] == n_apx and n_apx > 0


def line_of_four(B, xs, charges=None):
    """NP = 4 particles per box at x = xs (y = z = 0.5) in every box; charges
    [box][particle] or all 0.5."""
    NP = len(xs)
    nbox = B ** 3
    rq = np.zeros((4, nbox * NP))
    for b in range(nbox):
        for j, x in enumerate(xs):
            p = b * NP + j
            rq[:, p] = [x, 0.5, 0.5, 0.5 if charges is None else charges[b][j]]
    return rq


@pytest.mark.parametrize("level", [oracle.THREAD, oracle.WARP, oracle.BLOCK])
def test_iact_shared_table_writes_the_farthest_exact_lane(level):
    """Four particles on a line (x = 0.10, 0.11, 0.60, 0.90) in each of the 8
    boxes of a 2^3 grid, one table for the warp, threshold 0.2. The entries
    each rule stores, worked out by hand:
      k = 0: the table is empty, all compute; the writer is lane 0 (all
             distances +inf, lowest lane) -> entry A (x = 0.10).
      thread level: k = 1: lanes 0, 1 hit A; lanes 2, 3 compute; the writer is
             lane 3 (0.8 from A against 0.5) -> entry D. k = 2: lane 3 hits D,
             lane 2 (0.3 from D) computes and writes C. Later every lane hits.
      warp or block level (the block is the one warp): k = 1: 2 of 4 lanes
             want, no majority, all compute, lane 3 writes D. k = 2: lanes 0,
             1, 3 want; the majority makes lane 2 take its nearest entry, D.
    """
    B, xs = 2, [0.10, 0.11, 0.60, 0.90]
    rq = line_of_four(B, xs)
    fv, cnt, m = oracle.lavamd(B, 4, A2, rq, technique=oracle.LAVAMD_IACT, level=level, tsize=4,
                               tperwarp=1, thresh=0.2, mask=True)
    ys = per_invocation(B, 4, rq)
    P = 8 * 4
    for h in range(8):
        y = [ys[h * 4 + j] for j in range(4)]
        if level == oracle.THREAD:
            expect = [8 * y[0][0],
                      y[1][0] + 7 * y[0][0],
                      y[2][0] + y[2][1] + 6 * y[2][2],
                      y[3][0] + 7 * y[3][1]]
            apx = [[0] + [1] * 7, [0] + [1] * 7, [0, 0, 0] + [1] * 5, [0, 0] + [1] * 6]
        else:
            expect = [7 * y[0][0] + y[0][1],
                      y[1][0] + y[1][1] + 6 * y[0][0],
                      y[2][0] + y[2][1] + 6 * y[3][1],
                      y[3][0] + 7 * y[3][1]]
            apx = [[0, 0] + [1] * 6] * 4
        for j in range(4):
            p = h * 4 + j
            assert np.abs(fv[:, p] - expect[j]).max() <= 1e-13 * np.abs(expect[j]).max()
            assert [int(m[k * P + p]) for k in range(8)] == apx[j]


@pytest.mark.parametrize("steady", [3, 2])
@pytest.mark.parametrize("level", [oracle.THREAD, oracle.WARP, oracle.BLOCK])
def test_taf_majority_forces_the_minority(level, steady):
    """Four particles 0.2 apart with a2 = 1000, so each feels only its own
    index in every box (cross terms e^-40). Particle j's potential from box b
    is then its charge c[b][j]: 1 for j = 0, 1, 2 (window RSD ~ 0) and 2^b for
    j = 3 (any two boxes differ twofold: RSD >= 1/3). h = 2, p = 2, threshold
    0.1, 8 invocations each. Lanes 0-2 want to predict whenever their window
    is full: exact, exact, 2 predicted, exact, 2 predicted, exact. Lane 3
    never wants: at thread level it computes all 8; at warp and block level
    the 3-of-4 majority makes it follow the same pattern, repeating its
    newest exact output. With two steady lanes (2 of 4 is no majority) warp
    and block level predict nothing."""
    B, xs = 2, [0.1, 0.3, 0.5, 0.7]
    ch = [[1.0 if j < steady else 2.0 ** b for j in range(4)] for b in range(8)]
    rq = line_of_four(B, xs, ch)
    fv, cnt, m = oracle.lavamd(B, 4, 1000.0, rq, technique=oracle.LAVAMD_TAF, level=level, hsize=2, psize=2,
                               thresh=0.1, mask=True)
    ys = per_invocation(B, 4, rq, a2=1000.0)
    P = 32
    pattern = [0, 0, 1, 1, 0, 1, 1, 0]
    for h in range(8):
        for j in range(4):
            p = h * 4 + j
            if level == oracle.THREAD:
                pat = pattern if j < steady else [0] * 8
            else:
                pat = pattern if steady == 3 else [0] * 8
            acc, newest = np.zeros(4), None
            for k, a in enumerate(pat):
                if not a:
                    newest = ys[p][k]
                acc = acc + newest
            assert [int(m[k * P + p]) for k in range(8)] == pat
            assert np.abs(fv[:, p] - acc).max() <= 1e-13 * np.abs(acc).max()
    assert cnt[3] == 0


@pytest.mark.parametrize("h,p", [(1, 1), (2, 3), (3, 2), (4, 8)])
def test_taf_infinite_threshold_with_the_window_emptied_after_a_run(h, p):
    """The reset-on-exit reading: after p predictions the window is emptied,
    so h accurate outputs refill it before the next run. With thr = +inf the
    pattern is (h exact, p predicted) repeated."""
    B, NP = 3, 5
    rq = inputs(B, NP, 12)
    fv, cnt, m = oracle.lavamd(B, NP, A2, rq, technique=oracle.LAVAMD_TAF, hsize=h, psize=p,
                               thresh=np.inf, reset=1, mask=True)
    ys = per_invocation(B, NP, rq)
    P = B ** 3 * NP
    total = 0
    for q in range(P):
        nn = len(ys[q])
        pat = [0 if k % (h + p) < h else 1 for k in range(nn)]
        total += sum(pat)
        acc, newest = np.zeros(4), None
        for k, a in enumerate(pat):
            if not a:
                newest = ys[q][k]
            acc = acc + newest
            assert m[k * P + q] == a
        assert np.abs(fv[:, q] - acc).max() <= 1e-13 * np.abs(acc).max()
    assert cnt[1] == total


@pytest.mark.parametrize("level", [oracle.THREAD, oracle.WARP, oracle.BLOCK])
def test_iact_infinite_threshold_one_table_per_warp(level):
    """One table per warp and thr = +inf: at the first step the table is empty,
    every lane computes and the lowest lane writes (all distances +inf); from
    then on every lane hits that single entry, so nothing is written again and
    every later invocation repeats the warp's first lane's home-box output.
    40 particles per box: warps of 32 and 8 lanes."""
    B, NP = 3, 40
    rq = inputs(B, NP, 13)
    fv, cnt, m = oracle.lavamd(B, NP, A2, rq, technique=oracle.LAVAMD_IACT, level=level, tsize=4,
                               tperwarp=1, thresh=np.inf, mask=True)
    ys = per_invocation(B, NP, rq)
    P = B ** 3 * NP
    for q in range(P):
        lead = (q // NP) * NP + ((q % NP) // 32) * 32
        nn = len(ys[q])
        expect = ys[q][0] + (nn - 1) * ys[lead][0]
        assert np.abs(fv[:, q] - expect).max() <= 1e-13 * np.abs(expect).max()
        assert [int(m[k * P + q]) for k in range(nn)] == [0] + [1] * (nn - 1)
    assert cnt[1] == cnt[0] - P

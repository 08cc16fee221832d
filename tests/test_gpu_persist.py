"""Persistent approximation state on the GPU (TAF windows and iACT tables kept
across calls on a region): parity with the oracle's persistent state call by
call, with the oracle's single call over the concatenated iteration space,
and the handle's reset / reshape / disable behaviour."""
import numpy as np
import pytest

from paper_2308_16877_gb300 import workloads as W
from parity import source_index, taf_replay_check
from tolerances import EPS32, EPS64, output_tol

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
GAMMA = 5.0 / 3.0


@pytest.fixture(scope="module")
def H():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2308_16877_gb300 import hpac
    hpac.load()
    return hpac


def region_inputs(kind, n, dt=np.float64, seed=11):
    if kind == 0:
        return W.blackscholes_inputs(n, seed=seed).astype(dt), W.BS_RATE
    if kind == 1:
        return W.eos_inputs(n, seed=seed, smooth=16), GAMMA
    return W.identity_inputs(n, d=2, dtype=dt, kind="walk", seed=seed), 0.0


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


@pytest.mark.parametrize("dt", [np.float32, np.float64])
@pytest.mark.parametrize("level", [0, 1, 2])
@pytest.mark.parametrize("h,p,thr,reset", [(4, 8, 0.05, False), (3, 2, 0.5, True), (8, 4, 0.02, False)])
def test_taf_identity_persistent_bitexact(H, orc, dt, level, h, p, thr, reset):
    T, B, calls = 1280, 128, 4
    n = 6 * T
    x, param = region_inputs(3, n * calls, dt)
    tdt = torch.float32 if dt == np.float32 else torch.float64
    st = orc.taf_state(T, h)
    all_o, all_m = [], []
    with H.Region(3, dev(x[:, :n]), param=param, logical_threads=T, block_threads=B) as R:
        R.set_persistent(True)
        for c in range(calls):
            xs = np.ascontiguousarray(x[:, c * n:(c + 1) * n])
            out = torch.full((n,), float("nan"), dtype=tdt, device="cuda")
            mask = torch.full((n,), 255, dtype=torch.uint8, device="cuda")
            stat = torch.full((n,), -1.0, dtype=tdt, device="cuda")
            fast = c % 2 == 1   # alternate the fast-decision and statistic paths
            R.run_taf(dev(xs), out, h, p, thr, level, mask=mask, stat=None if fast else stat,
                      stats=not fast, reset_on_exit=reset)
            o, m, s, cnt = orc.run_taf(3, xs, param, h, p, thr, level=level, threads=T, block=B,
                                       reset=reset, state=st)
            assert np.array_equal(host(mask), m), c
            assert np.array_equal(host(out), o), c
            if not fast:
                assert np.array_equal(host(stat), s, equal_nan=True), c
            all_o.append(o)
            all_m.append(m)
    oc, mc, _, cc = orc.run_taf(3, x, param, h, p, thr, level=level, threads=T, block=B, reset=reset)
    assert np.array_equal(np.concatenate(all_m), mc) and np.array_equal(np.concatenate(all_o), oc)
    assert cc[1] > 0


@pytest.mark.parametrize("kind,dt", [(0, np.float32), (1, np.float64), (3, np.float32)])
@pytest.mark.parametrize("level", [0, 1, 2])
@pytest.mark.parametrize("ts,g", [(8, 32), (4, 4), (2, 1)])
def test_iact_persistent_tables(H, orc, kind, dt, level, ts, g):
    """iACT decisions depend on the inputs only: masks and distances equal the
    oracle's bit for bit, call after call."""
    T, B, calls = 1280, 128, 3
    n = 4 * T
    x, param = region_inputs(kind, n * calls, dt)
    sc = W.iact_scale(x, x.shape[1])
    thr = 0.05 if kind == 3 else 0.2   # thresholds at which every case has table hits
    tdt = torch.float32 if x.dtype == np.float32 else torch.float64
    st = orc.iact_state(T, ts, g, x.shape[0])
    with H.Region(kind, dev(x[:, :n]), param=param, logical_threads=T, block_threads=B) as R:
        R.set_persistent(True)
        total = 0
        for c in range(calls):
            xs = np.ascontiguousarray(x[:, c * n:(c + 1) * n])
            out = torch.full((n,), float("nan"), dtype=tdt, device="cuda")
            mask = torch.full((n,), 255, dtype=torch.uint8, device="cuda")
            stat = torch.full((n,), -1.0, dtype=tdt, device="cuda")
            R.run_iact(dev(xs), out, ts, g, thr, level, in_scale=sc, mask=mask, stat=stat)
            o, m, s, cnt = orc.run_iact(kind, xs, param, ts, g, thr, level=level, in_scale=sc,
                                        threads=T, block=B, state=st)
            assert np.array_equal(host(mask), m), c
            assert np.array_equal(host(stat), s), c
            go = host(out)
            if kind == 3:
                assert np.array_equal(go, o), c
            else:
                # an approximated output repeats the exact output of the slot's
                # writer (possibly from an earlier call), bounded by the largest
                # output bound of the stream
                tol = output_tol(kind, x.astype(np.float64), param, x.dtype)
                assert np.all(np.abs(go.astype(np.float64) - o.astype(np.float64)) <= tol.max()), c
            total += cnt[1]
    if level == 0:   # majorities are rare on these streams; thread level always hits
        assert total > 0


@pytest.mark.parametrize("kind,dt", [(0, np.float32), (1, np.float64)])
@pytest.mark.parametrize("level", [0, 1])
@pytest.mark.parametrize("ts,g", [(8, 1), (4, 4)])
def test_iact_persistent_tables_pipelined(H, orc, kind, dt, level, ts, g):
    """Kept tables at thread and warp level run on persistent warps that take
    several logical warps each, the next one's table image copied in while
    the current one runs: 7,813 logical warps (the last one ragged) outnumber
    the resident physical warps (a few thousand on 152 SMs), so most physical
    warps take two or more. Masks and distances equal the oracle's bit for
    bit, call after call."""
    T, B, calls = 250001, 256, 2
    n = 2 * T
    x, param = region_inputs(kind, n * calls, dt)
    sc = W.iact_scale(x, x.shape[1])
    thr = 0.2
    tdt = torch.float32 if x.dtype == np.float32 else torch.float64
    st = orc.iact_state(T, ts, g, x.shape[0])
    with H.Region(kind, dev(x[:, :n]), param=param, logical_threads=T, block_threads=B) as R:
        R.set_persistent(True)
        total = 0
        for c in range(calls):
            xs = np.ascontiguousarray(x[:, c * n:(c + 1) * n])
            out = torch.full((n,), float("nan"), dtype=tdt, device="cuda")
            mask = torch.full((n,), 255, dtype=torch.uint8, device="cuda")
            stat = torch.full((n,), -1.0, dtype=tdt, device="cuda")
            # the second call asks for counters (the counting instantiation)
            r = R.run_iact(dev(xs), out, ts, g, thr, level, in_scale=sc, mask=mask, stat=stat,
                           stats=c == 1)
            o, m, s, cnt = orc.run_iact(kind, xs, param, ts, g, thr, level=level, in_scale=sc,
                                        threads=T, block=B, state=st)
            assert np.array_equal(host(mask), m), c
            assert np.array_equal(host(stat), s), c
            if c == 1:
                assert r["approximated"] == cnt[1] and r["borderline"] == cnt[3]
            tol = output_tol(kind, x.astype(np.float64), param, x.dtype)
            assert np.all(np.abs(host(out).astype(np.float64) - o.astype(np.float64)) <= tol.max()), c
            total += cnt[1]
    if level == 0:   # warp majorities are rare on the Black-Scholes stream
        assert total > 0


@pytest.mark.parametrize("kind,dt", [(0, np.float32), (1, np.float64)])
@pytest.mark.parametrize("level", [0, 1])
def test_taf_regions_persistent_replay(H, orc, kind, dt, level):
    """Black-Scholes / EOS: the masks of three persistent calls, concatenated,
    are a valid trace of one call over the concatenated inputs, checked by
    replaying the oracle along them."""
    T, B, calls, h, p = 2048, 256, 3, 4, 8
    thr = 0.05 if kind == 0 else 0.01
    n = 8 * T
    x, param = region_inputs(kind, n * calls, dt)
    tdt = torch.float32 if dt == np.float32 else torch.float64
    outs, masks, stats = [], [], []
    with H.Region(kind, dev(x[:, :n]), param=param, logical_threads=T, block_threads=B) as R:
        R.set_persistent(True)
        for c in range(calls):
            xs = np.ascontiguousarray(x[:, c * n:(c + 1) * n])
            out = torch.zeros(n, dtype=tdt, device="cuda")
            mask = torch.zeros(n, dtype=torch.uint8, device="cuda")
            stat = torch.zeros(n, dtype=tdt, device="cuda")
            R.run_taf(dev(xs), out, h, p, thr, level, mask=mask, stat=stat)
            outs.append(host(out)), masks.append(host(mask)), stats.append(host(stat))
    g, gm, gs = np.concatenate(outs), np.concatenate(masks), np.concatenate(stats)
    N = n * calls
    o_r, s_r, dis, counts = orc.replay_taf(kind, x, param, h, p, thr, gm, level=level, threads=T, block=B)
    x64 = x.astype(np.float64)
    tol_x = output_tol(kind, x64, param, dt)
    ref64 = orc.run_exact(kind, x64, param)
    rel = tol_x / np.maximum(np.abs(ref64), 1e-300)
    eps = EPS32 if dt == np.float32 else EPS64
    src = source_index(N, T, gm)
    ndis = taf_replay_check(N, T, B, level, g, gm, gs, o_r, s_r, dis, counts, h, thr, 2 * tol_x[src],
                            2 * rel, eps)
    assert ndis <= max(1, counts[0] // 1000)


def test_reset_reshape_and_disable(H, orc):
    T, B, n, h, p = 1024, 128, 6 * 1024, 4, 4
    x, param = region_inputs(3, n, np.float64)
    xd = dev(x)

    def run(R, hh=h):
        out = torch.zeros(n, dtype=torch.float64, device="cuda")
        mask = torch.zeros(n, dtype=torch.uint8, device="cuda")
        R.run_taf(xd, out, hh, p, 0.05, 0, mask=mask)
        return host(mask)

    first = orc.run_taf(3, x, param, h, p, 0.05, threads=T, block=B)[1]
    with H.Region(3, xd, param=param, logical_threads=T, block_threads=B) as R:
        assert np.array_equal(run(R), first)                 # kernel-scoped by default
        assert np.array_equal(run(R), first)
        R.set_persistent(True)
        assert np.array_equal(run(R), first)                 # starts empty
        st = orc.taf_state(T, h)
        orc.run_taf(3, x, param, h, p, 0.05, threads=T, block=B, state=st)
        second = orc.run_taf(3, x, param, h, p, 0.05, threads=T, block=B, state=st)[1]
        assert np.array_equal(run(R), second)                # resumes
        assert not np.array_equal(second, first)
        R.reset_state()
        assert np.array_equal(run(R), first)                 # emptied
        run(R, hh=3)                                         # a new shape starts empty ...
        assert np.array_equal(run(R), first)                 # ... and so does the old one again
        R.set_persistent(False)
        assert np.array_equal(run(R), first)

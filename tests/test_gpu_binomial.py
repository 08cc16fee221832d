"""Binomial Options region on the GPU (one option per team of 32 lanes,
decisions per team) against the oracle's tree, which performs the same
single-precision operations in the same order: exact prices agree bit for bit
except where a leaf's double-precision exponential rounds differently, TAF is
checked by replay along the GPU's mask, iACT decisions and distances are
bit-exact, perforation masks are exact."""
import numpy as np
import pytest

from paper_2308_16877_gb300 import workloads as W
from parity import source_index, taf_replay_check
from tolerances import EPS32

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def H():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2308_16877_gb300 import hpac
    hpac.load()
    return hpac


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def price_tol(x):
    """A leaf S_j whose double exponential rounds to the other float moves the
    price by at most one float ulp of S_j times its probability weight, below
    4 eps S0 e^{rT} in all (the expected leaf), plus the tree's identical rest."""
    return 4 * EPS32 * x[0].astype(np.float64) * np.exp(W.BS_RATE * x[2].astype(np.float64)) + 1e-30


@pytest.mark.parametrize("steps", [1, 2, 31, 32, 33, 100, 287, 288, 543, 544, 1024])
def test_exact_prices(H, orc, steps):
    n = 700 if steps > 512 else 3000
    x = W.binomial_portfolio(100, n // 100, seed=steps)
    out = torch.full((x.shape[1],), float("nan"), device="cuda")
    with H.Region(H.HPAC_REGION_BINOMIAL, dev(x), param=W.BS_RATE, arg=steps, logical_threads=100) as R:
        R.run_exact(dev(x), out)
    g = host(out).astype(np.float64)
    o = orc.run_exact(orc.BINOMIAL, x, W.BS_RATE, steps=steps).astype(np.float64)
    assert np.all(np.abs(g - o) <= price_tol(x)), np.max(np.abs(g - o) / price_tol(x))
    assert np.mean(g == o) > 0.99


@pytest.mark.parametrize("h,p,thr", [(2, 8, 0.05), (4, 4, 0.02), (3, 16, 0.2), (1, 2, np.inf), (4, 8, 0.0)])
def test_taf_per_team_by_replay(H, orc, h, p, thr):
    M, K, steps = 256, 24, 128
    x = W.binomial_portfolio(M, K, seed=5)
    n = x.shape[1]
    out = torch.zeros(n, device="cuda")
    mask = torch.full((n,), 255, dtype=torch.uint8, device="cuda")
    stat = torch.zeros(n, device="cuda")
    with H.Region(H.HPAC_REGION_BINOMIAL, dev(x), param=W.BS_RATE, arg=steps, logical_threads=M) as R:
        st = R.run_taf(dev(x), out, h, p, thr, H.HPAC_LEVEL_BLOCK, mask=mask, stat=stat, stats=True)
        fast_mask = torch.zeros(n, dtype=torch.uint8, device="cuda")
        R.run_taf(dev(x), torch.zeros(n, device="cuda"), h, p, thr, H.HPAC_LEVEL_BLOCK, mask=fast_mask)
    g, gm, gs = host(out), host(mask), host(stat)
    assert np.array_equal(host(fast_mask), gm)
    o_r, s_r, dis, counts = orc.replay_taf(orc.BINOMIAL, x, W.BS_RATE, h, p, thr, gm, level=orc.THREAD,
                                           threads=M, block=256, steps=steps)
    ref = orc.run_exact(orc.BINOMIAL, x, W.BS_RATE, steps=steps).astype(np.float64)
    tol = price_tol(x)
    src = source_index(n, M, gm)
    ndis = taf_replay_check(n, M, 256, 0, g, gm, gs, o_r, s_r, dis, counts, h, thr, 2 * tol[src],
                            2 * tol / np.maximum(np.abs(ref), 1e-30), EPS32)
    assert ndis <= max(1, counts[0] // 1000)
    assert st["approximated"] == int((gm == 1).sum())
    if thr >= 0.05:
        assert st["approximated"] > 0


@pytest.mark.parametrize("ts,thr", [(8, 0.02), (1, 0.05), (64, 0.01)])
def test_iact_per_team(H, orc, ts, thr):
    M, K, steps = 256, 24, 64
    x = W.binomial_portfolio(M, K, seed=6)
    n = x.shape[1]
    sc = W.iact_scale(x, n)
    out = torch.zeros(n, device="cuda")
    mask = torch.full((n,), 255, dtype=torch.uint8, device="cuda")
    stat = torch.zeros(n, device="cuda")
    with H.Region(H.HPAC_REGION_BINOMIAL, dev(x), param=W.BS_RATE, arg=steps, logical_threads=M) as R:
        st = R.run_iact(dev(x), out, ts, 32, thr, H.HPAC_LEVEL_BLOCK, in_scale=sc, mask=mask, stat=stat,
                        stats=True)
    o, om, os_, cnt = orc.run_iact(orc.BINOMIAL, x, W.BS_RATE, ts, 32, thr, level=orc.THREAD, in_scale=sc,
                                   threads=M, block=256, steps=steps)
    assert np.array_equal(host(mask), om)
    assert np.array_equal(host(stat), os_)
    assert np.all(np.abs(host(out).astype(np.float64) - o) <= price_tol(x).max())
    assert st["approximated"] == cnt[1] > 0


@pytest.mark.parametrize("kind,m,rate,herded", [(0, 4, 0.0, 1), (1, 3, 0.0, 0), (2, 25, 0.0, 1), (3, 10, 0.0, 1),
                                                (4, 0, 0.3, 1), (4, 0, 0.3, 0)])
def test_perforation_per_team(H, orc, kind, m, rate, herded):
    M, K, steps = 160, 20, 50
    x = W.binomial_portfolio(M, K, seed=7)
    n = x.shape[1]
    out = torch.full((n,), float("nan"), device="cuda")
    mask = torch.full((n,), 255, dtype=torch.uint8, device="cuda")
    with H.Region(H.HPAC_REGION_BINOMIAL, dev(x), param=W.BS_RATE, arg=steps, logical_threads=M) as R:
        st = R.run_perfo(dev(x), out, kind, m, rate, 9, bool(herded), mask=mask, stats=True)
    prefill = np.full(n, np.nan, dtype=np.float32)
    o, om, cnt = orc.run_perfo(orc.BINOMIAL, x, W.BS_RATE, kind, m, rate, 9, herded, threads=M, out=prefill,
                               steps=steps)
    g = host(out)
    assert np.array_equal(host(mask), om) and st["skipped"] == cnt[2]
    assert np.array_equal(np.isnan(g), np.isnan(o))
    keep = ~np.isnan(o)
    assert np.all(np.abs(g[keep].astype(np.float64) - o[keep]) <= price_tol(x)[keep])


def test_portfolio_workload_sampled(H, orc):
    """The benchmark's workload (4096 members x 64 time points = 262,144
    American calls on 1024-step trees, one team per member) in its launch:
    exact prices of 256 sampled options against the oracle's tree, and a
    TAF run (h1 p2, per team) whose predicted outputs repeat the team's last
    exact price and whose exact ones equal the exact run's."""
    M, K, steps = 4096, 64, 1024
    x = W.binomial_portfolio(M, K)
    n = x.shape[1]
    xd = dev(x)
    exact = torch.zeros(n, device="cuda")
    out = torch.zeros(n, device="cuda")
    mask = torch.zeros(n, dtype=torch.uint8, device="cuda")
    with H.Region(H.HPAC_REGION_BINOMIAL, xd, param=W.BS_RATE, arg=steps, logical_threads=M) as R:
        R.run_exact(xd, exact)
        st = R.run_taf(xd, out, 1, 2, 0.05, H.HPAC_LEVEL_BLOCK, mask=mask, stats=True)
    g, o, m = host(exact), host(out), host(mask)
    idx = np.concatenate([np.random.default_rng(4).choice(n, 254, replace=False), [0, n - 1]])
    xs = np.ascontiguousarray(x[:, idx])
    ref = orc.run_exact(orc.BINOMIAL, xs, W.BS_RATE, steps=steps).astype(np.float64)
    assert np.all(np.abs(g[idx].astype(np.float64) - ref) <= price_tol(xs))
    assert 0 < st["approximated"] == int((m == 1).sum()) < n
    assert np.array_equal(o[m == 0], g[m == 0])
    # a predicted option repeats its team's previous output (column i - M)
    pred = np.nonzero(m == 1)[0]
    assert np.all(pred >= M) and np.array_equal(o[pred], o[pred - M])


def test_rejected_configurations(H):
    x = dev(W.binomial_portfolio(64, 2))
    n = x.shape[1]
    out = torch.zeros(n, device="cuda")
    with pytest.raises(H.HpacError):
        H.Region(H.HPAC_REGION_BINOMIAL, x, param=W.BS_RATE, arg=0)
    with pytest.raises(H.HpacError):
        H.Region(H.HPAC_REGION_BINOMIAL, x, param=W.BS_RATE, arg=1025)
    with pytest.raises(H.HpacError):
        H.Region(H.HPAC_REGION_BINOMIAL, x.double(), param=W.BS_RATE, arg=64)
    with pytest.raises(H.HpacError):
        H.Region(H.HPAC_REGION_BLACKSCHOLES, x, param=W.BS_RATE, arg=64)
    with H.Region(H.HPAC_REGION_BINOMIAL, x, param=W.BS_RATE, arg=64, logical_threads=64) as R:
        for lvl in (H.HPAC_LEVEL_THREAD, H.HPAC_LEVEL_WARP):
            with pytest.raises(H.HpacError):
                R.run_taf(x, out, 2, 2, 0.1, lvl)
        with pytest.raises(H.HpacError):
            R.run_iact(x, out, 4, 16, 0.1, H.HPAC_LEVEL_BLOCK)
        R.set_persistent(True)
        with pytest.raises(H.HpacError):
            R.run_taf(x, out, 2, 2, 0.1, H.HPAC_LEVEL_BLOCK)

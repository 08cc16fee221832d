"""K-Means region on the GPU against the oracle: the assignment (exact, TAF,
iACT, perforation) bit for bit on the same centroids, the centroid update to
the rounding of its double sums, and a whole exact K-Means run to the same
clusters in the same number of iterations."""
import numpy as np
import pytest

from paper_2308_16877_gb300 import workloads as W

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


def region(H, x, cent, T=0, B=256):
    R = H.Region(H.HPAC_REGION_KMEANS, x, arg=cent.shape[0], logical_threads=T, block_threads=B)
    R.set_aux(cent)
    return R


@pytest.mark.parametrize("n,K", [(1, 1), (33, 3), (4099, 16), (70001, 64), (0, 4)])
def test_exact_assignment(H, orc, n, K):
    x, labels, init = W.kmeans_blobs(max(n, K), K, seed=n + K)
    x = np.ascontiguousarray(x[:, :n]) if n else np.zeros((8, 0), dtype=np.float32)
    cent = (init + np.random.default_rng(1).normal(0, 1.5, init.shape)).astype(np.float32)
    out = torch.full((n,), float("nan"), device="cuda")
    with region(H, dev(x), dev(cent)) as R:
        R.run_exact(dev(x), out)
    if n:
        assert np.array_equal(host(out), orc.run_exact(orc.KMEANS, x, cent))


def test_misaligned_centroids_are_rejected(H):
    """Centroids are read as 16-byte vectors: a pointer off that boundary is
    refused when it is set, before any launch."""
    x = torch.zeros((8, 64), dtype=torch.float32, device="cuda")
    buf = torch.zeros(4 * 8 + 1, dtype=torch.float32, device="cuda")
    R = H.Region(H.HPAC_REGION_KMEANS, x, arg=4, logical_threads=0, block_threads=256)
    try:
        with pytest.raises(H.HpacError) as e:
            R.set_aux(buf[1:])
        assert e.value.status == H.HPAC_EINVAL
        R.set_aux(buf[:32])
    finally:
        R.close()


def test_assignment_at_4M_observations(H, orc):
    """The K-Means workload's size (4M observations, 16 clusters) in the
    benchmark's launch (T = N/8): every id against the oracle's nearest
    centroid (integer work, bit-exact)."""
    n, K = 1 << 22, 16
    x, _, _ = W.kmeans_blobs(n, K, spread=2.0)
    cent = np.ascontiguousarray(x[:, :K].T)
    out = torch.full((n,), float("nan"), device="cuda")
    with region(H, dev(x), dev(cent), T=n // 8) as R:
        R.run_exact(dev(x), out)
    assert np.array_equal(host(out), orc.run_exact(orc.KMEANS, x, cent))


@pytest.mark.parametrize("level", [0, 1, 2])
@pytest.mark.parametrize("h,p,thr", [(2, 4, 0.1), (4, 8, 0.5), (3, 2, np.inf)])
@pytest.mark.parametrize("K", [8, 7])
def test_taf_on_ids(H, orc, level, h, p, thr, K):
    """K odd takes the last centroid alone after the packed pairs."""
    n, T = 40000, 5000
    x, labels, init = W.kmeans_blobs(n, K, seed=9)
    idx = np.argsort(labels, kind="stable")       # clustered order: windows of equal ids
    x = np.ascontiguousarray(x[:, idx])
    out = torch.zeros(n, device="cuda")
    mask = torch.zeros(n, dtype=torch.uint8, device="cuda")
    stat = torch.zeros(n, device="cuda")
    with region(H, dev(x), dev(init), T=T, B=128) as R:
        st = R.run_taf(dev(x), out, h, p, thr, level, mask=mask, stat=stat, stats=True)
    o, m, s, cnt = orc.run_taf(orc.KMEANS, x, init, h, p, thr, level=level, threads=T, block=128)
    assert np.array_equal(host(mask), m) and np.array_equal(host(out), o)
    assert np.array_equal(host(stat), s, equal_nan=True)
    assert st["approximated"] == cnt[1] > 0


@pytest.mark.parametrize("level", [0, 1])
@pytest.mark.parametrize("ts,g,thr", [(8, 32, 0.05), (4, 4, 0.1)])
@pytest.mark.parametrize("K", [8, 5])
def test_iact_on_observations(H, orc, level, ts, g, thr, K):
    n, T = 30000, 3000
    x, labels, init = W.kmeans_blobs(n, K, seed=10)
    sc = W.iact_scale(x, n)
    out = torch.zeros(n, device="cuda")
    mask = torch.zeros(n, dtype=torch.uint8, device="cuda")
    stat = torch.zeros(n, device="cuda")
    with region(H, dev(x), dev(init), T=T, B=128) as R:
        st = R.run_iact(dev(x), out, ts, g, thr, level, in_scale=sc, mask=mask, stat=stat, stats=True)
    o, m, s, cnt = orc.run_iact(orc.KMEANS, x, init, ts, g, thr, level=level, in_scale=sc, threads=T,
                                block=128)
    assert np.array_equal(host(mask), m) and np.array_equal(host(stat), s)
    assert np.array_equal(host(out), o)
    assert st["approximated"] == cnt[1]


def test_perforation_keeps_previous_ids(H, orc):
    n, K = 20000, 6
    x, labels, init = W.kmeans_blobs(n, K, seed=11)
    prev = np.full(n, 7.0, dtype=np.float32)
    out = dev(prev)
    mask = torch.zeros(n, dtype=torch.uint8, device="cuda")
    with region(H, dev(x), dev(init), T=n // 4) as R:
        R.run_perfo(dev(x), out, H.HPAC_PERFO_SMALL, 3, herded=True, mask=mask)
    o, m, cnt = orc.run_perfo(orc.KMEANS, x, init, 0, 3, 0.0, 0, 1, threads=n // 4, out=prev.copy())
    assert np.array_equal(host(mask), m) and np.array_equal(host(out), o)


@pytest.mark.parametrize("K", [12, 24, 48, 64])
def test_update_and_changed_count(H, orc, K):
    """Centroid sums with thread-private columns (K <= 16: 64 threads per
    block, K <= 32: 32) and with per-warp shared atomics (K > 32); cluster
    K - 1 left empty keeps its centroid."""
    n = 100000
    x, labels, init = W.kmeans_blobs(n, K, seed=12)
    a = labels.astype(np.float32)
    a[a == K - 1] = 0                                # cluster K - 1 empty
    prev = np.roll(a, 1)
    cent = dev(init)
    work = H.kmeans_workspace(K)
    ch = H.kmeans_update(dev(x), dev(a), cent, work, prev=dev(prev))
    want, wch = orc.kmeans_update(x, a, init, prev=prev)
    assert ch == wch
    g = host(cent)
    assert np.all(np.abs(g - want) <= np.abs(want) * 2 ** -23 + 1e-7)
    assert np.array_equal(g[K - 1], init[K - 1])


def test_whole_run_matches_the_oracle(H, orc):
    n, K = 50000, 10
    x, labels, _ = W.kmeans_blobs(n, K, seed=13, spread=2.0)
    init = np.ascontiguousarray(x[:, :K].T)           # first observations: a harder start
    xo, co = x, init
    a_o, c_o, it_o = orc.kmeans(xo, co, max_iter=200)
    xd, cent = dev(x), dev(init)
    work = H.kmeans_workspace(K)
    a = torch.zeros(n, device="cuda")
    prev = torch.full((n,), -1.0, device="cuda")
    with region(H, xd, cent) as R:
        for it in range(1, 201):
            R.run_exact(xd, a)
            ch = H.kmeans_update(xd, a, cent, work, prev=prev if it > 1 else None)
            if it > 1 and ch == 0:
                break
            prev.copy_(a)
    assert it == it_o < 200
    assert np.array_equal(host(a), a_o)
    assert np.allclose(host(cent), c_o, rtol=2 ** -22, atol=1e-6)

"""The seeded input generators (no GPU): shapes, ranges, determinism, the
strike-sorted runs, and the sweep's region sizes and configuration list."""
import numpy as np

from paper_2308_16877_gb300 import workloads as W


def test_blackscholes_ranges_and_runs():
    x = W.blackscholes_inputs(1000 + 7)
    assert x.shape == (4, 1007) and x.dtype == np.float32
    for d, (lo, hi) in enumerate([W.BS_SPOT, W.BS_STRIKE, W.BS_EXPIRY, W.BS_VOL]):
        assert x[d].min() >= lo and x[d].max() <= hi
    runs = x[1, :992].reshape(-1, 32)
    assert np.all(np.diff(runs, axis=1) >= 0)
    assert np.array_equal(x, W.blackscholes_inputs(1007))


def test_sweep_sizes_and_configs():
    s = W.sweep_region_sizes()
    assert len(s) == 32 and s[0] == 1 << 12 and s[-1] == 1 << 22
    assert all(a <= b for a, b in zip(s, s[1:]))
    c = W.sweep_configs()
    assert len(c) == 256
    taf = [k for k in c if k["tech"] == "taf"]
    assert len(taf) == 128
    assert min(k["thresh"] for k in taf) == 1e-4 and max(k["thresh"] for k in taf) == 1.0
    perf = [k for k in c if k["tech"] == "perfo"]
    assert sum(k["herded"] for k in perf) == 64
    assert {k["kind"] for k in perf} == {0, 1, 2, 3, 4}
    rates = [k["rate"] for k in perf if k["kind"] == 4]
    assert min(rates) == 0.1 and abs(max(rates) - 0.5) < 1e-12


def test_sweep_inputs_layout():
    x, regions = W.sweep_inputs([100, 33, 4096])
    assert x.shape == (4, 4229)
    assert regions == [(100, 0, 12), (33, 100, 4), (4096, 133, 512)]
    assert np.array_equal(x[:, 100:133], W.blackscholes_inputs(33, seed=W.DEFAULT_SEED + 101))


def test_hydro_initial():
    x, y, z, e = W.hydro_initial(4)
    assert x.shape == (125,) and e.shape == (64,)
    assert e[0] == W.HYDRO_E0 and np.all(e[1:] == 0)
    g = x.reshape(5, 5, 5)
    assert np.all(g[:, :, 0] == 0) and np.all(g[:, :, 4] == 1.0)
    assert np.max(np.abs(g - np.arange(5) / 4.0)) <= 0.05 / 4 + 1e-15


def test_kmeans_coherent_layout():
    """Logical thread t's observations come from blob t mod K, but for the
    outlier share; generated deterministically."""
    n, K, T = 1 << 14, 16, 1024
    x, labels, cent = W.kmeans_coherent(n, K, T, outliers=0.05, seed=4)
    assert x.shape == (8, n) and x.dtype == np.float32 and cent.shape == (K, 8)
    own = labels == (np.arange(n) % T) % K
    assert 0.93 < own.mean() < 0.98
    assert np.array_equal(W.kmeans_coherent(n, K, T, outliers=0.05, seed=4)[0], x)

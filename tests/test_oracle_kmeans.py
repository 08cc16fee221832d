"""Pins of the oracle's K-Means region (Table 1: the cluster id of each
observation; the distance kernel is the approximated region) and its exact
centroid update, against numpy brute force and the generating labels of
well-separated blobs (no GPU)."""
import numpy as np

from paper_2308_16877_gb300 import workloads as W


def brute_assign(x, cent):
    """numpy float32, distances accumulated over d = 0..7 in order, argmin
    taking the lowest index on ties."""
    acc = np.zeros((cent.shape[0], x.shape[1]), dtype=np.float32)
    for d in range(8):
        df = x[d][None, :] - cent[:, d][:, None]
        acc = acc + df * df
    return np.argmin(acc, axis=0).astype(np.float32)


def test_assignment_equals_brute_force(orc):
    x, labels, init = W.kmeans_blobs(20000, 12, seed=3)
    rng = np.random.default_rng(0)
    for trial in range(3):
        cent = (init + rng.normal(0, 2, init.shape)).astype(np.float32)
        assert np.array_equal(orc.run_exact(orc.KMEANS, x, cent), brute_assign(x, cent))
    # ties go to the lowest index: duplicate centroids
    cent = np.repeat(init[:3], 2, axis=0)
    a = orc.run_exact(orc.KMEANS, x, cent)
    assert set(np.unique(a)) <= {0.0, 2.0, 4.0}


def test_update_is_the_cluster_mean(orc):
    x, labels, init = W.kmeans_blobs(5000, 6, seed=4)
    a = labels.astype(np.float32)
    a[a == 5] = 4                                   # cluster 5 empty: keeps its centroid
    new, ch = orc.kmeans_update(x, a, init, prev=labels.astype(np.float32))
    for k in range(5):
        m = x[:, a == k].astype(np.float64).mean(axis=1)
        assert np.allclose(new[k], m, rtol=2 ** -23, atol=1e-6)
    assert np.array_equal(new[5], init[5])
    assert ch == int((labels == 5).sum())


def test_kmeans_recovers_separated_blobs(orc):
    x, labels, init = W.kmeans_blobs(30000, 8, seed=5, spread=0.8)
    a, cent, it = orc.kmeans(x, init, max_iter=50)
    assert 2 <= it < 50
    # seeded with one observation per blob, the clusters are the blobs
    assert np.mean(a.astype(int) != labels) < 1e-3

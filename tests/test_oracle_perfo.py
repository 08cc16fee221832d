"""Pins of the oracle's loop perforation (Section 2.3, herded Section 3.1.5,
encounter counter Section 3.3) against closed-form counts, structural
invariants and the published SplitMix64 test vector (no GPU)."""
import itertools

import numpy as np
import pytest

from paper_2308_16877_gb300 import workloads as W

M64 = (1 << 64) - 1


def splitmix64(x):
    """SplitMix64 (Steele, Lea & Flood 2014), written from its published definition."""
    z = (x + 0x9E3779B97F4A7C15) & M64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & M64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & M64
    return z ^ (z >> 31)


def test_splitmix64_published_vector():
    # first output of a SplitMix64 stream seeded with 0
    assert splitmix64(0) == 0xE220A8397B1DCDAF


def executed_closed_form(pkind, n, T, m):
    """small:M keeps n_t - floor(n_t/M) per thread, large:M keeps ceil(n_t/M),
    ini/fini keep N - floor(N P / 100)."""
    if pkind in (2, 3):
        return n - (n * m) // 100
    tot = 0
    for t in range(min(T, n)):
        nt = (n - t + T - 1) // T
        tot += nt - nt // m if pkind == 0 else -(-nt // m)
    return tot


@pytest.mark.parametrize("n,T", [(1, 1), (37, 5), (100, 32), (1000, 96), (4096, 256), (513, 1000)])
def test_executed_counts_closed_form(orc, n, T):
    x = W.identity_inputs(n)
    for pkind, m in itertools.chain(((0, m) for m in (1, 2, 3, 4, 7)), ((1, m) for m in (1, 2, 4, 9)),
                                    ((2, p) for p in (0, 10, 33, 90, 100)),
                                    ((3, p) for p in (0, 10, 50, 99))):
        _, mask, cnt = orc.run_perfo(orc.IDENTITY, x, 0.0, pkind, m, threads=T, block=64)
        executed = int((mask == orc.EXACT).sum())
        assert executed == executed_closed_form(pkind, n, T, m), (pkind, m)
        assert cnt[2] == n - executed
        assert np.all((mask == orc.EXACT) | (mask == orc.SKIPPED))


def test_small_skips_every_mth_encounter(orc):
    """'skip every 4th': with one invocation per step index k, herded small:4
    drops k = 3, 7, 11, ...; large:4 keeps k = 0, 4, 8, ..."""
    n, T = 64, 4
    x = W.identity_inputs(n)
    _, mask, _ = orc.run_perfo(orc.IDENTITY, x, 0.0, orc.SMALL, 4, threads=T, block=32)
    k = np.arange(n) // T
    assert np.array_equal(mask == orc.SKIPPED, np.isin(k % 4, [3]))
    _, mask, _ = orc.run_perfo(orc.IDENTITY, x, 0.0, orc.LARGE, 4, threads=T, block=32)
    assert np.array_equal(mask == orc.EXACT, k % 4 == 0)


def test_herded_is_uniform_per_step_and_iteration_mode_diverges(orc):
    n, T = 96 * 20, 96
    x = W.identity_inputs(n)
    k = np.arange(n) // T
    for pkind, m, rate in ((0, 3, 0.0), (1, 2, 0.0), (4, 0, 0.3)):
        _, mask, _ = orc.run_perfo(orc.IDENTITY, x, 0.0, pkind, m, rate=rate, seed=9, herded=1,
                                   threads=T, block=32)
        per_step = mask.reshape(-1, T)
        assert np.all(per_step == per_step[:, :1]), pkind   # every thread drops the same steps
        _, mask2, _ = orc.run_perfo(orc.IDENTITY, x, 0.0, pkind, m, rate=rate, seed=9, herded=0,
                                    threads=T, block=32)
        lanes = mask2.reshape(-1, 32)
        assert np.any(lanes != lanes[:, :1]), pkind          # lanes of a warp diverge
    # per-iteration small:M depends on the iteration index only
    _, mask2, _ = orc.run_perfo(orc.IDENTITY, x, 0.0, orc.SMALL, 5, herded=0, threads=T, block=32)
    assert np.array_equal(mask2 == orc.SKIPPED, np.arange(n) % 5 == 4)


def test_random_pattern(orc):
    n, T, rate, seed = 50000, 50000, 0.3, 1234
    x = W.identity_inputs(n)
    _, mask, _ = orc.run_perfo(orc.IDENTITY, x, 0.0, orc.RANDOM, 0, rate=rate, seed=seed,
                               herded=0, threads=T, block=256)
    cut = int(np.floor(rate * 2 ** 24))
    expect = np.array([(splitmix64(seed ^ i) >> 40) < cut for i in range(n)])
    assert np.array_equal(mask == orc.SKIPPED, expect)
    sk = expect.sum()
    assert abs(sk - n * rate) < 5 * np.sqrt(n * rate * (1 - rate))
    # rate 0 keeps everything, rate 1 drops everything
    _, m0, _ = orc.run_perfo(orc.IDENTITY, x, 0.0, orc.RANDOM, 0, rate=0.0, seed=seed, herded=0)
    _, m1, _ = orc.run_perfo(orc.IDENTITY, x, 0.0, orc.RANDOM, 0, rate=1.0, seed=seed, herded=0)
    assert np.all(m0 == orc.EXACT) and np.all(m1 == orc.SKIPPED)


def test_dropped_outputs_untouched_kept_outputs_exact(orc):
    n = 3000
    x = W.blackscholes_inputs(n)
    exact = orc.run_exact(orc.BLACKSCHOLES, x, W.BS_RATE)
    out = np.full(n, np.nan, dtype=np.float32)
    out, mask, _ = orc.run_perfo(orc.BLACKSCHOLES, x, W.BS_RATE, orc.SMALL, 4, threads=n // 8,
                                 block=128, out=out)
    skip = mask == orc.SKIPPED
    assert np.all(np.isnan(out[skip]))
    assert np.array_equal(out[~skip], exact[~skip])
    assert 0.24 < skip.mean() < 0.26


def test_rejects_bad_knobs(orc):
    x = W.identity_inputs(10)
    for args in ((0, 0, 0.0), (1, 0, 0.0), (2, 101, 0.0), (3, -1, 0.0), (4, 0, 1.5), (7, 1, 0.0)):
        with pytest.raises(ValueError):
            orc.run_perfo(orc.IDENTITY, x, 0.0, args[0], args[1], rate=args[2])


def test_worked_masks(orc):
    """tests/golden/perfo_worked.txt: the masks of each pattern worked by hand."""
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "perfo_worked.txt")
    x = np.arange(12, dtype=np.float32)[None, :]
    for line in open(path):
        if not line.strip() or line.startswith("#"):
            continue
        kind, m, herded, want = line.split()
        _, mask, cnt = orc.run_perfo(orc.IDENTITY, x, 0.0, int(kind), int(m), 0.0, 0, int(herded), threads=4,
                                     out=np.zeros(12, dtype=np.float32))
        assert "".join(str(v) for v in mask) == want, line
        assert cnt[2] == want.count("2")

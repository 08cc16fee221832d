"""Parity of the batched knob sweep with the region API (same GPU arithmetic,
so counts agree exactly) and with the CPU oracle (counts up to borderline
decisions, error sums within rounding), independence of the schedule, and the
full 256-configuration x 32-region workload on sampled pairs."""
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


def build(H, sizes, seed=7):
    x, regions = W.sweep_inputs(sizes, seed=seed)
    xd = torch.from_numpy(x).cuda()
    x64 = xd.double().contiguous()
    ref = torch.zeros(x.shape[1], dtype=torch.float64, device="cuda")
    with H.Region(H.HPAC_REGION_BLACKSCHOLES, x64, param=W.BS_RATE) as R:
        R.run_exact(x64, ref)
    return x, xd, ref, regions


CONFIGS = [
    dict(tech="taf", hsize=2, psize=4, thresh=0.5),
    dict(tech="taf", hsize=4, psize=8, thresh=0.05),
    dict(tech="taf", hsize=3, psize=1, thresh=2.0),
    dict(tech="taf", hsize=1, psize=2, thresh=0.01),
    dict(tech="perfo", kind=0, m=4, herded=1),
    dict(tech="perfo", kind=0, m=3, herded=0),
    dict(tech="perfo", kind=1, m=2, herded=1),
    dict(tech="perfo", kind=2, m=30, herded=1),
    dict(tech="perfo", kind=3, m=15, herded=0),
    dict(tech="perfo", kind=4, m=0, rate=0.3, seed=11, herded=1),
    dict(tech="perfo", kind=4, m=0, rate=0.2, seed=12, herded=0),
]


def region_api(H, xd, ref, reg, cfg):
    """The same configuration through the region API: stats and error sums."""
    n, off, T = reg
    xs = xd[:, off:off + n].contiguous()
    rs = ref[off:off + n].contiguous()
    out = torch.zeros(n, dtype=torch.float32, device="cuda")
    with H.Region(H.HPAC_REGION_BLACKSCHOLES, xs, param=W.BS_RATE, logical_threads=T) as R:
        if cfg["tech"] == "taf":
            st = R.run_taf(xs, out, cfg["hsize"], cfg["psize"], cfg["thresh"], 0, stats=True)
        else:
            st = R.run_perfo(xs, out, cfg["kind"], cfg["m"], cfg.get("rate", 0.0), cfg.get("seed", 0),
                             bool(cfg.get("herded", 1)), stats=True)
    mape = H.quality(rs, out, H.HPAC_METRIC_MAPE)
    rmse = H.quality(rs, out, H.HPAC_METRIC_RMSE)
    return st, mape, rmse


def check_against_region_api(H, res, xd, ref, regions, configs, pairs):
    for c, r in pairs:
        st, mape, rmse = region_api(H, xd, ref, regions[r], configs[c])
        s = res[c, r]
        assert s["invocations"] == regions[r][0]
        assert s["approximated"] == st["approximated"], (c, r)
        assert s["skipped"] == st["skipped"], (c, r)
        assert s["mape_terms"] == mape["used"], (c, r)
        m = s["sum_abs_rel"] / max(s["mape_terms"], 1)
        assert m == pytest.approx(mape["value"], rel=1e-5, abs=1e-12), (c, r)
        rm = np.sqrt(s["sum_sq"] / s["invocations"])
        assert rm == pytest.approx(rmse["value"], rel=1e-5, abs=1e-9), (c, r)


def test_sweep_matches_region_api(H):
    sizes = [4096, 777, 20000, 65536, 1]
    x, xd, ref, regions = build(H, sizes)
    sw = H.Sweep(CONFIGS, regions, xd, ref, W.BS_RATE, block_threads=128, blocks_per_sm=2, tile_blocks=2)
    sw.run()
    res = sw.results()
    pairs = [(c, r) for c in range(len(CONFIGS)) for r in range(len(sizes))]
    check_against_region_api(H, res, xd, ref, regions, CONFIGS, pairs)
    # a second run of the graph gives the same sums
    sw.run()
    res2 = sw.results()
    assert np.array_equal(res["approximated"], res2["approximated"])
    assert np.allclose(res["sum_sq"], res2["sum_sq"], rtol=1e-12)
    sw.close()


def test_schedule_does_not_change_results(H):
    sizes = [30011, 4096]
    x, xd, ref, regions = build(H, sizes, seed=3)
    out = []
    for bt, bps, tb in ((64, 1, 1), (128, 4, 3), (256, 8, 1)):
        sw = H.Sweep(CONFIGS, regions, xd, ref, W.BS_RATE, block_threads=bt, blocks_per_sm=bps,
                     tile_blocks=tb)
        sw.run()
        out.append(sw.results())
        sw.close()
    for r in out[1:]:
        for f in ("invocations", "approximated", "skipped", "mape_terms"):
            assert np.array_equal(r[f], out[0][f]), f
        # the error sums group their single-precision terms by work item, so
        # they agree to single-precision rounding, not bit for bit
        assert np.allclose(r["sum_sq"], out[0]["sum_sq"], rtol=1e-5, atol=1e-20)
        assert np.allclose(r["sum_abs_rel"], out[0]["sum_abs_rel"], rtol=1e-5, atol=1e-20)


def test_sweep_against_oracle(H, orc):
    """Counts from the oracle's own runs; TAF counts may differ only where a
    window's RSD sits on the threshold (the exact prices differ by rounding
    between CUDA's and the C library's functions)."""
    sizes = [8192, 5000]
    x, xd, ref, regions = build(H, sizes, seed=5)
    sw = H.Sweep(CONFIGS, regions, xd, ref, W.BS_RATE)
    sw.run()
    res = sw.results()
    sw.close()
    ref_h = ref.cpu().numpy()
    for c, cfg in enumerate(CONFIGS):
        for r, (n, off, T) in enumerate(regions):
            xs = x[:, off:off + n]
            if cfg["tech"] == "taf":
                o, om, ost, cnt = orc.run_taf(orc.BLACKSCHOLES, xs, W.BS_RATE, cfg["hsize"], cfg["psize"],
                                              cfg["thresh"], threads=T)
                assert abs(res[c, r]["approximated"] - cnt[1]) <= max(2, n // 2000), (c, r)
            else:
                prefill = np.zeros(n, dtype=np.float32)
                o, om, cnt = orc.run_perfo(orc.BLACKSCHOLES, xs, W.BS_RATE, cfg["kind"], cfg["m"],
                                           cfg.get("rate", 0.0), cfg.get("seed", 0), cfg.get("herded", 1),
                                           threads=T, out=prefill)
                assert res[c, r]["skipped"] == cnt[2], (c, r)
                rm, _ = orc.quality(ref_h[off:off + n], o.astype(np.float64), orc.RMSE)
                assert np.sqrt(res[c, r]["sum_sq"] / n) == pytest.approx(rm, rel=1e-5, abs=1e-9)


def test_full_workload_sampled(H):
    """256 configurations over 32 regions of 2^12..2^22 options in one launch;
    sampled (configuration, region) pairs against the region API."""
    sizes = W.sweep_region_sizes()
    configs = W.sweep_configs()
    x, xd, ref, regions = build(H, sizes, seed=W.DEFAULT_SEED)
    sw = H.Sweep(configs, regions, xd, ref, W.BS_RATE)
    sw.run()
    res = sw.results()
    sw.close()
    assert np.all(res["invocations"] == np.array([r[0] for r in regions])[None, :])
    rng = np.random.default_rng(0)
    pairs = [(int(rng.integers(0, 256)), int(rng.integers(0, 32))) for _ in range(24)]
    pairs += [(0, 31), (127, 0), (128, 31), (255, 16)]
    check_against_region_api(H, res, xd, ref, regions, configs, pairs)


def test_tiny_zero_and_subnormal_prices(H):
    """Reference prices below 1e-30 (scaled far down, double subnormals),
    exactly zero, and one NaN: their relative terms leave the single-precision
    range, and ratios past 1e30 need double precision; sums and term counts
    still equal the region API followed by its quality."""
    sizes = [5000, 3001, 4096]
    x, xd, ref, regions = build(H, sizes, seed=9)
    r = ref.clone()
    idx = torch.arange(r.numel(), device="cuda")
    r[idx % 7 == 0] *= 1e-35
    r[idx % 11 == 0] *= 1e-290
    r[idx % 13 == 0] = 5e-324
    r[idx % 17 == 0] = 0.0
    r[idx % 19 == 0] = -r[idx % 19 == 0]
    sw = H.Sweep(CONFIGS, regions, xd, r, W.BS_RATE, block_threads=128, blocks_per_sm=2, tile_blocks=1)
    sw.run()
    res = sw.results()
    sw.close()
    pairs = [(c, g) for c in range(len(CONFIGS)) for g in range(len(sizes))]
    check_against_region_api(H, res, xd, r, regions, CONFIGS, pairs)
    # one NaN price: its MAPE term and sum are NaN in both
    r[regions[1][1] + 5] = float("nan")
    sw = H.Sweep(CONFIGS[:1], regions, xd, r, W.BS_RATE)
    sw.run()
    res = sw.results()
    sw.close()
    assert np.isnan(res[0, 1]["sum_abs_rel"]) and not np.isnan(res[0, 0]["sum_abs_rel"])
    assert res[0, 1]["mape_terms"] == H.quality(r[regions[1][1]:regions[1][1] + regions[1][0]].contiguous(),
                                                torch.zeros(regions[1][0], device="cuda"),
                                                H.HPAC_METRIC_MAPE)["used"]

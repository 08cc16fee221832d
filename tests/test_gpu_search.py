"""The genetic knob search on the GPU sweep: the evaluator reports exactly what
a direct sweep of the same configurations reports, the search is reproducible,
and its best configuration is feasible."""
import numpy as np
import pytest

from paper_2308_16877_gb300 import search as S
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


def workload(H, sizes=(4096, 20000, 65536, 131072)):
    x, regions = W.sweep_inputs(list(sizes), seed=21)
    xd = torch.from_numpy(x).cuda()
    x64 = xd.double().contiguous()
    ref = torch.zeros(x.shape[1], dtype=torch.float64, device="cuda")
    with H.Region(H.HPAC_REGION_BLACKSCHOLES, x64, param=W.BS_RATE) as R:
        R.run_exact(x64, ref)
    return xd, ref, regions


def test_evaluator_matches_a_direct_sweep(H):
    xd, ref, regions = workload(H)
    ev = S.sweep_evaluator(H, regions, xd, ref, W.BS_RATE)
    rng = np.random.default_rng(5)
    cfgs = [S.random_config(rng) for _ in range(24)]
    got = ev(cfgs)
    sw = H.Sweep(cfgs, regions, xd, ref, W.BS_RATE, 256, 4, 1)
    sw.run()
    res = sw.results()
    sw.close()
    inv = res["invocations"].sum(axis=1).astype(float)
    saved = (res["approximated"].sum(axis=1) + res["skipped"].sum(axis=1)) / inv
    rms = float(torch.sqrt(torch.mean(ref * ref)).item())
    nrmse = np.sqrt(res["sum_sq"].sum(axis=1) / inv) / rms
    assert np.array_equal(np.array([g[0] for g in got]), saved)     # counts: schedule independent
    assert np.allclose(np.array([g[1] for g in got]), nrmse, rtol=1e-5, atol=0)
    assert ev.calls == {"launches": 1, "configs": 24}


def test_search_on_the_sweep_is_reproducible_and_feasible(H):
    xd, ref, regions = workload(H)
    runs = []
    for _ in range(2):
        ev = S.sweep_evaluator(H, regions, xd, ref, W.BS_RATE)
        runs.append(S.genetic_search(ev, population=16, generations=5, seed=3) + (dict(ev.calls),))
    (b1, r1, h1, c1), (b2, r2, h2, c2) = runs
    assert b1 == b2 and r1[0] == r2[0] and np.isclose(r1[1], r2[1], rtol=1e-5)
    assert r1[1] <= 0.01 and r1[0] > 0
    assert c1["launches"] == 5 and c1["configs"] <= 5 * 16
    # the best configuration re-evaluated alone gives the same saved share
    ev = S.sweep_evaluator(H, regions, xd, ref, W.BS_RATE)
    alone = ev([b1])[0]
    assert alone[0] == r1[0] and np.isclose(alone[1], r1[1], rtol=1e-5)

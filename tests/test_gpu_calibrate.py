"""The calibrated fallback bound on the device (hpac_calibrate_floor, through
the C ABI) against the oracle's definition: the floor and the number of
invocations it serves agree exactly, on sizes below, at and above the sorting
chunk, with ties, NaN predictions, signed zeros and negative values; and the
surrogate's own floor on held-out Black-Scholes options."""
import math

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


def case(n, seed, ties=False, specials=False):
    rng = np.random.default_rng(seed)
    exact = rng.uniform(0.001, 30.0, n)
    # relative error grows as the price falls, as a surrogate's does
    rel = 0.002 + 0.05 * np.exp(-exact)
    pred = (exact * (1.0 + rng.normal(0.0, 1.0, n) * rel)).astype(np.float32)
    if ties and n > 4:
        pred[rng.integers(0, n, n // 4)] = np.float32(np.median(pred))
        pred[rng.integers(0, n, n // 8)] = np.float32(1.0)
    if specials and n > 8:
        pred[rng.integers(0, n, 3)] = np.nan
        pred[rng.integers(0, n, 2)] = -0.0
        pred[rng.integers(0, n, 2)] = 0.0
        pred[rng.integers(0, n, 3)] = -1.5
        exact[rng.integers(0, n, 2)] = 0.0
    return pred, exact


@pytest.mark.parametrize("n", [1, 5, 2047, 2048, 2049, 4097, 100_003, (1 << 20) + 3])
@pytest.mark.parametrize("variant", ["plain", "ties", "specials"])
@pytest.mark.parametrize("target,q", [(0.01, 0.99), (0.02, 0.9), (0.005, 1.0)])
def test_floor_matches_the_oracle(H, orc, n, variant, target, q):
    pred, exact = case(n, seed=n % 97 + len(variant), ties=variant == "ties", specials=variant == "specials")
    fl, kept = H.calibrate_floor(torch.from_numpy(pred).cuda(), torch.from_numpy(exact).cuda(), target, q)
    ofl, okept = orc.calibrate_floor(pred, exact, target, q)
    assert kept == okept
    assert (math.isinf(fl) and math.isinf(ofl)) or fl == ofl, (fl, ofl)


def test_empty_and_rejected_arguments(H):
    e = torch.zeros(0, dtype=torch.float64, device="cuda")
    p = torch.zeros(0, dtype=torch.float32, device="cuda")
    assert H.calibrate_floor(p, e) == (math.inf, 0)
    fl = H.C.c_float()
    for args in ((4, None, None, 0.01, 0.99), (4, 1, 1, -1.0, 0.99), (4, 1, 1, 0.01, 0.0),
                 (4, 1, 1, 0.01, 1.5), (-1, 1, 1, 0.01, 0.99)):
        n, a, b, t, q = args
        st = H.load().hpac_calibrate_floor(n, H.C.c_void_p(a) if a else None, H.C.c_void_p(b) if b else None,
                                           t, q, H.C.byref(fl), None, None)
        assert st == H.HPAC_EINVAL, args


def test_surrogate_floor_on_held_out_options(H, orc):
    """A briefly trained Black-Scholes surrogate: its predictions on 2^20
    held-out options, the exact prices in double precision, and the floor
    from the device equal to the oracle's; the options served above it meet
    the 99th-percentile bound."""
    dev = torch.device("cuda")
    xt = torch.from_numpy(W.blackscholes_inputs(1 << 18, seed=61)).to(dev)
    yt = torch.zeros(xt.shape[1], dtype=torch.float32, device=dev)
    with H.Region(H.HPAC_REGION_BLACKSCHOLES, xt, param=W.BS_RATE) as R:
        R.run_exact(xt, yt)
    S = H.Surrogate(H.blackscholes_desc(64), seed=5)
    S.fit_normalization(xt, yt, W.BS_RATE)
    S.train(xt, yt, W.BS_RATE, batch=4096, epochs=3, lr=3e-3)
    xc = torch.from_numpy(W.blackscholes_inputs(1 << 20, seed=62)).to(dev)
    pc = torch.zeros(xc.shape[1], dtype=torch.float32, device=dev)
    S.infer(xc, pc, W.BS_RATE)
    S.close()
    x64 = xc.double().contiguous()
    yc = torch.zeros(xc.shape[1], dtype=torch.float64, device=dev)
    with H.Region(H.HPAC_REGION_BLACKSCHOLES, x64, param=W.BS_RATE) as R:
        R.run_exact(x64, yc)
    fl, kept = H.calibrate_floor(pc, yc, 0.01, 0.99)
    p, y = pc.cpu().numpy(), yc.cpu().numpy()
    assert (fl, kept) == orc.calibrate_floor(p, y, 0.01, 0.99)
    served = p >= fl
    assert served.sum() == kept
    bad = np.abs(p[served].astype(np.float64) - y[served]) > 0.01 * np.abs(y[served])
    assert bad.sum() <= kept - math.ceil(0.99 * kept)

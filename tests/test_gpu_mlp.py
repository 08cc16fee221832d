"""The learned surrogate and the exact region's adjoint through the C ABI,
against the CPU oracle: forward within a bound propagated from bfloat16
rounding, parameter and input gradients, the training loop, the calibrated
exact fallback, and the adjoint against finite differences and a textbook
value."""
import os

import numpy as np
import pytest

from oracle import mlp as M
from paper_2308_16877_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
GOLD = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module")
def H():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2308_16877_gb300 import hpac
    hpac.load()
    return hpac


def dd(d):
    return M.desc_dict(d)


def forward_bound(p, desc, x, r):
    """Worst-case |net_gpu - net_oracle| from the arithmetic: every rounded
    activation may land one bfloat16 ulp (2^-7 relative) apart, the hardware
    tanh adds 2^-11 |z| to a GELU, FP32 accumulation 2^-20 of the absolute sum;
    propagated through |W2| and |W3| with |gelu'| <= 1.13."""
    params = M.unpack(p, desc["n_feat"], desc["hidden"])
    f, _ = M.features(0, x, r)
    _, (fn, z1, h1, z2, h2) = M.net(params, desc, f)
    W2 = M.bf16(params[2]).abs()
    W3 = M.bf16(params[4]).abs()
    dh1 = 2 ** -7 * h1.abs() + 2 ** -11 * z1.abs() + 1e-6 * (fn.abs() @ M.bf16(params[0]).abs().T)
    dz2 = dh1 @ W2.T + 2 ** -20 * (h1.abs() @ W2.T)
    dh2 = 1.13 * dz2 + 2 ** -7 * h2.abs() + 2 ** -11 * z2.abs()
    return (dh2 @ W3 + 2 ** -20 * (h2.abs() @ W3)).numpy()


@pytest.mark.parametrize("hidden", [64, 128])
def test_forward_matches_oracle(H, hidden):
    desc = H.blackscholes_desc(hidden)
    n = 3000
    x = W.blackscholes_inputs(n, seed=21)
    S = H.Surrogate(desc, seed=5)
    xd = torch.from_numpy(x).cuda()
    out = torch.zeros(n, dtype=torch.float32, device="cuda")
    S.infer(xd, out, W.BS_RATE)
    p = S.params()
    ref, net_ref, _ = M.forward(p, dd(desc), 0, x, W.BS_RATE)
    g = out.cpu().numpy().astype(np.float64)
    bound = forward_bound(p, dd(desc), x, W.BS_RATE) * desc.out_scale * x[0].astype(np.float64)
    assert np.all(np.abs(g - ref) <= bound + 1e-6 * np.abs(ref))
    rel = np.abs(g - ref) / np.maximum(np.abs(ref), 1e-3)
    assert np.median(rel) < 2 ** -9
    S.close()


def test_gradient_matches_oracle(H):
    desc = H.blackscholes_desc(64)
    n = 4096
    x = W.blackscholes_inputs(n, seed=22)
    xd = torch.from_numpy(x).cuda()
    target = M.forward(np.random.default_rng(1).uniform(-0.3, 0.3, M.n_params(5, 64)), dd(desc), 0, x,
                       W.BS_RATE)[0].astype(np.float32)
    td = torch.from_numpy(target).cuda()
    S = H.Surrogate(desc, seed=6)
    grad = torch.zeros(S.n_params, dtype=torch.float32, device="cuda")
    loss = S.grad(xd, td, W.BS_RATE, grad=grad, loss=True)
    p = S.params()
    l_ref, g_ref, *_ = M.loss_and_grad(p, dd(desc), 0, x.astype(np.float64), W.BS_RATE, target)
    g = grad.cpu().numpy().astype(np.float64)
    cos = float(g @ g_ref / (np.linalg.norm(g) * np.linalg.norm(g_ref)))
    assert cos > 0.999, cos
    assert np.linalg.norm(g - g_ref) / np.linalg.norm(g_ref) < 0.03
    assert loss == pytest.approx(l_ref, rel=0.02)
    S.close()


@pytest.mark.parametrize("kind,hidden,n", [(0, 64, 2048), (0, 128, 3 * 128 + 77), (1, 64, 5 * 128 + 1),
                                            (1, 128, 4096), (0, 64, 1)])
def test_input_gradient_matches_oracle(H, kind, hidden, n):
    """d(region output)/d(region inputs) of the surrogate (tcgen05 forward and
    backward products, chain rule per thread) against the oracle's FP64
    derivatives, within the bfloat16 rounding of the activations; sizes span
    several 128-sample tiles with a ragged tail, and a single sample."""
    if kind == 0:
        desc = H.blackscholes_desc(hidden)
        x = W.blackscholes_inputs(n, seed=23)
        param = W.BS_RATE
    else:
        desc = H.eos_desc(hidden)
        x = W.eos_inputs(n, seed=23)
        param = 5.0 / 3.0
    S = H.Surrogate(desc, seed=7)
    xd = torch.from_numpy(np.ascontiguousarray(x)).cuda()
    out = torch.full((4, n), np.nan, dtype=torch.float32, device="cuda")
    S.input_grad(xd, out, param)
    ref = M.input_grad(S.params(), dd(S.get_desc()), kind, x.astype(np.float64), param)
    g = out.cpu().numpy().astype(np.float64)
    assert np.all(np.isfinite(g))
    for d in range(4):
        nr = np.linalg.norm(ref[d])
        if nr == 0:
            assert np.all(g[d] == 0), d
            continue
        err = np.linalg.norm(g[d] - ref[d]) / nr
        assert err < 0.03, (d, err)
    S.close()


def test_training_reduces_loss_and_fallback_is_exact(H, orc):
    desc = H.blackscholes_desc(64)
    n = 1 << 18
    x = W.blackscholes_inputs(n, seed=24)
    xd = torch.from_numpy(x).cuda()
    tgt = torch.zeros(n, dtype=torch.float32, device="cuda")
    with H.Region(H.HPAC_REGION_BLACKSCHOLES, xd, param=W.BS_RATE) as R:
        R.run_exact(xd, tgt)
    S = H.Surrogate(desc, seed=8)
    l0 = S.grad(xd, tgt, W.BS_RATE, loss=True)
    l1 = S.train(xd, tgt, W.BS_RATE, batch=4096, epochs=4, lr=3e-3)
    assert l1 < 0.05 * l0, (l0, l1)
    # calibrated fallback: predictions below tau are recomputed exactly
    out = torch.zeros(n, dtype=torch.float32, device="cuda")
    mask = torch.zeros(n, dtype=torch.uint8, device="cuda")
    S.infer(xd, out, W.BS_RATE)
    pred = out.cpu().numpy()
    tau = float(np.quantile(pred, 0.3))
    st = S.infer(xd, out, W.BS_RATE, fallback_below=tau, mask=mask, stats=True)
    m = mask.cpu().numpy()
    o = out.cpu().numpy()
    ex = tgt.cpu().numpy()
    assert np.array_equal(m == 0, pred < tau)
    assert st["approximated"] == int((m == 1).sum())
    # fallback outputs are the exact region (within the single-precision
    # Black-Scholes bound of the double-precision price)
    from tolerances import blackscholes_tol
    idx = np.nonzero(m == 0)[0][:20000]
    ref = orc.run_exact(orc.BLACKSCHOLES, x[:, idx].astype(np.float64), W.BS_RATE)
    assert np.all(np.abs(o[idx] - ref) <= blackscholes_tol(x[:, idx], W.BS_RATE))
    assert np.all(np.abs(ex[idx] - ref) <= blackscholes_tol(x[:, idx], W.BS_RATE))
    assert np.array_equal(o[m == 1], pred[m == 1])
    S.close()


def test_inference_at_16M_options_sampled(H, orc):
    """The surrogate workload's inference size (2^24 options) with the
    calibrated fallback, in the benchmark's launch: sampled predictions within
    the bfloat16 forward bound of the oracle's network, the mask exactly the
    rule prediction < tau, sampled fallback outputs within the exact region's
    bar, approximated outputs equal to the plain predictions."""
    desc = H.blackscholes_desc(64)
    n = 1 << 24
    x = W.blackscholes_inputs(n, seed=25)
    xd = torch.from_numpy(x).cuda()
    S = H.Surrogate(desc, seed=9)
    m_tr = 1 << 18
    tgt = torch.zeros(m_tr, dtype=torch.float32, device="cuda")
    xt = xd[:, :m_tr].contiguous()
    with H.Region(H.HPAC_REGION_BLACKSCHOLES, xt, param=W.BS_RATE) as R:
        R.run_exact(xt, tgt)
    S.train(xt, tgt, W.BS_RATE, batch=4096, epochs=1, lr=3e-3)
    pred = torch.zeros(n, dtype=torch.float32, device="cuda")
    S.infer(xd, pred, W.BS_RATE)
    out = torch.zeros(n, dtype=torch.float32, device="cuda")
    mask = torch.zeros(n, dtype=torch.uint8, device="cuda")
    tau = 1.0
    st = S.infer(xd, out, W.BS_RATE, fallback_below=tau, mask=mask, stats=True)
    pr, o, m = pred.cpu().numpy(), out.cpu().numpy(), mask.cpu().numpy()
    assert np.array_equal(m == 0, pr < tau)
    assert st["approximated"] == int((m == 1).sum()) and 0 < st["approximated"] < n
    assert np.array_equal(o[m == 1], pr[m == 1])
    rng = np.random.default_rng(3)
    idx = np.concatenate([rng.choice(n, 4096, replace=False), [0, n - 1]])
    p = S.params()
    xs = np.ascontiguousarray(x[:, idx])
    ref, _, _ = M.forward(p, dd(desc), 0, xs, W.BS_RATE)
    bound = forward_bound(p, dd(desc), xs, W.BS_RATE) * desc.out_scale * xs[0].astype(np.float64)
    assert np.all(np.abs(pr[idx].astype(np.float64) - ref) <= bound + 1e-6 * np.abs(ref))
    from tolerances import blackscholes_tol
    fb = np.nonzero(m == 0)[0]
    fb = fb[rng.choice(fb.size, min(fb.size, 4096), replace=False)]
    exact = orc.run_exact(orc.BLACKSCHOLES, x[:, fb].astype(np.float64), W.BS_RATE)
    assert np.all(np.abs(o[fb] - exact) <= blackscholes_tol(x[:, fb], W.BS_RATE))
    S.close()


def test_adjoint_blackscholes_textbook_and_finite_differences(H, orc):
    rows = [l.split() for l in open(os.path.join(GOLD, "blackscholes_hull.txt"))
            if l.strip() and not l.startswith("#")]
    S0, K0, T0, sig0, r0 = map(float, rows[0][:5])
    x = np.array([[S0], [K0], [T0], [sig0]])
    with H.Region(H.HPAC_REGION_BLACKSCHOLES, torch.from_numpy(x).cuda(), param=r0) as R:
        g = torch.zeros(4, 1, dtype=torch.float64, device="cuda")
        H.region_adjoint(R, torch.from_numpy(x).cuda(), g)
    # Hull's worked example: delta N(d1) = 0.7791 (d1 = 0.7693)
    assert float(g[0, 0]) == pytest.approx(0.7791, abs=5e-5)
    n = 500
    for dt in (np.float32, np.float64):
        x = W.blackscholes_inputs(n, seed=25).astype(dt)
        xd = torch.from_numpy(x).cuda()
        gd = torch.zeros(4, n, dtype=torch.float32 if dt == np.float32 else torch.float64, device="cuda")
        with H.Region(H.HPAC_REGION_BLACKSCHOLES, xd, param=W.BS_RATE) as R:
            H.region_adjoint(R, xd, gd)
        got = gd.cpu().numpy().astype(np.float64)
        x64 = x.astype(np.float64)
        for d in range(4):
            h = 1e-6 * np.abs(x64[d])
            xp, xm = x64.copy(), x64.copy()
            xp[d] += h
            xm[d] -= h
            fd = (orc.run_exact(orc.BLACKSCHOLES, xp, W.BS_RATE) - orc.run_exact(orc.BLACKSCHOLES, xm, W.BS_RATE)) / (2 * h)
            scale = np.abs(fd).max()
            tol = 1e-4 if dt == np.float32 else 1e-6
            assert np.all(np.abs(got[d] - fd) <= tol * scale), (dt, d)


def test_adjoint_eos_finite_differences(H, orc):
    n = 1000
    x = W.eos_inputs(n, seed=26)
    xd = torch.from_numpy(x).cuda()
    g = torch.zeros(4, n, dtype=torch.float64, device="cuda")
    with H.Region(H.HPAC_REGION_EOS, xd, param=5 / 3) as R:
        H.region_adjoint(R, xd, g)
    got = g.cpu().numpy()
    for d in range(4):
        # the step scales with the column's magnitude so that the change of p
        # (about 1e5) stays far above its double-precision resolution
        h = 1e-7 * np.abs(x[d]).max()
        xp, xm = x.copy(), x.copy()
        xp[d] += h
        xm[d] -= h
        fd = (orc.run_exact(orc.EOS, xp, 5 / 3) - orc.run_exact(orc.EOS, xm, 5 / 3)) / (2 * h)
        # the central difference itself carries the rounding of p (a few ulps)
        # divided by the step, plus its O(h^2) truncation (relative 1e-5 here)
        p = orc.run_exact(orc.EOS, x, 5 / 3)
        noise = 8 * np.finfo(np.float64).eps * np.abs(p) / h
        assert np.all(np.abs(got[d] - fd) <= 1e-5 * np.abs(fd) + noise + 1e-300), d


def test_fit_normalization_matches_feature_moments(H):
    desc = H.blackscholes_desc(64)
    n = 100_000
    x = W.blackscholes_inputs(n, seed=27)
    xd = torch.from_numpy(x).cuda()
    y = torch.zeros(n, dtype=torch.float32, device="cuda")
    with H.Region(H.HPAC_REGION_BLACKSCHOLES, xd, param=W.BS_RATE) as R:
        R.run_exact(xd, y)
    S = H.Surrogate(desc, seed=1)
    d = S.fit_normalization(xd, y, W.BS_RATE)
    f, mult = M.features(0, x.astype(np.float64), W.BS_RATE)
    f = f.numpy()
    for k in range(5):
        assert d.feat_shift[k] == pytest.approx(f[:, k].mean(), rel=1e-4, abs=1e-5), k
        assert 1 / d.feat_scale[k] == pytest.approx(f[:, k].std(), rel=1e-3), k
    t = y.cpu().numpy().astype(np.float64) / mult.numpy()
    assert d.out_shift == pytest.approx(t.mean(), rel=1e-4)
    assert d.out_scale == pytest.approx(t.std(), rel=1e-3)
    S.close()


def test_eos_surrogate_forward_gradient_and_training(H):
    """The EOS surrogate (4 -> 128 -> 128 -> 1, double-precision region I/O):
    forward against the oracle, the parameter gradient, and training on EOS
    pairs; untouched elements (e = q = 0) come out exactly 0."""
    n = 8192
    x = W.eos_inputs(n, seed=28)
    x[:, :100] = np.array([[0.0], [1.0], [0.0], [0.0]])          # untouched elements
    xd = torch.from_numpy(x).cuda()
    y = torch.zeros(n, dtype=torch.float64, device="cuda")
    with H.Region(H.HPAC_REGION_EOS, xd, param=5 / 3) as R:
        R.run_exact(xd, y)
    S = H.Surrogate(H.eos_desc(128), seed=3)
    yf = y.float().contiguous()
    d = S.fit_normalization(xd, yf, 5 / 3)
    out = torch.zeros(n, dtype=torch.float64, device="cuda")
    S.infer(xd, out, 5 / 3)
    ref, _, _ = M.forward(S.params(), dd(d), 1, x, 5 / 3)
    g = out.cpu().numpy()
    assert np.all(g[:100] == 0.0)
    rel = np.abs(g - ref) / np.maximum(np.abs(ref), 1e-6 * np.abs(ref).max())
    assert np.median(rel) < 2 ** -8
    grad = torch.zeros(S.n_params, dtype=torch.float32, device="cuda")
    S.grad(xd, yf, 5 / 3, grad=grad)
    _, g_ref, *_ = M.loss_and_grad(S.params(), dd(d), 1, x, 5 / 3, yf.cpu().numpy())
    gg = grad.cpu().numpy().astype(np.float64)
    cos = float(gg @ g_ref / (np.linalg.norm(gg) * np.linalg.norm(g_ref)))
    assert cos > 0.999, cos
    l0 = S.grad(xd, yf, 5 / 3, loss=True)
    l1 = S.train(xd, yf, 5 / 3, batch=1024, epochs=20, lr=2e-3)
    assert l1 < 0.2 * l0, (l0, l1)
    S.close()


@pytest.mark.parametrize("kind", [0, 1])
def test_differentiable_exact_region(H, kind):
    """The exact region behind torch.autograd (forward hpac_run_exact, backward
    hpac_region_vjp): torch.autograd.gradcheck in double precision against
    central differences of the region itself, and the vector-Jacobian product
    equal to the adjoint times the upstream gradient."""
    n = 12
    if kind == 0:
        x = W.blackscholes_inputs(n, seed=31).astype(np.float64)
        param = W.BS_RATE
    else:
        x = W.eos_inputs(n, seed=31)
        x[0] += 1e3           # away from the energy clamp, where p is not differentiable
        param = 5.0 / 3.0
    xd = torch.from_numpy(np.ascontiguousarray(x)).cuda().requires_grad_(True)
    with H.Region(kind, xd.detach(), param=param) as R:
        f = lambda t: H.differentiable(R, t)
        if kind == 0:
            assert torch.autograd.gradcheck(f, (xd,), eps=1e-6, atol=1e-6, rtol=1e-4)
        else:
            # inputs of very different scales (e ~ 1e5, dv ~ 1e-2): central
            # differences with a step relative to each input row's magnitude
            (gx,) = torch.autograd.grad(f(xd).sum(), xd)
            for d in range(4):
                hstep = 1e-6 * max(float(xd.detach()[d].abs().max()), 1e-3)
                xp, xm = xd.detach().clone(), xd.detach().clone()
                xp[d] += hstep
                xm[d] -= hstep
                fd = (f(xp) - f(xm)) / (2 * hstep)
                assert torch.allclose(gx[d], fd, rtol=1e-5, atol=1e-9 * float(fd.abs().max())), d
        w = torch.randn(n, dtype=torch.float64, device="cuda")
        (f(xd) * w).sum().backward()
        adj = torch.zeros(4, n, dtype=torch.float64, device="cuda")
        H.region_adjoint(R, xd.detach(), adj)
    assert torch.allclose(xd.grad, adj * w, rtol=1e-12, atol=1e-300)


@pytest.mark.parametrize("kind,hidden", [(0, 64), (1, 128)])
def test_differentiable_surrogate(H, kind, hidden):
    """The surrogate behind torch.autograd with its parameters as a torch
    tensor (forward hpac_mlp_infer, backward hpac_mlp_vjp): the parameter and
    input gradients of sum_i w_i out_i against the oracle's, within the
    bfloat16 rounding of the activations (cosine > 0.999, < 3% relative)."""
    if kind == 0:
        desc = H.blackscholes_desc(hidden)
        n = 4096
        x = W.blackscholes_inputs(n, seed=32)
        param = W.BS_RATE
    else:
        desc = H.eos_desc(hidden)
        n = 4096
        x = W.eos_inputs(n, seed=32)
        param = 5.0 / 3.0
    S = H.Surrogate(desc, seed=12)
    p0 = S.params()
    xd = torch.from_numpy(np.ascontiguousarray(x)).cuda().requires_grad_(True)
    weights = torch.from_numpy(p0).cuda().requires_grad_(True)
    rng = np.random.default_rng(5)
    w = rng.normal(size=n)
    out = S.apply(xd, weights, param)
    (out * torch.from_numpy(w).cuda().to(out.dtype)).sum().backward()
    gp_ref, gx_ref = M.vjp(p0, dd(S.get_desc()), kind, x.astype(np.float64), param, w)
    gp = weights.grad.cpu().numpy().astype(np.float64)
    cos = float(gp @ gp_ref / (np.linalg.norm(gp) * np.linalg.norm(gp_ref)))
    assert cos > 0.999, cos
    assert np.linalg.norm(gp - gp_ref) / np.linalg.norm(gp_ref) < 0.03
    gx = xd.grad.cpu().numpy().astype(np.float64)
    for d in range(4):
        err = np.linalg.norm(gx[d] - gx_ref[d]) / max(np.linalg.norm(gx_ref[d]), 1e-300)
        assert err < 0.03, (d, err)
    # the parameters are the caller's: a changed tensor changes the output
    with torch.no_grad():
        w2 = weights.detach().clone()
        w2[-1] += 0.5
    out2 = S.apply(xd.detach(), w2, param)
    assert not torch.equal(out2, out.detach())
    S.close()


def test_surrogate_gains_over_taf_and_iact_at_one_percent(H):
    """What the trained network adds to the method: on the same Black-Scholes
    options, at the same quality bar (NRMSE <= 1% against the FP64 exact
    prices), the surrogate with its calibrated exact fallback replaces far more
    invocations than the best TAF or iACT configuration of a small knob sweep
    (independent random options give TAF windows no temporal stability and
    iACT tables no nearby inputs). Trained by the library's kernels on 4M
    exact pairs, calibrated on 1M held-out options, scored on another 1M."""
    dev = "cuda"

    def exact(x, dtype, T=0):
        out = torch.zeros(x.shape[1], dtype=dtype, device=dev)
        xx = x if dtype == torch.float32 else x.double().contiguous()
        with H.Region(H.HPAC_REGION_BLACKSCHOLES, xx, param=W.BS_RATE, logical_threads=T) as R:
            R.run_exact(xx, out)
        return out

    xt = torch.from_numpy(W.blackscholes_inputs(1 << 22, seed=31)).to(dev)
    yt = exact(xt, torch.float32)
    S = H.Surrogate(H.blackscholes_desc(64), seed=2308)
    S.fit_normalization(xt, yt, W.BS_RATE)
    S.train(xt, yt, W.BS_RATE, batch=8192, epochs=24, lr=3e-3)
    # calibration (hpac_calibrate_floor): the smallest price floor above which
    # the 99th percentile of the surrogate's relative error is within 1%
    xc = torch.from_numpy(W.blackscholes_inputs(1 << 20, seed=32)).to(dev)
    pc = torch.zeros(xc.shape[1], dtype=torch.float32, device=dev)
    S.infer(xc, pc, W.BS_RATE)
    tau, _ = H.calibrate_floor(pc, exact(xc, torch.float64), 0.01, 0.99)
    assert np.isfinite(tau), "no calibrated floor reaches the 1% bar"

    n = 1 << 20
    xs = W.blackscholes_inputs(n, seed=33)
    xi = torch.from_numpy(xs).to(dev)
    ref = exact(xi, torch.float64).cpu().numpy()
    rms = float(np.sqrt(np.mean(ref * ref)))
    nrmse = lambda o: float(np.sqrt(np.mean((o.cpu().numpy().astype(np.float64) - ref) ** 2)) / rms)

    out = torch.zeros(n, dtype=torch.float32, device=dev)
    st = S.infer(xi, out, W.BS_RATE, fallback_below=tau, stats=True)
    sur_frac, sur_q = st["approximated"] / n, nrmse(out)
    S.close()
    assert sur_q <= 0.01 and sur_frac >= 0.25, (sur_q, sur_frac, tau)

    best = {}
    sc = W.iact_scale(xs, n)
    with H.Region(H.HPAC_REGION_BLACKSCHOLES, xi, param=W.BS_RATE, logical_threads=n // 8) as R:
        for thr in (0.005, 0.02, 0.1):
            o = torch.zeros(n, dtype=torch.float32, device=dev)
            s = R.run_taf(xi, o, 4, 8, thr, H.HPAC_LEVEL_THREAD, stats=True)
            if nrmse(o) <= 0.01:
                best["taf"] = max(best.get("taf", 0.0), s["approximated"] / n)
        for thr in (1e-3, 1e-2, 5e-2):
            o = torch.zeros(n, dtype=torch.float32, device=dev)
            s = R.run_iact(xi, o, 8, 32, thr, H.HPAC_LEVEL_THREAD, in_scale=sc, stats=True)
            if nrmse(o) <= 0.01:
                best["iact"] = max(best.get("iact", 0.0), s["approximated"] / n)
    method = max(best.values(), default=0.0)
    assert sur_frac > 10 * method, (sur_frac, best)

"""LavaMD-style neighbour-box forces on the GPU (hpac_lavamd_run) against the
oracle (oracle/lavamd_oracle.c) on the same seeded particles.

Outputs: the GPU sums the same pair terms, fusing multiply-adds, with an
exponential within two ulps and each box's terms in four interleaved partial
sums, so each potential and force component agrees within 1e-12 of the
particle's potential: the FP64 parity bar, scaled by the potential because a
force component can cancel to near zero while the sum of its terms'
magnitudes stays below twice the potential. (A model of these roundings puts
the largest difference near 1e-15 at 16^3 boxes.) Masks: iACT distances are formed by the
same single-precision operations on both sides, so its decisions agree bit for
bit; TAF decisions compare an RSD of potentials that agree to ~1e-15, so its
masks agree except in the groups (particle, warp or box) of a decision whose
RSD lies within 1e-6 of the threshold, and outside those groups the outputs
agree as above."""
import numpy as np
import pytest

from paper_2308_16877_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

A2 = W.LAVAMD_A2
TOL = 1e-12


@pytest.fixture(scope="module")
def H():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2308_16877_gb300 import hpac
    hpac.load()
    return hpac


def run_both(H, orc, B, NP, seed, technique=0, **kn):
    rq = W.lavamd_inputs(B, NP, seed=seed)
    P = rq.shape[1]
    d = torch.from_numpy(rq).cuda()
    mask = torch.full((max(27 * P, 1),), 255, dtype=torch.uint8, device="cuda")
    fv, st = H.lavamd(d, B, NP, A2, technique=technique, mask=mask, stats=True, **kn)
    okn = {k: v for k, v in kn.items() if k != "reset_on_exit"}
    if "reset_on_exit" in kn:
        okn["reset"] = int(kn["reset_on_exit"])
    ofv, ocnt, om = orc.lavamd(B, NP, A2, rq, technique=technique, mask=True, **okn)
    torch.cuda.synchronize()
    return fv.cpu().numpy(), st, mask.cpu().numpy()[:27 * P], ofv, ocnt, om


def check_outputs(fv, ofv):
    pot = np.abs(ofv[0])
    err = np.abs(fv - ofv) / np.maximum(pot, 1e-300)
    assert np.all(np.isfinite(fv))
    assert err.size == 0 or err.max() <= TOL, err.max()


def check_taf(B, NP, level, fv, st, m, ofv, ocnt, om):
    """A decision whose RSD lies within 1e-6 of the threshold may go either way
    on either side; it changes the later decisions of its group only (the
    particle, its warp or its box). So at most one group per borderline
    decision may differ, and everything outside those groups agrees."""
    P = B ** 3 * NP
    diff = np.any(m.reshape(27, P) != om.reshape(27, P), axis=0)
    p = np.arange(P)
    box, lane = p // NP, p % NP
    gid = p if level == 0 else (box * 64 + lane // 32 if level == 1 else box)
    bad = np.unique(gid[diff])
    assert len(bad) <= max(int(ocnt[3]), int(st["borderline"]))
    keep = ~np.isin(gid, bad)
    check_outputs(fv[:, keep], ofv[:, keep])
    if len(bad) == 0:
        assert np.array_equal(m, om) and st["approximated"] == ocnt[1]


@pytest.mark.parametrize("B,NP", [(1, 1), (1, 100), (2, 33), (3, 100), (4, 37), (3, 128), (5, 64), (2, 257),
                                  (2, 1024)])
def test_exact(H, orc, B, NP):
    fv, st, m, ofv, ocnt, om = run_both(H, orc, B, NP, seed=B * 1000 + NP)
    check_outputs(fv, ofv)
    assert np.array_equal(m, om)
    assert st["invocations"] == ocnt[0] == (3 * B - 2) ** 3 * NP
    assert st["approximated"] == 0


TAF_CASES = [(4, 8, 0.02), (2, 3, 0.05), (3, 1, 0.1), (1, 2, 0.0), (5, 4, np.inf), (4, 0, 0.05), (8, 8, 0.03)]


@pytest.mark.parametrize("level", [0, 1, 2])
@pytest.mark.parametrize("h,p,thr", TAF_CASES)
def test_taf(H, orc, level, h, p, thr):
    B, NP = 4, 100
    fv, st, m, ofv, ocnt, om = run_both(H, orc, B, NP, seed=17, technique=1, level=level, hsize=h, psize=p,
                                        thresh=thr)
    check_taf(B, NP, level, fv, st, m, ofv, ocnt, om)
    assert st["borderline"] == ocnt[3]
    if 0 < thr < np.inf and p > 0 and h > 1:
        assert ocnt[1] > 0


@pytest.mark.parametrize("level", [0, 1, 2])
def test_taf_window_emptied_after_a_run(H, orc, level):
    fv, st, m, ofv, ocnt, om = run_both(H, orc, 3, 70, seed=4, technique=1, level=level, hsize=3, psize=2,
                                        thresh=0.05, reset_on_exit=True)
    assert ocnt[3] == 0 and ocnt[1] > 0
    check_taf(3, 70, level, fv, st, m, ofv, ocnt, om)


@pytest.mark.parametrize("level", [0, 1, 2])
@pytest.mark.parametrize("tsize,g,thr", [(8, 1, 0.05), (4, 4, 0.1), (16, 2, 0.2), (2, 32, 0.01), (8, 8, np.inf),
                                         (1, 1, 0.3), (8, 16, 0.0)])
def test_iact(H, orc, level, tsize, g, thr):
    B, NP = 4, 100
    fv, st, m, ofv, ocnt, om = run_both(H, orc, B, NP, seed=23, technique=2, level=level, tsize=tsize,
                                        tperwarp=g, thresh=thr)
    assert np.array_equal(m, om)
    assert st["approximated"] == ocnt[1] and st["borderline"] == ocnt[3]
    check_outputs(fv, ofv)


def test_iact_scaled_inputs(H, orc):
    fv, st, m, ofv, ocnt, om = run_both(H, orc, 3, 45, seed=8, technique=2, level=1, tsize=6, tperwarp=2,
                                        thresh=0.08, in_scale=[2.0, 0.5, 1.25])
    assert ocnt[1] > 0 and np.array_equal(m, om) and st["approximated"] == ocnt[1]
    check_outputs(fv, ofv)


@pytest.mark.parametrize("technique,kn", [(1, dict(hsize=3, psize=4, thresh=0.05)),
                                          (2, dict(tsize=4, tperwarp=1, thresh=0.3))])
def test_one_particle_per_box_all_levels_agree(H, orc, technique, kn):
    res = [run_both(H, orc, 5, 1, seed=31, technique=technique, level=lv, **kn) for lv in (0, 1, 2)]
    for fv, st, m, ofv, ocnt, om in res:
        assert ocnt[3] == 0
        assert np.array_equal(m, om) and st["approximated"] == ocnt[1]
        check_outputs(fv, ofv)
    assert np.array_equal(res[0][2], res[1][2]) and np.array_equal(res[0][2], res[2][2])


def test_bench_size(H, orc):
    """The benchmark's 16^3 boxes of 100 particles, exact and the two forms it
    times at warp level, against the whole oracle run."""
    B, NP = 16, W.LAVAMD_PAR_PER_BOX
    for technique, kn in ((0, {}), (1, dict(level=1, hsize=4, psize=8, thresh=0.04)),
                          (2, dict(level=1, tsize=8, tperwarp=1, thresh=0.05))):
        fv, st, m, ofv, ocnt, om = run_both(H, orc, B, NP, seed=W.DEFAULT_SEED, technique=technique, **kn)
        if technique == 1:
            check_taf(B, NP, 1, fv, st, m, ofv, ocnt, om)
        else:
            assert np.array_equal(m, om) and st["approximated"] == ocnt[1]
            check_outputs(fv, ofv)


def test_empty_grid_and_rejected_arguments(H):
    e = torch.zeros((4, 0), dtype=torch.float64, device="cuda")
    fv, st = H.lavamd(e, 0, 10, A2, stats=True)
    assert st["invocations"] == 0 and fv.numel() == 0
    rq = torch.from_numpy(W.lavamd_inputs(2, 4)).cuda()
    with pytest.raises(H.HpacError):
        H.lavamd(rq, 2, 4, A2, technique=1, hsize=0)
    with pytest.raises(H.HpacError):
        H.lavamd(rq, 2, 4, A2, technique=2, tperwarp=3)
    with pytest.raises(H.HpacError):
        H.lavamd(rq, 2, 4, -1.0)
    big = torch.from_numpy(W.lavamd_inputs(1, 1024)).cuda()
    with pytest.raises(H.HpacError):   # 64 x 4 x 1024 window doubles: beyond shared memory
        H.lavamd(big, 1, 1024, A2, technique=1, hsize=64)
    desc = H.hpac_lavamd_desc(2, 4, A2)
    base = rq.data_ptr()
    with pytest.raises(H.HpacError):   # misaligned input
        H.hpac_lavamd_run(desc, 0, None, base + 4, base, None)

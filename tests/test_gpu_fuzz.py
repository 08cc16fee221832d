"""Seeded random configurations of perforation, TAF and iACT on the identity
region (both sides see bit-identical values, so every mask, output and
statistic must equal the oracle's): random lengths (ragged against every
tile), logical-thread counts, block sizes, knobs over their whole ranges,
decision levels, value types and input kinds. Configurations the device
cannot hold (iACT tables beyond the shared memory of one block) must be
rejected with HPAC_EUNSUPPORTED before any launch."""
import numpy as np
import pytest

from paper_2308_16877_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

CASES = 160


@pytest.fixture(scope="module")
def H():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2308_16877_gb300 import hpac
    hpac.load()
    return hpac


def draw(rng):
    tech = ["perfo", "taf", "iact"][int(rng.integers(0, 3))]
    dt = [np.float32, np.float64][int(rng.integers(0, 2))]
    n = int(rng.integers(0, 20000))
    T = int(rng.choice([0, int(rng.integers(1, 64)), int(rng.integers(1, max(2, n + 1)))]))
    B = 32 * int(rng.integers(1, 33))
    level = int(rng.integers(0, 3))
    d = int(rng.integers(1, 5))
    ikind = ["walk", "levels", "uniform"][int(rng.integers(0, 3))]
    thr = float(rng.choice([0.0, np.inf, 10.0 ** rng.uniform(-5, 0), 10.0 ** rng.uniform(-1.5, 0.5),
                            10.0 ** rng.uniform(-1.5, 0.5)]))
    return dict(tech=tech, dt=dt, n=n, T=T, B=B, level=level, d=d, ikind=ikind, thr=thr,
                h=int(rng.integers(1, 17)), p=int(rng.integers(1, 65)),
                tsize=int(rng.integers(1, 65)), g=int(rng.choice([1, 2, 4, 8, 16, 32])),
                pk=int(rng.integers(0, 5)), m=int(rng.integers(1, 12)), pct=int(rng.integers(0, 101)),
                rate=float(rng.uniform(0, 1)), herded=int(rng.integers(0, 2)), seed=int(rng.integers(0, 1 << 30)))


@pytest.mark.parametrize("case", range(CASES))
def test_random_configuration(H, orc, case):
    c = draw(np.random.default_rng(1000 + case))
    n, dt = c["n"], c["dt"]
    x = W.identity_inputs(n, d=c["d"], dtype=dt, kind=c["ikind"], seed=case)
    xd = torch.from_numpy(np.ascontiguousarray(x)).cuda()
    tdt = torch.float32 if dt == np.float32 else torch.float64
    out = torch.full((n,), float("nan"), dtype=tdt, device="cuda")
    mask = torch.full((n,), 255, dtype=torch.uint8, device="cuda")
    with H.Region(3, xd, logical_threads=c["T"], block_threads=c["B"]) as R:
        if c["tech"] == "perfo":
            mo = c["m"] if c["pk"] in (0, 1) else c["pct"]
            st = R.run_perfo(xd, out, c["pk"], mo, c["rate"], c["seed"], bool(c["herded"]), mask=mask,
                             stats=True)
            o, om, cnt = orc.run_perfo(3, x, 0.0, c["pk"], mo, c["rate"], c["seed"], c["herded"],
                                       threads=c["T"], block=c["B"], out=np.full(n, np.nan, dtype=dt))
            assert st["skipped"] == cnt[2]
        elif c["tech"] == "taf":
            stat = torch.full((n,), -1.0, dtype=tdt, device="cuda")
            st = R.run_taf(xd, out, c["h"], c["p"], c["thr"], c["level"], mask=mask, stat=stat,
                           stats=True)
            o, om, os_, cnt = orc.run_taf(3, x, 0.0, c["h"], c["p"], c["thr"], level=c["level"],
                                          threads=c["T"], block=c["B"])
            assert np.array_equal(stat.cpu().numpy(), os_, equal_nan=True)
            assert st["approximated"] == cnt[1] and st["borderline"] == cnt[3]
            # the fast decision path (no statistic, no counters) takes the same decisions
            out2 = torch.zeros(n, dtype=tdt, device="cuda")
            mask2 = torch.zeros(n, dtype=torch.uint8, device="cuda")
            R.run_taf(xd, out2, c["h"], c["p"], c["thr"], c["level"], mask=mask2)
            assert np.array_equal(mask2.cpu().numpy(), om) and np.array_equal(out2.cpu().numpy(), o)
        else:
            sc = W.iact_scale(x, n)
            stat = torch.full((n,), -1.0, dtype=tdt, device="cuda")
            try:
                st = R.run_iact(xd, out, c["tsize"], c["g"], c["thr"], c["level"], in_scale=sc, mask=mask,
                                stat=stat, stats=True)
            except H.HpacError as e:
                assert e.status == H.HPAC_EUNSUPPORTED and c["level"] == 2, str(e)
                return
            o, om, os_, cnt = orc.run_iact(3, x, 0.0, c["tsize"], c["g"], c["thr"], level=c["level"],
                                           in_scale=sc, threads=c["T"], block=c["B"])
            assert np.array_equal(stat.cpu().numpy(), os_, equal_nan=True)
            assert st["approximated"] == cnt[1] and st["borderline"] == cnt[3]
    torch.cuda.synchronize()
    assert np.array_equal(mask.cpu().numpy(), om), c
    g = out.cpu().numpy()
    if c["tech"] == "perfo":
        assert np.array_equal(np.isnan(g), np.isnan(o)) and np.array_equal(g[~np.isnan(o)], o[~np.isnan(o)])
    else:
        assert np.array_equal(g, o), c


@pytest.mark.parametrize("case", range(48))
def test_random_persistent_sequence(H, orc, case):
    """Seeded random sequences of 2 to 5 calls on one region with state kept
    across calls (TAF or iACT on the identity region): a random length (rarely
    a multiple of T), knobs, level and block size, new inputs every call and a
    random reset between calls; every call's masks and outputs equal the
    oracle's persistent call."""
    rng = np.random.default_rng(5000 + case)
    tech = ["taf", "iact"][case % 2]
    dt = [np.float32, np.float64][int(rng.integers(0, 2))]
    T = int(rng.integers(1, 3000))
    B = 32 * int(rng.integers(1, 17))
    level = int(rng.integers(0, 3))
    thr = float(10.0 ** rng.uniform(-2, 0.3))
    h, p = int(rng.integers(1, 9)), int(rng.integers(1, 17))
    ts, g = int(rng.integers(1, 9)), int(rng.choice([1, 4, 16, 32]))
    calls = int(rng.integers(2, 6))
    n = int(rng.integers(1, 4 * T + 50))
    x = W.identity_inputs(n * calls, d=2, dtype=dt, kind="walk", seed=case)
    tdt = torch.float32 if dt == np.float32 else torch.float64
    fresh = lambda: orc.taf_state(T, h) if tech == "taf" else orc.iact_state(T, ts, g, 2)
    st = fresh()
    sc = W.iact_scale(x, x.shape[1])
    with H.Region(3, dev_(x[:, :n]), param=0.0, logical_threads=T, block_threads=B) as R:
        R.set_persistent(True)
        for c in range(calls):
            xs = np.ascontiguousarray(x[:, c * n:(c + 1) * n])
            if c > 0 and rng.random() < 0.25:
                R.reset_state()
                st = fresh()
            out = torch.full((n,), float("nan"), dtype=tdt, device="cuda")
            mask = torch.full((n,), 255, dtype=torch.uint8, device="cuda")
            if tech == "taf":
                R.run_taf(dev_(xs), out, h, p, thr, level, mask=mask)
                o, m, _, _ = orc.run_taf(3, xs, 0.0, h, p, thr, level=level, threads=T, block=B, state=st)
            else:
                R.run_iact(dev_(xs), out, ts, g, thr, level, in_scale=sc, mask=mask)
                o, m, _, _ = orc.run_iact(3, xs, 0.0, ts, g, thr, level=level, in_scale=sc, threads=T,
                                          block=B, state=st)
            torch.cuda.synchronize()
            assert np.array_equal(mask.cpu().numpy(), m), c
            assert np.array_equal(out.cpu().numpy(), o), c


def dev_(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()

"""Host-side logic of the benchmark that needs no GPU: the traffic record's
source digest, the compact formatting of the final line and the headline's
candidate forms."""
import os
import sys

import numpy as np

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402


def test_traffic_record_matches_the_current_element_kernel_source():
    # the committed DRAM-bytes record is only reported while its digest equals
    # the kernel source's; a stale record reads as null
    rec = {}
    for line in open(os.path.join(bench.ROOT, "profiles", "dram_traffic.txt")):
        f = line.split()
        if len(f) >= 3 and not line.startswith("#"):
            rec[f[0]] = f[2]
    assert set(rec) >= {"elem_kernel", "node_kernel"}
    for tag, dig in rec.items():
        assert (bench.dram_traffic(tag, 1) is not None) == (dig == bench.source_digest(tag))


def test_compact_rounding():
    assert bench.sig(1.23456789) == 1.235
    assert bench.sig({"a": [2.0 / 3.0, 7]}) == {"a": [0.6667, 7]}
    assert bench.sig(float("nan")) is None


def test_headline_forms_and_oracle_knobs():
    import oracle
    names = [f[0] for f in bench.HEAD_FORMS]
    assert len(set(names)) == len(names)
    for f in bench.HEAD_FORMS:
        k = bench.form_oracle_knobs(oracle, f, 8)
        assert k.mode == f[1] and (k.st[0] is not None) == f[2]


def test_lavamd_section_plumbing(monkeypatch):
    """The LavaMD section's bookkeeping on a 3^3 grid, with the library
    replaced by the oracle and CUDA events by a fixed clock: every form is
    timed at every level and scored against the exact run, and the roofline
    counts the pair terms the oracle reports."""
    import types

    import torch

    import oracle

    class Event:
        def __init__(self, enable_timing=False):
            pass

        def record(self, stream=None):
            pass

        def elapsed_time(self, other):
            return 12.0

    monkeypatch.setattr(torch.cuda, "Event", Event)
    monkeypatch.setattr(torch.cuda, "synchronize", lambda *a, **k: None)
    monkeypatch.setattr(torch.cuda, "get_device_properties",
                        lambda d: types.SimpleNamespace(multi_processor_count=152))

    class Lib:
        LAVAMD_TAF, LAVAMD_IACT = oracle.LAVAMD_TAF, oracle.LAVAMD_IACT
        HPAC_LEVEL_THREAD, HPAC_LEVEL_WARP, HPAC_LEVEL_BLOCK = oracle.THREAD, oracle.WARP, oracle.BLOCK
        HPAC_METRIC_MAPE, HPAC_METRIC_RMSE = oracle.MAPE, oracle.RMSE

        @staticmethod
        def lavamd(rq, B, NP, a2, technique=0, fv=None, stats=False, stream=None, level=0, **kn):
            kn = {k: v for k, v in kn.items() if k != "reset_on_exit"}
            out, cnt, _ = oracle.lavamd(B, NP, a2, rq.numpy(), technique=technique, level=level, **kn)
            fv.copy_(torch.from_numpy(out))
            st = {"invocations": int(cnt[0]), "approximated": int(cnt[1]), "skipped": 0,
                  "borderline": int(cnt[3])}
            return (fv, st) if stats else fv

        @staticmethod
        def quality(a, b, metric, stream=None):
            return {"value": oracle.quality(a.numpy(), b.numpy(), metric)[0]}

        @staticmethod
        def hpac_device_fp64_rate(stream=None):
            return 1.0

    r = bench.bench_lavamd(Lib, torch, torch.device("cpu"), types.SimpleNamespace(cuda_stream=None),
                           boxes1d=3)
    assert r["invocations"] == 7 ** 3 * 100 and r["pair_terms"] == r["invocations"] * 100
    assert len(r["table"]) == 12
    assert {(t["technique"], t["level"]) for t in r["table"]} == {
        (t, lv) for t in ("taf", "iact") for lv in ("thread", "warp", "block")}
    for t in r["table"]:
        assert t["speedup_vs_exact"] == 1.0 and 0.0 <= t["approximated"] <= 1.0
        assert t["potential_mape"] >= 0.0 and t["force_nrmse"] >= 0.0
    rl = r["roofline"]
    assert abs(rl["frac"] - rl["achieved"] / rl["peak"]) <= 1e-12
    assert r["exact_ms"] == 12.0 / 3       # three timed repetitions in 12 ms
    expect = bench.LAVAMD_PAIR_FP64_INSTR * r["pair_terms"] / (r["exact_ms"] * 1e-3)
    assert abs(rl["achieved"] * 1e12 - expect) <= 1e-9 * expect

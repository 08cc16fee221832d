"""Benchmark of the approximate-region hot path on GB300.

One step runs every technique of the hot path over one resident batch of the
workload: the accurate region, herded perforation, TAF and iACT (the paper's
three techniques, Section 2.3, with the GPU algorithms of Section 3.1), and the
quality loss of each against a double-precision exact run (Section 4). It
prints one JSON line: `value` is region invocations per second over the whole
step (all passes), per-pass timings give the speedup of each technique over the
accurate kernel on the same GPU, `roofline` covers the dominant kernel and
`cpu_baseline` the CPU oracle on a bounded sample of the same workload.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Under torchrun (N > 1) every rank runs an independent replica of the whole
step (the path shards by region with no exchange), `value` sums the ranks'
invocations over the slowest rank's time.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_2308_16877_gb300 import workloads as W  # noqa: E402

METRIC = "region elements/s and speedup vs exact kernel on 1 GB300 at <=1% quality loss"

# Black-Scholes batch: the option distributions, history/prediction/threshold
# and perforation of the 65,536-option configuration, at 2^24 options so that
# the 256 MB of inputs exceed the 129 MB L2 and every pass streams from HBM.
BS_N = 1 << 24
BS_IPT = 8                      # items per logical thread (T = N / 8)
TAF_KNOBS = dict(hsize=4, psize=8, thresh=0.005, level=0)
PERFO_KNOBS = dict(kind=0, m_or_percent=4, herded=True)     # skip every 4th
IACT_KNOBS = dict(tsize=8, tperwarp=32, thresh=0.05, level=1)


def env_rank():
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)),
            int(os.environ.get("LOCAL_RANK", 0)))


class ClockSampler:
    """Samples SM clocks and throttle reasons with nvidia-smi during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in self.lines:
            f = [c.strip() for c in l.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


KERNEL_TAGS = {"exact": "map_kernel<BlackScholes32,4>", "perfo": "map_kernel<BlackScholes32,4>",
               "taf": "taf_kernel<BlackScholes32,thread>", "iact": "iact_kernel<BlackScholes32,warp>"}
KERNEL_SOURCES = {"map_kernel": ["exact_perfo.cu", "regions.cuh"], "taf_kernel": ["taf.cu", "regions.cuh"],
                  "iact_kernel": ["iact.cu", "regions.cuh"]}


def source_digest(tag):
    import hashlib
    h = hashlib.sha1()
    for f in KERNEL_SOURCES[tag.split("<")[0]]:
        with open(os.path.join(ROOT, "paper_2308_16877_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:12]


def dram_traffic(tag, n):
    """DRAM bytes (read + write) per launch of `tag` at n invocations, scaled
    from the ncu capture recorded in profiles/dram_traffic.txt; None when the
    kernel's sources changed since that capture."""
    p = os.path.join(ROOT, "profiles", "dram_traffic.txt")
    if not os.path.exists(p):
        return None
    for line in open(p):
        f = line.split()
        if len(f) >= 4 and not line.startswith("#") and f[0] == tag:
            per_inv, digest = float(f[1]), f[2]
            return per_inv * n if digest == source_digest(tag) else None
    return None


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d.get("hbm_gbs", 6800.0), "measured"
    return 6800.0, "fallback"


# ---------------------------------------------------------------- CPU oracle

def cpu_baseline(sample_n=1 << 22):
    """The oracle as it stands, timed on the host cores on a bounded sample of
    the same workload (the same four passes on `sample_n` options)."""
    import oracle
    x = W.blackscholes_inputs(sample_n)
    T = sample_n // BS_IPT
    sc = W.iact_scale(x, sample_n)
    t0 = time.perf_counter()
    oracle.run_exact(oracle.BLACKSCHOLES, x, W.BS_RATE)
    oracle.run_perfo(oracle.BLACKSCHOLES, x, W.BS_RATE, PERFO_KNOBS["kind"], PERFO_KNOBS["m_or_percent"],
                     herded=1, threads=T)
    oracle.run_taf(oracle.BLACKSCHOLES, x, W.BS_RATE, TAF_KNOBS["hsize"], TAF_KNOBS["psize"],
                   TAF_KNOBS["thresh"], level=TAF_KNOBS["level"], threads=T)
    oracle.run_iact(oracle.BLACKSCHOLES, x, W.BS_RATE, IACT_KNOBS["tsize"], IACT_KNOBS["tperwarp"],
                    IACT_KNOBS["thresh"], level=IACT_KNOBS["level"], in_scale=sc, threads=T)
    dt = time.perf_counter() - t0
    return {"value": 4 * sample_n / dt, "unit": "elements/s", "cores": oracle.num_threads(),
            "kind": "oracle",
            "sample": f"{sample_n} options, the step's four passes (exact, perforation, TAF, iACT)",
            "seconds": dt}


def run_reference(args):
    rank, world, _ = env_rank()
    if rank != 0:
        return 0
    import oracle
    oracle.lib()
    sample_n = 1 << 21
    times = []
    for i in range(args.warmup + args.steps):
        cb = cpu_baseline(sample_n)
        if i >= args.warmup:
            times.append(cb["seconds"])
    v = 4 * sample_n * len(times) / sum(times)
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "elements/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * sum(times) / len(times), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"blackscholes {sample_n} options (bounded CPU sample)",
                       "parallelism": "oracle on host cores"},
            "cpu_baseline": {"value": v, "unit": "elements/s", "cores": oracle.num_threads(),
                             "kind": "oracle", "sample": f"{sample_n} options per step, four passes"},
            "e2e": {"value": v, "unit": "elements/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


# ---------------------------------------------------------------- GPU arm

def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--n", type=int, default=BS_N)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args(argv)
    if args.impl == "reference":
        return run_reference(args)

    import torch
    import torch.distributed as dist

    from paper_2308_16877_gb300 import hpac

    rank, world, local = env_rank()
    if world > 1:
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    hpac.load()

    n = args.n
    T = n // BS_IPT
    x_h = W.blackscholes_inputs(n, seed=W.DEFAULT_SEED + rank)
    x = torch.from_numpy(x_h).to(dev)
    out = {k: torch.zeros(n, dtype=torch.float32, device=dev) for k in ("exact", "perfo", "taf", "iact")}
    sc = W.iact_scale(x_h, n)
    stream = torch.cuda.current_stream(dev)

    R = hpac.Region(hpac.HPAC_REGION_BLACKSCHOLES, x, param=W.BS_RATE, logical_threads=T,
                    block_threads=256, stream=stream)
    # double-precision exact reference for the quality loss (computed once)
    ref = torch.zeros(n, dtype=torch.float64, device=dev)
    x64 = x.double().contiguous()
    with hpac.Region(hpac.HPAC_REGION_BLACKSCHOLES, x64, param=W.BS_RATE, stream=stream) as R64:
        R64.run_exact(x64, ref)
    del x64

    passes = ["exact", "perfo", "taf", "iact"]
    launches_per_pass = {"exact": 1, "perfo": 1, "taf": 1, "iact": 1}

    def run_pass(p):
        if p == "exact":
            R.run_exact(x, out[p])
        elif p == "perfo":
            R.run_perfo(x, out[p], PERFO_KNOBS["kind"], PERFO_KNOBS["m_or_percent"],
                        herded=PERFO_KNOBS["herded"])
        elif p == "taf":
            R.run_taf(x, out[p], **TAF_KNOBS)
        else:
            R.run_iact(x, out[p], in_scale=sc, **IACT_KNOBS)

    def step(events=None):
        for j, p in enumerate(passes):
            if events is not None:
                events[j][0].record(stream)
            run_pass(p)
            if events is not None:
                events[j][1].record(stream)
        q = {p: hpac.quality(ref, out[p], hpac.HPAC_METRIC_MAPE, stream=stream)["value"] for p in passes}
        return q

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    clk = ClockSampler(local).__enter__()
    # untimed pre-heat of about one second so that the clock record has samples
    # under load on both sides of the timed region
    t_end = time.perf_counter() + 1.0
    while time.perf_counter() < t_end:
        step()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()

    ev = [[[torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)]
           for _ in passes] for _ in range(args.steps)]
    start, stop = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    start.record(stream)
    for s in range(args.steps):
        quality = step(ev[s])
    stop.record(stream)
    torch.cuda.synchronize()
    t_end = time.perf_counter() + 0.5
    while time.perf_counter() < t_end:
        step()
    torch.cuda.synchronize()
    clk.__exit__()
    total_ms = start.elapsed_time(stop)
    if world > 1:
        t = torch.tensor([total_ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    pass_ms = {p: float(np.mean([ev[s][j][0].elapsed_time(ev[s][j][1]) for s in range(args.steps)]))
               for j, p in enumerate(passes)}
    ms_per_step = total_ms / args.steps
    value = world * len(passes) * n / (ms_per_step * 1e-3)

    # statistics of the approximated passes (outside the timed region)
    stats = {
        "perfo": R.run_perfo(x, out["perfo"], PERFO_KNOBS["kind"], PERFO_KNOBS["m_or_percent"],
                             herded=True, stats=True),
        "taf": R.run_taf(x, out["taf"], stats=True, **TAF_KNOBS),
        "iact": R.run_iact(x, out["iact"], in_scale=sc, stats=True, **IACT_KNOBS),
    }
    rmse = {p: hpac.quality(ref, out[p], hpac.HPAC_METRIC_RMSE, stream=stream)["value"] for p in passes}
    rms_ref = float(torch.sqrt(torch.mean(ref * ref)).item())
    nrmse = {p: rmse[p] / rms_ref for p in passes}

    # algorithmic bytes per pass: 16 B of inputs + 4 B of output per evaluated
    # invocation; a TAF prediction writes 4 B; a dropped invocation moves none
    def bytes_of(p):
        if p == "exact" or p == "iact":
            return 20 * n
        if p == "perfo":
            return 20 * (n - stats["perfo"]["skipped"])
        a = stats["taf"]["approximated"]
        return 20 * (n - a) + 4 * a

    dom = max(passes, key=lambda p: pass_ms[p])
    peak, peak_src = measured_peaks()
    achieved = bytes_of(dom) / (pass_ms[dom] * 1e-3) / 1e9
    traffic = dram_traffic(KERNEL_TAGS[dom], n)
    roofline = {"bound": "hbm", "kernel": KERNEL_TAGS[dom], "achieved": achieved, "peak": peak,
                "unit": "GB/s", "frac": achieved / peak, "peak_source": peak_src,
                "traffic": traffic, "bytes_per_launch": bytes_of(dom)}
    exact_achieved = bytes_of("exact") / (pass_ms["exact"] * 1e-3) / 1e9

    # end to end through the public API with host buffers: pinned inputs copied
    # in, the TAF pass, outputs copied back, every step
    x_pin = torch.from_numpy(x_h).pin_memory()
    o_pin = torch.empty(n, dtype=torch.float32).pin_memory()
    xd = torch.empty_like(x)
    for _ in range(2):
        xd.copy_(x_pin, non_blocking=True)
        R.run_taf(xd, out["taf"], **TAF_KNOBS)
        o_pin.copy_(out["taf"], non_blocking=True)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        xd.copy_(x_pin, non_blocking=True)
        R.run_taf(xd, out["taf"], **TAF_KNOBS)
        o_pin.copy_(out["taf"], non_blocking=True)
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = e0.elapsed_time(e1) / args.steps
    e2e = {"value": world * n / (e2e_ms * 1e-3), "unit": "elements/s", "pass": "taf",
           "h2d_bytes_per_step": int(x_h.nbytes), "d2h_bytes_per_step": int(4 * n)}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline()
        cpu.pop("seconds", None)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "elements/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": f"blackscholes {n} options (uniform S,K,T,sigma; strike-sorted runs of 32), "
                                   "exact + perforation small:4 + TAF h4/p8/0.5% + iACT t8/warp",
                       "logical_threads": T, "block_threads": 256,
                       "l2": "inputs (256 MB) larger than L2", "parallelism": f"replicas{world}"},
            "roofline": roofline,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": args.steps * (sum(launches_per_pass.values()) + 2 * len(passes)),
            "clocks": clk.summary(),
            "passes_ms": pass_ms,
            "speedup_vs_exact": {p: pass_ms["exact"] / pass_ms[p] for p in passes},
            "exact_kernel_roofline_frac": exact_achieved / peak,
            "quality_mape": quality, "quality_rmse": rmse, "quality_nrmse": nrmse,
            "approximated": {k: v for k, v in stats.items()},
        }
        print(json.dumps(line))
    R.close()
    if world > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())

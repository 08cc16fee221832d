"""Schedule autotuner for the batched knob sweep.

The sweep's results do not depend on its schedule (TAF runs at thread level and
perforation per invocation, so neither the physical block size nor the work-item
size changes a decision); only its speed does. This picks, by timing with CUDA
events on the real workload, the physical block size, persistent blocks per SM
and logical blocks per work item, and caches the choice on disk keyed by the
device name, the region sizes and the configuration count.
"""
from __future__ import annotations

import hashlib
import json
import os

CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_build", "autotune.json")
CANDIDATES = [(bt, bps, tb) for bt in (128, 256) for bps in (4, 8) for tb in (1, 2, 4)]


def _kernel_digest():
    """Digest of the sweep kernel's source, so that a changed kernel is re-tuned."""
    src = os.path.join(os.path.dirname(os.path.abspath(__file__)), "csrc", "sweep.cu")
    try:
        with open(src, "rb") as f:
            return hashlib.sha1(f.read()).hexdigest()[:12]
    except OSError:
        return ""


def _key(device_name, regions, n_configs):
    h = hashlib.sha1(json.dumps([device_name, [r[0] for r in regions], n_configs,
                                 _kernel_digest()]).encode())
    return h.hexdigest()[:16]


def _load():
    try:
        with open(CACHE) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def tune_sweep(make, regions, n_configs, reps=3, candidates=None, use_cache=True):
    """make(block_threads, blocks_per_sm, tile_blocks) -> Sweep. Returns
    (best (bt, bps, tb), {candidate: ms}) and records the best in the cache."""
    import torch
    name = torch.cuda.get_device_name()
    key = _key(name, regions, n_configs)
    cache = _load()
    if use_cache and key in cache:
        return tuple(cache[key]["best"]), cache[key]["ms"]
    timings = {}
    for cand in candidates or CANDIDATES:
        sw = make(*cand)
        sw.run()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            sw.run()
        e1.record()
        torch.cuda.synchronize()
        timings[",".join(map(str, cand))] = e0.elapsed_time(e1) / reps
        sw.close()
    best = min(timings, key=timings.get)
    cache[key] = {"best": [int(v) for v in best.split(",")], "ms": timings, "device": name}
    os.makedirs(os.path.dirname(CACHE), exist_ok=True)
    tmp = CACHE + f".{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(cache, f, indent=1)
    os.replace(tmp, CACHE)
    return tuple(cache[key]["best"]), timings

"""Schedule autotuner for the batched knob sweep.

The sweep's results do not depend on its schedule (TAF runs at thread level and
perforation per invocation, so neither the physical block size nor the work-item
size changes a decision); only its speed does. The schedule space is the
physical block size (64, 128, 256 threads), the persistent blocks per SM
(1 to 16) and the logical blocks per work item (1 to 16): 90 points. The tuner
times candidates with CUDA events on the real workload and searches the space
by coordinate descent: from a starting point it times every value of one
coordinate with the others fixed, moves to the best, and cycles through the
coordinates until a full cycle improves nothing (typically 20 to 30 timed
points instead of 90). The choice is cached on disk keyed by the device name,
the region sizes, the configuration count and the kernel's source.
"""
from __future__ import annotations

import hashlib
import json
import os

CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_build", "autotune.json")
AXES = ((64, 128, 256), (1, 2, 4, 8, 12, 16), (1, 2, 4, 8, 16))
START = (128, 8, 4)


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


def coordinate_descent(cost, axes=AXES, start=START, max_cycles=6):
    """Minimise cost(point) over the grid axes[0] x axes[1] x ... by
    coordinate descent from `start`; every point is evaluated at most once.
    Returns (best point, {point: cost})."""
    seen = {}

    def f(pt):
        if pt not in seen:
            seen[pt] = cost(pt)
        return seen[pt]

    best = tuple(start)
    best_c = f(best)
    for _ in range(max_cycles):
        moved = False
        for ax, values in enumerate(axes):
            for v in values:
                pt = best[:ax] + (v,) + best[ax + 1:]
                c = f(pt)
                if c < best_c:
                    best, best_c, moved = pt, c, True
        if not moved:
            break
    return best, seen


def tune_sweep(make, regions, n_configs, reps=3, use_cache=True):
    """make(block_threads, blocks_per_sm, tile_blocks) -> Sweep. Returns
    (best (bt, bps, tb), {candidate: ms}) and records the best in the cache."""
    import torch
    name = torch.cuda.get_device_name()
    key = _key(name, regions, n_configs)
    cache = _load()
    if use_cache and key in cache:
        return tuple(cache[key]["best"]), cache[key]["ms"]

    def timed(cand):
        sw = make(*cand)
        sw.run()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            sw.run()
        e1.record()
        torch.cuda.synchronize()
        sw.close()
        return e0.elapsed_time(e1) / reps

    best, seen = coordinate_descent(timed)
    timings = {",".join(map(str, k)): v for k, v in seen.items()}
    cache[key] = {"best": list(best), "ms": timings, "device": name}
    os.makedirs(os.path.dirname(CACHE), exist_ok=True)
    tmp = CACHE + f".{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(cache, f, indent=1)
    os.replace(tmp, CACHE)
    return tuple(best), timings

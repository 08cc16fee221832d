"""Knob search with the batched sweep as the evaluator.

The paper explores its design space exhaustively (one build and run per
configuration, Section 4.3) and names search as the way out. Here a seeded
genetic search proposes a population of configurations (TAF and perforation
knobs over continuous and integer ranges, not a fixed grid), evaluates the
whole population in one batched sweep launch, and breeds the next generation
from the best. A configuration is scored by the share of invocations it does
not compute exactly (approximated or skipped: the work the approximation
removes) subject to a quality bound on the normalised RMSE of the outputs;
infeasible ones are ranked below every feasible one by their excess loss.

Host logic only: `evaluate(configs) -> [(saved_fraction, nrmse), ...]` is the
caller's (bench.py and the tests pass the GPU sweep; the CPU tests a closed
form).
"""
from __future__ import annotations

import math

import numpy as np

THRESH_RANGE = (1e-4, 1.0)      # TAF RSD threshold, log-uniform
HSIZE_RANGE = (1, 16)
PSIZE_RANGE = (1, 64)
M_RANGE = (2, 10)               # small / large perforation
PERCENT_RANGE = (5, 50)         # ini / fini perforation
RATE_RANGE = (0.05, 0.5)        # random perforation


def _clip(v, lo, hi):
    return lo if v < lo else hi if v > hi else v


def _q(v, rng_=None):
    """Continuous knobs live on a grid of 1/256 octave: a step computed from a
    measured loss then does not depend on the loss's last bits (the sweep's
    sums are reduced with atomics, so they vary in their final digits)."""
    q = float(2.0 ** (round(math.log2(v) * 256) / 256))
    return q if rng_ is None else _clip(q, *rng_)


def random_config(rng: np.random.Generator) -> dict:
    """One configuration drawn from the whole space (half TAF, half perforation)."""
    if rng.random() < 0.5:
        lo, hi = np.log(THRESH_RANGE)
        return {"tech": "taf", "hsize": int(rng.integers(HSIZE_RANGE[0], HSIZE_RANGE[1] + 1)),
                "psize": int(rng.integers(PSIZE_RANGE[0], PSIZE_RANGE[1] + 1)),
                "thresh": _q(float(np.exp(rng.uniform(lo, hi))), THRESH_RANGE), "level": 0}
    kind = int(rng.integers(0, 5))
    d = {"tech": "perfo", "kind": kind, "herded": int(rng.integers(0, 2)), "seed": int(rng.integers(0, 1 << 30)),
         "m": 0, "rate": 0.0}
    if kind in (0, 1):
        d["m"] = int(rng.integers(M_RANGE[0], M_RANGE[1] + 1))
    elif kind in (2, 3):
        d["m"] = int(rng.integers(PERCENT_RANGE[0], PERCENT_RANGE[1] + 1))
    else:
        d["rate"] = _q(float(rng.uniform(*RATE_RANGE)), RATE_RANGE)
    return d


def mutate(cfg: dict, rng: np.random.Generator, strength: float = 1.0) -> dict:
    """A neighbour: each knob moves with probability 1/2 by a step scaled by strength."""
    d = dict(cfg)
    if d["tech"] == "taf":
        if rng.random() < 0.5:
            d["thresh"] = _q(float(np.exp(np.log(d["thresh"]) + rng.normal(0, 0.7 * strength))), THRESH_RANGE)
        if rng.random() < 0.5:
            d["hsize"] = int(_clip(d["hsize"] + rng.integers(-2, 3), *HSIZE_RANGE))
        if rng.random() < 0.5:
            d["psize"] = int(_clip(round(d["psize"] * math.exp(rng.normal(0, 0.5 * strength))), *PSIZE_RANGE))
        return d
    if d["kind"] in (0, 1):
        d["m"] = int(_clip(d["m"] + rng.integers(-1, 2), *M_RANGE))
    elif d["kind"] in (2, 3):
        d["m"] = int(_clip(d["m"] + rng.integers(-5, 6), *PERCENT_RANGE))
    else:
        d["rate"] = _q(float(_clip(d["rate"] + rng.normal(0, 0.05 * strength), *RATE_RANGE)), RATE_RANGE)
    if rng.random() < 0.1:
        d["herded"] = 1 - d["herded"]
    return d


def toward_bound(cfg: dict, loss: float, bound: float, rng: np.random.Generator) -> dict:
    """Move the configuration's aggressiveness knob (TAF threshold, skip rate,
    M or percentage) so that its loss would land near the bound if the loss
    scaled in proportion: the feasible frontier is where the best ones sit."""
    d = dict(cfg)
    if not (np.isfinite(loss) and loss > 0):
        f = 2.0
    else:
        f = _q(float(np.clip((bound / loss) ** 0.8 * rng.uniform(0.85, 1.0), 0.25, 4.0)))
    if d["tech"] == "taf":
        d["thresh"] = _q(d["thresh"] * f, THRESH_RANGE)
    elif d["kind"] == 4:
        d["rate"] = _q(float(_clip(d["rate"] * f, *RATE_RANGE)), RATE_RANGE)
    elif d["kind"] == 0:      # skips 1/M
        d["m"] = int(_clip(round(d["m"] / f), *M_RANGE))
    elif d["kind"] == 1:      # skips (M-1)/M
        d["m"] = int(_clip(round(1.0 / max(1e-9, 1.0 - f * (1.0 - 1.0 / d["m"]))), *M_RANGE))
    else:
        d["m"] = int(_clip(round(d["m"] * f), *PERCENT_RANGE))
    return d


def crossover(a: dict, b: dict, rng: np.random.Generator) -> dict:
    """Uniform crossover of two configurations of the same technique and pattern;
    otherwise a copy of one parent."""
    same = a["tech"] == b["tech"] and (a["tech"] == "taf" or a["kind"] == b["kind"])
    if not same:
        return dict(a if rng.random() < 0.5 else b)
    return {k: (a[k] if rng.random() < 0.5 else b[k]) for k in a}


def score(saved: float, loss: float, bound: float) -> float:
    """Feasible (loss <= bound): the saved share in [0, 1]. Infeasible: below
    every feasible score, ordered by the excess loss."""
    if not np.isfinite(loss):
        return -np.inf
    return saved if loss <= bound else -(loss - bound) / bound - 1e-9


def key(cfg: dict) -> tuple:
    return tuple(sorted((k, round(v, 12) if isinstance(v, float) else v) for k, v in cfg.items()))


def genetic_search(evaluate, population: int = 32, generations: int = 12, bound: float = 0.01,
                   elite: int = 6, seed: int = 0, tournament: int = 3):
    """Seeded genetic search. evaluate(list of configs) -> list of (saved, loss).
    Each generation is one call of evaluate on `population` configurations (the
    elite are carried and re-scored from memory, not re-evaluated). Returns
    (best config, its (saved, loss), history: per generation the best score)."""
    rng = np.random.default_rng(seed)
    seen: dict = {}
    pop = [random_config(rng) for _ in range(population)]
    history = []
    for gen in range(generations):
        fresh = [c for c in pop if key(c) not in seen]
        if fresh:
            for c, r in zip(fresh, evaluate(fresh)):
                seen[key(c)] = (c, (float(r[0]), float(r[1])))
        ranked = sorted((seen[key(c)] for c in pop), key=lambda cr: score(*cr[1], bound), reverse=True)
        history.append(score(*ranked[0][1], bound))
        if gen == generations - 1:
            break
        parents = [c for c, _ in ranked]
        losses = [r[1] for _, r in ranked]
        nxt = [dict(c) for c in parents[:elite]]
        # the elite's frontier moves: each elite nudged toward the quality bound
        for c, l in zip(parents[:elite], losses[:elite]):
            if len(nxt) < population:
                nxt.append(toward_bound(c, l, bound, rng))
        strength = 1.0 - 0.6 * gen / max(1, generations - 1)
        while len(nxt) < population:
            def pick():
                idx = int(min(rng.choice(len(parents), size=min(tournament, len(parents)), replace=False)))
                return parents[idx], losses[idx]    # ranked list: a lower index is fitter
            (a, la), (b, _) = pick(), pick()
            child = crossover(a, b, rng)
            u = rng.random()
            if u < 0.3:
                child = toward_bound(child, la, bound, rng)
            elif u < 0.85:
                child = mutate(child, rng, strength)
            if rng.random() < 0.1:
                child = random_config(rng)          # immigrants keep the search global
            nxt.append(child)
        pop = nxt
    best_cfg, best_r = max(seen.values(), key=lambda cr: score(*cr[1], bound))
    return best_cfg, best_r, history


def sweep_evaluator(hpac, regions, x, ref, rate, schedule=(128, 8, 4), stream=None):
    """evaluate(configs) through one batched sweep launch: the saved share (approximated +
    skipped over invocations) and the normalised RMSE over every region."""
    import torch
    ref_rms = float(torch.sqrt(torch.mean(ref * ref)).item())
    calls = {"launches": 0, "configs": 0}

    def evaluate(configs):
        sw = hpac.Sweep(configs, regions, x, ref, rate, *schedule, stream=stream)
        sw.run()
        res = sw.results()
        sw.close()
        calls["launches"] += 1
        calls["configs"] += len(configs)
        inv = res["invocations"].sum(axis=1).astype(np.float64)
        saved = (res["approximated"].sum(axis=1) + res["skipped"].sum(axis=1)) / inv
        nrmse = np.sqrt(res["sum_sq"].sum(axis=1) / inv) / ref_rms
        return list(zip(saved.tolist(), nrmse.tolist()))

    evaluate.calls = calls
    return evaluate

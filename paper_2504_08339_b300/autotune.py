"""Autotuner for the launch shapes of a plan.

Times `neat_forward` on the caller's own population and inputs under a small
set of candidate tunings (the per-warp batch byte budget and CTA size of the
level-synchronous form, warps of a sample-parallel CTA, samples per lane, the
small-S switch point), applies the
fastest, and caches the choice per workload signature in a JSON file
(`$NEAT_TUNE_CACHE`, default `~/.cache/neat_b300/tune.json`).  Changing the
batch budget rebuilds the level batches, so the population is re-transformed.
"""
from __future__ import annotations

import json
import os

import torch

from .api import Plan


def _cache_path():
    return os.environ.get("NEAT_TUNE_CACHE",
                          os.path.join(os.path.expanduser("~"), ".cache", "neat_b300", "tune.json"))


def _signature(plan: Plan, S: int, n_edges: float, n_nodes: float) -> str:
    name = torch.cuda.get_device_name(plan.device)
    return (f"{name}|P={plan.P}|N={plan.N}|C={plan.C}|I={plan.I}|O={plan.O}|S={S}"
            f"|E~{int(round(n_edges, -1))}|V~{int(round(n_nodes, -1))}")


def candidates(plan: Plan, S: int):
    """Candidate tunings for S samples per genome."""
    out = []
    if S <= 8:
        out.append(dict())  # the default: batches cut to the resident warps
        for kb in (8, 10, 12, 16, 18, 24):
            out.append(dict(lvl_budget_kb=kb))
        out.append(dict(lvl_budget_kb=12, lvl_threads=64))
        out.append(dict(lvl_budget_kb=16, lvl_threads=128))
    for spl in (1, 2, 4):
        if spl > 1 and S < 32 * spl:
            continue
        for w in (4, 8, 16):
            out.append(dict(small_s_max=-1, warps_per_cta=w, samples_per_lane=spl))
    return out


def _time_forward(plan: Plan, inputs, out, reps: int, saved=None) -> float:
    for _ in range(3):
        plan.forward(inputs, out=out, saved=saved)
    torch.cuda.synchronize()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(reps):
        plan.forward(inputs, out=out, saved=saved)
    b.record()
    torch.cuda.synchronize()
    return a.elapsed_time(b) / reps


def autotune(plan: Plan, nodes, conns, inputs, reps: int = 20, use_cache: bool = True,
             verbose: bool = False, base: dict | None = None, saved: bool = False) -> dict:
    """Pick and apply the fastest tuning for this population and input shape.
    `base` holds knobs every candidate keeps (e.g. prune_dead=1); `saved`
    times the forward that also writes the aggregates a backward reads (the
    position walk) instead of the outputs-only forward (the compiled walk).
    Returns {"tuning": {...}, "ms": best forward time, "trials": [...]}."""
    base = dict(base or {})
    S = inputs.shape[1]
    en = (~torch.isnan(conns[..., 0])) & (conns[..., 3] != 0) & ~torch.isnan(conns[..., 3])
    n_edges = float(en.sum(dim=1).float().mean())
    n_nodes = float((~torch.isnan(nodes[..., 0])).sum(dim=1).float().mean())
    sig = (_signature(plan, S, n_edges, n_nodes) + "|" + json.dumps(base, sort_keys=True) +
           ("|saved" if saved else ""))
    path = _cache_path()
    cache = {}
    if use_cache and os.path.exists(path):
        try:
            with open(path) as f:
                cache = json.load(f)
        except (OSError, ValueError):
            cache = {}
    if use_cache and sig in cache:
        best = cache[sig]
        plan.set_tuning(**best["tuning"])
        plan.transform(nodes, conns)
        return best
    out = torch.empty((plan.P, S, plan.O), dtype=torch.float32, device=inputs.device)
    sv = (torch.empty((plan.P, plan.N, S), dtype=torch.float32, device=inputs.device)
          if saved else None)
    trials = []
    for cand in candidates(plan, S):
        cand = {**base, **cand}
        plan.set_tuning(**cand)
        plan.transform(nodes, conns)
        ms = _time_forward(plan, inputs, out, reps, sv)
        trials.append({"tuning": cand, "ms": ms})
        if verbose:
            print(f"autotune {cand} -> {ms * 1e3:.2f} us")
    best = min(trials, key=lambda t: t["ms"])
    plan.set_tuning(**best["tuning"])
    plan.transform(nodes, conns)
    result = {"tuning": best["tuning"], "ms": best["ms"], "trials": trials}
    if use_cache:
        cache[sig] = result
        try:
            os.makedirs(os.path.dirname(path), exist_ok=True)
            with open(path, "w") as f:
                json.dump(cache, f, indent=1)
        except OSError:
            pass
    return result

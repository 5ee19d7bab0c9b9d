#!/usr/bin/env python
"""Throughput of population-wide NEAT network evaluation on B300.

Metric: connection evaluations per second, conn-evals/s = pop x samples x
enabled connections / time (every enabled connection of every genome is
evaluated once per input vector).

Default workload (--config locomotion): 10,000 genomes with 27 inputs and
8 outputs (N=128, C=512), one rollout of 1,000 sequential steps with one
input vector per genome per step.  One benchmark step is the whole hot path
on one batch: the transformation stage (validate, sort, layers, pack, queue)
followed by the 1,000-step forward rollout, captured in one CUDA graph.  The
step inputs (1.08 GB) exceed the 126 MB L2, so no step starts warm except
for the population's programs, which a rollout re-reads by design.

Legs of the JSON line:
  value        device-resident throughput over K timed steps (CUDA events)
  e2e          same metric through the public Rollout API from pinned host
               buffers (H2D population + inputs, D2H outputs inside the timing,
               pipelined by chunks of steps so the copies overlap the kernels)
  roofline     forward kernel: algorithmic bytes / average launch duration
  plain        the padded one-launch-per-step form on the same workload
  cpu_baseline the FP64 oracle on the host cores, on a bounded sample

--impl reference times the FP64 oracle (the method's reference is the paper's
text, so the plain definition written out is the comparison arm) on the same
workload, one bounded sample per step.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "conn-evals/s (pop×samples×enabled conns), % roofline; batched/fwd+bwd vs plain"
UNIT = "conn-evals/s"
PEAKS_FALLBACK = {"hbm_gbs": 6400.0, "source": "fallback"}

# DRAM bytes (read + write) per launch of the timed kernel from one ncu
# capture (summaries under profiles/), keyed by workload and kernel: (bytes,
# population of the capture, hash prefixes of the sources it was taken on:
# the kernel's, and the library's where that picks the kernel's instantiation
# and launch shape).  A capture on a smaller population is scaled by
# population (the traffic grows with the genomes processed); the figure is
# reported only while those sources are unchanged.
_INTERNAL = ("paper_2504_08339_b300/csrc/neat_internal.cuh", "0d5d940c51250188")
TRAFFIC = {
    ("locomotion", "k_forward_lvl"): (32806656, 10000, dict([
        ("paper_2504_08339_b300/csrc/level.cu", "9c35aa382f0efee0"), _INTERNAL])),
    ("uneven", "k_forward_sp"): (106514944, 2048, dict([
        ("paper_2504_08339_b300/csrc/forward.cu", "5829aa1bc16b8561"),
        ("paper_2504_08339_b300/csrc/api.cu", "a5479abbfff12c07"), _INTERNAL])),
    ("differentiation", "k_backward"): (359663104, 512, dict([
        ("paper_2504_08339_b300/csrc/backward.cu", "ae1c59197d133899"), _INTERNAL])),
}


def measured_traffic(name, kernel, pop):
    import hashlib
    rec = TRAFFIC.get((name, kernel))
    if rec is None:
        return None
    nbytes, ref_pop, srcs = rec
    for path, prefix in srcs.items():
        with open(os.path.join(ROOT, path), "rb") as f:
            if hashlib.sha256(f.read()).hexdigest()[:16] != prefix:
                return None
    return int(round(nbytes * pop / ref_pop))


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        d["source"] = "measured"
        return d
    return dict(PEAKS_FALLBACK)


def roofline(hbm_bytes, chip_bytes, launch_us, peaks, dev):
    """Roofline of one launch: t_roof = max(HBM bytes / HBM peak, on-chip
    bytes / shared-memory peak); the larger term names the bound.  The HBM
    peak is the measured copy bandwidth, the shared-memory peak is measured
    here, now, by the library's probe kernel (same clocks as the run)."""
    from paper_2504_08339_b300.probe import smem_read_gbs
    sm = smem_read_gbs(dev.index)
    hbm_peak = float(peaks["hbm_gbs"])
    t = launch_us * 1e-6
    terms = {
        "hbm": {"bytes": int(hbm_bytes), "achieved": round(hbm_bytes / t / 1e9, 1),
                "peak": hbm_peak, "t_roof_us": round(hbm_bytes / hbm_peak / 1e3, 3),
                "peak_source": f"{peaks.get('source')} (MEASURED_PEAKS.json hbm_gbs, copy)"},
        "smem": {"bytes": int(chip_bytes), "achieved": round(chip_bytes / t / 1e9, 1),
                 "peak": round(sm["gbs"], 1), "t_roof_us": round(chip_bytes / sm["gbs"] / 1e3, 3),
                 "peak_source": f"measured now: shared-memory read probe, {sm['blocks']} CTAs"},
    }
    bound = max(terms, key=lambda k: terms[k]["t_roof_us"])
    b = terms[bound]
    return {"bound": bound, "achieved": b["achieved"], "peak": b["peak"], "unit": "GB/s",
            "frac": round(b["achieved"] / b["peak"], 4),
            "algorithmic_bytes_per_launch": b["bytes"], "terms": terms}


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=40)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--config", default="locomotion",
                    choices=["locomotion", "uneven", "differentiation", "hyperneat", "tiny",
                             "recurrent", "distance", "mutate", "substrate"])
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--tune", default="auto", choices=["auto", "default"],
                    help="auto: run the autotuner on the workload before timing "
                         "(the chosen tuning is recorded in config.tuning)")
    ap.add_argument("--tuning", default=None,
                    help="a given tuning, as JSON (e.g. '{\"samples_per_lane\": 2}'), "
                         "instead of the autotuner (profiling captures of a small case in the "
                         "full-size launch shape); recorded in config.tuning")
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--prune", action="store_true",
                    help="skip the nodes no output depends on (prune_dead = 1): the same "
                         "outputs; the value still counts every enabled connection")
    ap.add_argument("--recompute", action="store_true",
                    help="differentiation at S = 65,536 with the forward values recomputed in the "
                         "backward (no saved aggregates)")
    ap.add_argument("--pop", type=int, default=None,
                    help="population override (profiling captures and small cases; the line's "
                         "config then says so)")
    ap.add_argument("--horizon", type=int, default=None,
                    help="rollout steps override (profiling captures of the full population "
                         "with a short rollout; the line's config then says so)")
    return ap.parse_args()


# ---------------------------------------------------------------------------
# distributed plumbing (one process per GPU; no collective on the data path)
def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    pg = None
    if world > 1:
        import torch.distributed as dist
        backend = "nccl" if args.impl == "ours" else "gloo"
        dist.init_process_group(backend)
        pg = dist
    return rank, world, local, pg


def barrier(pg, device=None):
    if pg is not None:
        if device is not None:
            pg.barrier(device_ids=[device.index])
        else:
            pg.barrier()


def allreduce_max(pg, x, device):
    if pg is None:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    return float(t.item())


def allreduce_sum(pg, x, device):
    if pg is None:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    pg.all_reduce(t, op=pg.ReduceOp.SUM)
    return float(t.item())


# ---------------------------------------------------------------------------
class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during a region."""
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.proc = None
        try:
            import torch
            uuid = "GPU-" + str(torch.cuda.get_device_properties(device_index).uuid)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100", "-i", uuid], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL,
                text=True)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except Exception:
            self.proc.kill()
            out = ""
        sm, mx, power = [], [], []
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 8:
                continue
            try:
                sm.append(float(f[0]))
                mx.append(float(f[1]))
                power.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[4:8]):
                if v == "Active":
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "samples": len(sm),
                "power_w_max": max(power), "reasons": sorted(reasons)}


# ---------------------------------------------------------------------------
def enabled_counts(nodes, conns):
    """Enabled connections and valid nodes of every genome (host-side count of
    the workload's size; padding rows have a NaN key)."""
    valid_c = ~np.isnan(conns[..., 0]) & ~np.isnan(conns[..., 1])
    en = valid_c & ~np.isnan(conns[..., 3]) & (conns[..., 3] != 0)
    return en.sum(axis=1).astype(np.int64), (~np.isnan(nodes[..., 0])).sum(axis=1).astype(np.int64)


def live_counts(nodes, conns, I, O):
    """Per genome, the enabled connections into and the non-input nodes of the
    part of the network the outputs depend on: one breadth-first search over
    the reversed connections of the whole population from a root joined to
    every output row."""
    from scipy.sparse import csr_matrix
    from scipy.sparse.csgraph import breadth_first_order
    P, N = nodes.shape[:2]
    keys = nodes[..., 0]
    valid_n = ~np.isnan(keys)
    # row of each connection key: sort every genome's valid keys
    kk = np.where(valid_n, keys, 3.0e7)  # keys are below 2^24
    order = np.argsort(kk, axis=1, kind="stable")
    skeys = np.take_along_axis(kk, order, axis=1)
    c = conns
    en = ~np.isnan(c[..., 0]) & ~np.isnan(c[..., 1]) & ~np.isnan(c[..., 3]) & (c[..., 3] != 0)
    g, j = np.nonzero(en)
    a_key, b_key = c[g, j, 0], c[g, j, 1]

    ra, rb = _rows(skeys, order, g, a_key), _rows(skeys, order, g, b_key)
    ok = (ra >= 0) & (rb >= 0)
    g, ra, rb = g[ok], ra[ok], rb[ok]
    root = P * N
    src = np.concatenate([g * N + rb, np.full(P * O, root)])
    dst = np.concatenate([g * N + ra, (np.arange(P)[:, None] * N + np.arange(I, I + O)).ravel()])
    m = csr_matrix((np.ones(len(src), np.int8), (src, dst)), shape=(root + 1, root + 1))
    reach = breadth_first_order(m, root, directed=True, return_predecessors=False)
    live = np.zeros(root + 1, bool)
    live[reach] = True
    live = live[:root].reshape(P, N) & valid_n
    live[:, :I] = False
    V_live = live.sum(axis=1).astype(np.int64)
    E_live = np.bincount(g[live.ravel()[g * N + rb]], minlength=P).astype(np.int64)
    return E_live, V_live


def _rows(skeys, order, g, key):
    """Row of each (genome, key) pair, -1 where the genome has no such key."""
    P, N = skeys.shape
    flat = (skeys.astype(np.float64) + (np.arange(P)[:, None] * 4.0e7)).ravel()  # genomes disjoint
    q = key.astype(np.float64) + g * 4.0e7
    pos = np.searchsorted(flat, q)
    pos = np.minimum(pos, flat.size - 1)
    hit = (flat[pos] == q) & (key < 3.0e7)
    return np.where(hit, order.ravel()[pos] % N, -1)


def walked_counts(prune, nodes, conns, spec, E, Vn, extra):
    """Connections and non-input nodes an evaluation visits, per genome: all
    of them, or with pruning the part some output depends on (noted in the
    line's extra)."""
    if not prune:
        return E, Vn - spec.I
    E_live, V_live = live_counts(nodes, conns, spec.I, spec.O)
    extra["live_subgraph"] = live_note(E, E_live, V_live)
    return E_live, V_live


def live_note(E, E_live, V_live):
    return {"conns_per_genome_mean": round(float(E_live.mean()), 2),
            "conns_fraction_of_enabled": round(float(E_live.sum() / max(1, E.sum())), 4),
            "nodes_per_genome_mean": round(float(V_live.mean()), 2),
            "note": "--prune: nodes no output depends on are not evaluated (identical "
                    "outputs); value counts every enabled connection, the roofline only "
                    "the live part"}


def workload(name, seed, pop=None, horizon=None):
    from workloads import CONFIGS, make_population
    # the distance workload is the locomotion population, all pairs
    base = {"distance": "locomotion", "mutate": "locomotion", "substrate": "hyperneat"}
    cfg = dict(CONFIGS[base.get(name, name)])
    if pop is not None:
        cfg["P"] = pop
    if horizon is not None and "steps" in cfg:
        cfg["steps"] = horizon
    spec = cfg["spec"]
    nodes, conns = make_population(spec, cfg["P"], seed=seed)
    return cfg, spec, nodes, conns


def describe(name, cfg, spec):
    if name == "locomotion":
        return (f"locomotion rollout: pop={cfg['P']}, {spec.I} in / {spec.O} out, N={spec.N}, "
                f"C={spec.C}, {cfg['steps']} sequential steps x S=1, transform + rollout per step")
    if name == "uneven":
        return (f"uneven batching: pop={cfg['P']}, V~logU[23,1024], E~logU[8,4096], S={cfg['S']}, "
                f"{cfg['steps']} steps per rollout")
    if name == "differentiation":
        mode = "recompute" if cfg.get("recompute") else "saved aggregates"
        return (f"differentiation: pop={cfg['P']}, S={cfg['S']}, forward+backward (MSE), "
                f"{mode}")
    if name == "hyperneat":
        return f"HyperNEAT query: pop={cfg['P']} CPPNs, 32x32 substrate (2^20 queries each)"
    if name == "substrate":
        return (f"HyperNEAT query + two-sheet substrate: pop={cfg['P']} CPPNs, 32x32 grid "
                f"(2^20 weights each), S=64 input patterns per substrate, tanh")
    if name == "mutate":
        return (f"one generation's structural edits: pop={cfg['P']} locomotion genomes, "
                f"16 Sec. 3.2 operations each, then the transform (population restored "
                f"on the device before every step)")
    if name == "distance":
        return (f"compatibility distance of every pair: the locomotion population "
                f"(pop={cfg['P']}, N={spec.N}, C={spec.C}), {cfg['P']}^2 pairs per step")
    if name == "recurrent":
        return (f"recurrent networks: pop={cfg['P']}, {spec.I} in / {spec.O} out, N={spec.N}, "
                f"C={spec.C}, 15 % back edges / self-loops, S={cfg['S']}, T={cfg['T']} "
                f"synchronous iterations; conn-evals count every iteration")
    return f"tiny XOR: pop={cfg['P']}, S=4"


# ---------------------------------------------------------------------------
def accuracy(g, r, bound=None):
    """Error of the GPU results g against the FP64 oracle's r: max absolute
    error, max relative error (over |r| >= 1e-3), the elements beyond the
    stated tolerance (1e-5 relative + 1e-6 absolute) and, with the oracle's
    fp32 error bound, those beyond max(tolerance, 2 x bound) -- the parity
    tests' criterion (0 expected)."""
    g = np.asarray(g, np.float64)
    r = np.asarray(r, np.float64)
    fin = np.isfinite(r)
    same_nf = (np.isnan(g) & np.isnan(r)) | (g == r)
    with np.errstate(invalid="ignore"):  # inf - inf on the non-finite class
        err = np.abs(g - r)
    ar = np.abs(r)
    tol = 1e-6 + 1e-5 * ar
    big = fin & (ar >= 1e-3)
    res = {"n": int(fin.sum()),
           "max_abs_err": float(err[fin].max()) if fin.any() else 0.0,
           "max_rel_err": float((err[big] / ar[big]).max()) if big.any() else 0.0,
           "beyond_tolerance": int((fin & (err > tol)).sum()),
           "nonfinite_mismatch": int((~fin & ~same_nf).sum())}
    if bound is not None:
        lim = np.maximum(tol, 2.0 * np.asarray(bound, np.float64))
        res["beyond_bound"] = int((fin & (err > lim)).sum())
    return res


def grad_accuracy(g, r):
    """Gradients: max error relative to each genome's largest |gradient|."""
    g = np.asarray(g, np.float64).reshape(r.shape[0], -1)
    r = np.asarray(r, np.float64).reshape(r.shape[0], -1)
    scale = np.maximum(np.abs(r).max(axis=1, keepdims=True), 1e-30)
    rel = np.abs(g - r) / scale
    return {"n": int(r.size), "max_err_rel_to_genome_max": float(rel.max()),
            "beyond_1e-4": int((rel > 1e-4).sum())}


def cpu_model():
    """The host CPU's model name (from /proc/cpuinfo), or None."""
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.startswith("model name"):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return None


def cpu_baseline(name, cfg, spec, nodes, conns, seed, budget_steps=None, gpu=None, threads=None):
    """The FP64 oracle as it stands on a bounded sample, its genomes split
    over `threads` host threads (default: every core); with `gpu` (callables
    returning the GPU's results for the same sample) also the GPU's error
    against it, outside the timing."""
    import oracle
    from workloads import locomotion_inputs, regression_batch, uneven_inputs
    threads = int(threads or os.cpu_count() or 1)
    scale = max(1, threads // 2)  # sample sizes grow with the cores (10-30 s of work)
    E, _ = enabled_counts(nodes, conns)
    gpu = gpu or {}
    acc = None
    th = dict(threads=threads)
    t0 = time.perf_counter()
    if name == "locomotion":
        R = budget_steps or min(cfg["steps"], 200 * scale)
        x = np.concatenate([locomotion_inputs(seed, t, cfg["P"], spec.I) for t in range(R)], axis=1)
        t0 = time.perf_counter()
        oracle.forward(nodes, conns, x, spec.I, spec.O, **th)
        units = float(E.sum()) * R
        sample = f"all {cfg['P']} genomes x {R} of the {cfg['steps']} rollout steps"
        if "out" in gpu:
            dt = time.perf_counter() - t0
            ref, bnd = oracle.forward(nodes, conns, x, spec.I, spec.O, with_bound=True, **th)
            acc = {"outputs": accuracy(gpu["out"](R), ref, bnd)}
            if "plain" in gpu:
                acc["plain_outputs"] = accuracy(gpu["plain"](R), ref, bnd)
    elif name == "uneven":
        k = budget_steps or min(cfg["P"], 1500 * scale)
        sel = np.arange(k)
        x = uneven_inputs(seed, 0, cfg["P"])[sel]
        t0 = time.perf_counter()
        oracle.forward(nodes[sel], conns[sel], x, spec.I, spec.O, **th)
        units = float(E[sel].sum()) * cfg["S"]
        sample = f"{k} of {cfg['P']} genomes x 1 step (S={cfg['S']})"
        if "out" in gpu:
            dt = time.perf_counter() - t0
            ref, bnd = oracle.forward(nodes[sel], conns[sel], x, spec.I, spec.O, with_bound=True,
                                      **th)
            acc = {"outputs": accuracy(gpu["out"](k), ref, bnd)}
            if "plain" in gpu:
                acc["plain_outputs"] = accuracy(gpu["plain"](k), ref, bnd)
    elif name == "differentiation":
        k = budget_steps or min(cfg["P"], (64 if cfg["S"] <= 4096 else 4) * scale)
        x, y = regression_batch(seed, cfg["S"])
        t0 = time.perf_counter()
        out = oracle.forward(nodes[:k], conns[:k], x, spec.I, spec.O, **th)
        go = (2.0 / cfg["S"]) * (out[..., 0] - y[None].astype(np.float64))
        grads = oracle.backward(nodes[:k], conns[:k], x, spec.I, spec.O, go[..., None],
                                want_inputs=True, **th)
        units = float(E[:k].sum()) * cfg["S"]
        sample = f"{k} of {cfg['P']} genomes, forward + backward at S={cfg['S']}"
        if "out" in gpu:
            dt = time.perf_counter() - t0
            _, bnd = oracle.forward(nodes[:k], conns[:k], x, spec.I, spec.O, with_bound=True, **th)
            acc = {"outputs": accuracy(gpu["out"](k), out, bnd)}
            gg = gpu["grads"](k)
            for nm, a_, b_ in zip(("grad_weight", "grad_bias", "grad_response", "grad_inputs"),
                                  gg, grads):
                if a_ is not None and b_ is not None and np.size(a_) == np.size(b_):
                    acc[nm] = grad_accuracy(a_, b_)
    elif name == "substrate":
        k = budget_steps or min(cfg["P"], scale)
        G, S = 32, 64
        q = np.arange(G ** 4)
        t0 = time.perf_counter()
        w = oracle.hyperneat(nodes[:k], conns[:k], grid=G, qidx=q, **th).reshape(k, G * G, G * G)
        x = np.random.default_rng(seed).standard_normal((k, S, G * G)).astype(np.float32)
        oracle.substrate(w, x, 2)
        units = float(E[:k].sum()) * G ** 4 + float(k) * S * G ** 4
        sample = f"{k} of {cfg['P']} CPPNs: full query + substrate at S={S}"
    elif name == "mutate":
        from workloads import random_ops
        k = budget_steps or 2000
        ops = random_ops(seed, nodes[:k], conns[:k], spec.I, 16)
        t0 = time.perf_counter()
        n2, c2, _ = oracle.apply_ops(nodes[:k], conns[:k], ops)
        oracle.transform(n2, c2, spec.I, spec.O, **th)
        dt = time.perf_counter() - t0
        res = {"value": k / dt, "unit": "genomes/s", "cores": threads, "kind": "oracle",
               "cpu_model": cpu_model(),
               "note": "operations on one thread, the transform on every core",
               "sample": f"{k} of {cfg['P']} genomes: 16 operations + transform",
               "seconds": round(dt, 3)}
        if "pop" in gpu:
            gn, gc = gpu["pop"](k)
            same = lambda a, b: ((a == b) | (np.isnan(a) & np.isnan(b))).reshape(k, -1).all(1)  # noqa: E731
            res["gpu_vs_oracle"] = {"genomes": k, "nodes_bit_exact": int(same(gn, n2).sum()),
                                    "conns_bit_exact": int(same(gc, c2).sum())}
        return res
    elif name == "distance":
        k = budget_steps or 300
        t0 = time.perf_counter()
        ref = oracle.distance(nodes[:k], conns[:k], spec.I, spec.O)
        units = float(k) * k
        sample = f"all pairs of {k} of {cfg['P']} genomes"
        dt = time.perf_counter() - t0
        res = {"value": units / dt, "unit": "genome-pairs/s", "cores": 1, "kind": "oracle",
               "cpu_model": cpu_model(), "sample": sample, "seconds": round(dt, 3),
               "note": "one thread: the oracle computes the pair matrix in one call"}
        if "dist" in gpu:
            res["gpu_vs_oracle"] = {"distances": accuracy(gpu["dist"](k), ref)}
        return res
    elif name == "recurrent":
        k = budget_steps or min(cfg["P"], 300 * scale)
        x = np.random.default_rng(seed).standard_normal((k, cfg["S"], spec.I)).astype(np.float32)
        t0 = time.perf_counter()
        oracle.forward_recurrent(nodes[:k], conns[:k], x, spec.I, spec.O, cfg["T"], **th)
        units = float(E[:k].sum()) * cfg["S"] * cfg["T"]
        sample = f"{k} of {cfg['P']} genomes x S={cfg['S']} x T={cfg['T']}"
        if "out" in gpu:
            dt = time.perf_counter() - t0
            ref, bnd = oracle.forward_recurrent(nodes[:k], conns[:k], x, spec.I, spec.O,
                                                cfg["T"], with_bound=True, **th)
            acc = {"outputs": accuracy(gpu["out"](k), ref, bnd)}
    elif name == "hyperneat":
        k = budget_steps or min(cfg["P"], 2 * scale)
        q = np.arange(32 ** 4 // 4)
        t0 = time.perf_counter()
        oracle.hyperneat(nodes[:k], conns[:k], grid=32, qidx=q, **th)
        units = float(E[:k].sum()) * q.size
        sample = f"{k} of {cfg['P']} CPPNs x a quarter of the 2^20 queries"
        if "weights" in gpu:
            dt = time.perf_counter() - t0
            ref, raw, bnd = oracle.hyperneat(nodes[:k], conns[:k], grid=32,
                                             thresh=cfg["thresh"], qidx=q, with_raw=True,
                                             with_bound=True, **th)
            g = gpu["weights"](k, q)
            # queries whose raw value lies within the error band of the
            # threshold may be kept or zeroed either way: left out
            near = np.abs(np.abs(raw) - cfg["thresh"]) <= np.maximum(1e-6 + 1e-5 * np.abs(raw),
                                                                      2 * bnd)
            acc = {"weights": accuracy(np.where(near, 0.0, g), np.where(near, 0.0, ref),
                                       np.where(near, 0.0, bnd)),
                   "threshold_ties_left_out": int(near.sum())}
    else:
        from workloads import xor_inputs
        t0 = time.perf_counter()
        for _ in range(200):
            oracle.forward(nodes, conns, xor_inputs(), spec.I, spec.O, **th)
        units = float(E.sum()) * 4 * 200
        sample = "200 repetitions of the whole population"
        if "out" in gpu:
            dt = time.perf_counter() - t0
            ref, bnd = oracle.forward(nodes, conns, xor_inputs(), spec.I, spec.O, with_bound=True)
            acc = {"outputs": accuracy(gpu["out"](None), ref, bnd)}
            if "plain" in gpu:
                acc["plain_outputs"] = accuracy(gpu["plain"](None), ref, bnd)
    if acc is None:
        dt = time.perf_counter() - t0
    res = {"value": units / dt, "unit": UNIT, "cores": threads, "kind": "oracle",
           "cpu_model": cpu_model(), "sample": sample, "seconds": round(dt, 3)}
    if acc is not None:
        res["gpu_vs_oracle"] = acc
    return res


# ---------------------------------------------------------------------------
def bench_ours(args, rank, world, local, pg):
    import torch
    from paper_2504_08339_b300.api import Plan
    from paper_2504_08339_b300.rollout import Rollout
    from workloads import locomotion_inputs, regression_batch, uneven_inputs

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    peaks = load_peaks()
    name = args.config
    cfg, spec, nodes, conns = workload(name, args.seed + rank, args.pop, args.horizon)
    if name == "differentiation" and args.recompute:
        cfg["S"], cfg["recompute"] = cfg["S_recompute"], True
    P = cfg["P"]
    E, Vn = enabled_counts(nodes, conns)
    plan = Plan(P, spec.N, spec.C, spec.I, spec.O, device=dev)
    if args.prune:
        plan.set_tuning(prune_dead=1)
    launches_per_step = 4  # transform, rank, offsets, pack
    extra = {}
    tuning = {"mode": args.tune, "chosen": {}}
    if args.tuning is not None:
        given = json.loads(args.tuning)
        plan.set_tuning(**given, **({"prune_dead": 1} if args.prune else {}))
        tuning = {"mode": "given", "chosen": given}

    def autotune_on(x_dev, saved=False):
        """Run the autotuner on this population and one step's inputs (no
        cache: every run measures), keeping the prune setting; `saved`: on
        the forward that writes the aggregates (the one a training step runs)."""
        if args.tune != "auto" or args.tuning is not None:
            return
        from paper_2504_08339_b300.autotune import autotune
        d_n = torch.from_numpy(nodes).to(dev)
        d_c = torch.from_numpy(conns).to(dev)
        base = {"prune_dead": 1} if args.prune else {}
        r = autotune(plan, d_n, d_c, x_dev, use_cache=False, base=base, saved=saved)
        tuning["chosen"] = r["tuning"]
        tuning["trials_us"] = {json.dumps(t["tuning"], sort_keys=True): round(1e3 * t["ms"], 2)
                               for t in r["trials"]}

    if name in ("locomotion", "uneven", "tiny"):
        if name == "locomotion":
            T, S, ring = cfg["steps"], 1, cfg["steps"]
            host_in = np.stack([locomotion_inputs(args.seed + rank, t, P, spec.I) for t in range(T)])
        elif name == "uneven":
            T, S, ring = cfg["steps"], cfg["S"], 8
            host_in = np.stack([uneven_inputs(args.seed + rank, t, P) for t in range(ring)])
        else:
            from workloads import xor_inputs
            T, S, ring = 1, 4, 1
            host_in = np.repeat(xor_inputs(), P, 0)[None]
        autotune_on(torch.from_numpy(np.ascontiguousarray(host_in[0])).to(dev))
        ro = Rollout(plan, T, S=S, ring=ring)
        ro.load(torch.from_numpy(nodes), torch.from_numpy(conns), torch.from_numpy(host_in),
                non_blocking=False)
        ro.capture_split()
        units_per_step = float(E.sum()) * S * T
        launches_per_step += T
        # a step: the transform graph, then the graph of the T forward launches;
        # the events between them time the forward launches (no event node
        # among the kernels), in every timed step
        fwd_ev = []

        def run():
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            ro.run_split(a, b)
            fwd_ev.append((a, b))
            if len(fwd_ev) > 4 * max(1, args.steps):
                del fwd_ev[0]
        fwd_launches = T
        # an outputs-only forward evaluates only the nodes some output depends
        # on: its algorithmic traffic counts that part (program: 8 B per edge,
        # 12 B per node; inputs and outputs; on chip a value read per edge and
        # written per node, per sample)
        E_live, V_live = walked_counts(args.prune, nodes, conns, spec, E, Vn, extra)
        alg_bytes = float((8 * E_live + 12 * (V_live + spec.I)).sum() +
                          4 * S * (spec.I + spec.O) * P)
        chip_bytes = float(4 * S * (E_live + V_live).sum())
    elif name == "differentiation":
        S = cfg["S"]
        x, y = regression_batch(args.seed + rank, S)
        d_nodes = torch.from_numpy(nodes).to(dev)
        d_conns = torch.from_numpy(conns).to(dev)
        d_x = torch.from_numpy(x).to(dev)
        d_y = torch.from_numpy(y).to(dev)
        saved = None if cfg.get("recompute") else torch.empty((P, spec.N, S), device=dev)
        out = torch.empty((P, S, spec.O), device=dev)
        go = torch.empty((P, S, spec.O), device=dev)
        autotune_on(d_x, saved=saved is not None)
        tr = plan.transform(d_nodes, d_conns)
        # ev[0]: the backward (the dominant kernel, the roofline's); ev_f: the forward
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))]
        ev_f = (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))

        def run():
            plan.transform(d_nodes, d_conns, out=tr)
            ev_f[0].record()
            plan.forward(d_x, out=out, saved=saved)
            ev_f[1].record()
            torch.sub(out[..., 0], d_y, out=go[..., 0])
            go.mul_(2.0 / S)
            ev[0][0].record()
            g = plan.backward(d_x, go, saved=saved)
            ev[0][1].record()
            return g

        units_per_step = float(E.sum()) * S
        launches_per_step += 2
        fwd_launches = 1
        ro = None
        # backward: program again, grads out, saved aggregates in, dL/dO in,
        # dL/dx out, the shared inputs in; on chip 12 S E + 8 S V
        # (recompute: no saved aggregates; the forward's on-chip traffic again)
        # The backward visits only the nodes some output depends on (the others
        # have a zero adjoint): its program, saved-aggregate and on-chip terms
        # count that part; the gradients of every row are written.
        rec = saved is None
        E_live, V_live = walked_counts(args.prune, nodes, conns, spec, E, Vn, extra)
        Vl = V_live + spec.I
        alg_bytes = float((8 * E_live + 12 * Vl).sum() + (4 * E + 8 * Vn).sum() +
                          (0 if rec else 4 * S * V_live.sum()) +
                          4 * S * spec.O * P + 4 * S * spec.I * P + 4 * S * spec.I)
        chip_bytes = float((12 * S * E_live + 8 * S * Vl).sum() +
                           (4 * S * (E_live + V_live).sum() if rec else 0))
        fwd_hbm = float((8 * E + 12 * Vn).sum() + 4 * S * spec.I + 4 * S * spec.O * P +
                        (0 if rec else 4 * S * Vn.sum()))
        fwd_chip = float(4 * S * (E + Vn).sum())
    elif name == "substrate":
        G, S = 32, 64
        K = G * G
        d_nodes = torch.from_numpy(nodes).to(dev)
        d_conns = torch.from_numpy(conns).to(dev)
        tr = plan.transform(d_nodes, d_conns)
        x = np.random.default_rng(args.seed + rank).standard_normal((P, S, K)).astype(np.float32)
        d_x = torch.from_numpy(x).to(dev)
        wts = torch.empty((P, K, K), device=dev)
        sub_out = torch.empty((P, S, K), device=dev)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))]
        ev_s = (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
        from paper_2504_08339_b300.api import substrate_forward

        def run():
            plan.transform(d_nodes, d_conns, out=tr)
            ev[0][0].record()
            plan.hyperneat(G, cfg["thresh"], out=wts)
            ev[0][1].record()
            ev_s[0].record()
            substrate_forward(wts, d_x, act=2, out=sub_out)
            ev_s[1].record()

        units_per_step = float(E.sum()) * 2 ** 20 + float(P) * S * K * K
        launches_per_step += 2
        fwd_launches = 1
        ro = None
        E_live, V_live = walked_counts(args.prune, nodes, conns, spec, E, Vn, extra)
        alg_bytes = float((8 * E + 12 * Vn).sum() + 4.0 * 2 ** 20 * P)
        chip_bytes = float(4.0 * 2 ** 20 * (E_live + V_live).sum())
    elif name == "mutate":
        from workloads import random_ops
        K = 16
        ops = random_ops(args.seed + rank, nodes, conns, spec.I, K)
        d_nodes0 = torch.from_numpy(nodes).to(dev)
        d_conns0 = torch.from_numpy(conns).to(dev)
        d_nodes = d_nodes0.clone()
        d_conns = d_conns0.clone()
        d_ops = torch.from_numpy(ops).to(dev)
        tr, op_st = plan.mutate_transform(d_nodes, d_conns, d_ops)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))]

        def run():
            d_nodes.copy_(d_nodes0)
            d_conns.copy_(d_conns0)
            ev[0][0].record()
            plan.mutate_transform(d_nodes, d_conns, d_ops, op_status=op_st, out=tr)
            ev[0][1].record()

        units_per_step = float(P)
        launches_per_step = 1 + 4 + 3  # operations, transform pipeline, level batches
        fwd_launches = 1
        ro = None
        # the operations list in; the population read by the operations and by
        # the transform; order / layer and the packed programs written
        pop_bytes = P * (spec.N * 5 + spec.C * 4) * 4
        alg_bytes = float(P * K * 32 + 2 * pop_bytes + P * spec.N * 8 +
                          (16 * Vn + 8 * E).sum())
        chip_bytes = 0.0
    elif name == "distance":
        from paper_2504_08339_b300.api import distance
        d_nodes = torch.from_numpy(nodes).to(dev)
        d_conns = torch.from_numpy(conns).to(dev)
        tr = plan.transform(d_nodes, d_conns)
        dist = torch.empty((P, P), device=dev)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))]

        def run():
            ev[0][0].record()
            distance(d_nodes, d_conns, spec.I, spec.O, status=tr.status, out=dist)
            ev[0][1].record()

        units_per_step = float(P) * P
        launches_per_step = 2
        fwd_launches = 1
        ro = None
        # HBM: the padded genomes in, the distance matrix out; on chip: both
        # genomes' sorted keys streamed through once per unordered pair (the
        # distance is symmetric: P (P + 1) / 2 merges for the P^2 entries; 4 B
        # a node key, 8 B a connection key; the attributes of shared keys on
        # top)
        alg_bytes = float(P * (spec.N * 5 + spec.C * 4) * 4 + 4.0 * P * P)
        M = (~np.isnan(conns[:, :, 0]) & ~np.isnan(conns[:, :, 1])).sum(1)  # connection genes
        chip_bytes = (float(P) * (P + 1) / 2) * 2 * (4.0 * float(Vn.mean()) + 8.0 * float(M.mean()))
    elif name == "recurrent":
        S, T = cfg["S"], cfg["T"]
        x = np.random.default_rng(args.seed + rank).standard_normal((P, S, spec.I)).astype(
            np.float32)
        d_nodes = torch.from_numpy(nodes).to(dev)
        d_conns = torch.from_numpy(conns).to(dev)
        d_x = torch.from_numpy(x).to(dev)
        out = torch.empty((P, S, spec.O), device=dev)
        status = plan.transform_recurrent(d_nodes, d_conns)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))]

        def run():
            plan.transform_recurrent(d_nodes, d_conns, status=status)
            ev[0][0].record()
            plan.forward_recurrent(d_x, T, out=out)
            ev[0][1].record()

        units_per_step = float(E.sum()) * S * T
        launches_per_step += 1
        fwd_launches = 1
        ro = None
        # HBM: program once, inputs, outputs; on chip: every iteration reads a
        # value per enabled connection and writes one per node
        alg_bytes = float((8 * E + 12 * Vn).sum() + 4 * S * (spec.I + spec.O) * P)
        chip_bytes = float(4 * S * T * (E + Vn).sum())
    else:  # hyperneat
        d_nodes = torch.from_numpy(nodes).to(dev)
        d_conns = torch.from_numpy(conns).to(dev)
        tr = plan.transform(d_nodes, d_conns)
        w = torch.empty((P, 1024, 1024), device=dev)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))]

        def run():
            plan.transform(d_nodes, d_conns, out=tr)
            ev[0][0].record()
            plan.hyperneat(32, cfg["thresh"], out=w)
            ev[0][1].record()

        units_per_step = float(E.sum()) * 2 ** 20
        launches_per_step += 1
        fwd_launches = 1
        ro = None
        # the query evaluates only the nodes the output depends on: program
        # bytes once, a weight written per query; on chip a value read per
        # live connection and written per live node, per query
        E_live, V_live = walked_counts(args.prune, nodes, conns, spec, E, Vn, extra)
        alg_bytes = float((8 * E + 12 * Vn).sum() + 4.0 * 2 ** 20 * P)
        chip_bytes = float(4.0 * 2 ** 20 * (E_live + V_live).sum())

    # ---- timed region (device-resident inputs)
    for _ in range(max(3, args.warmup)):
        run()
    torch.cuda.synchronize()
    barrier(pg, dev)
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record()
    launch_ms = []
    if ro is not None:
        fwd_ev.clear()
    for _ in range(args.steps):
        run()
    t1.record()
    torch.cuda.synchronize()
    ms = t0.elapsed_time(t1)
    clk = clocks.stop()
    barrier(pg, dev)
    # per-launch duration of the forward kernel: the T forward launches of
    # every timed step (one graph, no event among them) divided by T
    if ro is not None:
        launch_ms = [a.elapsed_time(b) / fwd_launches for a, b in fwd_ev]
    else:
        launch_ms = [ev[0][0].elapsed_time(ev[0][1])]
    ms_max = allreduce_max(pg, ms, dev)
    units_total = allreduce_sum(pg, units_per_step * args.steps, dev)
    value = units_total / (ms_max / 1e3)

    avg_launch_us = 1e3 * float(np.mean(launch_ms)) if launch_ms else None
    roof = None
    if avg_launch_us:
        if name == "hyperneat":
            kernel = "k_hyperneat"
        elif name == "recurrent":
            kernel = "k_forward_rec"
        elif name == "distance":
            kernel = "k_distance"
        elif name == "mutate":
            kernel = "k_apply_ops + transform pipeline"
        elif name == "substrate":
            kernel = "k_hyperneat"
            sub_us = 1e3 * ev_s[0].elapsed_time(ev_s[1])
            flops = 2.0 * P * 64 * 1024 * 1024
            sm_mhz = float((clk or {}).get("sm_mhz") or 2032.0)
            sms = torch.cuda.get_device_properties(dev).multi_processor_count
            peak = sms * 128 * 2 * sm_mhz * 1e6 / 1e12
            ach = flops / (sub_us * 1e-6) / 1e12
            extra["substrate"] = {
                "kernel": "k_substrate (fp32 SIMT, tanh fused)", "launch_us": round(sub_us, 3),
                "bound": "alu", "achieved": round(ach, 2), "unit": "TFLOP/s",
                "peak": round(peak, 2), "frac": round(ach / peak, 4),
                "peak_source": f"derived: {sms} SMs x 128 fp32 lanes x 2 flop x {sm_mhz:.0f} MHz"}
        elif name == "differentiation":
            kernel = "k_backward<recompute>" if cfg.get("recompute") else "k_backward"
            fwd_us = 1e3 * ev_f[0].elapsed_time(ev_f[1])
            extra["forward"] = roofline(fwd_hbm, fwd_chip, fwd_us, peaks, dev)
            extra["forward"].update({"kernel": "k_forward_sp (with the saved aggregates)",
                                     "launch_us": round(fwd_us, 3)})
        else:
            tune = plan.get_tuning()
            kernel = "k_forward_lvl" if S <= tune["small_s_max"] else "k_forward_sp"
        roof = roofline(alg_bytes, chip_bytes, avg_launch_us, peaks, dev)
        roof.update({"traffic": None if args.prune else measured_traffic(name, kernel, P),
                     "kernel": kernel,
                     "avg_launch_us": round(avg_launch_us, 3), "launches_timed":
                         len(launch_ms) * (fwd_launches if ro is not None else 1),
                     "launch_time": "CUDA events around the graph of the step's forward "
                                    "launches (no event among them), per launch"
                                    if ro is not None else "CUDA events around the launch"})
        extra["launch_us_min"] = round(1e3 * min(launch_ms), 3)
        extra["launch_us_max"] = round(1e3 * max(launch_ms), 3)

    # ---- plain padded one-launch-per-step form (eager launches, no graph)
    plain = None
    if not args.no_plain and name in ("locomotion", "uneven", "tiny"):
        K = max(1, min(3, args.steps))
        d_in = ro.inputs
        out_p = torch.empty_like(ro.outputs[0])

        def run_plain():
            plan.transform(ro.nodes, ro.conns, out=ro.tr)
            for t in range(ro.T):
                plan.forward(d_in[t % ro.ring], out=out_p, plain=True)

        run_plain()
        torch.cuda.synchronize()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(K):
            run_plain()
        b.record()
        torch.cuda.synchronize()
        pms = a.elapsed_time(b) / K
        plain = {"value": units_per_step / (pms / 1e3), "ms_per_step": round(pms, 3),
                 "form": ("padded programs, all N positions, one warp per (genome, sample) "
                          "with lanes over a node's incoming edges"
                          if S <= 8 else
                          "padded programs, all N positions, one warp per (genome, 32 samples)")
                 + ", one launch per rollout step, eager (no graph)", "steps": K}

    # ---- end to end through the public API from pinned host buffers
    e2e = None
    if not args.no_e2e and ro is not None:
        h_nodes = torch.from_numpy(nodes).pin_memory()
        h_conns = torch.from_numpy(conns).pin_memory()
        h_in = torch.from_numpy(host_in).pin_memory()
        h_out = torch.empty(ro.outputs.shape, dtype=torch.float32).pin_memory()
        K = max(1, min(10, args.steps))
        ro.run_host(h_nodes, h_conns, h_in, h_out)
        torch.cuda.synchronize()
        w0 = time.perf_counter()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(K):
            ro.run_host(h_nodes, h_conns, h_in, h_out)
        b.record()
        torch.cuda.synchronize()
        wall = (time.perf_counter() - w0) / K
        ems = max(a.elapsed_time(b) / K, wall * 1e3)
        h2d = h_nodes.numel() * 4 + h_conns.numel() * 4 + h_in.numel() * 4
        d2h = h_out.numel() * 4
        e2e = {"value": allreduce_sum(pg, units_per_step, dev) / (allreduce_max(pg, ems, dev) / 1e3),
               "unit": UNIT, "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
               "ms_per_step": round(ems, 3), "steps": K,
               "form": f"Rollout.run_host: chunks of {ro.chunk} steps, each a graph; input "
                       "and output copies on two streams overlap the kernels (open loop: "
                       "every step's inputs are given)"}

    if not args.no_e2e and name == "differentiation":
        # through the public differentiable API (torch.autograd.Function):
        # population and batch H2D, transform + forward + MSE + backward,
        # gradients of nodes, conns and inputs and the loss D2H
        from paper_2504_08339_b300.api import evaluate
        h_nodes = torch.from_numpy(nodes).pin_memory()
        h_conns = torch.from_numpy(conns).pin_memory()
        h_x = torch.from_numpy(x).pin_memory()
        h_y = torch.from_numpy(y).pin_memory()
        g_nodes = torch.empty(h_nodes.shape, dtype=torch.float32).pin_memory()
        g_conns = torch.empty(h_conns.shape, dtype=torch.float32).pin_memory()
        g_x = torch.empty(h_x.shape, dtype=torch.float32).pin_memory()
        h_loss = torch.empty((1,), dtype=torch.float32).pin_memory()
        store = not cfg.get("recompute")

        def step_e2e():
            n_ = h_nodes.to(dev, non_blocking=True).requires_grad_()
            c_ = h_conns.to(dev, non_blocking=True).requires_grad_()
            x_ = h_x.to(dev, non_blocking=True).requires_grad_()
            y_ = h_y.to(dev, non_blocking=True)
            o_ = evaluate(plan, n_, c_, x_, store=store)
            loss = ((o_[..., 0] - y_) ** 2).mean(dim=1).sum()
            loss.backward()
            g_nodes.copy_(n_.grad, non_blocking=True)
            g_conns.copy_(c_.grad, non_blocking=True)
            g_x.copy_(x_.grad, non_blocking=True)
            h_loss.copy_(loss.detach().reshape(1), non_blocking=True)

        step_e2e()
        torch.cuda.synchronize()
        K = max(1, min(5, args.steps))
        w0 = time.perf_counter()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(K):
            step_e2e()
        b.record()
        torch.cuda.synchronize()
        wall = (time.perf_counter() - w0) / K
        ems = max(a.elapsed_time(b) / K, wall * 1e3)
        h2d = (h_nodes.numel() + h_conns.numel() + h_x.numel() + h_y.numel()) * 4
        d2h = (g_nodes.numel() + g_conns.numel() + g_x.numel() + 1) * 4
        e2e = {"value": allreduce_sum(pg, units_per_step, dev) / (allreduce_max(pg, ems, dev) / 1e3),
               "unit": UNIT, "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
               "ms_per_step": round(ems, 3), "steps": K,
               "path": "paper_2504_08339_b300.api.evaluate (torch.autograd.Function), MSE loss"}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        # the GPU's results for the oracle's sample, read after the timing
        gpu = {}
        np_ = lambda t: t.float().cpu().numpy()  # noqa: E731
        if name == "locomotion":
            gpu["out"] = lambda R: np_(ro.outputs[:R, :, 0, :].permute(1, 0, 2))
        elif name == "uneven":
            gpu["out"] = lambda k: np_(ro.outputs[0][:k])
        elif name == "tiny":
            gpu["out"] = lambda _: np_(ro.outputs[0])
        elif name == "differentiation":
            gpu["out"] = lambda k: np_(out[:k])
            gpu["grads"] = lambda k: [None if t is None else np_(t[:k]) for t in run()]
        elif name == "recurrent":
            gpu["out"] = lambda k: np_(out[:k])
        elif name == "hyperneat":
            gpu["weights"] = lambda k, q: np_(w[:k].reshape(k, -1)[:, torch.from_numpy(q).to(dev)])
        elif name == "distance":
            gpu["dist"] = lambda k: np_(dist[:k, :k])
        elif name == "mutate":
            gpu["pop"] = lambda k: (np_(d_nodes[:k]), np_(d_conns[:k]))
        if plain is not None:
            # the plain form's outputs for the same sample (the plan holds the
            # population's programs after the rollout)
            def plain_out(k):
                if name == "locomotion":
                    o = torch.stack([plan.forward(ro.inputs[t], plain=True) for t in range(k)])
                    return np_(o[:, :, 0, :].permute(1, 0, 2))
                o = plan.forward(ro.inputs[0], plain=True)
                return np_(o if name == "tiny" else o[:k])
            gpu["plain"] = plain_out
        cpu = cpu_baseline(name, cfg, spec, nodes, conns, args.seed, gpu=gpu)

    gpu_launches = launches_per_step * args.steps
    line = {
        "metric": {"distance": "genome-pairs/s (compatibility distance)",
                   "mutate": "genomes/s (operations + transform)"}.get(name, METRIC),
        "value": value, "unit": {"distance": "genome-pairs/s", "mutate": "genomes/s"}.get(name, UNIT),
        "n_gpus": world, "steps": args.steps,
        "warmup": max(3, args.warmup), "ms_per_step": round(ms_max / args.steps, 4),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic (seeded generators; random genomes shaped like the workload)",
        "config": {"workload": describe(name, cfg, spec), "name": name, "pop": P,
                   "pop_override": args.pop is not None,
                   "horizon_override": args.horizon is not None,
                   "prune_dead": bool(args.prune), "tuning": tuning,
                   "enabled_conns_per_genome_mean": round(float(E.mean()), 2),
                   "valid_nodes_per_genome_mean": round(float(Vn.mean()), 2),
                   "form": "batched: persistent size-sorted queue over ragged-packed programs, "
                           "CUDA graph", "parallelism": f"dp{world} (independent populations)",
                   "l2": "step inputs exceed L2 (126 MB); programs L2-resident within a rollout"},
        "clocks": clk, "gpu_launches": gpu_launches, "roofline": roof,
        "cpu_baseline": cpu, "e2e": e2e, "plain": plain, "extra": extra,
        "fwd_launches_per_step": fwd_launches,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)


def bench_reference(args, rank, world):
    """The FP64 oracle, as it stands, on the host cores: every step is a
    bounded sample of the same workload."""
    if rank != 0:
        return
    name = args.config
    cfg, spec, nodes, conns = workload(name, args.seed, args.pop, args.horizon)
    # per-step samples of about a second of single-core work, grown with the
    # cores the oracle's genome split uses
    scale = max(1, (os.cpu_count() or 1) // 2)
    budget = {"locomotion": 8, "uneven": 150, "differentiation": 4, "hyperneat": 1, "tiny": None,
              "recurrent": 40, "distance": 200, "mutate": 2000, "substrate": 1}[name]
    if budget is not None and name not in ("distance", "mutate"):
        budget *= scale
    for _ in range(max(3, args.warmup)):
        cpu_baseline(name, cfg, spec, nodes, conns, args.seed, budget)
    vals, secs = [], 0.0
    rec = None
    for _ in range(args.steps):
        rec = cpu_baseline(name, cfg, spec, nodes, conns, args.seed, budget)
        vals.append(rec["value"])
        secs += rec["seconds"]
    value = float(np.mean(vals))
    line = {
        "impl": "reference",
        "metric": {"distance": "genome-pairs/s (compatibility distance)",
                   "mutate": "genomes/s (operations + transform)"}.get(name, METRIC),
        "value": value, "unit": rec["unit"], "n_gpus": world,
        "steps": args.steps, "warmup": max(3, args.warmup),
        "ms_per_step": round(1e3 * secs / args.steps, 3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": describe(name, cfg, spec), "name": name, "pop": cfg["P"],
                   "pop_override": args.pop is not None},
        "cpu_baseline": {"kind": "oracle", "cores": rec["cores"], "cpu_model": rec.get("cpu_model"),
                         "sample": rec["sample"], "value": value, "unit": rec["unit"]},
        "e2e": {"value": value, "unit": rec["unit"], "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def main():
    args = parse_args()
    rank, world, local, pg = dist_setup(args)
    try:
        if args.impl == "reference":
            bench_reference(args, rank, world)
        else:
            bench_ours(args, rank, world, local, pg)
    finally:
        if pg is not None:
            pg.destroy_process_group()


if __name__ == "__main__":
    main()

"""Seeded generators for padded NEAT populations (Sec. 3.1 encoding).

Layout written here (float32, row-major):
  nodes[P, N, 5]  = (key, bias, response, activation id, aggregation id)
  conns[P, C, 4]  = (in key, out key, weight, enabled)
An invalid (padding) row has NaN in every column.  Rows 0..I-1 are the input
nodes and rows I..I+O-1 the output nodes (the genome interface of App. B fixes
input_idx = arange(I), output_idx = arange(I, I+O)); their keys equal their row.
Hidden nodes get distinct random keys in [I+O, 8N), so keys and rows differ and
a key->row lookup is exercised.  Holes (NaN rows) are left between valid rows,
as node/connection removal in Sec. 3.2 leaves them.

The DAG recipe: a position order [inputs, shuffled hidden, outputs]; an edge
(a -> b) is a candidate iff pos(a) < pos(b) and b is not an input.  Enabled
edges are distinct candidates; about one disabled row per nine enabled ones is
added (p_enabled ~ 0.9).  Nothing here evaluates a network.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

# Column ids of the activation / aggregation options (the interface ids that
# the node rows carry; each consumer defines its own functions for them).
ACT = dict(identity=0, sigmoid=1, tanh=2, relu=3, sin=4, gaussian=5, abs=6)
AGG = dict(sum=0, product=1, max=2, mean=3)


@dataclass
class GenomeSpec:
    I: int
    O: int
    N: int
    C: int
    hidden: tuple | None = None          # hidden count ~ U{lo..hi}
    V_loguniform: tuple | None = None    # valid node count ~ logU[lo, hi]
    E_uniform: tuple | None = None       # enabled conns ~ U{lo..hi}
    E_loguniform: tuple | None = None    # enabled conns ~ logU[lo, hi]
    edge_p: float | None = None          # keep each candidate with prob p
    p_enabled: float = 0.9
    acts: tuple = ("sigmoid",)
    out_acts: tuple | None = None
    aggs: tuple = ("sum",)
    w_std: float = 1.0
    b_std: float = 1.0
    r_mean: float = 1.0
    r_std: float = 0.0
    hole_frac: float = 0.05
    back_frac: float = 0.0               # extra enabled back-edges / self-loops (recurrent)


def _distinct_ints(rng, n: int, k: int) -> np.ndarray:
    """k distinct integers from [0, n) in random order."""
    if k <= 0:
        return np.zeros(0, dtype=np.int64)
    if n <= 65536 or 4 * k > n:
        return rng.permutation(n)[:k].astype(np.int64)
    out = np.zeros(0, dtype=np.int64)
    while out.size < k:
        draw = rng.integers(0, n, size=int(1.3 * (k - out.size)) + 16)
        allv = np.concatenate([out, draw])
        _, first = np.unique(allv, return_index=True)
        out = allv[np.sort(first)]
    return out[:k]


def _scatter_rows(rng, n_items: int, lo: int, hi: int, hole_frac: float) -> np.ndarray:
    """Distinct rows in [lo, hi) for n_items items, spread over a span with
    about hole_frac holes; the remaining rows stay padding."""
    avail = hi - lo
    if n_items == 0:
        return np.zeros(0, dtype=np.int64)
    span = min(avail, int(math.ceil(n_items * (1.0 + hole_frac))) + 1)
    return lo + _distinct_ints(rng, span, n_items)


def random_genome(rng, spec: GenomeSpec):
    """One padded genome: (nodes [N,5] f32, conns [C,4] f32)."""
    I, O, N, C = spec.I, spec.O, spec.N, spec.C
    max_h = N - I - O
    if spec.V_loguniform is not None:
        lo, hi = spec.V_loguniform
        V = int(round(math.exp(rng.uniform(math.log(lo), math.log(hi)))))
        h = V - I - O
    else:
        h = int(rng.integers(spec.hidden[0], spec.hidden[1] + 1))
    h = max(0, min(h, max_h))
    M = I + h + O

    # node ids: 0..I-1 inputs, I..I+O-1 outputs, I+O.. hidden
    hid_keys = I + O + _distinct_ints(rng, 8 * N - I - O, h)
    keys = np.concatenate([np.arange(I + O), hid_keys]).astype(np.int64)
    hid_rows = _scatter_rows(rng, h, I + O, N, spec.hole_frac)
    rows = np.concatenate([np.arange(I + O), hid_rows]).astype(np.int64)
    # position order [inputs, shuffled hidden, outputs] -> node id
    pos_node = np.concatenate([np.arange(I), I + O + rng.permutation(h),
                               I + np.arange(O)]).astype(np.int64)

    # candidate pairs (a < b in position, b >= I): index x -> (a, b)
    dst_pos = np.arange(I, M, dtype=np.int64)
    cum = np.concatenate([[0], np.cumsum(dst_pos)])  # start index per dst
    n_cand = int(cum[-1])
    if spec.edge_p is not None:
        b_all = np.repeat(dst_pos, dst_pos)
        a_all = np.arange(n_cand, dtype=np.int64) - np.repeat(cum[:-1], dst_pos)
        keep = rng.random(n_cand) < spec.edge_p
        sel = np.flatnonzero(keep)
        sel = sel[rng.permutation(sel.size)]
        if sel.size > C:
            sel = sel[:C]
        en = rng.random(sel.size) < spec.p_enabled
        a_pos, b_pos = a_all[sel], b_all[sel]
    else:
        if spec.E_loguniform is not None:
            lo, hi = spec.E_loguniform
            E = int(round(math.exp(rng.uniform(math.log(lo), math.log(hi)))))
        else:
            E = int(rng.integers(spec.E_uniform[0], spec.E_uniform[1] + 1))
        E = max(0, min(E, n_cand, C))
        n_dis = int(round(E * (1.0 - spec.p_enabled) / spec.p_enabled))
        n_dis = max(0, min(n_dis, n_cand - E, C - E))
        x = _distinct_ints(rng, n_cand, E + n_dis)
        bi = np.searchsorted(cum, x, side="right") - 1
        b_pos = I + bi
        a_pos = x - cum[bi]
        en = np.zeros(x.size, dtype=bool)
        en[:E] = True

    if spec.back_frac > 0.0:
        # recurrent genomes: extra enabled pairs with pos(a) >= pos(b) (back
        # edges and self-loops), b not an input; index x -> (a, b)
        nb = (M - dst_pos).astype(np.int64)
        cumb = np.concatenate([[0], np.cumsum(nb)])
        n_back = int(round(int(en.sum()) * spec.back_frac))
        n_back = max(0, min(n_back, int(cumb[-1]), C - a_pos.size))
        xb = _distinct_ints(rng, int(cumb[-1]), n_back)
        bi = np.searchsorted(cumb, xb, side="right") - 1
        b_b = I + bi
        a_b = b_b + (xb - cumb[bi])
        a_pos = np.concatenate([a_pos, a_b])
        b_pos = np.concatenate([b_pos, b_b])
        en = np.concatenate([en, np.ones(n_back, dtype=bool)])

    nodes = np.full((N, 5), np.nan, dtype=np.float32)
    conns = np.full((C, 4), np.nan, dtype=np.float32)

    nv = I + O + h
    bias = rng.normal(0.0, spec.b_std, size=nv)
    resp = spec.r_mean + spec.r_std * rng.normal(size=nv) if spec.r_std > 0 \
        else np.full(nv, spec.r_mean)
    act_ids = np.array([ACT[a] for a in spec.acts])
    agg_ids = np.array([AGG[a] for a in spec.aggs])
    act = act_ids[rng.integers(0, act_ids.size, size=nv)]
    agg = agg_ids[rng.integers(0, agg_ids.size, size=nv)]
    if spec.out_acts is not None:
        oa = np.array([ACT[a] for a in spec.out_acts])
        act[I:I + O] = oa[rng.integers(0, oa.size, size=O)]
    bias[:I] = 0.0
    resp[:I] = 1.0
    act[:I] = 0
    agg[:I] = 0
    nodes[rows, 0] = keys
    nodes[rows, 1] = bias
    nodes[rows, 2] = resp
    nodes[rows, 3] = act
    nodes[rows, 4] = agg

    k = a_pos.size
    crow = _scatter_rows(rng, k, 0, C, spec.hole_frac)
    src_node = pos_node[a_pos]
    dst_node = pos_node[b_pos]
    conns[crow, 0] = keys[src_node]
    conns[crow, 1] = keys[dst_node]
    conns[crow, 2] = rng.normal(0.0, spec.w_std, size=k)
    conns[crow, 3] = en.astype(np.float32)
    return nodes, conns


def make_population(spec: GenomeSpec, P: int, seed: int = 0):
    """P independent genomes from one seeded stream: (nodes [P,N,5], conns [P,C,4])."""
    rng = np.random.default_rng(seed)
    nodes = np.empty((P, spec.N, 5), dtype=np.float32)
    conns = np.empty((P, spec.C, 4), dtype=np.float32)
    for g in range(P):
        nodes[g], conns[g] = random_genome(rng, spec)
    return nodes, conns


# ---------------------------------------------------------------------------
# The workloads.  Sizes follow the benchmark definitions; where a workload
# leaves a choice open (activation/aggregation sets of the uneven and HyperNEAT
# populations, edge-count ranges) the choice is written here.
CONFIGS = {
    # XOR-sized: 3 inputs (x1, x2, bias), 1 output, hidden U{0..8}, each
    # forward pair kept with p=0.3 and enabled with p=0.9, sigmoid/sum.
    "tiny": dict(P=100, S=4, spec=GenomeSpec(
        I=3, O=1, N=16, C=32, hidden=(0, 8), edge_p=0.3, p_enabled=0.9,
        acts=("sigmoid",), aggs=("sum",), w_std=1.0, b_std=1.0)),
    # Locomotion-control-sized (Ant-shaped 27 obs / 8 actions), one input
    # vector per genome per step, 1000 sequential steps.
    "locomotion": dict(P=10000, S=1, steps=1000, spec=GenomeSpec(
        I=27, O=8, N=128, C=512, hidden=(0, 90), E_uniform=(50, 500),
        acts=("sigmoid", "tanh", "relu", "identity", "sin"),
        aggs=("sum", "product", "max", "mean"), w_std=1.0, b_std=0.5)),
    # Uneven sizes: valid nodes logU[I+O, 1024], enabled conns logU[8, 4096].
    # Bounded activations and no product aggregation keep fp32 finite on
    # genomes with thousands of edges and hundreds of layers.
    "uneven": dict(P=16384, S=64, steps=200, spec=GenomeSpec(
        I=17, O=6, N=1024, C=4096, V_loguniform=(23, 1024),
        E_loguniform=(8, 4096), acts=("sigmoid", "tanh", "sin", "gaussian"),
        aggs=("sum", "mean", "max"), w_std=1.0, b_std=0.5)),
    # Supervised fwd+bwd: tanh/sigmoid hidden, identity output, sum.
    "differentiation": dict(P=2048, S=4096, S_recompute=65536, spec=GenomeSpec(
        I=8, O=1, N=64, C=256, hidden=(0, 55), E_uniform=(32, 256),
        acts=("tanh", "sigmoid"), out_acts=("identity",), aggs=("sum",),
        w_std=1.0, b_std=0.5)),
    # HyperNEAT CPPNs: inputs (x1, y1, x2, y2, bias), 1 output.
    "hyperneat": dict(P=256, grid=32, thresh=0.2, spec=GenomeSpec(
        I=5, O=1, N=64, C=256, hidden=(0, 58), E_uniform=(32, 256),
        acts=("sin", "gaussian", "tanh", "abs", "identity"), aggs=("sum",),
        w_std=1.0, b_std=0.5)),
    # Recurrent ("concurrent") networks: the locomotion shape plus 15 % extra
    # enabled back-edges and self-loops; T synchronous iterations per input
    # vector, S = 64 vectors per genome.  Bounded activations, no product.
    "recurrent": dict(P=10000, S=64, T=8, spec=GenomeSpec(
        I=27, O=8, N=128, C=512, hidden=(0, 90), E_uniform=(50, 400),
        acts=("sigmoid", "tanh", "sin", "gaussian"), aggs=("sum", "mean", "max"),
        w_std=1.0, b_std=0.5, back_frac=0.15)),
}


def population_for(name: str, seed: int = 0, P: int | None = None):
    """(nodes, conns, spec) for a named workload; P overrides the size."""
    cfg = CONFIGS[name]
    spec = cfg["spec"]
    return (*make_population(spec, cfg["P"] if P is None else P, seed), spec)


def xor_inputs() -> np.ndarray:
    """The four XOR points with a constant bias input, shared by all genomes:
    shape [1, 4, 3] (population stride 0)."""
    return np.array([[[0, 0, 1], [0, 1, 1], [1, 0, 1], [1, 1, 1]]], dtype=np.float32)


def locomotion_inputs(seed: int, step: int, P: int, I: int = 27) -> np.ndarray:
    """Observation vectors of one rollout step, N(0,1): [P, 1, I] f32.
    Each step has its own seeded stream, so any step can be regenerated alone."""
    rng = np.random.default_rng([seed, 1, step])
    return rng.standard_normal((P, 1, I), dtype=np.float32)


def uneven_inputs(seed: int, step: int, P: int, S: int = 64, I: int = 17) -> np.ndarray:
    """S input vectors per genome for one step, N(0,1): [P, S, I] f32."""
    rng = np.random.default_rng([seed, 2, step])
    return rng.standard_normal((P, S, I), dtype=np.float32)


def regression_batch(seed: int, S: int):
    """Supervised batch x ~ U(-1,1)^8, target y = sin(x1*x2) + 0.5*x3^2.
    Returns (x [1, S, 8] f32 shared by all genomes, y [S] f32)."""
    rng = np.random.default_rng([seed, 3])
    x = rng.uniform(-1.0, 1.0, size=(S, 8)).astype(np.float32)
    xd = x.astype(np.float64)
    y = (np.sin(xd[:, 0] * xd[:, 1]) + 0.5 * xd[:, 2] ** 2).astype(np.float32)
    return x[None], y


def random_ops(seed: int, nodes: np.ndarray, conns: np.ndarray, I: int, K: int):
    """Seeded operation lists ops [P, K, 8] for the Sec. 3.2 operation kernel
    (kind, row, v0..v5), drawn like a NEAT generation: an enabled connection
    split by a new node (disable it, add the node, add the two connections),
    connections added between existing keys, connections removed or disabled,
    fresh weights and biases (drawn, not computed from the old values), and a
    few operations that must fail (no free row or a bad column).  Only input
    generation: no network arithmetic."""
    rng = np.random.default_rng([seed, 11])
    P, N = nodes.shape[0], nodes.shape[1]
    ops = np.zeros((P, K, 8), np.float32)
    for g in range(P):
        live = np.flatnonzero(~np.isnan(conns[g, :, 0]) & ~np.isnan(conns[g, :, 1]))
        en = live[conns[g, live, 3] != 0]
        keys = nodes[g, ~np.isnan(nodes[g, :, 0]), 0]
        hid = np.flatnonzero(~np.isnan(nodes[g, :, 0]))
        hid = hid[hid >= I]
        new_key = float(8 * N + g % 1000)
        k = 0

        def put(kind, row=0.0, *v):
            nonlocal k
            if k < K:
                ops[g, k, 0], ops[g, k, 1] = kind, row
                ops[g, k, 2:2 + len(v)] = v
                k += 1

        if en.size and K - k >= 4:  # split an enabled connection
            r = int(rng.choice(en))
            a, b, w = conns[g, r, 0], conns[g, r, 1], conns[g, r, 2]
            put(6, r, 3, 0.0)
            put(1, 0, new_key, rng.normal(0, 0.5), 1.0, rng.integers(0, 5), rng.integers(0, 4))
            put(3, 0, a, new_key, 1.0, 1.0)
            put(3, 0, new_key, b, w, 1.0)
        while k < K:
            u = rng.random()
            if u < 0.25 and live.size:
                put(6, int(rng.choice(live)), 2, rng.normal())           # weight
            elif u < 0.4 and hid.size:
                put(5, int(rng.choice(hid)), 1, rng.normal(0, 0.5))      # bias
            elif u < 0.55 and live.size:
                put(4, int(rng.choice(live)))                            # remove a connection
            elif u < 0.7 and keys.size >= 2 and hid.size:
                a = rng.choice(keys)
                b = nodes[g, int(rng.choice(hid)), 0]                    # not an input
                put(3, 0, a, b, rng.normal(), 1.0)                       # add a connection
            elif u < 0.8 and live.size:
                put(6, int(rng.choice(live)), 3, 0.0)                    # disable
            elif u < 0.9:
                put(5, int(rng.integers(0, N)), 0, 1.0)                  # key column: fails
            else:
                put(2, float(N + rng.integers(0, 4)))                    # row out of range: fails
    return ops

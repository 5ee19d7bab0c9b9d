"""Hand-built genomes for tests (padded Sec. 3.1 encoding), plus the textbook
activation functions used to write closed forms.  No network evaluation here."""
import json
import math
import os

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")

IDENTITY, SIGMOID, TANH, RELU, SIN, GAUSS, ABS = range(7)
SUM, PRODUCT, MAX, MEAN = range(4)


def blank(N, C):
    return (np.full((N, 5), np.nan, np.float32), np.full((C, 4), np.nan, np.float32))


def genome(N, C, nodes, conns):
    """nodes: [(row, key, bias, resp, act, agg)], conns: [(row, in_key, out_key, w, en)]."""
    n, c = blank(N, C)
    for row, key, b, r, a, g in nodes:
        n[row] = (key, b, r, a, g)
    for row, ki, ko, w, en in conns:
        c[row] = (ki, ko, w, en)
    return n, c


def load_xor():
    with open(os.path.join(GOLDEN, "xor_network.json")) as f:
        d = json.load(f)
    nodes = [tuple(x) for x in d["nodes"]]
    conns = [tuple(x) for x in d["conns"]]
    n, c = genome(d["N"], d["C"], nodes, conns)
    return d, n, c


def act_ref(a, z):
    """Textbook unscaled activations (sigmoid 1/(1+e^-z), gaussian e^{-z^2})."""
    if a == IDENTITY:
        return z
    if a == SIGMOID:
        return 1.0 / (1.0 + math.exp(-z)) if z >= 0 else math.exp(z) / (1.0 + math.exp(z))
    if a == TANH:
        return math.tanh(z)
    if a == RELU:
        return z if z > 0 else 0.0
    if a == SIN:
        return math.sin(z)
    if a == GAUSS:
        return math.exp(-z * z)
    if a == ABS:
        return abs(z)
    raise ValueError(a)


def stack(genomes):
    ns = np.stack([g[0] for g in genomes])
    cs = np.stack([g[1] for g in genomes])
    return ns, cs


def mlp_genome(rng, I, H, O, W1, b1, W2, b2, r1, r2, act, N, C):
    """Dense layered network I -> H -> O (sum aggregation) with random hidden
    keys, shuffled hidden rows and scattered connection rows.  Returns
    (nodes, conns, hidden_rows) with hidden unit h at row hidden_rows[h]."""
    keys_h = rng.choice(np.arange(I + O, 200), H, replace=False)
    rows_h = I + O + rng.choice(N - I - O, H, replace=False)
    nodes = [(i, i, 0, 1, 0, 0) for i in range(I)]
    nodes += [(I + o, I + o, b2[o], r2[o], act, SUM) for o in range(O)]
    nodes += [(int(rows_h[h]), int(keys_h[h]), b1[h], r1[h], act, SUM) for h in range(H)]
    conns = []
    for h in range(H):
        for i in range(I):
            conns.append((int(keys_h[h]), i, W1[h, i]))
    for o in range(O):
        for h in range(H):
            conns.append((I + o, int(keys_h[h]), W2[o, h]))
    crow = rng.permutation(C)[:len(conns)]
    n, c = genome(N, C, nodes, [(int(crow[k]), src, dst, w, 1)
                                for k, (dst, src, w) in enumerate(conns)])
    return n, c, [int(r) for r in rows_h]

"""Pins of the oracle's transformation stage (Sec. 3.3: topological order,
plus layer indices) against hand derivations, brute force and invariants."""
import itertools

import numpy as np
import pytest

import oracle
from genome_builders import SIGMOID, SUM, genome, load_xor, stack
from workloads import CONFIGS, GenomeSpec, make_population, population_for


def test_xor_order_and_layers():
    d, n, c = load_xor()
    order, layer, nl, st = oracle.transform(n[None], c[None], d["I"], d["O"])
    assert st[0] == 0
    assert order[0].tolist() == d["expected_order_rows"]
    assert layer[0].tolist() == d["expected_layer_per_row"]
    assert nl[0] == d["expected_n_layers"]


def _edges(n, c):
    """enabled (src_row, dst_row) pairs, resolved by key (test-side decoding)."""
    key_row = {float(n[r, 0]): r for r in range(n.shape[0]) if not np.isnan(n[r, 0])}
    out = []
    for j in range(c.shape[0]):
        if np.isnan(c[j, 0]) or np.isnan(c[j, 1]) or np.isnan(c[j, 3]) or c[j, 3] == 0:
            continue
        out.append((key_row[float(c[j, 0])], key_row[float(c[j, 1])]))
    return out


def _longest_path_layers(rows, edges):
    """layer(k) = number of edges on the longest path ending at k, by explicit
    enumeration of all paths (exponential; tiny graphs only)."""
    preds = {r: [s for s, d in edges if d == r] for r in rows}

    def all_paths_to(k):
        if not preds[k]:
            return [[k]]
        paths = [[k]]
        for s in preds[k]:
            paths += [p + [k] for p in all_paths_to(s)]
        return paths

    return {r: max(len(p) - 1 for p in all_paths_to(r)) for r in rows}


def _random_tiny_dag(rng, n_valid, I, O, N, C):
    """random DAG on n_valid nodes with random keys / rows (test-local recipe)."""
    h = n_valid - I - O
    keys = list(range(I + O)) + list(rng.choice(np.arange(I + O, 40), h, replace=False))
    rows = list(range(I + O)) + list(I + O + rng.choice(N - I - O, h, replace=False))
    perm = [0] * I + list(rng.permutation(h) + 1)  # rank for hidden
    # position order: inputs, hidden (random), outputs
    pos = {}
    hid = list(rng.permutation(h))
    seq = list(range(I)) + [I + O + x for x in hid] + list(range(I, I + O))
    for p, node in enumerate(seq):
        pos[node] = p
    cand = [(a, b) for a in seq for b in seq if pos[a] < pos[b] and b >= I]
    k = min(len(cand), C, int(rng.integers(1, len(cand) + 1)))
    pick = rng.choice(len(cand), k, replace=False)
    nodes = [(rows[i], keys[i], float(rng.normal()), 1.0, SIGMOID, SUM) for i in range(n_valid)]
    crow = rng.choice(C, k, replace=False)
    conns = [(int(crow[t]), keys[cand[pi][0]], keys[cand[pi][1]], float(rng.normal()),
              1.0 if rng.random() < 0.85 else 0.0) for t, pi in enumerate(pick)]
    del perm
    return genome(N, C, nodes, conns)


@pytest.mark.parametrize("seed", range(6))
def test_bruteforce_all_topological_orders(seed):
    rng = np.random.default_rng(100 + seed)
    I, O, N, C = 2, 1, 10, 24
    gens = [_random_tiny_dag(rng, int(rng.integers(3, 8)), I, O, N, C) for _ in range(25)]
    n, c = stack(gens)
    order, layer, nl, st = oracle.transform(n, c, I, O)
    x = rng.normal(size=(len(gens), 3, I)).astype(np.float32)
    out = oracle.forward(n, c, x, I, O)
    for g in range(len(gens)):
        assert st[g] == 0
        rows = [r for r in range(N) if not np.isnan(n[g, r, 0])]
        edges = _edges(n[g], c[g])
        valid_orders = [p for p in itertools.permutations(rows)
                        if all(p.index(s) < p.index(d) for s, d in edges)]
        got = [r for r in order[g] if r >= 0]
        assert tuple(got) in valid_orders
        lp = _longest_path_layers(rows, edges)
        for r in rows:
            assert layer[g, r] == lp[r]
        canon = sorted(rows, key=lambda r: (lp[r], float(n[g, r, 0])))
        assert got == canon
        assert nl[g] == max(lp.values()) + 1
        # canonical = lexicographically smallest (layer, key) sequence among valid orders
        best = min(valid_orders, key=lambda p: [(lp[r], float(n[g, r, 0])) for r in p])
        assert list(best) == got
    # relabelling hidden keys changes tie order but never the values
    n2 = n.copy()
    for g in range(len(gens)):
        hid = [r for r in range(I + O, N) if not np.isnan(n2[g, r, 0])]
        old = [float(n2[g, r, 0]) for r in hid]
        new = list(rng.permutation(np.arange(50, 50 + len(hid))).astype(float))
        remap = dict(zip(old, new))
        for r, k in zip(hid, new):
            n2[g, r, 0] = k
        for j in range(C):
            for col in (0, 1):
                v = float(c[g, j, col])
                if v in remap:
                    c[g, j, col] = remap[v]
    out2 = oracle.forward(n2, c, x, I, O)
    np.testing.assert_array_equal(out, out2)


@pytest.mark.parametrize("name", ["tiny", "locomotion", "uneven", "differentiation", "hyperneat"])
def test_every_enabled_edge_points_forward(name):
    nodes, conns, spec = population_for(name, seed=3, P=40)
    order, layer, nl, st = oracle.transform(nodes, conns, spec.I, spec.O)
    assert (st == 0).all()
    for g in range(nodes.shape[0]):
        pos = {int(r): p for p, r in enumerate(order[g]) if r >= 0}
        valid = [r for r in range(spec.N) if not np.isnan(nodes[g, r, 0])]
        assert sorted(pos) == valid
        for s, d in _edges(nodes[g], conns[g]):
            assert layer[g, s] < layer[g, d]
            assert pos[s] < pos[d]
        # layers are dense: every layer index below n_layers is used
        assert set(layer[g][layer[g] >= 0].tolist()) == set(range(nl[g]))
        # inputs sit in layer 0
        assert (layer[g, :spec.I] == 0).all()


def test_row_permutation_relabels_order():
    spec = CONFIGS["locomotion"]["spec"]
    nodes, conns = make_population(spec, 30, seed=7)
    order, layer, nl, st = oracle.transform(nodes, conns, spec.I, spec.O)
    rng = np.random.default_rng(1)
    for g in range(nodes.shape[0]):
        rp = np.arange(spec.N)
        rp[spec.I + spec.O:] = spec.I + spec.O + rng.permutation(spec.N - spec.I - spec.O)
        n2 = nodes[g][rp]          # new row i holds old row rp[i]
        c2 = conns[g][rng.permutation(spec.C)]
        o2, l2, nl2, st2 = oracle.transform(n2[None], c2[None], spec.I, spec.O)
        inv = np.empty_like(rp)
        inv[rp] = np.arange(spec.N)
        expect = [int(inv[r]) if r >= 0 else -1 for r in order[g]]
        assert o2[0].tolist() == expect
        np.testing.assert_array_equal(l2[0], layer[g][rp])
        assert nl2[0] == nl[g]


def _xor_variant(mutate):
    d, n, c = load_xor()
    n, c = n.copy(), c.copy()
    mutate(n, c)
    _, _, _, st = oracle.transform(n[None], c[None], d["I"], d["O"])
    return int(st[0]), n, c


B = oracle


@pytest.mark.parametrize("mutate,bits", [
    (lambda n, c: c.__setitem__(3, (3, 7, 1.0, 1)), B.CYCLE),                  # 3 -> 7 -> 3
    (lambda n, c: c.__setitem__(3, (7, 7, 1.0, 1)), B.CYCLE),                  # self-loop
    (lambda n, c: c.__setitem__(3, (99, 3, 1.0, 1)), B.DANGLING_KEY),
    (lambda n, c: c.__setitem__(3, (0, 99, 1.0, 1)), B.DANGLING_KEY),
    (lambda n, c: c.__setitem__(3, (0.5, 3, 1.0, 1)), B.DANGLING_KEY),         # non-integral key
    (lambda n, c: n.__setitem__(6, (5, 0, 1, 1, 0)), B.DUP_KEY),
    (lambda n, c: c.__setitem__(3, (0, 7, 2.0, 1)), B.DUP_EDGE),
    (lambda n, c: c.__setitem__(3, (7, 0, 1.0, 1)), B.EDGE_INTO_INPUT),
    (lambda n, c: n.__setitem__((4, 3), 9), B.BAD_ATTR),                       # act id
    (lambda n, c: n.__setitem__((4, 4), 4), B.BAD_ATTR),                       # agg id
    (lambda n, c: n.__setitem__((4, 3), 1.5), B.BAD_ATTR),
    (lambda n, c: n.__setitem__((4, 1), np.nan), B.BAD_ATTR),                  # NaN bias
    (lambda n, c: n.__setitem__((4, 2), np.nan), B.BAD_ATTR),                  # NaN response
    (lambda n, c: c.__setitem__((0, 2), np.nan), B.BAD_ATTR),                  # NaN weight, enabled
    (lambda n, c: n.__setitem__(6, (2.0 ** 24, 0, 1, 1, 0)), B.BAD_ATTR),      # key range
    (lambda n, c: n.__setitem__(6, (-1, 0, 1, 1, 0)), B.BAD_ATTR),
    (lambda n, c: n.__setitem__(6, (8.25, 0, 1, 1, 0)), B.BAD_ATTR),
    (lambda n, c: n.__setitem__((3, 0), np.nan), B.IO_ROW_INVALID | B.DANGLING_KEY),
    (lambda n, c: n.__setitem__((1, 0), np.nan), B.IO_ROW_INVALID | B.DANGLING_KEY),
    (lambda n, c: c.__setitem__((10, 2), np.nan), 0),                          # NaN weight, disabled
    (lambda n, c: c.__setitem__((10, 3), np.nan), 0),                          # NaN enabled = off
    (lambda n, c: n.__setitem__((0, 3), 99), 0),                               # input attrs ignored
    (lambda n, c: n.__setitem__((1, 1), np.nan), 0),
    (lambda n, c: c.__setitem__(3, (np.nan, 3, 5.0, 1)), 0),                   # half-NaN row = padding
])
def test_malformed_status_bits(mutate, bits):
    st, n, c = _xor_variant(mutate)
    assert st == bits
    out = oracle.forward(n[None], c[None], np.zeros((1, 2, 3), np.float32), 3, 1)
    assert np.isnan(out).all() == (bits != 0)


def test_cycle_keeps_partial_order():
    st, n, c = _xor_variant(lambda n, c: c.__setitem__(3, (3, 7, 1.0, 1)))
    order, layer, nl, _ = oracle.transform(n[None], c[None], 3, 1)
    # 7 and 3 sit on the cycle and so does nothing downstream; 0,1,2 then 5 are emitted
    assert order[0].tolist()[:4] == [0, 1, 2, 5] and (order[0][4:] == -1).all()
    assert layer[0].tolist() == [0, 0, 0, -1, -1, 1, -1, -1]
    assert nl[0] == 2


def test_non_cycle_errors_give_no_order():
    st, n, c = _xor_variant(lambda n, c: c.__setitem__(3, (99, 3, 1.0, 1)))
    order, layer, nl, _ = oracle.transform(n[None], c[None], 3, 1)
    assert (order == -1).all() and (layer == -1).all() and nl[0] == 0


def test_empty_and_degenerate_genomes():
    # only inputs and outputs, no connections: every output is an orphan at layer 0
    n, c = genome(6, 4, [(0, 0, 0, 1, 0, 0), (1, 1, 0, 1, 0, 0), (2, 2, 0.3, 1, SIGMOID, SUM)], [])
    order, layer, nl, st = oracle.transform(n[None], c[None], 2, 1)
    assert st[0] == 0 and order[0].tolist()[:3] == [0, 1, 2] and nl[0] == 1
    # zero-size population
    o, l, nl, st = oracle.transform(np.zeros((0, 6, 5), np.float32), np.zeros((0, 4, 4), np.float32), 2, 1)
    assert o.shape == (0, 6)


def test_long_chain_layers():
    N = 40
    nodes = [(0, 0, 0, 1, 0, 0), (1, 1, 0, 1, 0, 0)]
    keys = list(range(1000, 1000 + N - 2))
    for i, k in enumerate(keys):
        nodes.append((2 + i, k, 0.1, 1, 0, 0))
    chain = [0] + keys + [1]
    conns = [(i, chain[i], chain[i + 1], 1.0, 1) for i in range(len(chain) - 1)]
    n, c = genome(N, N, nodes, conns)
    order, layer, nl, st = oracle.transform(n[None], c[None], 1, 1)
    assert st[0] == 0 and nl[0] == N and layer[0, 1] == N - 1
    assert order[0].tolist() == [0] + list(range(2, N)) + [1]

"""Pins of the oracle's calculation stage (Sec. 3.3 forward rule
v[k] = act(b + r * agg_e(w_e * v[src_e]))) against closed forms, a library
special case and invariants."""
import math

import numpy as np
import pytest

import oracle
from genome_builders import (ABS, GAUSS, IDENTITY, MAX, MEAN, PRODUCT, RELU, SIGMOID, SIN, SUM,
                             TANH, act_ref, genome, load_xor, mlp_genome, stack)
from workloads import CONFIGS, make_population, population_for

ACTS = [IDENTITY, SIGMOID, TANH, RELU, SIN, GAUSS, ABS]


def test_xor_closed_form():
    d, n, c = load_xor()
    x = np.array(d["inputs"], np.float32)[None]
    out = oracle.forward(n[None], c[None], x, 3, 1)

    def s(z):
        return 1.0 / (1.0 + math.exp(-z))

    for k, (x1, x2, _) in enumerate(d["inputs"]):
        expect = s(20 * s(20 * x1 + 20 * x2 - 10) + 20 * s(-20 * x1 - 20 * x2 + 30) - 30)
        assert out[0, k, 0] == pytest.approx(expect, rel=1e-14, abs=1e-300)
    # XOR truth table
    assert out[0, 0, 0] < 1e-3 and out[0, 3, 0] < 1e-3
    assert out[0, 1, 0] > 1 - 1e-3 and out[0, 2, 0] > 1 - 1e-3


@pytest.mark.parametrize("agg", [SUM, PRODUCT, MAX, MEAN])
def test_single_path_chain_closed_form(agg):
    """x -> h1 -> h2 -> h3 -> out; every node aggregates one term, so any
    aggregation is the identity on it and y is a composition of scalars."""
    rng = np.random.default_rng(agg)
    for trial in range(30):
        acts = rng.choice(ACTS, 4)
        b = rng.normal(size=4)
        r = rng.normal(1.0, 0.5, size=4)
        w = rng.normal(size=4)
        keys = [0, 1, 17, 9, 30]           # x, out, h1, h2, h3
        rows = [0, 1, 5, 3, 2]
        nodes = [(0, 0, 0, 1, 0, 0)]
        chain = [keys[2], keys[3], keys[4], keys[1]]
        crow = rng.permutation(6)[:4]
        for i, k in enumerate(chain):
            row = rows[[2, 3, 4, 1][i]]
            nodes.append((row, k, b[i], r[i], int(acts[i]), agg))
        prev = [0] + chain[:-1]
        conns = [(int(crow[i]), prev[i], chain[i], w[i], 1) for i in range(4)]
        n, c = genome(8, 6, nodes, conns)
        xs = rng.normal(size=5)
        out = oracle.forward(n[None], c[None], xs.reshape(1, 5, 1).astype(np.float32), 1, 1)
        for s, x in enumerate(xs.astype(np.float32).astype(np.float64)):
            v = float(x)
            for i in range(4):
                f = lambda a: float(np.float32(a))   # the fp32 values stored in the genome
                v = act_ref(int(acts[i]), f(b[i]) + f(r[i]) * (f(w[i]) * v))
            assert out[0, s, 0] == pytest.approx(v, rel=1e-13, abs=1e-13)


@pytest.mark.parametrize("agg", [SUM, PRODUCT, MAX, MEAN])
@pytest.mark.parametrize("act", ACTS)
def test_two_input_aggregations(agg, act):
    rng = np.random.default_rng(10 * agg + act)
    b, r, w1, w2 = (float(np.float32(v)) for v in rng.normal(size=4))
    # out node (row 2, key 2) with edges from x1 (key 0) and x2 (key 1), rows swapped
    n, c = genome(4, 4, [(0, 0, 0, 1, 0, 0), (1, 1, 0, 1, 0, 0), (2, 2, b, r, act, agg)],
                  [(3, 1, 2, w2, 1), (1, 0, 2, w1, 1), (0, 0, 2, 55.0, 0)])
    xs = rng.normal(size=(7, 2)).astype(np.float32)
    out = oracle.forward(n[None], c[None], xs[None], 2, 1)
    for s, (x1, x2) in enumerate(xs.astype(np.float64)):
        t1, t2 = w1 * x1, w2 * x2
        a = {SUM: t1 + t2, PRODUCT: t1 * t2, MAX: max(t1, t2), MEAN: (t1 + t2) / 2}[agg]
        assert out[0, s, 0] == pytest.approx(act_ref(act, b + r * a), rel=1e-13, abs=1e-14)


@pytest.mark.parametrize("agg", [SUM, PRODUCT, MAX, MEAN])
@pytest.mark.parametrize("act", ACTS)
def test_orphan_node_is_activation_of_bias(agg, act):
    """A node without enabled incoming connections aggregates to 0 (reading R5)."""
    n, c = genome(4, 2, [(0, 0, 0, 1, 0, 0), (1, 1, 0.37, 2.0, act, agg)], [(0, 0, 1, 3.0, 0)])
    out = oracle.forward(n[None], c[None], np.ones((1, 2, 1), np.float32), 1, 1)
    assert out[0, 0, 0] == pytest.approx(act_ref(act, float(np.float32(0.37))), rel=1e-15)


@pytest.mark.parametrize("act", [TANH, SIGMOID, IDENTITY, RELU, SIN])
def test_layered_mlp_matches_numpy_matmul(act):
    rng = np.random.default_rng(act)
    I, H, O, N, C = 5, 7, 3, 20, 64
    f = lambda a: a.astype(np.float32).astype(np.float64)
    W1, b1, r1 = f(rng.normal(size=(H, I))), f(rng.normal(size=H)), f(rng.normal(1, .3, size=H))
    W2, b2, r2 = f(rng.normal(size=(O, H))), f(rng.normal(size=O)), f(rng.normal(1, .3, size=O))
    n, c, _ = mlp_genome(rng, I, H, O, W1, b1, W2, b2, r1, r2, act, N, C)
    x = rng.normal(size=(1, 11, I)).astype(np.float32)
    out = oracle.forward(n[None], c[None], x, I, O)
    fn = {TANH: np.tanh, SIGMOID: lambda z: 1 / (1 + np.exp(-z)), IDENTITY: lambda z: z,
          RELU: lambda z: np.maximum(z, 0), SIN: np.sin}[act]
    X = x[0].astype(np.float64).T                      # [I, S]
    hid = fn(b1[:, None] + r1[:, None] * (W1 @ X))
    ref = fn(b2[:, None] + r2[:, None] * (W2 @ hid)).T
    np.testing.assert_allclose(out[0], ref, rtol=1e-12, atol=1e-12)


def test_disabled_and_padding_rows_change_nothing():
    spec = CONFIGS["locomotion"]["spec"]
    nodes, conns = make_population(spec, 20, seed=5)
    x = np.random.default_rng(0).normal(size=(20, 3, spec.I)).astype(np.float32)
    ref = oracle.forward(nodes, conns, x, spec.I, spec.O)
    rng = np.random.default_rng(1)
    n2, c2 = nodes.copy(), conns.copy()
    c3 = conns.copy()
    for g in range(20):
        en = np.flatnonzero((~np.isnan(conns[g, :, 0])) & (conns[g, :, 3] == 1))
        kill = rng.choice(en, 5, replace=False)
        c2[g, kill, 3] = 0.0                 # disable ...
        c3[g, kill] = np.nan                 # ... is the same as removing the row
        dis = np.flatnonzero(c2[g, :, 3] == 0)
        c2[g, dis, 2] = rng.choice([np.nan, np.inf, 1e30], dis.size)   # garbage weights
        pad = np.flatnonzero(np.isnan(c2[g, :, 0]))
        c2[g, pad, 1:] = rng.normal(size=(pad.size, 3))                 # garbage after NaN key
        npad = np.flatnonzero(np.isnan(nodes[g, :, 0]))
        n2[g, npad, 1:] = rng.normal(size=(npad.size, 4)) * 100
        n2[g, :spec.I, 1:] = np.nan                                     # input attrs unused
    a = oracle.forward(n2, c2, x, spec.I, spec.O)
    b = oracle.forward(nodes, c3, x, spec.I, spec.O)
    np.testing.assert_array_equal(a, b)
    assert not np.array_equal(a, ref)


def test_population_permutation_permutes_outputs():
    nodes, conns, spec = population_for("differentiation", seed=2, P=40)
    x = np.random.default_rng(0).normal(size=(40, 4, spec.I)).astype(np.float32)
    ref = oracle.forward(nodes, conns, x, spec.I, spec.O)
    perm = np.random.default_rng(3).permutation(40)
    out = oracle.forward(nodes[perm], conns[perm], x[perm], spec.I, spec.O)
    np.testing.assert_array_equal(out, ref[perm])


def test_row_permutation_changes_nothing():
    nodes, conns, spec = population_for("locomotion", seed=4, P=25)
    x = np.random.default_rng(0).normal(size=(25, 3, spec.I)).astype(np.float32)
    ref = oracle.forward(nodes, conns, x, spec.I, spec.O)
    rng = np.random.default_rng(9)
    n2, c2 = nodes.copy(), conns.copy()
    fixed = spec.I + spec.O
    for g in range(25):
        n2[g, fixed:] = nodes[g, fixed + rng.permutation(spec.N - fixed)]
        c2[g] = conns[g, rng.permutation(spec.C)]
    out = oracle.forward(n2, c2, x, spec.I, spec.O)
    # connection order inside a sum changes fp64 rounding only
    np.testing.assert_allclose(out, ref, rtol=1e-12, atol=1e-12)


def test_shared_inputs_equal_broadcast():
    nodes, conns, spec = population_for("tiny", seed=0)
    from workloads import xor_inputs
    x = xor_inputs()
    a = oracle.forward(nodes, conns, x, 3, 1)
    b = oracle.forward(nodes, conns, np.repeat(x, nodes.shape[0], 0), 3, 1)
    np.testing.assert_array_equal(a, b)


def _fp32_forward(n, c, order, x, I, O, rng):
    """Independent fp32 evaluation (numpy float32 scalars, shuffled sums)."""
    f = np.float32
    key_row = {float(n[r, 0]): r for r in range(n.shape[0]) if not np.isnan(n[r, 0])}
    ins = {}
    for j in range(c.shape[0]):
        if np.isnan(c[j, 0]) or np.isnan(c[j, 1]) or np.isnan(c[j, 3]) or c[j, 3] == 0:
            continue
        ins.setdefault(key_row[float(c[j, 1])], []).append((key_row[float(c[j, 0])], f(c[j, 2])))
    acts = {0: lambda z: z, 1: lambda z: f(1) / (f(1) + np.exp(-z)), 2: np.tanh,
            3: lambda z: max(z, f(0)), 4: np.sin, 5: lambda z: np.exp(-(z * z)), 6: abs}
    v = {}
    for i in range(I):
        v[i] = f(x[i])
    for r in order:
        if r < 0 or r < I:
            continue
        terms = [w * v[s] for s, w in ins.get(r, [])]
        terms = [terms[k] for k in rng.permutation(len(terms))]
        agg = int(n[r, 4])
        if not terms:
            a = f(0)
        elif agg == SUM or agg == MEAN:
            a = f(0)
            for t in terms:
                a = f(a + t)
            if agg == MEAN:
                a = f(a / f(len(terms)))
        elif agg == PRODUCT:
            a = f(1)
            for t in terms:
                a = f(a * t)
        else:
            a = terms[0]
            for t in terms[1:]:
                a = max(a, t)
        v[r] = f(acts[int(n[r, 3])](f(n[r, 1]) + f(n[r, 2]) * a))
    return [v[I + j] for j in range(O)]


def test_fp32_error_bound_covers_independent_fp32_evaluation():
    nodes, conns, spec = population_for("locomotion", seed=11, P=60)
    x = np.random.default_rng(0).normal(size=(60, 4, spec.I)).astype(np.float32)
    ref, bnd = oracle.forward(nodes, conns, x, spec.I, spec.O, with_bound=True)
    order, _, _, _ = oracle.transform(nodes, conns, spec.I, spec.O)
    rng = np.random.default_rng(2)
    worst = 0.0
    with np.errstate(all="ignore"):
        for g in range(60):
            for s in range(4):
                got = np.array(_fp32_forward(nodes[g], conns[g], order[g], x[g, s], spec.I, spec.O,
                                             rng), np.float64)
                err = np.abs(got - ref[g, s])
                fin = np.isfinite(ref[g, s])
                assert (err[fin] <= 2 * bnd[g, s][fin] + 1e-30).all(), (g, s, err, bnd[g, s])
                worst = max(worst, float((err[fin] / (bnd[g, s][fin] + 1e-300)).max(initial=0)))
    # the bound is tight: an independent fp32 evaluation reaches 0.96 of it on
    # this population, so a bound four times too loose fails here
    assert worst > 0.25

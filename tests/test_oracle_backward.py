"""Pins of the oracle's reverse mode (dL/dw, dL/db, dL/dr, dL/dx for
L = sum_{s,o} g[s,o] * O[s,o]) against FP64 central differences of the oracle
forward and against hand back-propagation of a layered MLP."""
import numpy as np
import pytest

import oracle
from genome_builders import (ABS, GAUSS, IDENTITY, MAX, MEAN, PRODUCT, RELU, SIGMOID, SIN, SUM,
                             TANH, genome, mlp_genome)
from workloads import CONFIGS, make_population, regression_batch

H = 1e-6


def _loss(n, c, x, I, O, g):
    return float((oracle.forward(n, c, x, I, O) * g).sum())


def _fd_check(n, c, x, I, O, rng, n_probe=12, rtol=2e-6):
    """Compare oracle.backward with central differences on random probes.
    A probe where the two one-sided differences disagree sits on a kink
    (relu, abs, max switch) and is skipped."""
    n = n.astype(np.float64)
    c = c.astype(np.float64)
    x = x.astype(np.float64)
    P, S = n.shape[0], x.shape[1]
    g = rng.normal(size=(P, S, O))
    gw, gb, gr, gi = oracle.backward(n, c, x, I, O, g)
    scale = max(np.abs(gw).max(), np.abs(gb).max(), np.abs(gr).max(), np.abs(gi).max(), 1e-30)
    l0 = _loss(n, c, x, I, O, g)

    def check(arr, idx, analytic, what):
        a0 = arr[idx]
        arr[idx] = a0 + H
        lp = _loss(n, c, x, I, O, g)
        arr[idx] = a0 - H
        lm = _loss(n, c, x, I, O, g)
        arr[idx] = a0
        fwd, bwd = (lp - l0) / H, (l0 - lm) / H
        if abs(fwd - bwd) > 1e-3 * max(abs(fwd), abs(bwd), scale):
            return 0                                   # kink
        fd = (lp - lm) / (2 * H)
        assert abs(fd - analytic) <= rtol * max(abs(fd), scale), (what, idx, fd, analytic)
        return 1

    checked = 0
    for p in range(P):
        en = np.flatnonzero((~np.isnan(c[p, :, 0])) & (c[p, :, 3] != 0))
        for j in rng.choice(en, min(n_probe, en.size), replace=False):
            checked += check(c, (p, j, 2), gw[p, j], "w")
        valid = [r for r in range(I, n.shape[1]) if not np.isnan(n[p, r, 0])]
        for r in rng.choice(valid, min(max(n_probe // 2, 1), len(valid)), replace=False):
            checked += check(n, (p, r, 1), gb[p, r], "b")
            checked += check(n, (p, r, 2), gr[p, r], "r")
        for s in range(min(S, 3)):
            for i in range(I):
                checked += check(x, (p, s, i), gi[p, s, i], "x")
        off = np.setdiff1d(np.arange(c.shape[1]), en)
        assert (gw[p, off] == 0).all()                  # disabled / padding rows
        assert (gb[p, :I] == 0).all() and (gr[p, :I] == 0).all()
    return checked


def test_fd_differentiation_population():
    """The supervised-workload genomes: tanh/sigmoid hidden, identity output, sum."""
    spec = CONFIGS["differentiation"]["spec"]
    n, c = make_population(spec, 32, seed=0)
    x = np.repeat(regression_batch(0, 6)[0], 32, 0)
    assert _fd_check(n, c, x, spec.I, spec.O, np.random.default_rng(0), n_probe=6) > 500


@pytest.mark.parametrize("agg", [SUM, PRODUCT, MAX, MEAN])
@pytest.mark.parametrize("act", [IDENTITY, SIGMOID, TANH, RELU, SIN, GAUSS, ABS])
def test_fd_hand_cases(agg, act):
    """Small three-level genomes per (activation, aggregation)."""
    rng = np.random.default_rng(7 * agg + act)
    done = 0
    for trial in range(12):
        nodes = [(0, 0, 0, 1, 0, 0), (1, 1, 0, 1, 0, 0), (2, 2, 0, 1, 0, 0),
                 (3, 3, rng.normal(), rng.normal(1, .3), act, agg),
                 (4, 11, rng.normal(), rng.normal(1, .3), act, agg),
                 (6, 8, rng.normal(), rng.normal(1, .3), act, agg)]
        conns = [(0, 0, 11, rng.normal(), 1), (2, 1, 11, rng.normal(), 1),
                 (3, 2, 8, rng.normal(), 1), (5, 11, 8, rng.normal(), 1),
                 (6, 11, 3, rng.normal(), 1), (7, 8, 3, rng.normal(), 1),
                 (8, 1, 3, rng.normal(), 1), (9, 0, 8, 4.0, 0)]
        n, c = genome(8, 10, nodes, conns)
        x = rng.normal(size=(1, 4, 3))
        done += _fd_check(n[None], c[None], x, 3, 1, rng, n_probe=8, rtol=5e-6)
    assert done > 100


def test_product_gradient_with_zero_factor():
    """Product with a zero factor: o = (2 x0)(3 x1) at x0 = 0."""
    n, c = genome(4, 4, [(0, 0, 0, 1, 0, 0), (1, 1, 0, 1, 0, 0),
                         (2, 2, 0.0, 1.0, IDENTITY, PRODUCT)],
                  [(0, 0, 2, 2.0, 1), (1, 1, 2, 3.0, 1)])
    x = np.array([[[0.0, 5.0]]], np.float32)
    gw, gb, gr, gi = oracle.backward(n[None], c[None], x, 2, 1, np.ones((1, 1, 1)))
    # do/dw0 = x0 * 3 x1 = 0, do/dw1 = 2 x0 * x1 = 0, do/dx0 = 2 * 3 x1 = 30, do/dx1 = 0
    assert gw[0, 0] == 0 and gw[0, 1] == 0
    assert gi[0, 0, 0] == 30.0 and gi[0, 0, 1] == 0.0
    assert gr[0, 2] == 0.0 and gb[0, 2] == 1.0


def test_max_tie_goes_to_lowest_row():
    n, c = genome(4, 4, [(0, 0, 0, 1, 0, 0), (1, 1, 0, 1, 0, 0), (2, 2, 0.0, 1.0, IDENTITY, MAX)],
                  [(2, 0, 2, 1.0, 1), (1, 1, 2, 1.0, 1)])
    x = np.array([[[0.5, 0.5]]], np.float32)
    gw, gb, gr, gi = oracle.backward(n[None], c[None], x, 2, 1, np.ones((1, 1, 1)))
    assert gw[0, 1] == 0.5 and gw[0, 2] == 0.0      # row 1 (key 1 -> 2) wins the tie
    assert gi[0, 0].tolist() == [0.0, 1.0]


def test_mlp_backprop_matches_numpy():
    rng = np.random.default_rng(3)
    I, Hd, O, N, C = 4, 6, 2, 16, 48
    f = lambda a: a.astype(np.float32).astype(np.float64)
    W1, b1, r1 = f(rng.normal(size=(Hd, I))), f(rng.normal(size=Hd)), f(rng.normal(1, .3, size=Hd))
    W2, b2, r2 = f(rng.normal(size=(O, Hd))), f(rng.normal(size=O)), f(rng.normal(1, .3, size=O))
    n, c, hrows = mlp_genome(rng, I, Hd, O, W1, b1, W2, b2, r1, r2, TANH, N, C)
    x = rng.normal(size=(1, 9, I)).astype(np.float32)
    G = rng.normal(size=(1, 9, O))
    gw, gb, gr, gi = oracle.backward(n[None], c[None], x, I, O, G)
    X = x[0].astype(np.float64).T
    a1 = W1 @ X
    h = np.tanh(b1[:, None] + r1[:, None] * a1)
    a2 = W2 @ h
    y = np.tanh(b2[:, None] + r2[:, None] * a2)
    dz2 = G[0].T * (1 - y ** 2)
    dW2 = (r2[:, None] * dz2) @ h.T
    dh = W2.T @ (r2[:, None] * dz2)
    dz1 = dh * (1 - h ** 2)
    dW1 = (r1[:, None] * dz1) @ X.T
    dX = W1.T @ (r1[:, None] * dz1)
    np.testing.assert_allclose(gb[0, I:I + O], dz2.sum(1), rtol=1e-11, atol=1e-12)
    np.testing.assert_allclose(gr[0, I:I + O], (dz2 * a2).sum(1), rtol=1e-11, atol=1e-12)
    np.testing.assert_allclose(gb[0, hrows], dz1.sum(1), rtol=1e-11, atol=1e-12)
    np.testing.assert_allclose(gr[0, hrows], (dz1 * a1).sum(1), rtol=1e-11, atol=1e-12)
    np.testing.assert_allclose(gi[0], dX.T, rtol=1e-11, atol=1e-12)
    key_row = {float(n[r, 0]): r for r in range(N) if not np.isnan(n[r, 0])}
    for j in range(C):
        if np.isnan(c[j, 0]):
            assert gw[0, j] == 0
            continue
        s, d = key_row[float(c[j, 0])], key_row[float(c[j, 1])]
        expect = dW2[d - I, hrows.index(s)] if d < I + O else dW1[hrows.index(d), s]
        assert gw[0, j] == pytest.approx(expect, rel=1e-10, abs=1e-12)


def test_malformed_genome_has_zero_gradients():
    n, c = genome(4, 4, [(0, 0, 0, 1, 0, 0), (1, 1, 0, 1, 0, 0), (2, 2, 0.0, 1.0, TANH, SUM)],
                  [(0, 0, 2, 2.0, 1), (1, 2, 2, 3.0, 1)])      # self-loop -> cycle
    gw, gb, gr, gi = oracle.backward(n[None], c[None], np.ones((1, 2, 2), np.float32), 2, 1,
                                     np.ones((1, 2, 1)))
    assert not gw.any() and not gb.any() and not gr.any() and not gi.any()

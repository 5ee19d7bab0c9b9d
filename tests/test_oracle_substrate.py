"""Pins of the oracle's HyperNEAT substrate evaluation (reading R14: the
two-sheet substrate of the query grid, y_t = act(sum_s w[s, t] x_s)):
the identity case against numpy matmul, a one-connection closed form, a
closed-form CPPN through the query, and the fp32 bound."""
import math

import numpy as np

import oracle
from genome_builders import genome

IDENTITY, SIGMOID, TANH, SIN = 0, 1, 2, 4


def test_identity_substrate_is_a_matrix_product():
    rng = np.random.default_rng(0)
    P, K, S = 3, 49, 5
    w = rng.standard_normal((P, K, K))
    w[np.abs(w) < 0.2] = 0.0
    x = rng.standard_normal((P, S, K))
    np.testing.assert_allclose(oracle.substrate(w, x, IDENTITY), x @ w, rtol=1e-12, atol=1e-12)
    xs = rng.standard_normal((1, S, K))  # one pattern set shared by every genome
    np.testing.assert_allclose(oracle.substrate(w, xs, IDENTITY), xs @ w, rtol=1e-12,
                               atol=1e-12)


def test_single_connection_closed_form():
    K = 16
    w = np.zeros((1, K, K))
    w[0, 3, 11] = 0.75
    x = np.linspace(-1, 1, K)[None, None]
    y = oracle.substrate(w, x, TANH)[0, 0]
    for t in range(K):
        want = math.tanh(0.75 * x[0, 0, 3]) if t == 11 else 0.0
        assert math.isclose(y[t], want, rel_tol=1e-14, abs_tol=1e-15)


def test_closed_form_cppn_through_the_query():
    """CPPN o = sin(x_s + y_t) (one hidden-free node): the query's thresholded
    weights in closed form, then the substrate sum in closed form."""
    G, thr = 5, 0.2
    n, c = genome(8, 8, [(r, r, 0, 1, 0, 0) for r in range(5)] + [(5, 5, 0.0, 1.0, SIN, 0)],
                  [(0, 0, 5, 1.0, 1.0), (1, 3, 5, 1.0, 1.0)])
    w = oracle.hyperneat(n[None], c[None], grid=G, thresh=thr).reshape(1, G * G, G * G)
    coord = [-1 + 2 * i / (G - 1) for i in range(G)]
    x = np.random.default_rng(3).standard_normal((1, 2, G * G))
    y = oracle.substrate(w, x, SIGMOID)
    for s_ in range(2):
        for t in range(G * G):
            tot = 0.0
            for src in range(G * G):
                o = math.sin(coord[src % G] + coord[t // G])
                wt = o if abs(o) > thr else 0.0
                tot += wt * x[0, s_, src]
            assert math.isclose(y[0, s_, t], 1 / (1 + math.exp(-tot)), rel_tol=1e-12,
                                abs_tol=1e-14)


def test_fp32_products_stay_inside_the_bound():
    rng = np.random.default_rng(5)
    P, K, S = 2, 1024, 4
    w = rng.standard_normal((P, K, K)).astype(np.float32)
    w[np.abs(w) < 0.2] = 0.0
    x = rng.standard_normal((P, S, K)).astype(np.float32)
    for act in (IDENTITY, TANH, SIN):
        ref, bnd = oracle.substrate(w, x, act, with_bound=True)
        f32 = np.matmul(x, w)  # float32 arithmetic, its own summation order
        if act == TANH:
            f32 = np.tanh(f32)
        elif act == SIN:
            f32 = np.sin(f32)
        err = np.abs(f32.astype(np.float64) - ref)
        assert (err <= 2 * bnd).all(), float((err / bnd).max())
        # not vacuous: at most about the textbook (K + 1) u sum_s |w x|
        # (u = 2^-24), and of that order where the activation does not
        # saturate (tanh of sums near +-30 has a vanishing slope)
        sabs = np.abs(x.astype(np.float64)) @ np.abs(w.astype(np.float64))
        assert (bnd <= 1e-4 * sabs + 1e-30).all()
        if act != TANH:
            assert (bnd >= 1e-5 * sabs).mean() > 0.5

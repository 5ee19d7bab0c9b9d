"""Pins of the oracle's recurrent ("concurrent") calculation, reading R11:
T synchronous iterations, inputs clamped, v^0 = 0 on non-input nodes, outputs
v^T.  Each check is independent of the oracle's own per-node loop: matrix
powers of the linear special case, a hand-derived closed form, and the
(separately pinned) feed-forward calculation on acyclic genomes."""
import math

import numpy as np
import pytest

import oracle
from genome_builders import genome, stack
from workloads import CONFIGS, GenomeSpec, make_population, population_for

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")

IDENTITY, TANH = 0, 2
SUM = 0


def _linear_recurrent(rng, I, O, H, N, C, p_edge=0.35, scale=0.4):
    """Identity/sum genome over I inputs, O outputs and H hidden nodes with
    random edges between any nodes (back edges and self-loops included),
    random biases and responses.  Returns (nodes, conns, W, b, r) with W[d, s]
    the weight of edge s -> d over node ids 0..M-1 (inputs first, then
    outputs, then hidden; node id = row)."""
    M = I + O + H
    keys = list(range(I + O)) + [int(k) for k in rng.choice(np.arange(I + O, 400), H,
                                                             replace=False)]
    f32 = lambda a: np.asarray(a, np.float32).astype(np.float64)  # noqa: E731 (table precision)
    b = f32(rng.normal(0, 0.3, M))
    r = f32(rng.uniform(0.5, 1.5, M))
    b[:I] = 0.0
    r[:I] = 1.0
    nodes = [(m, keys[m], b[m], r[m], IDENTITY, SUM) for m in range(M)]
    W = np.zeros((M, M))
    conns = []
    row = 0
    for d in range(I, M):
        for s_ in range(M):
            if rng.random() < p_edge and row < C:
                w = float(f32(rng.normal(0, scale)))
                W[d, s_] = w
                conns.append((row, keys[s_], keys[d], w, 1.0))
                row += 1
    n, c = genome(N, C, nodes, conns)
    return n, c, W, b, r


@pytest.mark.parametrize("seed", range(8))
def test_linear_recurrent_matches_matrix_powers(seed):
    """Identity activations with sum aggregation make every iteration affine:
    h^t = M h^{t-1} + u with M = diag(r) W_hh, u = b + diag(r) W_hx x, h^0 = 0,
    so h^T = sum_{k<T} M^k u (numpy matrix powers)."""
    rng = np.random.default_rng(seed)
    I, O, H, N, C = 3, 2, 5, 16, 128
    n, c, W, b, r = _linear_recurrent(rng, I, O, H, N, C)
    x = rng.standard_normal((1, 4, I))
    idx = np.arange(I, I + O + H)
    Mh = np.diag(r[idx]) @ W[np.ix_(idx, idx)]
    for T in (0, 1, 2, 5, 9):
        out = oracle.forward_recurrent(n[None], c[None], x, I, O, T)
        for s in range(4):
            u = b[idx] + r[idx] * (W[np.ix_(idx, np.arange(I))] @ x[0, s])
            h = sum((np.linalg.matrix_power(Mh, k) @ u for k in range(T)),
                    np.zeros(idx.size))
            np.testing.assert_allclose(out[0, s], h[:O], rtol=1e-12, atol=1e-12)


def test_self_loop_closed_form():
    """x -> h (w1), h -> h (w2), h -> o (w3), identity/sum, b = 0, r = 1:
    h^t = w1 x (1 - w2^t) / (1 - w2) and o^t = w3 h^{t-1}, o^0 = 0."""
    w1, w2, w3 = 0.75, -0.375, 1.25  # exact in fp32
    n, c = genome(8, 8, [(0, 0, 0, 1, IDENTITY, SUM), (1, 1, 0, 1, IDENTITY, SUM),
                         (5, 40, 0, 1, IDENTITY, SUM)],
                  [(2, 0, 40, w1, 1.0), (4, 40, 40, w2, 1.0), (6, 40, 1, w3, 1.0)])
    for x in (0.5, -2.0):
        for T in range(0, 8):
            out = oracle.forward_recurrent(n[None], c[None], np.array([[[x]]]), 1, 1, T)
            want = 0.0 if T == 0 else w3 * w1 * x * (1 - w2 ** (T - 1)) / (1 - w2)
            assert math.isclose(out[0, 0, 0], want, rel_tol=1e-13, abs_tol=1e-15), (x, T)


def test_acyclic_genomes_reach_the_feedforward_values():
    """On a DAG the node of layer l is final from iteration l on, so T >=
    depth gives exactly the feed-forward outputs (bit for bit in FP64); one
    iteration fewer than a deep genome's depth generally does not."""
    nodes, conns, spec = population_for("locomotion", seed=4, P=40)
    x = np.random.default_rng(2).standard_normal((40, 3, spec.I))
    ff = oracle.forward(nodes, conns, x, spec.I, spec.O)
    _, _, n_layers, _ = oracle.transform(nodes, conns, spec.I, spec.O)
    differs = 0
    for g in range(40):
        T = int(n_layers[g])
        rec = oracle.forward_recurrent(nodes[g:g + 1], conns[g:g + 1], x[g:g + 1], spec.I,
                                       spec.O, T)
        np.testing.assert_array_equal(rec[0], ff[g])
        rec2 = oracle.forward_recurrent(nodes[g:g + 1], conns[g:g + 1], x[g:g + 1], spec.I,
                                        spec.O, T + 3)
        np.testing.assert_array_equal(rec2[0], ff[g])
        if T >= 3:
            short = oracle.forward_recurrent(nodes[g:g + 1], conns[g:g + 1], x[g:g + 1],
                                             spec.I, spec.O, T - 2)
            differs += int(not np.array_equal(short[0], ff[g]))
    assert differs >= 5


def test_status_bits_are_those_of_the_transform_without_cycle():
    """Cycles and self-loops are legal here; every other malformation keeps its
    bit (and NaN outputs), exactly as the feed-forward transform reports it."""
    nodes, conns, spec = population_for("recurrent", seed=1, P=30)
    _, _, _, st_ff = oracle.transform(nodes, conns, spec.I, spec.O)
    assert (st_ff == 1).sum() >= 20  # the workload is cyclic
    x = np.zeros((1, 1, spec.I))
    out, st = oracle.forward_recurrent(nodes, conns, x, spec.I, spec.O, 3, with_status=True)
    assert (st == 0).all() and np.isfinite(out).all()
    bad_n, bad_c = nodes[:4].copy(), conns[:4].copy()
    live = np.flatnonzero(~np.isnan(bad_c[0, :, 0]) & (bad_c[0, :, 3] != 0))
    bad_c[0, live[0], 1] = 7777.0                     # dangling key
    bad_c[1, live[0], 1] = 0.0                        # edge into an input
    bad_n[2, spec.I + spec.O - 1, 0] = bad_n[2, 0, 0]   # duplicate key
    bad_n[3, spec.I, 3] = 11.0                        # activation id out of range
    out, st = oracle.forward_recurrent(bad_n, bad_c, x, spec.I, spec.O, 3, with_status=True)
    _, _, _, st_ff = oracle.transform(bad_n, bad_c, spec.I, spec.O)
    np.testing.assert_array_equal(st, st_ff & ~np.uint32(1))
    assert (st != 0).all() and np.isnan(out).all()


def test_fp32_iterations_stay_inside_the_bound():
    """An independent fp32 evaluation (numpy float32 matrix form, its own
    summation order) of tanh/sum recurrent genomes stays within 2x the
    oracle's first-order bound, and the bound is not vacuous."""
    rng = np.random.default_rng(11)
    I, O, H, N, C, T = 4, 2, 10, 24, 256, 6
    worst, tight = 0.0, 0
    for trial in range(12):
        n, c, W, b, r = _linear_recurrent(rng, I, O, H, N, C, p_edge=0.3, scale=0.6)
        n[I:I + O + H, 3] = TANH
        x = rng.standard_normal((1, 5, I)).astype(np.float32).astype(np.float64)
        ref, bnd = oracle.forward_recurrent(n[None], c[None], x, I, O, T, with_bound=True)
        idx = np.arange(I, I + O + H)
        Wf = W.astype(np.float32)
        for s in range(5):
            v = np.zeros(I + O + H, np.float32)
            v[:I] = x[0, s]
            for _ in range(T):
                a = Wf[idx] @ v
                vn = v.copy()
                vn[idx] = np.tanh(b[idx].astype(np.float32) + r[idx].astype(np.float32) * a)
                v = vn
            err = np.abs(v[I:I + O].astype(np.float64) - ref[0, s])
            assert (err <= 2 * bnd[0, s] + 1e-30).all(), (trial, s, err, bnd[0, s])
            worst = max(worst, float((err / np.maximum(bnd[0, s], 1e-300)).max()))
            tight += int((bnd[0, s] < 1e-4).all())
    assert tight >= 30 and worst > 0.0


def test_generator_draws_back_edges_only_when_asked():
    """The recurrent option adds enabled pairs with pos(src) >= pos(dst); the
    other workloads' genomes are unchanged by its presence."""
    spec = CONFIGS["recurrent"]["spec"]
    n, c = make_population(spec, 20, seed=3)
    _, _, _, st = oracle.transform(n, c, spec.I, spec.O)
    assert (st == 1).sum() >= 15
    plain = GenomeSpec(**{**spec.__dict__, "back_frac": 0.0})
    n2, c2 = make_population(plain, 20, seed=3)
    _, _, _, st2 = oracle.transform(n2, c2, spec.I, spec.O)
    assert (st2 == 0).all()
    _ = stack  # builder module shared with the other oracle tests

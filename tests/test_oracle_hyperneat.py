"""Pins of the oracle's HyperNEAT substrate query: CPPNs whose output is a
known function of the coordinates, evaluated over the whole 32x32 grid."""
import numpy as np
import pytest

import oracle
from genome_builders import GAUSS, IDENTITY, SIN, SUM, TANH, genome

G = 32


def _grid():
    lin = np.linspace(-1.0, 1.0, G)          # x_i = -1 + 2 i / (G - 1)
    cell_x = np.tile(lin, G)                 # cell c = j * G + i
    cell_y = np.repeat(lin, G)
    return cell_x, cell_y


def _cppn(act, edges, bias=0.0):
    """inputs rows 0..4 = (x1, y1, x2, y2, bias), output row 5 (key 5)."""
    nodes = [(i, i, 0, 1, 0, 0) for i in range(5)] + [(5, 5, bias, 1.0, act, SUM)]
    conns = [(j, src, 5, w, 1) for j, (src, w) in enumerate(edges)]
    return genome(8, 8, nodes, conns)


@pytest.mark.parametrize("act,edges,bias,fn", [
    (IDENTITY, [(0, 1.0)], 0.0, lambda xs, ys, xd, yd: xs),
    (IDENTITY, [(3, 1.0)], 0.0, lambda xs, ys, xd, yd: yd),
    (SIN, [(0, 1.0), (3, 1.0)], 0.0, lambda xs, ys, xd, yd: np.sin(xs + yd)),
    (GAUSS, [(2, 1.5), (1, -1.5)], 0.0, lambda xs, ys, xd, yd: np.exp(-(1.5 * xd - 1.5 * ys) ** 2)),
    (TANH, [(4, 0.5), (0, 2.0)], 0.1, lambda xs, ys, xd, yd: np.tanh(0.1 + 0.5 + 2 * xs)),
])
def test_single_node_cppn_closed_form(act, edges, bias, fn):
    n, c = _cppn(act, edges, bias)
    out, raw = oracle.hyperneat(n[None], c[None], grid=G, thresh=0.2, with_raw=True)
    cx, cy = _grid()
    xs, ys = cx[:, None], cy[:, None]          # source cell varies along rows
    xd, yd = cx[None, :], cy[None, :]
    f32 = lambda a: float(np.float32(a))
    bias = f32(bias)
    expect = fn(xs, ys, xd, yd) * np.ones((G * G, G * G))
    if act == TANH:
        expect = np.tanh(bias + f32(0.5) + 2 * xs) * np.ones((G * G, G * G))
    np.testing.assert_allclose(raw[0].reshape(G * G, G * G), expect, rtol=1e-12, atol=1e-12)
    thr = np.where(np.abs(expect) > 0.2, expect, 0.0)
    np.testing.assert_allclose(out[0].reshape(G * G, G * G), thr, rtol=1e-12, atol=1e-12)


def test_query_subset_matches_full_grid():
    from workloads import population_for
    nodes, conns, spec = population_for("hyperneat", seed=1, P=3)
    full = oracle.hyperneat(nodes, conns, grid=8)
    q = np.random.default_rng(0).choice(8 ** 4, 100, replace=False)
    sub = oracle.hyperneat(nodes, conns, grid=8, qidx=q)
    np.testing.assert_array_equal(sub, full[:, q])


def test_threshold_is_strict():
    # o = x_s exactly; the grid has no |x| == 0.2 point, so use bias to hit 0.2 exactly
    n, c = _cppn(IDENTITY, [], bias=0.25)
    out = oracle.hyperneat(n[None], c[None], grid=4, thresh=0.25)
    assert (out == 0).all()
    out = oracle.hyperneat(n[None], c[None], grid=4, thresh=0.2499)
    assert (out == np.float32(0.25)).all()

"""Pins of the oracle's tensorized operations (Sec. 3.2, reading R13): node and
connection addition at the first NaN row, removal by writing NaN, attribute
assignment; expected tensors written out by hand."""
import numpy as np

import oracle
from workloads import population_for

NAN = np.nan


def _op(kind, row=0, *v):
    o = [kind, row] + list(v)
    return o + [0.0] * (8 - len(o))


def _run(n, c, ops):
    return oracle.apply_ops(n[None], c[None], np.array([ops], np.float64))


def test_add_and_remove_use_the_first_nan_row():
    n = np.array([[0, 0, 1, 0, 0],
                  [1, 0.5, 1, 1, 0],
                  [NAN, NAN, NAN, NAN, NAN],
                  [7, -0.5, 1, 2, 3],
                  [NAN, NAN, NAN, NAN, NAN]], np.float32)
    c = np.array([[0, 1, 0.25, 1],
                  [NAN, NAN, NAN, NAN],
                  [0, 7, -1.0, 0]], np.float32)
    ops = [_op(1, 0, 9, 0.1, 1.0, 4, 2),    # node -> row 2
           _op(2, 1),                       # remove row 1
           _op(1, 0, 11, 0.2, 1.0, 5, 1),   # node -> row 1 (the freed lower row)
           _op(1, 0, 12, 0.3, 1.0, 6, 0),   # node -> row 4
           _op(1, 0, 13, 0.4, 1.0, 1, 0),   # no free row: fails (bit 4)
           _op(3, 0, 9, 7, 0.5, 1),         # connection -> row 1
           _op(4, 0),                       # remove connection row 0
           _op(3, 0, 11, 9, -2.0, 1),       # connection -> row 0
           _op(3, 0, 1, 1, 1.0, 1)]         # no free row: fails (bit 8)
    nn, cc, st = _run(n, c, ops)
    want_n = np.array([[0, 0, 1, 0, 0],
                       [11, 0.2, 1, 5, 1],
                       [9, 0.1, 1, 4, 2],
                       [7, -0.5, 1, 2, 3],
                       [12, 0.3, 1, 6, 0]], np.float64)
    want_c = np.array([[11, 9, -2.0, 1],
                       [9, 7, 0.5, 1],
                       [0, 7, -1.0, 0]], np.float64)
    np.testing.assert_array_equal(nn[0], want_n.astype(np.float64))
    np.testing.assert_array_equal(cc[0], want_c)
    assert st[0] == (1 << 4) | (1 << 8)


def test_a_connection_row_is_free_when_either_key_is_nan():
    n = np.zeros((3, 5), np.float32)
    n[:, 0] = [0, 1, 2]
    c = np.array([[0, 1, 1, 1], [5, NAN, 3, 1], [0, 2, 1, 1]], np.float32)
    nn, cc, st = _run(n, c, [_op(3, 0, 1, 2, 0.75, 0)])
    np.testing.assert_array_equal(cc[0, 1], [1, 2, 0.75, 0])
    assert st[0] == 0


def test_attribute_assignment_and_ranges():
    n = np.array([[0, 0, 1, 0, 0], [4, 0.5, 1, 1, 0]], np.float32)
    c = np.array([[0, 4, 0.25, 1]], np.float32)
    ops = [_op(5, 1, 1, 2.5),       # bias of row 1
           _op(5, 1, 3, 6),         # activation id of row 1
           _op(6, 0, 2, -3.0),      # weight of conn row 0
           _op(6, 0, 3, 0.0),       # disable it
           _op(5, 1, 0, 99),        # the key column is not an attribute: fails (bit 4)
           _op(6, 0, 1, 5),         # nor the out key: fails (bit 5)
           _op(5, 2, 1, 1.0),       # row out of range: fails (bit 6)
           _op(2, -1),              # fails (bit 7)
           _op(4, 0.5),             # not an integer row: fails (bit 8)
           _op(0, 0, 1, 2, 3),      # nothing
           _op(17, 0)]              # unknown kind: nothing
    nn, cc, st = _run(n, c, ops)
    np.testing.assert_array_equal(nn[0], [[0, 0, 1, 0, 0], [4, 2.5, 1, 6, 0]])
    np.testing.assert_array_equal(cc[0], [[0, 4, -3.0, 0.0]])
    assert st[0] == sum(1 << b for b in (4, 5, 6, 7, 8))


def test_empty_and_noop_lists_change_nothing():
    nodes, conns, spec = population_for("locomotion", seed=2, P=5)
    for ops in (np.zeros((5, 0, 8)), np.zeros((5, 6, 8))):
        nn, cc, st = oracle.apply_ops(nodes, conns, ops)
        np.testing.assert_array_equal(nn, nodes.astype(np.float64))
        np.testing.assert_array_equal(cc, conns.astype(np.float64))
        assert (st == 0).all()


def test_operations_feed_the_transform():
    """Split an enabled connection a -> b by a new node h (NEAT's add-node
    mutation written as Sec. 3.2 operations): disable the row, add h, add
    a -> h and h -> b; the result still transforms and h sits between a and b."""
    nodes, conns, spec = population_for("locomotion", seed=3, P=1)
    live = np.flatnonzero(~np.isnan(conns[0, :, 0]) & (conns[0, :, 3] != 0))
    r = int(live[0])
    a, b, w = (float(x) for x in conns[0, r, :3])
    ops = [_op(6, r, 3, 0.0), _op(1, 0, 5000, 0.0, 1.0, 0, 0),
           _op(3, 0, a, 5000, 1.0, 1), _op(3, 0, 5000, b, w, 1)]
    nn, cc, st = oracle.apply_ops(nodes, conns, np.array([ops], np.float64))
    assert st[0] == 0
    order, layer, _, status = oracle.transform(nn, cc, spec.I, spec.O)
    assert status[0] == 0
    key_row = {float(k): i for i, k in enumerate(nn[0, :, 0]) if not np.isnan(k)}
    la, lh, lb = layer[0, key_row[a]], layer[0, key_row[5000.0]], layer[0, key_row[b]]
    assert la < lh < lb

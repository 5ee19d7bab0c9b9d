"""GPU parity of the Sec. 3.2 tensorized operations (node / connection
addition at the first NaN row, removal, attribute assignment) and of the fused
operations + transform call, bit for bit against the oracle."""
import numpy as np
import pytest
import torch

import oracle
from workloads import population_for, random_ops

pytestmark = pytest.mark.gpu


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _same(gpu, ref):
    np.testing.assert_array_equal(gpu.cpu().numpy().astype(np.float64), ref)


@pytest.mark.parametrize("name,P,K", [("locomotion", 300, 16), ("uneven", 40, 24),
                                      ("tiny", 100, 6)])
def test_apply_ops_bit_exact(name, P, K):
    from paper_2504_08339_b300.api import apply_ops
    nodes, conns, spec = population_for(name, seed=7, P=P)
    ops = random_ops(7, nodes, conns, spec.I, K)
    dn, dc = _dev(nodes), _dev(conns)
    st = apply_ops(dn, dc, _dev(ops))
    rn, rc, rst = oracle.apply_ops(nodes, conns, ops)
    _same(dn, rn)
    _same(dc, rc)
    np.testing.assert_array_equal(st.cpu().numpy().view(np.uint32), rst)
    assert rst.any()  # the lists include operations that must fail


def test_first_free_row_reuse_and_full_tables():
    from paper_2504_08339_b300.api import apply_ops
    nan = np.nan
    n = np.array([[[0, 0, 1, 0, 0], [1, 0.5, 1, 1, 0], [nan] * 5, [7, -0.5, 1, 2, 3],
                   [nan] * 5]], np.float32)
    c = np.array([[[0, 1, 0.25, 1], [nan] * 4, [0, 7, -1.0, 0]]], np.float32)

    def op(kind, row=0, *v):
        o = [kind, row] + list(v)
        return o + [0.0] * (8 - len(o))

    ops = np.array([[op(1, 0, 9, 0.1, 1.0, 4, 2), op(2, 1), op(1, 0, 11, 0.2, 1.0, 5, 1),
                     op(1, 0, 12, 0.3, 1.0, 6, 0), op(1, 0, 13, 0.4, 1.0, 1, 0),
                     op(3, 0, 9, 7, 0.5, 1), op(4, 0), op(3, 0, 11, 9, -2.0, 1),
                     op(3, 0, 1, 1, 1.0, 1), op(5, 1, 0, 3), op(6, 2, 3, 1.0), op(9, 0)]],
                   np.float32)
    dn, dc = _dev(n), _dev(c)
    st = apply_ops(dn, dc, _dev(ops))
    rn, rc, rst = oracle.apply_ops(n, c, ops)
    _same(dn, rn)
    _same(dc, rc)
    assert st.cpu().numpy().view(np.uint32)[0] == rst[0] == (1 << 4) | (1 << 8) | (1 << 9)


def test_mutate_transform_matches_oracle():
    from paper_2504_08339_b300.api import Plan
    nodes, conns, spec = population_for("locomotion", seed=8, P=500)
    ops = random_ops(8, nodes, conns, spec.I, 16)
    plan = Plan(500, spec.N, spec.C, spec.I, spec.O)
    dn, dc = _dev(nodes), _dev(conns)
    tr, st = plan.mutate_transform(dn, dc, _dev(ops))
    rn, rc, rst = oracle.apply_ops(nodes, conns, ops)
    _same(dn, rn)
    _same(dc, rc)
    np.testing.assert_array_equal(st.cpu().numpy().view(np.uint32), rst)
    o, l, nl, gs = oracle.transform(rn, rc, spec.I, spec.O)
    np.testing.assert_array_equal(tr.order.cpu().numpy(), o)
    np.testing.assert_array_equal(tr.layer.cpu().numpy(), l)
    np.testing.assert_array_equal(tr.n_layers.cpu().numpy(), nl)
    np.testing.assert_array_equal(tr.status.cpu().numpy().view(np.uint32), gs)
    # the mutated population evaluates like the oracle's
    x = np.random.default_rng(1).standard_normal((500, 2, spec.I)).astype(np.float32)
    from parity_util import compare_outputs
    ref, bnd = oracle.forward(rn, rc, x, spec.I, spec.O, with_bound=True)
    compare_outputs(plan.forward(_dev(x)).cpu().numpy(), ref, bnd)


def test_empty_operation_lists():
    from paper_2504_08339_b300.api import apply_ops
    nodes, conns, spec = population_for("tiny", seed=1, P=20)
    dn, dc = _dev(nodes), _dev(conns)
    st = apply_ops(dn, dc, torch.zeros((20, 0, 8), device="cuda"))
    _same(dn, nodes.astype(np.float64))
    assert (st.cpu().numpy() == 0).all()

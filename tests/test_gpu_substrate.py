"""GPU parity of the HyperNEAT two-sheet substrate evaluation (y_t =
act(sum_s w[s, t] x_s)) against the FP64 oracle, alone and fused with the
CPPN query."""
import numpy as np
import pytest
import torch

import oracle
from parity_util import compare_outputs
from workloads import population_for

pytestmark = pytest.mark.gpu

IDENTITY, TANH, SIN = 0, 2, 4


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("G,S,act,shared", [(7, 33, TANH, False), (32, 33, IDENTITY, True),
                                            (32, 70, SIN, False), (2, 5, TANH, True)])
def test_substrate_forward_parity(G, S, act, shared):
    from paper_2504_08339_b300.api import substrate_forward
    rng = np.random.default_rng(G * 100 + S)
    P, K = 5, G * G
    w = rng.standard_normal((P, K, K)).astype(np.float32)
    w[np.abs(w) <= 0.2] = 0.0  # thresholded like the query's weights
    x = rng.standard_normal((1 if shared else P, S, K)).astype(np.float32)
    out = substrate_forward(_dev(w), _dev(x), act=act).cpu().numpy()
    ref, bnd = oracle.substrate(w, x, act, with_bound=True)
    stats = compare_outputs(out, ref, bnd, what=f"G={G} act={act}")
    assert stats["n"] == P * S * K


def test_hyperneat_substrate_fused_matches_the_oracle():
    """Query + substrate in one call; outputs whose column holds a weight
    within the error band of the threshold (where 0 and the raw value are
    both correct) are left out of the comparison."""
    from paper_2504_08339_b300.api import Plan
    G, S, thr = 12, 17, 0.2
    K = G * G
    nodes, conns, spec = population_for("hyperneat", seed=6, P=10)
    plan = Plan(10, spec.N, spec.C, spec.I, spec.O)
    plan.transform(_dev(nodes), _dev(conns))
    x = np.random.default_rng(2).standard_normal((10, S, K)).astype(np.float32)
    out, wts = plan.hyperneat_substrate(_dev(x), grid=G, thresh=thr, act=TANH)
    # the fused call's weights are the query's, bit for bit
    q = plan.hyperneat(G, thr)
    assert torch.equal(wts.view(torch.int32), q.view(torch.int32))
    w_ref, raw, bnd_q = oracle.hyperneat(nodes, conns, grid=G, thresh=thr, with_raw=True,
                                         with_bound=True)
    w_ref = w_ref.reshape(10, K, K)
    raw = raw.reshape(10, K, K)
    lim = np.maximum(1e-6 + 1e-5 * np.abs(raw), 2 * bnd_q.reshape(10, K, K))
    near = np.abs(np.abs(raw) - thr) <= lim            # [g, s, t]
    ref, bnd = oracle.substrate(w_ref, x, TANH, with_bound=True)
    # an output column t is unambiguous when none of its weights is near
    keep = ~near.any(axis=1)                             # [g, t]
    mask = np.broadcast_to(keep[:, None, :], out.shape)
    assert mask.mean() > 0.9
    o = out.cpu().numpy()
    # the substrate sums also carry the query's own weight errors
    wb = bnd_q.reshape(10, K, K) * (~near)
    extra = np.abs(x.astype(np.float64)) @ wb
    compare_outputs(o[mask], ref[mask], (bnd + extra)[mask], what="fused substrate")


def test_substrate_arguments():
    from paper_2504_08339_b300 import _lib
    lib = _lib.load()
    assert lib.neat_substrate_forward(None, 2, 4, None, 0, 3, 0, None, None) == _lib.NEAT_ERR_ARG
    assert lib.neat_substrate_forward(None, 2, 4, None, 0, 3, 9, None, None) == _lib.NEAT_ERR_ARG
    assert lib.neat_substrate_forward(None, 0, 4, None, 0, 3, 0, None, None) == _lib.NEAT_OK

"""Device-side failures reach the caller, and the autograd function survives a
plan that was transformed again between its forward and backward.

The failure path of the level-synchronous forward is exercised without any
fault: the tuning knob wait_polls = -1 makes every warp give up on its staged
batch program at once (no poll), as a wait that ran out would.  The warp then
waits (with the full limit) for its bulk copies to land, NaNs the batch's
outputs and sets the plan's NEAT_DEV_TIMEOUT bit, which neat_plan_device_errors
and neat_plan_check report."""
import ctypes

import numpy as np
import pytest
import torch

import oracle
from parity_util import compare_grads, compare_outputs
from workloads import locomotion_inputs, population_for, regression_batch

pytestmark = pytest.mark.gpu


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def test_level_wait_timeout_is_reported_and_outputs_are_nan():
    from paper_2504_08339_b300 import NeatError, _lib
    from paper_2504_08339_b300.api import Plan
    P = 700
    nodes, conns, spec = population_for("locomotion", seed=5, P=P)
    x = locomotion_inputs(5, 0, P, spec.I)
    plan = Plan(P, spec.N, spec.C, spec.I, spec.O)
    plan.transform(_dev(nodes), _dev(conns))
    assert plan.device_errors() == 0
    plan.set_tuning(wait_polls=-1)  # every staging wait gives up at once
    out = plan.forward(_dev(x))
    torch.cuda.synchronize()
    assert torch.isnan(out).all()  # every batch was given up on: no stale output
    assert plan.device_errors(clear=False) == _lib.DEV_TIMEOUT
    with pytest.raises(NeatError, match="-6"):
        plan.check()  # NEAT_ERR_TIMEOUT, and the word is cleared
    assert plan.device_errors() == 0
    # through the C ABI: the status code itself, then the copy into a device word
    plan.forward(_dev(x))
    s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    word = torch.zeros((1,), dtype=torch.int32, device="cuda")
    assert plan._lib.neat_plan_device_errors(plan._h, ctypes.c_void_p(word.data_ptr()), 0, s) == 0
    torch.cuda.synchronize()
    assert int(word.item()) == _lib.DEV_TIMEOUT
    assert plan._lib.neat_plan_check(plan._h, s) == _lib.NEAT_ERR_TIMEOUT
    assert plan._lib.neat_plan_check(plan._h, s) == _lib.NEAT_OK
    # the default limit: the same plan evaluates correctly and reports nothing
    plan.set_tuning(wait_polls=0)
    out = plan.forward(_dev(x)).cpu().numpy()
    ref, bnd = oracle.forward(nodes, conns, x, spec.I, spec.O, with_bound=True)
    compare_outputs(out, ref, bnd)
    plan.check()
    assert plan.device_errors() == 0


def test_transform_clears_the_failure_word():
    from paper_2504_08339_b300.api import Plan
    P = 64
    nodes, conns, spec = population_for("tiny", seed=1, P=P)
    plan = Plan(P, spec.N, spec.C, spec.I, spec.O)
    plan.set_tuning(wait_polls=-1)
    plan.transform(_dev(nodes), _dev(conns))
    from workloads import xor_inputs
    plan.forward(_dev(xor_inputs()))
    torch.cuda.synchronize()
    assert plan.device_errors(clear=False) != 0
    plan.transform(_dev(nodes), _dev(conns))
    assert plan.device_errors() == 0


def test_autograd_backward_after_another_evaluate_on_the_same_plan():
    """Two evaluates on one plan (population A, then B), then the backward of
    A's loss: A's gradients, not gradients taken on B's programs."""
    from paper_2504_08339_b300.api import Plan, evaluate
    P, S = 48, 64
    na, ca, spec = population_for("differentiation", seed=3, P=P)
    nb, cb, _ = population_for("differentiation", seed=4, P=P)
    x, y = regression_batch(3, S)
    plan = Plan(P, spec.N, spec.C, spec.I, spec.O)
    for store in (True, False):
        tna = _dev(na).requires_grad_()
        tca = _dev(ca).requires_grad_()
        out_a = evaluate(plan, tna, tca, _dev(x), store=store)
        out_b = evaluate(plan, _dev(nb), _dev(cb), _dev(x), store=store)
        del out_b
        go = (2.0 / S) * (out_a.detach()[..., 0] - _dev(y)[None])
        loss = ((out_a[..., 0] - _dev(y)[None]) ** 2).mean(dim=1).sum()
        loss.backward()
        out_r = oracle.forward(na, ca, x, spec.I, spec.O)
        go_r = (2.0 / S) * (out_r[..., 0] - y[None].astype(np.float64))
        rw, rb, rr, _ = oracle.backward(na, ca, x, spec.I, spec.O, go_r[..., None],
                                        want_inputs=False)
        compare_grads(tca.grad[..., 2].cpu().numpy(), rw, "grad_weight")
        compare_grads(tna.grad[..., 1].cpu().numpy(), rb, "grad_bias")
        compare_grads(tna.grad[..., 2].cpu().numpy(), rr, "grad_response")
        del go

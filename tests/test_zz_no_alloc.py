"""neat_forward_noalloc: the entry point for callers that cannot allocate
device memory when they evaluate (an allocator-free real-time loop, a plugin
handed only its input and output buffers).  Its working memory is a fixed
device array inside the library; these checks call it through the C ABI and
compare it with the plan-based neat_forward.

This file is collected last on purpose: a run that stops at the first failure
has run every other test before it."""
import ctypes

import numpy as np
import pytest
import torch

from parity_util import compare_outputs
from workloads import population_for

pytestmark = pytest.mark.gpu


def _vp(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def _reference(nodes, conns, x, spec):
    from paper_2504_08339_b300.api import Plan
    plan = Plan(nodes.shape[0], spec.N, spec.C, spec.I, spec.O)
    plan.set_tuning(small_s_max=-1)  # the sample-parallel form, as the no-alloc call uses
    tr = plan.transform(nodes, conns)
    return plan.forward(x), tr.status


@pytest.mark.parametrize("name,P,S,shared", [("locomotion", 600, 1, False),
                                             ("differentiation", 256, 77, True),
                                             ("tiny", 100, 4, True)])
def test_noalloc_matches_plan_forward_twice(name, P, S, shared):
    from paper_2504_08339_b300 import _lib
    lib = _lib.load()
    nodes_np, conns_np, spec = population_for(name, seed=12, P=P)
    rng = np.random.default_rng(3)
    x_np = rng.standard_normal((1 if shared else P, S, spec.I)).astype(np.float32)
    nodes = torch.from_numpy(nodes_np).cuda()
    conns = torch.from_numpy(conns_np).cuda()
    x = torch.from_numpy(x_np).cuda()
    ref, ref_status = _reference(nodes, conns, x, spec)
    stride = 0 if shared else S * spec.I
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for call in range(2):  # two calls in a row share (and overwrite) the array
        out = torch.full((P, S, spec.O), float("nan"), device="cuda")
        status = torch.full((P,), -1, dtype=torch.int32, device="cuda")
        code = lib.neat_forward_noalloc(_vp(nodes), _vp(conns), P, spec.N, spec.C, spec.I, spec.O,
                                        _vp(x), stride, S, _vp(out), _vp(status), stream)
        assert code == 0, (call, code, lib.neat_last_cuda_error())
        torch.cuda.synchronize()
        assert torch.equal(status, ref_status)
        compare_outputs(out.cpu().numpy(), ref.cpu().numpy().astype(np.float64),
                        what=f"{name} call {call}")


def test_noalloc_rejects_populations_beyond_the_array():
    from paper_2504_08339_b300 import _lib
    lib = _lib.load()
    n = torch.zeros((1, 128, 5), device="cuda")
    c = torch.zeros((1, 512, 4), device="cuda")
    o = torch.zeros((1, 1, 8), device="cuda")
    s = torch.zeros((1,), dtype=torch.int32, device="cuda")
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    code = lib.neat_forward_noalloc(_vp(n), _vp(c), 1_000_000, 128, 512, 27, 8, _vp(o), 0, 1,
                                    _vp(o), _vp(s), stream)
    assert code == _lib.NEAT_ERR_WORKSPACE

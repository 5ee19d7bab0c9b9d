"""neat_forward_noalloc: the entry point for callers that cannot allocate
device memory when they evaluate (an allocator-free real-time loop, a plugin
handed only its input and output buffers).  Its working memory is a fixed
device array inside the library; these checks call it through the C ABI and
compare it with the FP64 oracle and with the plan-based neat_forward.

This file is collected last on purpose: a run that stops at the first failure
has run every other test before it."""
import ctypes

import numpy as np
import pytest
import torch

import oracle
from parity_util import compare_outputs
from workloads import population_for

pytestmark = pytest.mark.gpu

SCRATCH = 32 << 20  # NEAT_NOALLOC_SCRATCH_BYTES


def _vp(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def _reference(nodes, conns, x, spec):
    from paper_2504_08339_b300.api import Plan
    plan = Plan(nodes.shape[0], spec.N, spec.C, spec.I, spec.O)
    plan.set_tuning(small_s_max=-1)  # the sample-parallel form, as the no-alloc call uses
    tr = plan.transform(nodes, conns)
    return plan.forward(x), tr.status


def _call(lib, nodes, conns, P, spec, x, stride, S, out, status):
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return lib.neat_forward_noalloc(_vp(nodes), _vp(conns), P, spec.N, spec.C, spec.I, spec.O,
                                    _vp(x), stride, S, _vp(out), _vp(status), stream)


@pytest.mark.parametrize("name,P,S,shared", [("locomotion", 600, 1, False),
                                             ("differentiation", 256, 77, True),
                                             ("tiny", 100, 4, True),
                                             ("uneven", 24, 64, False)])
def test_noalloc_matches_oracle_and_plan_forward_twice(name, P, S, shared):
    from paper_2504_08339_b300 import _lib
    lib = _lib.load()
    nodes_np, conns_np, spec = population_for(name, seed=12, P=P)
    rng = np.random.default_rng(3)
    x_np = rng.standard_normal((1 if shared else P, S, spec.I)).astype(np.float32)
    nodes = torch.from_numpy(nodes_np).cuda()
    conns = torch.from_numpy(conns_np).cuda()
    x = torch.from_numpy(x_np).cuda()
    ref, bnd = oracle.forward(nodes_np, conns_np, x_np, spec.I, spec.O, with_bound=True)
    plan_out, ref_status = _reference(nodes, conns, x, spec)
    stride = 0 if shared else S * spec.I
    for call in range(2):  # two calls in a row share (and overwrite) the array
        out = torch.full((P, S, spec.O), float("nan"), device="cuda")
        status = torch.full((P,), -1, dtype=torch.int32, device="cuda")
        code = _call(lib, nodes, conns, P, spec, x, stride, S, out, status)
        assert code == 0, (call, code, lib.neat_last_cuda_error())
        torch.cuda.synchronize()
        assert torch.equal(status, ref_status)
        compare_outputs(out.cpu().numpy(), ref, bnd, what=f"{name} call {call} vs oracle")
        compare_outputs(out.cpu().numpy(), plan_out.cpu().numpy().astype(np.float64),
                        what=f"{name} call {call} vs neat_forward")


def _needed(P, N, C, I, O):
    """Bytes of the array a call uses, as include/neat.h states them: 16
    regions, each rounded up to 256 bytes."""
    a = lambda x: (x + 255) // 256 * 256  # noqa: E731
    regions = [48 * P, 16 * P * N, 8 * P * C, 4 * P * C, 4 * P * N, 4 * P * N, 4 * P * (I + O),
               4 * (P + 1), 4 * (P + 1), 16 * P * N, 8 * P * C, 4 * P * C, 256,
               4 * P * N, 4 * P * N, 4 * P]
    return sum(a(r) for r in regions)


def test_noalloc_capacity_boundary():
    """The largest locomotion-shaped population that fits (1,800 genomes)
    runs and matches the oracle; one more genome is refused before any launch."""
    from paper_2504_08339_b300 import _lib
    lib = _lib.load()
    nodes_np, conns_np, spec = population_for("locomotion", seed=13, P=1801)
    pmax = max(p for p in range(1700, 1900) if _needed(p, spec.N, spec.C, spec.I, spec.O) <= SCRATCH)
    assert pmax == 1800
    assert _needed(pmax, spec.N, spec.C, spec.I, spec.O) <= (
        pmax * (48 * spec.N + 24 * spec.C + 4 * (spec.I + spec.O) + 60) + 4352)
    nodes = torch.from_numpy(nodes_np).cuda()
    conns = torch.from_numpy(conns_np).cuda()
    x_np = np.random.default_rng(4).standard_normal((1801, 1, spec.I)).astype(np.float32)
    x = torch.from_numpy(x_np).cuda()
    out = torch.full((1801, 1, spec.O), 7.0, device="cuda")
    status = torch.full((1801,), -1, dtype=torch.int32, device="cuda")
    assert _call(lib, nodes, conns, 1801, spec, x, spec.I, 1, out, status) == _lib.NEAT_ERR_WORKSPACE
    torch.cuda.synchronize()
    assert (out == 7.0).all() and (status == -1).all()  # nothing was launched
    assert _call(lib, nodes, conns, 1800, spec, x, spec.I, 1, out, status) == 0
    torch.cuda.synchronize()
    ref, bnd = oracle.forward(nodes_np[:1800], conns_np[:1800], x_np[:1800], spec.I, spec.O,
                              with_bound=True)
    compare_outputs(out[:1800].cpu().numpy(), ref, bnd, what="1800 genomes")
    assert (out[1800] == 7.0).all()


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

"""neat_sum_genomes: the gradient of an input set that every genome shares is
the sum over genomes of their per-genome input gradients (chain rule through
the one tensor all of them read).  Checked against the exactly rounded sum
(math.fsum), for determinism, for P = 0 and for its argument errors."""
import ctypes
import math

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


def _vp(t):
    return ctypes.c_void_p(t.data_ptr())


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


@pytest.mark.parametrize("P,n", [(1, 5), (7, 33), (2048, 8192), (13, 100_003)])
def test_sum_genomes_against_exact_sum(P, n):
    from paper_2504_08339_b300 import _lib
    lib = _lib.load()
    rng = np.random.default_rng(P + n)
    # mixed magnitudes and signs, so that the summation order matters in f32
    x = (rng.standard_normal((P, n)) * 10.0 ** rng.integers(-3, 4, (P, n))).astype(np.float32)
    xd = torch.from_numpy(x).cuda()
    out = torch.full((n,), float("nan"), device="cuda")
    assert lib.neat_sum_genomes(_vp(xd), P, n, _vp(out), _stream()) == 0
    again = torch.full((n,), float("nan"), device="cuda")
    assert lib.neat_sum_genomes(_vp(xd), P, n, _vp(again), _stream()) == 0
    got = out.cpu().numpy().astype(np.float64)
    assert torch.equal(out, again)  # deterministic
    cols = range(n) if n <= 8192 else np.random.default_rng(1).choice(n, 4096, replace=False)
    for j in cols:
        exact = math.fsum(x[:, j].astype(np.float64).tolist())
        # double accumulation of P terms, one rounding to f32: within one
        # f32 unit of the exact sum (plus the double error, far below it)
        ulp = np.spacing(np.float32(abs(exact))).astype(np.float64)
        assert abs(got[j] - exact) <= ulp + P * 2.0 ** -52 * np.abs(x[:, j]).sum(), (j, got[j], exact)


def test_sum_genomes_empty_and_errors():
    from paper_2504_08339_b300 import _lib
    lib = _lib.load()
    out = torch.full((10,), 3.0, device="cuda")
    x = torch.ones((4, 10), device="cuda")
    assert lib.neat_sum_genomes(None, 0, 10, _vp(out), _stream()) == 0
    torch.cuda.synchronize()
    assert (out == 0).all()
    assert lib.neat_sum_genomes(_vp(x), 4, 10, _vp(out), _stream()) == 0
    torch.cuda.synchronize()
    assert (out == 4).all()
    # overlapping ranges, negative sizes, null pointers: refused, nothing written
    out.fill_(3.0)
    assert lib.neat_sum_genomes(_vp(x), 4, 10, _vp(x[2]), _stream()) == _lib.NEAT_ERR_ARG
    assert lib.neat_sum_genomes(_vp(x), -1, 10, _vp(out), _stream()) == _lib.NEAT_ERR_ARG
    assert lib.neat_sum_genomes(_vp(x), 4, -1, _vp(out), _stream()) == _lib.NEAT_ERR_ARG
    assert lib.neat_sum_genomes(_vp(x), 4, 10, None, _stream()) == _lib.NEAT_ERR_ARG
    torch.cuda.synchronize()
    assert (out == 3.0).all() and (x == 1).all()

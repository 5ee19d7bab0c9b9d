"""Accuracy of the activation functions the kernels evaluate, through the C
ABI: the level-synchronous kernel's own exp / reciprocal / tanh series / sine
(act_math.cuh) and the CUDA math library of the one-activation-per-warp
kernels.

Each genome is one input connected to the single output node (weight 1,
bias 0, response 1, sum aggregation), so its output is act(x) for the input
x.  The inputs sweep every activation over small, moderate, large and
special arguments; the result must be within the error the oracle's fp32
bound allows an activation: 8 * 2^-24 relative for sigmoid, tanh and sin,
(8 + x^2) * 2 * 2^-24 for gaussian (the rounding of x^2 included), exact for
identity, relu and abs; for sin beyond |x| = 1 the absolute error may also be
that of the argument's own rounding (|x| 2^-24).  The level-synchronous form
evaluates several nodes of different activations in one warp with branch-free
functions of its own; the sample-parallel form (one node per warp step)
calls the CUDA math library; both are checked."""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

U = 2.0 ** -24
ACTS = ["identity", "sigmoid", "tanh", "relu", "sin", "gaussian", "abs"]


def _genomes():
    """7 genomes, genome a: input row 0 -> output row 1 with activation a."""
    P, N, C = len(ACTS), 2, 1
    nodes = np.full((P, N, 5), np.nan, np.float32)
    conns = np.full((P, C, 4), np.nan, np.float32)
    for a in range(P):
        nodes[a, 0] = (0, 0, 1, 0, 0)
        nodes[a, 1] = (1, 0, 1, a, 0)
        conns[a, 0] = (0, 1, 1.0, 1)
    return nodes, conns


def _arguments():
    rng = np.random.default_rng(0)
    mag = np.concatenate([np.linspace(0, 12, 4001), np.geomspace(1e-8, 1e5, 4000),
                          rng.uniform(0, 100, 4000), [0.55, np.nextafter(0.55, 0), 0.5499],
                          np.pi / 2 * np.arange(1, 200), [88.7, 88.8, 87.0, 86.9, 104.0]])
    x = np.concatenate([mag, -mag]).astype(np.float32)
    return x


def _reference(a, x):
    z = x.astype(np.float64)
    return {"identity": z, "sigmoid": 1.0 / (1.0 + np.exp(-z)), "tanh": np.tanh(z),
            "relu": np.maximum(z, 0.0), "sin": np.sin(z), "gaussian": np.exp(-z * z),
            "abs": np.abs(z)}[ACTS[a]]


@pytest.mark.parametrize("path", ["sample", "level"])
def test_activation_accuracy(path):
    """Every argument through the sample-parallel form (one launch) or the
    level-synchronous form (launches of 64 samples: tiles of 4 per lane)."""
    from paper_2504_08339_b300.api import Plan
    nodes, conns = _genomes()
    x = _arguments()
    P, S = nodes.shape[0], x.size
    plan = Plan(P, 2, 1, 1, 1)
    plan.set_tuning(small_s_max=-1 if path == "sample" else 64)
    plan.transform(torch.from_numpy(nodes).cuda(), torch.from_numpy(conns).cuda())
    xd = torch.from_numpy(x).cuda()
    if path == "sample":
        out = plan.forward(xd.reshape(1, S, 1)).cpu().numpy()[:, :, 0]
    else:
        out = torch.cat([plan.forward(xd[i:i + 64].reshape(1, -1, 1))
                         for i in range(0, S, 64)], dim=1).cpu().numpy()[:, :, 0]
    for a in range(P):
        g, r = out[a].astype(np.float64), _reference(a, x)
        if ACTS[a] in ("identity", "relu", "abs"):
            assert np.array_equal(g, r.astype(np.float32).astype(np.float64)), ACTS[a]
            continue
        if ACTS[a] == "gaussian":
            lim = (8.0 + x.astype(np.float64) ** 2) * 2.0 * U * np.abs(r)
        else:
            lim = 8.0 * U * np.abs(r)
        if ACTS[a] == "sin":
            lim = np.maximum(lim, 2.0 * U * np.abs(x.astype(np.float64)))
        lim = np.maximum(lim, 1e-37)  # results below 2^-125 flush to zero
        err = np.abs(g - r)
        bad = err > lim
        assert not bad.any(), (ACTS[a], x[bad][:5], g[bad][:5], r[bad][:5])

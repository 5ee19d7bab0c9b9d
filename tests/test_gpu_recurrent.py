"""GPU parity of the recurrent ("concurrent") calculation, T synchronous
iterations, against the FP64 oracle on the same seeded inputs."""
import numpy as np
import pytest
import torch

import oracle
from parity_util import compare_outputs
from workloads import population_for

pytestmark = pytest.mark.gpu


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _plan(spec, P):
    from paper_2504_08339_b300.api import Plan
    return Plan(P, spec.N, spec.C, spec.I, spec.O)


@pytest.mark.parametrize("T", [0, 1, 3, 8])
@pytest.mark.parametrize("shared", [False, True])
def test_recurrent_parity(T, shared):
    """Cyclic genomes (back edges and self-loops), S = 45 (a ragged tile)."""
    P, S = 300, 45
    nodes, conns, spec = population_for("recurrent", seed=5, P=P)
    x = np.random.default_rng(7).standard_normal((1 if shared else P, S, spec.I)).astype(
        np.float32)
    plan = _plan(spec, P)
    status = plan.transform_recurrent(_dev(nodes), _dev(conns))
    out = plan.forward_recurrent(_dev(x), T).cpu().numpy()
    ref, bnd, st = oracle.forward_recurrent(nodes, conns, x, spec.I, spec.O, T, with_bound=True,
                                            with_status=True)
    np.testing.assert_array_equal(status.cpu().numpy().view(np.uint32), st)
    assert (st == 0).all()
    compare_outputs(out, ref, bnd, what=f"T={T}")


@pytest.mark.parametrize("spl", [1, 2])
def test_recurrent_samples_per_lane(spl):
    """One or two samples per lane (the tuning's samples_per_lane): the same
    outputs, against the oracle; S = 77 leaves a ragged last tile for both."""
    P, S, T = 200, 77, 5
    nodes, conns, spec = population_for("recurrent", seed=9, P=P)
    x = np.random.default_rng(3).standard_normal((P, S, spec.I)).astype(np.float32)
    plan = _plan(spec, P)
    plan.set_tuning(samples_per_lane=spl)
    plan.transform_recurrent(_dev(nodes), _dev(conns))
    out = plan.forward_recurrent(_dev(x), T).cpu().numpy()
    plan.check()
    ref, bnd = oracle.forward_recurrent(nodes, conns, x, spec.I, spec.O, T, with_bound=True)
    compare_outputs(out, ref, bnd, what=f"spl={spl}")


def test_recurrent_status_bits_match_the_oracle():
    nodes, conns, spec = population_for("recurrent", seed=6, P=8)
    live = np.flatnonzero(~np.isnan(conns[0, :, 0]) & (conns[0, :, 3] != 0))
    conns[0, live[0], 1] = 7777.0                           # dangling key
    conns[1, live[0], 1] = 0.0                              # edge into an input
    nodes[2, spec.I + spec.O - 1, 0] = nodes[2, 0, 0]       # duplicate key
    nodes[3, spec.I, 3] = 11.0                              # activation id
    src = conns[4, live[0], 0]                              # duplicate enabled edge
    conns[4, live[1], 0], conns[4, live[1], 1] = src, conns[4, live[0], 1]
    x = np.random.default_rng(1).standard_normal((8, 4, spec.I)).astype(np.float32)
    plan = _plan(spec, 8)
    status = plan.transform_recurrent(_dev(nodes), _dev(conns)).cpu().numpy().view(np.uint32)
    out = plan.forward_recurrent(_dev(x), 4).cpu().numpy()
    ref, st = oracle.forward_recurrent(nodes, conns, x, spec.I, spec.O, 4, with_status=True)
    np.testing.assert_array_equal(status, st)
    assert (st[:5] != 0).all() and (st[5:] == 0).all()
    compare_outputs(out, ref)


def test_acyclic_population_reaches_the_feedforward_outputs():
    """On DAGs, T = depth gives the feed-forward values; also valid after the
    feed-forward transform, where the feed-forward calls stay available."""
    P, S = 200, 3
    nodes, conns, spec = population_for("locomotion", seed=9, P=P)
    x = np.random.default_rng(3).standard_normal((P, S, spec.I)).astype(np.float32)
    ref, bnd = oracle.forward(nodes, conns, x, spec.I, spec.O, with_bound=True)
    _, _, n_layers, _ = oracle.transform(nodes, conns, spec.I, spec.O)
    T = int(n_layers.max())
    plan = _plan(spec, P)
    plan.transform_recurrent(_dev(nodes), _dev(conns))
    compare_outputs(plan.forward_recurrent(_dev(x), T).cpu().numpy(), ref, bnd)
    plan.transform(_dev(nodes), _dev(conns))
    compare_outputs(plan.forward_recurrent(_dev(x), T).cpu().numpy(), ref, bnd)
    compare_outputs(plan.forward(_dev(x)).cpu().numpy(), ref, bnd)


def test_network_type_state_and_arguments():
    from paper_2504_08339_b300 import NeatError
    nodes, conns, spec = population_for("recurrent", seed=2, P=16)
    plan = _plan(spec, 16)
    x = _dev(np.zeros((16, 2, spec.I), np.float32))
    with pytest.raises(NeatError):
        plan.forward_recurrent(x, 2)          # nothing transformed yet
    plan.transform_recurrent(_dev(nodes), _dev(conns))
    with pytest.raises(NeatError):
        plan.forward(x)                       # feed-forward calls need neat_transform
    with pytest.raises(NeatError):
        plan.forward_recurrent(x, -1)
    assert plan.forward_recurrent(x, 2).shape == (16, 2, spec.O)


def test_recurrent_full_population_sampled():
    """The full 10,000-genome recurrent workload in the benchmark's launch shape
    (S = 64, T = 8); a sample of genomes vs the oracle."""
    nodes, conns, spec = population_for("recurrent", seed=0)
    P, S, T = nodes.shape[0], 64, 8
    x = np.random.default_rng(0).standard_normal((P, S, spec.I)).astype(np.float32)
    plan = _plan(spec, P)
    plan.transform_recurrent(_dev(nodes), _dev(conns))
    out = plan.forward_recurrent(_dev(x), T).cpu().numpy()
    sel = np.random.default_rng(1).choice(P, 150, replace=False)
    ref, bnd = oracle.forward_recurrent(nodes[sel], conns[sel], x[sel], spec.I, spec.O, T,
                                        with_bound=True)
    compare_outputs(out[sel], ref, bnd)

"""neat_plan_validate: the structure check of a transformed population.

Every structure the transform writes (queues, headers, packed position
programs, input / output positions, compiled programs, level batch programs)
must hold only in-range indices after any transform: every workload, with and
without pruning, malformed genomes, the library's maximum sizes and the
recurrent transform.  A workspace overwritten with garbage must be reported,
and the check itself reads only inside the workspace (no fault whatever the
bytes)."""
import numpy as np
import pytest
import torch

from paper_2504_08339_b300 import NeatError, _lib
from paper_2504_08339_b300.api import Plan
from workloads import GenomeSpec, make_population, population_for

pytestmark = pytest.mark.gpu


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("prune", [0, 1])
@pytest.mark.parametrize("name,P", [("tiny", 100), ("locomotion", 2000), ("uneven", 400),
                                    ("differentiation", 512), ("hyperneat", 128)])
def test_every_workload_validates(name, P, prune):
    nodes, conns, spec = population_for(name, seed=3, P=P)
    plan = Plan(P, spec.N, spec.C, spec.I, spec.O)
    with pytest.raises(NeatError):
        plan.validate()  # no transform yet
    plan.set_tuning(prune_dead=prune)
    plan.transform(_dev(nodes), _dev(conns))
    assert plan.validate() == 0
    # a fixed batch budget (the cut without the budget search) as well
    plan.set_tuning(prune_dead=prune, lvl_budget_kb=8)
    plan.transform(_dev(nodes), _dev(conns))
    assert plan.validate() == 0


def test_malformed_and_maximum_sized_genomes_validate():
    # rejected genomes among valid ones: cycles, dangling keys, bad ids
    nodes, conns, spec = population_for("locomotion", seed=9, P=64)
    nodes, conns = nodes.copy(), conns.copy()
    rng = np.random.default_rng(0)
    for g in range(0, 64, 4):
        r = int(rng.integers(0, spec.C))
        conns[g, r] = (float(spec.I), float(spec.I), 0.5, 1.0)  # a self-loop on an output
    nodes[1, spec.I, 3] = 99.0                                   # activation id out of range
    conns[2, :, 0] = np.where(np.isnan(conns[2, :, 0]), np.nan, 12345.0)  # dangling keys
    plan = Plan(64, spec.N, spec.C, spec.I, spec.O)
    tr = plan.transform(_dev(nodes), _dev(conns))
    assert (tr.status.cpu().numpy() != 0).sum() >= 3
    assert plan.validate() == 0
    # the library maxima
    big = GenomeSpec(I=9, O=3, N=1024, C=8192, V_loguniform=(700, 1024),
                     E_loguniform=(6000, 8192), acts=("tanh", "sigmoid", "sin"),
                     aggs=("sum", "mean", "max"), w_std=1.0, b_std=0.5)
    n2, c2 = make_population(big, 5, seed=2)
    plan2 = Plan(5, 1024, 8192, 9, 3)
    plan2.transform(_dev(n2), _dev(c2))
    assert plan2.validate() == 0


def test_recurrent_transform_validates():
    nodes, conns, spec = population_for("recurrent", seed=1, P=300)
    plan = Plan(300, spec.N, spec.C, spec.I, spec.O)
    plan.transform_recurrent(_dev(nodes), _dev(conns))
    assert plan.validate() == 0


@pytest.mark.parametrize("fill", ["ones", "zeros", "random"])
def test_garbage_workspace_is_reported(fill):
    """After a transform the whole workspace is overwritten: the check reports
    it (the plan itself is not used again) and the device stays usable."""
    nodes, conns, spec = population_for("locomotion", seed=5, P=500)
    plan = Plan(500, spec.N, spec.C, spec.I, spec.O)
    plan.transform(_dev(nodes), _dev(conns))
    assert plan.validate() == 0
    ws = plan.workspace
    if fill == "ones":
        ws.fill_(0xFF)
    elif fill == "zeros":
        ws.zero_()
    else:
        g = torch.Generator(device="cuda").manual_seed(7)
        ws.copy_(torch.randint(0, 256, ws.shape, generator=g, device="cuda", dtype=torch.int32)
                 .to(torch.uint8))
    bits = plan.validate()
    assert bits != 0
    assert bits & ~(_lib.BAD_QUEUE | _lib.BAD_PACKED | _lib.BAD_COMPILED | _lib.BAD_BATCHES) == 0
    # every genome header and the batch count are garbage
    assert bits & _lib.BAD_PACKED
    assert bits & _lib.BAD_BATCHES
    # a new plan on the same device evaluates normally
    fresh = Plan(500, spec.N, spec.C, spec.I, spec.O)
    fresh.transform(_dev(nodes), _dev(conns))
    assert fresh.validate() == 0
    x = np.random.default_rng(1).standard_normal((500, 1, spec.I)).astype(np.float32)
    assert torch.isfinite(fresh.forward(_dev(x))).all()

"""GPU parity: the CUDA path through the C ABI against the FP64 oracle on the
same seeded inputs.  Orders, layers and status bits must be bit-exact; outputs
and gradients within the tolerances of parity_util."""
import numpy as np
import pytest
import torch

import oracle
from genome_builders import load_xor, stack
from parity_util import compare_grads, compare_outputs
from workloads import (CONFIGS, locomotion_inputs, population_for, regression_batch,
                       uneven_inputs, xor_inputs)

pytestmark = pytest.mark.gpu


def _plan(spec, P):
    from paper_2504_08339_b300.api import Plan
    return Plan(P, spec.N, spec.C, spec.I, spec.O)


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _transform_both(nodes, conns, spec):
    P = nodes.shape[0]
    plan = _plan(spec, P)
    tr = plan.transform(_dev(nodes), _dev(conns))
    torch.cuda.synchronize()
    ref = oracle.transform(nodes, conns, spec.I, spec.O)
    return plan, tr, ref


def _assert_transform_equal(tr, ref):
    o, l, nl, st = ref
    np.testing.assert_array_equal(tr.order.cpu().numpy(), o)
    np.testing.assert_array_equal(tr.layer.cpu().numpy(), l)
    np.testing.assert_array_equal(tr.n_layers.cpu().numpy(), nl)
    np.testing.assert_array_equal(tr.status.cpu().numpy().astype(np.uint32), st)


SIZES = {"tiny": 100, "locomotion": 3000, "uneven": 600, "differentiation": 2048, "hyperneat": 256}


@pytest.mark.parametrize("name", list(SIZES))
def test_transform_bit_exact(name):
    nodes, conns, spec = population_for(name, seed=1, P=SIZES[name])
    plan, tr, ref = _transform_both(nodes, conns, spec)
    _assert_transform_equal(tr, ref)
    assert (ref[3] == 0).all()


def _malformed_population():
    d, n, c = load_xor()
    variants = []

    def v(f):
        nn, cc = n.copy(), c.copy()
        f(nn, cc)
        variants.append((nn, cc))

    v(lambda n, c: None)
    v(lambda n, c: c.__setitem__(3, (3, 7, 1.0, 1)))            # cycle
    v(lambda n, c: c.__setitem__(3, (7, 7, 1.0, 1)))            # self loop
    v(lambda n, c: c.__setitem__(3, (99, 3, 1.0, 1)))           # dangling
    v(lambda n, c: c.__setitem__(3, (0.5, 3, 1.0, 1)))          # non-integral conn key
    v(lambda n, c: n.__setitem__(6, (5, 0, 1, 1, 0)))           # duplicate key
    v(lambda n, c: c.__setitem__(3, (0, 7, 2.0, 1)))            # duplicate edge
    v(lambda n, c: c.__setitem__(3, (7, 0, 1.0, 1)))            # edge into input
    v(lambda n, c: n.__setitem__((4, 3), 9))                    # act id
    v(lambda n, c: n.__setitem__((4, 4), 1.5))                  # agg id
    v(lambda n, c: n.__setitem__((4, 1), np.nan))               # NaN bias
    v(lambda n, c: c.__setitem__((0, 2), np.nan))               # NaN weight enabled
    v(lambda n, c: c.__setitem__((10, 2), np.nan))              # NaN weight disabled: fine
    v(lambda n, c: n.__setitem__(6, (2.0 ** 24, 0, 1, 1, 0)))   # key range
    v(lambda n, c: n.__setitem__(6, (-3, 0, 1, 1, 0)))
    v(lambda n, c: n.__setitem__((3, 0), np.nan))               # output row padding
    v(lambda n, c: n.__setitem__((0, 3), 99))                   # input attrs ignored
    v(lambda n, c: c.__setitem__(3, (np.nan, 3, 5.0, 1)))       # half-NaN row = padding
    v(lambda n, c: c.__setitem__((10, 3), np.nan))              # NaN enabled = disabled
    return stack(variants), d


def test_transform_and_forward_malformed_genomes():
    (nodes, conns), d = _malformed_population()
    spec = CONFIGS["tiny"]["spec"]
    from paper_2504_08339_b300.api import Plan
    P = nodes.shape[0]
    plan = Plan(P, nodes.shape[1], conns.shape[1], 3, 1)
    tr = plan.transform(_dev(nodes), _dev(conns))
    ref = oracle.transform(nodes, conns, 3, 1)
    _assert_transform_equal(tr, ref)
    assert (ref[3] != 0).sum() >= 12
    x = xor_inputs()
    out = plan.forward(_dev(x)).cpu().numpy()
    r = oracle.forward(nodes, conns, x, 3, 1)
    compare_outputs(out, r)
    plain = plan.forward(_dev(x), plain=True).cpu().numpy()
    compare_outputs(plain, r)
    del spec


def _fwd_case(name, P, S, seed=2):
    nodes, conns, spec = population_for(name, seed=seed, P=P)
    rng = np.random.default_rng(seed)
    if name == "tiny":
        x = xor_inputs()
    elif name == "differentiation":
        x = regression_batch(seed, S)[0]
    else:
        x = rng.standard_normal((P, S, spec.I), dtype=np.float32)
    return nodes, conns, spec, x


@pytest.mark.parametrize("name,P,S", [
    ("tiny", 100, 4),
    ("locomotion", 1000, 1),
    ("locomotion", 400, 37),
    ("uneven", 300, 64),
    ("differentiation", 256, 100),
    ("hyperneat", 128, 33),
])
@pytest.mark.parametrize("path", ["auto", "level", "sample", "plain"])
def test_forward_parity(name, P, S, path):
    nodes, conns, spec, x = _fwd_case(name, P, S)
    plan = _plan(spec, P)
    if path == "level":
        plan.set_tuning(small_s_max=64)
    elif path == "sample":
        plan.set_tuning(small_s_max=-1)
    plan.transform(_dev(nodes), _dev(conns))
    out = plan.forward(_dev(x), plain=path == "plain").cpu().numpy()
    ref, bnd = oracle.forward(nodes, conns, x, spec.I, spec.O, with_bound=True)
    stats = compare_outputs(out, ref, bnd)
    if name in ("tiny", "differentiation"):
        # well-conditioned populations: inside the plain tolerance everywhere
        assert stats["ill_conditioned"] == 0, stats


def _live_cost(n, c, I, O):
    """Enabled connections into, plus twice the count of, the non-input nodes
    some output depends on (reverse reachability from the output rows)."""
    row = {float(k): r for r, k in enumerate(n[:, 0]) if not np.isnan(k)}
    en = ~np.isnan(c[:, 0]) & ~np.isnan(c[:, 1]) & ~np.isnan(c[:, 3]) & (c[:, 3] != 0)
    preds = {}
    for a, b in c[en, :2]:
        preds.setdefault(row[float(b)], []).append(row[float(a)])
    live, stack = set(range(I, I + O)), list(range(I, I + O))
    while stack:
        for a in preds.get(stack.pop(), ()):
            if a not in live:
                live.add(a)
                stack.append(a)
    return sum(len(preds.get(r, ())) + 2 for r in live if r >= I)


@pytest.mark.parametrize("prune", [0, 1])
@pytest.mark.parametrize("name,P,S", [("uneven", 300, 77), ("locomotion", 200, 45),
                                      ("differentiation", 128, 100)])
def test_sample_parallel_shapes_agree_bitwise(name, P, S, prune):
    """Samples per lane and warps per CTA change which lane and which value
    slot evaluate a sample, not the arithmetic: every shape gives the same
    bits, and the saved aggregates too; the outputs-only calls (compiled
    programs, with or without the nodes no output depends on) give the bits
    of the position walk.  S = 77, 45, 100 leave a ragged last tile for 1, 2
    and 4 samples per lane."""
    nodes, conns, spec, x = _fwd_case(name, P, S)
    if name == "uneven":
        # genomes of cost E + 2V >= 2048 (>= 512 for the part the outputs
        # depend on, with pruning) are evaluated by whole CTAs (layer by
        # layer); the others by single warps: both run here
        if prune:
            cost = np.array([_live_cost(nodes[g], conns[g], spec.I, spec.O) for g in range(P)])
        else:
            en = (~np.isnan(conns[:, :, 0]) & ~np.isnan(conns[:, :, 1]) &
                  ~np.isnan(conns[:, :, 3]) & (conns[:, :, 3] != 0))
            cost = en.sum(1) + 2 * ((~np.isnan(nodes[:, :, 0])).sum(1) - spec.I)
        big = 512 if prune else 2048
        assert (cost >= big).sum() >= 10 and (cost < big).sum() >= 10
    plan = _plan(spec, P)
    plan.set_tuning(small_s_max=-1, prune_dead=prune)
    plan.transform(_dev(nodes), _dev(conns))
    dx = _dev(x)
    base_saved = torch.full((P, spec.N, S), float("nan"), device="cuda")
    base = plan.forward(dx, saved=base_saved)
    ref, bnd = oracle.forward(nodes, conns, x, spec.I, spec.O, with_bound=True)
    compare_outputs(base.cpu().numpy(), ref, bnd)
    shapes = [dict(samples_per_lane=2), dict(samples_per_lane=4),
              dict(samples_per_lane=1, warps_per_cta=1),
              dict(samples_per_lane=2, warps_per_cta=4),
              dict(samples_per_lane=4, warps_per_cta=16),
              dict(samples_per_lane=1, warps_per_cta=16)]
    for sh in shapes:
        plan.set_tuning(small_s_max=-1, prune_dead=prune, **sh)
        saved = torch.full((P, spec.N, S), float("nan"), device="cuda")
        out = plan.forward(dx, saved=saved)
        bits = lambda t: t.view(torch.int32)  # noqa: E731  (NaN-safe equality)
        assert torch.equal(bits(out), bits(base)), sh
        # (positions the forward does not write stay NaN on both sides)
        assert torch.equal(bits(saved), bits(base_saved)), sh
        assert torch.equal(bits(plan.forward(dx)), bits(base)), sh


@pytest.mark.parametrize("name,P,S", [("locomotion", 500, 1), ("uneven", 200, 64),
                                      ("differentiation", 64, 100), ("tiny", 100, 4)])
def test_pruning_changes_no_result(name, P, S):
    """Skipping the nodes no output depends on (prune_dead = 1) gives the
    bits of evaluating every node: the level-synchronous, compiled
    sample-parallel and HyperNEAT paths, and the gradients' values (the
    skipped nodes' gradients are 0 either way)."""
    nodes, conns, spec, x = _fwd_case(name, P, S)
    dn, dc, dx = _dev(nodes), _dev(conns), _dev(x)
    res = []
    for prune in (0, 1):
        plan = _plan(spec, P)
        plan.set_tuning(prune_dead=prune)
        plan.transform(dn, dc)
        out = plan.forward(dx)
        plan.set_tuning(prune_dead=prune, small_s_max=-1)
        out_sp = plan.forward(dx)
        go = torch.ones((P, S, spec.O), device="cuda")
        # (uneven genomes, N = 1024 and C = 4096, take the backward whose
        # per-warp arrays sit in workspace slots)
        grads = plan.backward(dx, go)
        res.append((out, out_sp, grads))
    bits = lambda t: t.view(torch.int32)  # noqa: E731
    assert torch.equal(bits(res[0][0]), bits(res[1][0]))
    assert torch.equal(bits(res[0][1]), bits(res[1][1]))
    for a, b in zip(res[0][2], res[1][2]):
        assert torch.equal(a, b)
    ref, bnd = oracle.forward(nodes, conns, x, spec.I, spec.O, with_bound=True)
    compare_outputs(res[1][0].cpu().numpy(), ref, bnd)


def test_pruning_changes_no_hyperneat_weight():
    nodes, conns, spec = population_for("hyperneat", seed=6, P=24)
    outs = []
    for prune in (0, 1):
        plan = _plan(spec, 24)
        plan.set_tuning(prune_dead=prune)
        plan.transform(_dev(nodes), _dev(conns))
        outs.append(plan.hyperneat(grid=9, thresh=0.2).view(torch.int32).clone())
    assert torch.equal(outs[0], outs[1])


def test_forward_saved_aggregates_match_oracle_values():
    nodes, conns, spec, x = _fwd_case("differentiation", 64, 45)
    plan = _plan(spec, 64)
    tr = plan.transform(_dev(nodes), _dev(conns))
    saved = torch.empty((64, spec.N, 45), device="cuda")
    out = plan.forward(_dev(x), saved=saved)
    out2 = plan.forward(_dev(x))
    assert torch.equal(out, out2)
    # the saved aggregate a at position p gives v = act(b + r a); check it on outputs
    order = tr.order.cpu().numpy()
    _, vals = oracle.forward(nodes, conns, x, spec.I, spec.O, with_values=True)
    sv = saved.cpu().numpy()
    for g in range(64):
        pos_out = int(np.flatnonzero(order[g] == spec.I)[0])      # output row I
        a = sv[g, pos_out, :].astype(np.float64)
        b, r = float(nodes[g, spec.I, 1]), float(nodes[g, spec.I, 2])
        np.testing.assert_allclose(b + r * a, vals[g, :, spec.I], rtol=1e-4, atol=1e-5)


def test_locomotion_full_population_sampled_steps():
    """The full 10,000-genome locomotion population, in the launch shape of the
    rollout (S = 1 per step); a sample of steps and all genomes vs the oracle."""
    name = "locomotion"
    nodes, conns, spec = population_for(name, seed=0)
    P = nodes.shape[0]
    plan = _plan(spec, P)
    tr = plan.transform(_dev(nodes), _dev(conns))
    ref_t = oracle.transform(nodes, conns, spec.I, spec.O)
    _assert_transform_equal(tr, ref_t)
    for step in (0, 1, 517, 999):
        x = locomotion_inputs(0, step, P, spec.I)
        out = plan.forward(_dev(x)).cpu().numpy()
        ref, bnd = oracle.forward(nodes, conns, x, spec.I, spec.O, with_bound=True)
        compare_outputs(out, ref, bnd, what=f"step {step}")


def test_uneven_full_population_sampled_genomes():
    """The full 16,384-genome uneven population: transform bit-exact on every
    genome; forward on one step checked on a 400-genome sample."""
    nodes, conns, spec = population_for("uneven", seed=0)
    P = nodes.shape[0]
    plan = _plan(spec, P)
    tr = plan.transform(_dev(nodes), _dev(conns))
    ref_t = oracle.transform(nodes, conns, spec.I, spec.O)
    _assert_transform_equal(tr, ref_t)
    x = uneven_inputs(0, 3, P)
    out = plan.forward(_dev(x)).cpu().numpy()
    sel = np.random.default_rng(0).choice(P, 400, replace=False)
    ref, bnd = oracle.forward(nodes[sel], conns[sel], x[sel], spec.I, spec.O, with_bound=True)
    compare_outputs(out[sel], ref, bnd)


@pytest.mark.parametrize("stored", [True, False])
@pytest.mark.parametrize("name,P,S", [("differentiation", 96, 77), ("locomotion", 48, 40),
                                      ("hyperneat", 32, 20), ("differentiation", 40, 300)])
def test_backward_parity(name, P, S, stored):
    nodes, conns, spec, x = _fwd_case(name, P, S, seed=5)
    plan = _plan(spec, P)
    plan.transform(_dev(nodes), _dev(conns))
    xd = _dev(x)
    saved = None
    if stored:
        saved = torch.empty((P, spec.N, S), device="cuda")
        plan.forward(xd, saved=saved)
    go = np.random.default_rng(9).standard_normal((P, S, spec.O)).astype(np.float32)
    gw, gb, gr, gi = plan.backward(xd, _dev(go), saved=saved)
    rw, rb, rr, ri = oracle.backward(nodes, conns, x, spec.I, spec.O, go)
    compare_grads(gw.cpu().numpy(), rw, "grad_weight")
    compare_grads(gb.cpu().numpy(), rb, "grad_bias")
    compare_grads(gr.cpu().numpy(), rr, "grad_response")
    compare_grads(gi.cpu().numpy(), ri, "grad_inputs")


@pytest.mark.parametrize("stored", [True, False])
@pytest.mark.parametrize("name,P,S", [("differentiation", 96, 77), ("locomotion", 48, 40)])
def test_backward_parity_workspace_slots(name, P, S, stored):
    """bwd_global = 1: the per-warp arrays in workspace slots (the path of
    genomes too large for shared memory) on genomes that also fit in shared
    memory: the same gradients against the oracle, and with the records and
    sort keys reused across the genomes a CTA walks."""
    nodes, conns, spec, x = _fwd_case(name, P, S, seed=5)
    plan = _plan(spec, P)
    plan.set_tuning(bwd_global=1)
    plan.transform(_dev(nodes), _dev(conns))
    xd = _dev(x)
    saved = None
    if stored:
        saved = torch.empty((P, spec.N, S), device="cuda")
        plan.forward(xd, saved=saved)
    go = np.random.default_rng(9).standard_normal((P, S, spec.O)).astype(np.float32)
    gw, gb, gr, gi = plan.backward(xd, _dev(go), saved=saved)
    plan.check()
    rw, rb, rr, ri = oracle.backward(nodes, conns, x, spec.I, spec.O, go)
    compare_grads(gw.cpu().numpy(), rw, "grad_weight")
    compare_grads(gb.cpu().numpy(), rb, "grad_bias")
    compare_grads(gr.cpu().numpy(), rr, "grad_response")
    compare_grads(gi.cpu().numpy(), ri, "grad_inputs")


@pytest.mark.parametrize("stored", [True, False])
def test_backward_parity_uneven_largest_genomes(stored):
    """Uneven-shaped genomes (N = 1024, C = 4096: too large for the backward's
    shared-memory arrays) through the workspace-slot backward, against the
    oracle; the largest genomes of the population included."""
    P, S = 40, 70
    nodes, conns, spec = population_for("uneven", seed=14, P=P)
    assert (spec.N, spec.C) == (1024, 4096)
    en = (~np.isnan(conns[:, :, 0]) & ~np.isnan(conns[:, :, 1]) & ~np.isnan(conns[:, :, 3]) &
          (conns[:, :, 3] != 0)).sum(1)
    assert en.max() >= 2000  # some genomes near the size limit
    x = np.random.default_rng(14).standard_normal((P, S, spec.I)).astype(np.float32)
    go = np.random.default_rng(15).standard_normal((P, S, spec.O)).astype(np.float32)
    plan = _plan(spec, P)
    plan.transform(_dev(nodes), _dev(conns))
    xd = _dev(x)
    saved = None
    if stored:
        saved = torch.empty((P, spec.N, S), device="cuda")
        plan.forward(xd, saved=saved)
    gw, gb, gr, gi = plan.backward(xd, _dev(go), saved=saved)
    plan.check()
    rw, rb, rr, ri = oracle.backward(nodes, conns, x, spec.I, spec.O, go)
    compare_grads(gw.cpu().numpy(), rw, "grad_weight")
    compare_grads(gb.cpu().numpy(), rb, "grad_bias")
    compare_grads(gr.cpu().numpy(), rr, "grad_response")
    compare_grads(gi.cpu().numpy(), ri, "grad_inputs")


@pytest.mark.parametrize("S", [77, 300])
def test_backward_parity_every_aggregation(S):
    """Product and max nodes (per-sample factors, summed with warp reductions
    during the reverse walk) next to sum and mean nodes, with kinked
    activations (relu, abs); S = 77 and 300 leave ragged last tiles."""
    from workloads import GenomeSpec, make_population
    spec = GenomeSpec(I=4, O=2, N=32, C=128, hidden=(4, 20), E_uniform=(12, 80),
                      acts=("tanh", "sigmoid", "relu", "abs", "sin", "identity"),
                      aggs=("sum", "product", "max", "mean"), w_std=0.8, b_std=0.3,
                      r_mean=1.0, r_std=0.3)
    P = 48
    nodes, conns = make_population(spec, P, seed=21)
    x = np.random.default_rng(4).uniform(-1, 1, (P, S, spec.I)).astype(np.float32)
    go = np.random.default_rng(6).standard_normal((P, S, spec.O)).astype(np.float32)
    plan = _plan(spec, P)
    plan.transform(_dev(nodes), _dev(conns))
    xd = _dev(x)
    rw, rb, rr, ri = oracle.backward(nodes, conns, x, spec.I, spec.O, go)
    for stored in (True, False):
        saved = None
        if stored:
            saved = torch.empty((P, spec.N, S), device="cuda")
            plan.forward(xd, saved=saved)
        gw, gb, gr, gi = plan.backward(xd, _dev(go), saved=saved)
        compare_grads(gw.cpu().numpy(), rw, f"grad_weight stored={stored}")
        compare_grads(gb.cpu().numpy(), rb, f"grad_bias stored={stored}")
        compare_grads(gr.cpu().numpy(), rr, f"grad_response stored={stored}")
        compare_grads(gi.cpu().numpy(), ri, f"grad_inputs stored={stored}")


def test_backward_recompute_at_65536_samples():
    """The differentiation configuration's recompute mode (S = 65,536: the saved
    aggregates would take P x 64 x 65,536 floats): gradients summed over every
    sample of 12 genomes against the oracle."""
    P, S = 12, 65536
    nodes, conns, spec = population_for("differentiation", seed=8, P=P)
    x, _ = regression_batch(8, S)
    go = (np.random.default_rng(5).standard_normal((P, S, spec.O)) / S).astype(np.float32)
    plan = _plan(spec, P)
    plan.transform(_dev(nodes), _dev(conns))
    gw, gb, gr, gi = plan.backward(_dev(x), _dev(go), saved=None)
    rw, rb, rr, ri = oracle.backward(nodes, conns, x, spec.I, spec.O, go)
    compare_grads(gw.cpu().numpy(), rw, "grad_weight")
    compare_grads(gb.cpu().numpy(), rb, "grad_bias")
    compare_grads(gr.cpu().numpy(), rr, "grad_response")
    sel = np.random.default_rng(2).choice(S, 2048, replace=False)
    compare_grads(gi.cpu().numpy()[:, sel], ri[:, sel], "grad_inputs")


def test_backward_and_forward_are_deterministic():
    nodes, conns, spec, x = _fwd_case("differentiation", 128, 300, seed=3)
    plan = _plan(spec, 128)
    plan.transform(_dev(nodes), _dev(conns))
    xd = _dev(x)
    go = _dev(np.random.default_rng(1).standard_normal((128, 300, 1)).astype(np.float32))
    a = plan.forward(xd)
    b = plan.forward(xd)
    assert torch.equal(a, b)
    g1 = plan.backward(xd, go)
    g2 = plan.backward(xd, go)
    for u, v in zip(g1, g2):
        assert torch.equal(u, v)


def test_autograd_function_matches_oracle():
    from paper_2504_08339_b300.api import evaluate
    nodes, conns, spec, x = _fwd_case("differentiation", 40, 64, seed=4)
    plan = _plan(spec, 40)
    n = _dev(nodes).requires_grad_(True)
    c = _dev(conns).requires_grad_(True)
    xi = _dev(x).requires_grad_(True)
    y = _dev(regression_batch(4, 64)[1])
    for store in (True, False):
        out = evaluate(plan, n, c, xi, store)
        loss = ((out[..., 0] - y) ** 2).mean(dim=1).sum()
        gn, gc, gx = torch.autograd.grad(loss, (n, c, xi))
        ref = oracle.forward(nodes, conns, x, spec.I, spec.O)
        gout = (2.0 / 64) * (ref[..., 0] - y.cpu().numpy()[None].astype(np.float64))
        rw, rb, rr, ri = oracle.backward(nodes, conns, x, spec.I, spec.O, gout[..., None])
        compare_grads(gc[..., 2].cpu().numpy(), rw, "w")
        compare_grads(gn[..., 1].cpu().numpy(), rb, "b")
        compare_grads(gn[..., 2].cpu().numpy(), rr, "r")
        compare_grads(gx.cpu().numpy(), ri.sum(0, keepdims=True), "x")
        assert torch.count_nonzero(gn[..., 0]) == 0 and torch.count_nonzero(gc[..., 3]) == 0


def test_autograd_switches_to_recompute_above_the_budget():
    """evaluate() without `store`: the aggregates are kept while 4 P N S bytes
    fit the budget and recomputed in the backward above it; the gradients
    match the oracle either way."""
    from paper_2504_08339_b300.api import evaluate, saved_bytes
    P, S = 24, 96
    nodes, conns, spec, x = _fwd_case("differentiation", P, S, seed=9)
    plan = _plan(spec, P)
    y = _dev(regression_batch(9, S)[1])
    need = saved_bytes(plan, S)
    assert need == 4 * P * spec.N * S
    ref = oracle.forward(nodes, conns, x, spec.I, spec.O)
    gout = (2.0 / S) * (ref[..., 0] - y.cpu().numpy()[None].astype(np.float64))
    rw, rb, rr, _ = oracle.backward(nodes, conns, x, spec.I, spec.O, gout[..., None])
    for budget, kept in ((need, True), (need - 1, False), (None, True)):
        n = _dev(nodes).requires_grad_(True)
        c = _dev(conns).requires_grad_(True)
        out = evaluate(plan, n, c, _dev(x), budget=budget)
        assert (out.grad_fn.saved_agg is not None) == kept, budget
        loss = ((out[..., 0] - y) ** 2).mean(dim=1).sum()
        gn, gc = torch.autograd.grad(loss, (n, c))
        compare_grads(gc[..., 2].cpu().numpy(), rw, "w")
        compare_grads(gn[..., 1].cpu().numpy(), rb, "b")
        compare_grads(gn[..., 2].cpu().numpy(), rr, "r")


def test_back_to_back_level_forwards_each_match_the_oracle():
    """Consecutive level-synchronous forwards on one plan (programmatic
    dependent launch: each may start while the previous one ends), eager and
    in a captured graph, with a transform of another population in between:
    every launch's outputs match the oracle on its own inputs."""
    P = 1500
    na, ca, spec = population_for("locomotion", seed=21, P=P)
    nb, cb, _ = population_for("locomotion", seed=22, P=P)
    xs = [locomotion_inputs(21, t, P, spec.I) for t in range(6)]
    plan = _plan(spec, P)
    for nodes, conns in ((na, ca), (nb, cb)):
        plan.transform(_dev(nodes), _dev(conns))
        outs = [plan.forward(_dev(x)) for x in xs[:3]]
        torch.cuda.synchronize()
        for x, o in zip(xs[:3], outs):
            ref, bnd = oracle.forward(nodes, conns, x, spec.I, spec.O, with_bound=True)
            compare_outputs(o.cpu().numpy(), ref, bnd)
    # captured: three launches in one graph, replayed after a fresh transform
    xd = [_dev(x) for x in xs[3:]]
    od = [torch.empty((P, 1, spec.O), device="cuda") for _ in xd]
    plan.transform(_dev(na), _dev(ca))
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        plan.forward(xd[0], out=od[0])  # the first after the transform, outside the graph
        s.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=s):
            for x, o in zip(xd, od):
                plan.forward(x, out=o)
    for o in od:
        o.fill_(float("nan"))
    g.replay()
    torch.cuda.synchronize()
    plan.check()
    for x, o in zip(xs[3:], od):
        ref, bnd = oracle.forward(na, ca, x, spec.I, spec.O, with_bound=True)
        compare_outputs(o.cpu().numpy(), ref, bnd)


def test_hyperneat_full_grid_small():
    nodes, conns, spec = population_for("hyperneat", seed=6, P=12)
    plan = _plan(spec, 12)
    plan.transform(_dev(nodes), _dev(conns))
    G = 12
    out = plan.hyperneat(grid=G, thresh=0.2).cpu().numpy().reshape(12, -1)
    ref, raw, bnd = oracle.hyperneat(nodes, conns, grid=G, thresh=0.2, with_raw=True,
                                     with_bound=True)
    _check_threshold(out, ref, raw, bnd)


def _check_threshold(out, ref, raw, bnd):
    # the threshold decision is unique only away from |o| = thresh; near it
    # either 0 or the raw value is correct
    lim = np.maximum(1e-6 + 1e-5 * np.abs(raw), 2 * bnd)
    near = np.abs(np.abs(raw) - 0.2) <= lim
    compare_outputs(out[~near], ref[~near], None if bnd is None else bnd[~near])
    ok = (out[near] == 0) | (np.abs(out[near] - raw[near]) <= lim[near])
    assert ok.all()


def test_hyperneat_every_aggregation_and_shape():
    """CPPNs with every activation and aggregation (the staged walk pads odd
    in-degrees with an edge that leaves each aggregate unchanged) and many
    nodes the output does not depend on (not evaluated): every launch shape
    gives the same bits, and those match the oracle."""
    from workloads import GenomeSpec, make_population
    spec = GenomeSpec(I=5, O=1, N=48, C=160, hidden=(0, 40), E_uniform=(10, 160),
                      acts=("identity", "sigmoid", "tanh", "relu", "sin", "gaussian", "abs"),
                      aggs=("sum", "product", "max", "mean"), w_std=0.9, b_std=0.4)
    P, G = 40, 7
    nodes, conns = make_population(spec, P, seed=31)
    plan = _plan(spec, P)
    plan.transform(_dev(nodes), _dev(conns))
    outs = []
    for spl in (1, 2, 4):
        for warps in (1, 4, 8, 16):
            plan.set_tuning(samples_per_lane=spl, warps_per_cta=warps)
            outs.append(plan.hyperneat(grid=G, thresh=0.2).view(torch.int32).clone())
    for o in outs[1:]:
        assert torch.equal(o, outs[0])
    out = outs[0].view(torch.float32).cpu().numpy().reshape(P, -1)
    ref, raw, bnd = oracle.hyperneat(nodes, conns, grid=G, thresh=0.2, with_raw=True,
                                     with_bound=True)
    _check_threshold(out, ref, raw, bnd)


def test_hyperneat_maximum_sizes():
    """N = 1024, C = 8192 CPPNs: the staged walk where a genome's value rows fit
    in shared memory, the workspace-slot walk where they do not."""
    from workloads import GenomeSpec, make_population
    spec = GenomeSpec(I=5, O=1, N=1024, C=8192, V_loguniform=(20, 1024),
                      E_loguniform=(30, 8192), acts=("tanh", "sin", "gaussian"),
                      aggs=("sum", "mean", "max"), w_std=0.5, b_std=0.5)
    P, G = 7, 5
    nodes, conns = make_population(spec, P - 1, seed=12)
    # plus one wide genome: 1000 hidden nodes between the inputs and the output,
    # all live at once (more value rows than shared memory holds per warp)
    from genome_builders import genome
    H = 1000
    rng = np.random.default_rng(4)
    nl = [(r, r, 0.0, 1.0, 0, 0) for r in range(5)] + [(5, 5, 0.1, 1.0, 2, 0)]
    nl += [(6 + h, 6 + h, float(rng.normal()), 1.0, int(rng.choice([2, 4, 5])), 0)
           for h in range(H)]
    cl = [(2 * h, h % 5, 6 + h, float(rng.normal()), 1.0) for h in range(H)]
    cl += [(2 * h + 1, 6 + h, 5, float(rng.normal()) * 0.05, 1.0) for h in range(H)]
    n1, c1 = genome(spec.N, spec.C, nl, cl)
    nodes = np.concatenate([nodes, n1[None]])
    conns = np.concatenate([conns, c1[None]])
    plan = _plan(spec, P)
    plan.transform(_dev(nodes), _dev(conns))
    out = plan.hyperneat(grid=G, thresh=0.2).cpu().numpy().reshape(P, -1)
    ref, raw, bnd = oracle.hyperneat(nodes, conns, grid=G, thresh=0.2, with_raw=True,
                                     with_bound=True)
    _check_threshold(out, ref, raw, bnd)


def test_hyperneat_full_size_sampled():
    """All 256 CPPNs on the 32x32 substrate (268M queries, 1 GiB of weights);
    every query of 4 genomes and a 1% sample of 8 more are checked."""
    nodes, conns, spec = population_for("hyperneat", seed=0)
    P = nodes.shape[0]
    plan = _plan(spec, P)
    plan.transform(_dev(nodes), _dev(conns))
    out = plan.hyperneat(grid=32, thresh=0.2).view(P, -1)
    rng = np.random.default_rng(0)
    full = rng.choice(P, 4, replace=False)
    got = out[torch.from_numpy(full).cuda()].cpu().numpy()
    ref, raw, bnd = oracle.hyperneat(nodes[full], conns[full], grid=32, with_raw=True,
                                     with_bound=True)
    _check_threshold(got, ref, raw, bnd)
    samp = rng.choice(np.setdiff1d(np.arange(P), full), 8, replace=False)
    q = rng.choice(32 ** 4, 32 ** 4 // 100, replace=False)
    got = out[torch.from_numpy(samp).cuda()][:, torch.from_numpy(q).cuda()].cpu().numpy()
    ref, raw, bnd = oracle.hyperneat(nodes[samp], conns[samp], grid=32, qidx=q, with_raw=True,
                                     with_bound=True)
    _check_threshold(got, ref, raw, bnd)


def test_edge_cases():
    from paper_2504_08339_b300.api import Plan
    spec = CONFIGS["differentiation"]["spec"]
    # zero genomes, zero samples
    plan = Plan(0, spec.N, spec.C, spec.I, spec.O)
    e = torch.empty((0, spec.N, 5), device="cuda")
    tr = plan.transform(e, torch.empty((0, spec.C, 4), device="cuda"))
    assert tr.order.shape == (0, spec.N)
    nodes, conns, spec = population_for("differentiation", seed=7, P=5)
    plan = _plan(spec, 5)
    plan.transform(_dev(nodes), _dev(conns))
    out = plan.forward(torch.empty((5, 0, spec.I), device="cuda"))
    assert out.shape == (5, 0, 1)
    # shared inputs equal broadcast inputs
    x = regression_batch(0, 50)[0]
    a = plan.forward(_dev(x))
    b = plan.forward(_dev(np.repeat(x, 5, 0)))
    assert torch.equal(a, b)
    # genome without any connection and hidden nodes: outputs are act(b) constants
    n = np.full((1, spec.N, 5), np.nan, np.float32)
    c = np.full((1, spec.C, 4), np.nan, np.float32)
    for r in range(spec.I):
        n[0, r] = (r, 0, 1, 0, 0)
    n[0, spec.I] = (spec.I, 0.3, 1.0, 2, 0)
    p1 = _plan(spec, 1)
    p1.transform(_dev(n), _dev(c))
    o = p1.forward(_dev(x)).cpu().numpy()
    compare_outputs(o, oracle.forward(n, c, x, spec.I, spec.O))


def test_maximum_sizes():
    """N = 1024 node rows, C = 8192 connection rows (the library maxima)."""
    from workloads import GenomeSpec, make_population
    spec = GenomeSpec(I=9, O=3, N=1024, C=8192, V_loguniform=(700, 1024),
                      E_loguniform=(6000, 8192), acts=("tanh", "sigmoid", "sin"),
                      aggs=("sum", "mean", "max"), w_std=1.0, b_std=0.5)
    nodes, conns = make_population(spec, 6, seed=11)
    plan, tr, ref = _transform_both(nodes, conns, spec)
    _assert_transform_equal(tr, ref)
    x = np.random.default_rng(0).standard_normal((6, 40, 9)).astype(np.float32)
    out = plan.forward(_dev(x)).cpu().numpy()
    r, bnd = oracle.forward(nodes, conns, x, 9, 3, with_bound=True)
    compare_outputs(out, r, bnd)
    # one sample per genome (the rollout step's call) and the saved aggregates
    x1 = np.ascontiguousarray(x[:, :1])
    r1, b1 = oracle.forward(nodes, conns, x1, 9, 3, with_bound=True)
    compare_outputs(plan.forward(_dev(x1)).cpu().numpy(), r1, b1)
    saved = torch.empty((6, spec.N, 40), device="cuda")
    compare_outputs(plan.forward(_dev(x), saved=saved).cpu().numpy(), r, bnd)
    plan.check()
    # the backward at the maxima (per-warp arrays in workspace slots), both modes
    go = np.random.default_rng(1).standard_normal((6, 40, 3)).astype(np.float32)
    rw, rb, rr, ri = oracle.backward(nodes, conns, x, 9, 3, go)
    for sv in (saved, None):
        gw, gb, gr, gi = plan.backward(_dev(x), _dev(go), saved=sv)
        plan.check()
        compare_grads(gw.cpu().numpy(), rw, "grad_weight")
        compare_grads(gb.cpu().numpy(), rb, "grad_bias")
        compare_grads(gr.cpu().numpy(), rr, "grad_response")
        compare_grads(gi.cpu().numpy(), ri, "grad_inputs")


def test_abi_argument_errors():
    import ctypes
    from paper_2504_08339_b300 import _lib
    lib = _lib.load()
    assert lib.neat_workspace_bytes(10, 3, 4, 2, 2) == 0           # N < I + O
    assert lib.neat_workspace_bytes(10, 1025, 4, 2, 2) == 0        # N too large
    h = ctypes.c_void_p()
    nb = lib.neat_workspace_bytes(4, 16, 32, 3, 1)
    ws = torch.empty(nb + 512, dtype=torch.uint8, device="cuda")
    base = (ws.data_ptr() + 255) // 256 * 256
    assert lib.neat_plan_create(ctypes.byref(h), 4, 16, 32, 3, 1, ctypes.c_void_p(base + 16),
                                nb) == _lib.NEAT_ERR_ARG
    assert lib.neat_plan_create(ctypes.byref(h), 4, 16, 32, 3, 1, ctypes.c_void_p(base),
                                nb - 1) == _lib.NEAT_ERR_WORKSPACE
    assert lib.neat_plan_create(ctypes.byref(h), 4, 16, 32, 3, 1, ctypes.c_void_p(base),
                                nb) == _lib.NEAT_OK
    x = torch.zeros((4, 2, 3), device="cuda")
    out = torch.zeros((4, 2, 1), device="cuda")
    s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    assert lib.neat_forward(h, ctypes.c_void_p(x.data_ptr()), 6, 2,
                            ctypes.c_void_p(out.data_ptr()), None, s) == _lib.NEAT_ERR_STATE
    nodes = torch.full((4, 16, 5), float("nan"), device="cuda")
    conns = torch.full((4, 32, 4), float("nan"), device="cuda")
    i32 = [torch.zeros(64, dtype=torch.int32, device="cuda") for _ in range(4)]
    assert lib.neat_transform(h, ctypes.c_void_p(nodes.data_ptr()),
                              ctypes.c_void_p(conns.data_ptr() + 4), *[
                                  ctypes.c_void_p(t.data_ptr()) for t in i32], s) == _lib.NEAT_ERR_ARG
    assert lib.neat_transform(h, ctypes.c_void_p(nodes.data_ptr()),
                              ctypes.c_void_p(conns.data_ptr()), *[
                                  ctypes.c_void_p(t.data_ptr()) for t in i32], s) == _lib.NEAT_OK
    assert lib.neat_forward(h, ctypes.c_void_p(x.data_ptr()), 5, 2,
                            ctypes.c_void_p(out.data_ptr()), None, s) == _lib.NEAT_ERR_ARG
    assert lib.neat_forward(h, ctypes.c_void_p(x.data_ptr() + 2), 6, 2,
                            ctypes.c_void_p(out.data_ptr()), None, s) == _lib.NEAT_ERR_ARG
    assert lib.neat_hyperneat_query(h, 32, 0.2, ctypes.c_void_p(out.data_ptr()), s) == \
        _lib.NEAT_ERR_UNSUPPORTED
    torch.cuda.synchronize()
    # every genome was all-padding: IO rows invalid
    st = i32[3][:4].cpu().numpy()
    assert (st == 64).all()
    lib.neat_plan_destroy(h)


def test_cuda_graph_replay_matches_direct_calls():
    nodes, conns, spec = population_for("locomotion", seed=2, P=500)
    plan = _plan(spec, 500)
    plan.transform(_dev(nodes), _dev(conns))
    T = 7
    xs = _dev(np.stack([locomotion_inputs(2, t, 500) for t in range(T)]))
    outs = torch.empty((T, 500, 1, spec.O), device="cuda")
    direct = torch.stack([plan.forward(xs[t]) for t in range(T)])
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        plan.forward(xs[0], out=outs[0])       # warm-up on the capture stream
    torch.cuda.current_stream().wait_stream(s)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        for t in range(T):
            plan.forward(xs[t], out=outs[t])
    for _ in range(3):
        outs.zero_()
        graph.replay()
        torch.cuda.synchronize()
        assert torch.equal(outs, direct)


@pytest.mark.parametrize("name,T,S,ring,chunk", [("locomotion", 23, 1, 23, 5),
                                                  ("uneven", 9, 33, 4, 2),
                                                  ("locomotion", 4, 1, 4, 8)])
def test_rollout_from_host_buffers_matches_device_rollout(name, T, S, ring, chunk):
    """The pipelined host-buffer rollout (chunks of steps, copies on their own
    streams) gives the device-resident rollout's outputs bit for bit; chunks
    that do not divide T, a ring shorter than T and a chunk longer than T;
    repeated calls reuse the buffers."""
    from paper_2504_08339_b300.rollout import Rollout
    P = 300
    nodes, conns, spec = population_for(name, seed=4, P=P)
    plan = _plan(spec, P)
    rng = np.random.default_rng(1)
    x = rng.standard_normal((ring, P, S, spec.I)).astype(np.float32)
    ro = Rollout(plan, T, S=S, ring=ring, chunk=chunk)
    ro.load(torch.from_numpy(nodes), torch.from_numpy(conns), torch.from_numpy(x),
            non_blocking=False)
    dev_out = ro.run().clone()
    torch.cuda.synchronize()
    ro2 = Rollout(plan, T, S=S, ring=ring, chunk=chunk)
    h_nodes = torch.from_numpy(nodes).pin_memory()
    h_conns = torch.from_numpy(conns).pin_memory()
    h_in = torch.from_numpy(x).pin_memory()
    h_out = torch.full((T, P, S, spec.O), 7.0).pin_memory()
    for _ in range(2):
        h_out.fill_(7.0)
        ro2.run_host(h_nodes, h_conns, h_in, h_out)
        torch.cuda.synchronize()
        assert torch.equal(h_out.view(torch.int32), dev_out.cpu().view(torch.int32))
    # the outputs are the plan's own forward of each step's inputs
    plan.transform(_dev(nodes), _dev(conns))
    for t in (0, T - 1):
        assert torch.equal(h_out[t], plan.forward(_dev(x[t % ring])).cpu())


def test_tuning_knobs_and_autotuner(tmp_path, monkeypatch):
    from paper_2504_08339_b300 import NeatError
    from paper_2504_08339_b300.autotune import autotune
    nodes, conns, spec = population_for("locomotion", seed=8, P=600)
    plan = _plan(spec, 600)
    t = plan.get_tuning()
    assert t["lvl_threads"] in (32, 64, 128, 256) and t["small_s_max"] == 8
    assert t["lvl_budget_kb"] == 0 and t["wait_polls"] == 1 << 22  # 0: chosen per population
    with pytest.raises(NeatError):
        plan.set_tuning(lvl_threads=100)
    with pytest.raises(NeatError):
        plan.set_tuning(lvl_budget_kb=1)
    with pytest.raises(NeatError):
        plan.set_tuning(samples_per_lane=3)
    with pytest.raises(NeatError):
        plan.set_tuning(wait_polls=-2)
    with pytest.raises(NeatError):
        plan.set_tuning(samples_per_lanes=2)  # a misspelt knob is not ignored
    x = np.random.default_rng(0).standard_normal((600, 1, spec.I)).astype(np.float32)
    ref, bnd = oracle.forward(nodes, conns, x, spec.I, spec.O, with_bound=True)
    monkeypatch.setenv("NEAT_TUNE_CACHE", str(tmp_path / "tune.json"))
    dn, dc, dx = _dev(nodes), _dev(conns), _dev(x)
    res = autotune(plan, dn, dc, dx, reps=3)
    assert res["trials"] and isinstance(res["tuning"], dict)  # {}: the defaults
    compare_outputs(plan.forward(dx).cpu().numpy(), ref, bnd)
    # every candidate tuning gives a correct result
    for tr in res["trials"]:
        plan.set_tuning(**tr["tuning"])
        plan.transform(dn, dc)
        compare_outputs(plan.forward(dx).cpu().numpy(), ref, bnd, what=str(tr["tuning"]))
    # the cache answers the second call
    res2 = autotune(plan, dn, dc, dx, reps=3)
    assert res2["tuning"] == res["tuning"]


def test_autotuner_on_the_saved_aggregates_forward(tmp_path, monkeypatch):
    """With saved=True the autotuner times the forward that writes the
    aggregates (S = 64: one and two samples a lane among the candidates);
    its choice gives the oracle's outputs and aggregates, and the cache keeps
    the two kinds of timing apart."""
    from paper_2504_08339_b300.autotune import autotune
    P, S = 96, 64
    nodes, conns, spec = population_for("differentiation", seed=3, P=P)
    plan = _plan(spec, P)
    x = np.random.default_rng(2).standard_normal((P, S, spec.I)).astype(np.float32)
    monkeypatch.setenv("NEAT_TUNE_CACHE", str(tmp_path / "tune.json"))
    dn, dc, dx = _dev(nodes), _dev(conns), _dev(x)
    res = autotune(plan, dn, dc, dx, reps=2, saved=True)
    assert {t["tuning"].get("samples_per_lane") for t in res["trials"]} >= {1, 2}
    saved = torch.empty((P, spec.N, S), device="cuda")
    out = plan.forward(dx, saved=saved).cpu().numpy()
    ref, bnd = oracle.forward(nodes, conns, x, spec.I, spec.O, with_bound=True)
    compare_outputs(out, ref, bnd)
    autotune(plan, dn, dc, dx, reps=2)  # outputs only: its own cache entry
    import json
    with open(tmp_path / "tune.json") as f:
        assert len(json.load(f)) == 2

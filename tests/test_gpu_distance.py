"""GPU parity of the population-wide compatibility distance against the FP64
oracle (reading R12): node and connection genes matched by key, disjoint
counts, homologous attribute differences."""
import numpy as np
import pytest
import torch

import oracle
from workloads import population_for

pytestmark = pytest.mark.gpu


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _close(got, ref):
    both_nan = np.isnan(got) & np.isnan(ref)
    ok = both_nan | (np.abs(got - ref) <= 1e-6 + 1e-5 * np.abs(ref))
    assert ok.all(), (np.argwhere(~ok)[:5], got[~ok][:5], ref[~ok][:5])


def _family(seed, name="locomotion", P=24):
    """Strangers plus perturbed copies (shared genes, changed weights, deleted
    and disabled rows, a repeated disabled key), rows shuffled."""
    rng = np.random.default_rng(seed)
    nodes, conns, spec = population_for(name, seed=seed, P=P)
    for g in range(P // 2, P):
        src = g - P // 2
        n, c = nodes[src].copy(), conns[src].copy()
        live = np.flatnonzero(~np.isnan(c[:, 0]))
        if live.size >= 4:
            pick = rng.choice(live, max(1, live.size // 5), replace=False)
            c[pick, 2] += rng.normal(0, 0.3, pick.size).astype(np.float32)
            c[rng.choice(live, 2, replace=False), 3] = 0.0
            c[rng.choice(live, 1), :] = np.nan
        free = np.flatnonzero(np.isnan(c[:, 0]))
        if free.size and live.size:
            c[free[0]] = c[live[0]]
            c[free[0], 3] = 0.0
        c = c[rng.permutation(c.shape[0])]
        nodes[g], conns[g] = n, c
    return nodes, conns, spec


@pytest.mark.parametrize("name", ["locomotion", "tiny", "uneven"])
def test_distance_parity(name):
    from paper_2504_08339_b300.api import Plan, distance
    P = {"locomotion": 24, "tiny": 40, "uneven": 12}[name]
    nodes, conns, spec = _family(3, name, P)
    dn, dc = _dev(nodes), _dev(conns)
    plan = Plan(P, spec.N, spec.C, spec.I, spec.O)
    tr = plan.transform(dn, dc)
    d = distance(dn, dc, spec.I, spec.O, status=tr.status).cpu().numpy()
    ref = oracle.distance(nodes, conns, spec.I, spec.O)
    _close(d, ref)
    np.testing.assert_array_equal(d.view(np.int32), d.T.view(np.int32))
    np.testing.assert_array_equal(np.diag(d), 0.0)


def test_distance_malformed_and_coefficients():
    from paper_2504_08339_b300.api import Plan, distance
    nodes, conns, spec = population_for("tiny", seed=4, P=10)
    nodes[2, 3, 0] = nodes[2, 0, 0]                        # duplicate key
    live = np.flatnonzero(~np.isnan(conns[5, :, 0]) & (conns[5, :, 3] != 0))
    conns[5, live[0], 1] = 777.0                           # dangling key
    dn, dc = _dev(nodes), _dev(conns)
    plan = Plan(10, spec.N, spec.C, spec.I, spec.O)
    tr = plan.transform(dn, dc)
    d = distance(dn, dc, spec.I, spec.O, status=tr.status, c_disjoint=2.0,
                 c_homologous=0.25).cpu().numpy()
    ref = oracle.distance(nodes, conns, spec.I, spec.O, c_disjoint=2.0, c_homologous=0.25)
    _close(d, ref)
    for bad in (2, 5):
        assert np.isnan(d[bad]).all() and np.isnan(d[:, bad]).all()
    # without status words every genome is taken as valid
    d2 = distance(dn, dc, spec.I, spec.O, c_disjoint=2.0, c_homologous=0.25).cpu().numpy()
    ok = [g for g in range(10) if g not in (2, 5)]
    np.testing.assert_array_equal(d2[np.ix_(ok, ok)], d[np.ix_(ok, ok)])


def test_distance_full_population_sampled():
    """All 10,000 x 10,000 pairs of the locomotion population; a 120-genome
    sub-matrix against the oracle."""
    from paper_2504_08339_b300.api import distance
    nodes, conns, spec = population_for("locomotion", seed=0)
    P = nodes.shape[0]
    d = distance(_dev(nodes), _dev(conns), spec.I, spec.O)
    sel = np.sort(np.random.default_rng(1).choice(P, 120, replace=False))
    ref = oracle.distance(nodes[sel], conns[sel], spec.I, spec.O)
    _close(d[sel][:, sel].cpu().numpy(), ref)


def test_distance_arguments():
    from paper_2504_08339_b300 import _lib
    lib = _lib.load()
    assert lib.neat_distance_scratch_bytes(10, 16, 32) > 10 * (16 + 32) * 16
    assert lib.neat_distance_scratch_bytes(10, 2000, 32) == 0
    assert lib.neat_distance(None, None, None, 4, 16, 32, 3, 1, 1.0, 0.5, None, None, 0,
                             None) == _lib.NEAT_ERR_ARG

"""Pins of the oracle's compatibility distance (reading R12): an independent
brute force written with Python sets and dicts, closed forms of genomes one
gene apart, and invariants (symmetry, zero self-distance, row permutations,
malformed genomes)."""
import math

import numpy as np
import pytest

import oracle
from workloads import population_for

CD, CH = 1.0, 0.5


def _brute(nodes, conns, I, cd=CD, ch=CH):
    """Distance of two genomes straight from the definition (dict joins)."""
    def genes(n, c):
        ng = {}
        for r in range(n.shape[0]):
            if np.isnan(n[r, 0]):
                continue
            ng[float(n[r, 0])] = (r < I, float(n[r, 1]), float(n[r, 2]), n[r, 3], n[r, 4])
        cg = {}
        for r in range(c.shape[0]):
            if np.isnan(c[r, 0]) or np.isnan(c[r, 1]):
                continue
            k = (float(c[r, 0]), float(c[r, 1]))
            if k not in cg:  # the lowest row of a repeated key
                en = not np.isnan(c[r, 3]) and c[r, 3] != 0
                cg[k] = (float(c[r, 2]), en)
        return ng, cg

    (na, ca), (nb, cb) = genes(*nodes), genes(*conns)
    shared = set(na) & set(nb)
    dn = len(set(na) ^ set(nb))
    hn = 0.0
    for k in shared:
        a, b = na[k], nb[k]
        if not a[0] and not b[0]:
            hn += abs(a[1] - b[1]) + abs(a[2] - b[2]) + (a[3] != b[3]) + (a[4] != b[4])
    d = (cd * dn + ch * hn) / max(len(na), len(nb)) if max(len(na), len(nb)) else 0.0
    sc = set(ca) & set(cb)
    dc = len(set(ca) ^ set(cb))
    hc = sum(abs(ca[k][0] - cb[k][0]) + (ca[k][1] != cb[k][1]) for k in sc)
    m = max(len(ca), len(cb))
    return d + ((cd * dc + ch * hc) / m if m else 0.0)


def _relatives(rng, n0, c0, count):
    """Genomes sharing most genes with (n0, c0): weights, biases and flags
    perturbed, rows deleted, a duplicate disabled row added, rows shuffled."""
    out = []
    for _ in range(count):
        n, c = n0.copy(), c0.copy()
        live = np.flatnonzero(~np.isnan(c[:, 0]))
        pick = rng.choice(live, max(1, live.size // 4), replace=False)
        c[pick, 2] += rng.normal(0, 0.5, pick.size).astype(np.float32)
        c[rng.choice(live, 2, replace=False), 3] = 0.0
        c[rng.choice(live, 2, replace=False), :] = np.nan        # deleted connections
        hid = np.flatnonzero(~np.isnan(n[:, 0]))[8:]
        if hid.size:
            n[rng.choice(hid, min(3, hid.size), replace=False), 1] += 0.25
            n[rng.choice(hid, 1), 3] = 4.0
        free = np.flatnonzero(np.isnan(c[:, 0]))
        if free.size:                                           # a disabled duplicate
            src = live[0]
            c[free[0]] = c[src]
            c[free[0], 2] = 9.0
            c[free[0], 3] = 0.0
        out.append((n, c))
    return out


def test_distance_matches_brute_force():
    rng = np.random.default_rng(0)
    nodes, conns, spec = population_for("locomotion", seed=3, P=3)
    gen = [(nodes[i], conns[i]) for i in range(3)]
    gen += _relatives(rng, nodes[0], conns[0], 4) + _relatives(rng, nodes[1], conns[1], 3)
    n = np.stack([g[0] for g in gen])
    c = np.stack([g[1] for g in gen])
    d = oracle.distance(n, c, spec.I, spec.O)
    for a in range(len(gen)):
        for b in range(len(gen)):
            want = _brute(gen[a], gen[b], spec.I)
            assert math.isclose(d[a, b], want, rel_tol=1e-12, abs_tol=1e-12), (a, b)
    assert d[0, 3] < d[0, 1]  # relatives are closer than strangers


def test_closed_forms_one_gene_apart():
    nodes, conns, spec = population_for("locomotion", seed=5, P=1)
    n, c = nodes[0], conns[0]
    live = np.flatnonzero(~np.isnan(c[:, 0]))
    m = live.size                                # connection genes (keys distinct here)
    nv = int((~np.isnan(n[:, 0])).sum())
    # one weight changed by 0.75
    c2 = c.copy()
    c2[live[3], 2] += np.float32(0.75)
    d = oracle.distance(np.stack([n, n]), np.stack([c, c2]), spec.I, spec.O)
    delta = float(c2[live[3], 2]) - float(c[live[3], 2])
    assert math.isclose(d[0, 1], CH * abs(delta) / m, rel_tol=1e-12)
    # one extra hidden node without connections
    n3 = n.copy()
    free = np.flatnonzero(np.isnan(n3[:, 0]))[0]
    n3[free] = (9999.0, 0.1, 1.0, 1.0, 0.0)
    d = oracle.distance(np.stack([n, n3]), np.stack([c, c]), spec.I, spec.O)
    assert math.isclose(d[0, 1], CD * 1.0 / (nv + 1), rel_tol=1e-12)
    # one connection disabled: enabled flag differs
    c4 = c.copy()
    c4[live[0], 3] = 0.0
    d = oracle.distance(np.stack([n, n]), np.stack([c, c4]), spec.I, spec.O)
    assert math.isclose(d[0, 1], CH * 1.0 / m, rel_tol=1e-12)


def test_invariants():
    rng = np.random.default_rng(2)
    nodes, conns, spec = population_for("uneven", seed=2, P=6)
    d = oracle.distance(nodes, conns, spec.I, spec.O)
    np.testing.assert_array_equal(d, d.T)
    np.testing.assert_array_equal(np.diag(d), 0.0)
    assert (d[~np.eye(6, dtype=bool)] > 0).all()
    # shuffling a genome's rows (node rows past the inputs and outputs, all
    # connection rows) changes no distance
    n2, c2 = nodes.copy(), conns.copy()
    k = spec.I + spec.O
    perm = k + rng.permutation(spec.N - k)
    n2[2, k:] = nodes[2, perm]
    c2[2] = conns[2, rng.permutation(spec.C)]
    np.testing.assert_array_equal(oracle.distance(n2, c2, spec.I, spec.O), d)


def test_malformed_genomes_get_nan():
    nodes, conns, spec = population_for("tiny", seed=1, P=4)
    nodes[1, 3, 0] = nodes[1, 0, 0]  # duplicate key
    d = oracle.distance(nodes, conns, spec.I, spec.O)
    assert np.isnan(d[1]).all() and np.isnan(d[:, 1]).all()
    ok = [0, 2, 3]
    assert np.isfinite(d[np.ix_(ok, ok)]).all()

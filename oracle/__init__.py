"""FP64 CPU oracle for tensorized NEAT evaluation (Sec. 3.1-3.3).

TEST INFRASTRUCTURE ONLY: tests, the smoke check and the benchmark's CPU
baseline / reference legs use it; the CUDA library never does.  The arithmetic
lives in ``neat_oracle.c`` (plain C, double precision); this module compiles it
with gcc and marshals numpy arrays through ctypes.

Parity status of each function (what pins it, in tests/test_oracle_*.py):
  transform  -- XOR worked example, brute force over all topological orders of
                tiny DAGs, longest-path layers, relabelling invariants, status
                bits of malformed genomes.
  forward    -- XOR closed form, single-path chains per activation, closed forms
                of two-input aggregations, layered-MLP special case vs numpy,
                invariants (disabled/padding rows, genome and row permutations).
  bound      -- checked empirically against independent fp32 evaluations.
  backward   -- central finite differences of the forward; MLP special case
                against numpy back-propagation.
  hyperneat  -- single-node CPPNs with closed forms over the grid.
  distance   -- brute force with Python sets and dicts on small genomes,
                closed forms (one weight / one extra gene apart), symmetry,
                zero self-distance, row-permutation invariance, NaN for
                malformed genomes.
  substrate  -- the identity-activation case against numpy matmul, a single
                connection closed form, the threshold pipeline with a
                closed-form CPPN, the fp32 bound against float32 matmuls.
  apply_ops  -- hand-written expected tensors of operation sequences (first
                NaN row, reuse of a freed lower row, full tensors, ranges),
                no-op invariance, transform of the result.
  forward_recurrent -- linear (identity, sum) recurrent genomes against numpy
                matrix powers, a self-loop closed form, equality with the
                feed-forward forward on DAGs once T reaches their depth,
                status bits without CYCLE.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "neat_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

# status bits (the oracle's own copy; the CUDA library defines its own)
CYCLE, DANGLING_KEY, DUP_KEY, DUP_EDGE, EDGE_INTO_INPUT, BAD_ATTR, IO_ROW_INVALID = (
    1, 2, 4, 8, 16, 32, 64)


def build(force: bool = False) -> str:
    """Compile neat_oracle.c into liboracle.so next to it (gcc -O2, IEEE math)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-Wall",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            P = ctypes.c_void_p
            i32, i64, dbl = ctypes.c_int, ctypes.c_int64, ctypes.c_double
            lib.or_transform.argtypes = [i32, i32, i32, i32, i32, P, P, P, P, P, P]
            lib.or_forward.argtypes = [i32, i32, i32, i32, i32, P, P, P, i64, i32, P, P, P]
            lib.or_backward.argtypes = [i32, i32, i32, i32, i32, P, P, P, i64, i32, P, P, P, P, P]
            lib.or_forward_recurrent.argtypes = [i32, i32, i32, i32, i32, P, P, P, i64, i32, i32,
                                                 P, P, P]
            lib.or_distance.argtypes = [i32, i32, i32, i32, i32, P, P, dbl, dbl, P]
            lib.or_apply_ops.argtypes = [i32, i32, i32, P, P, P, i32, P]
            lib.or_substrate.argtypes = [i32, i32, P, P, i64, i32, i32, P, P]
            lib.or_hyperneat.argtypes = [i32, i32, i32, P, P, i32, dbl, P, i64, P, P, P]
            for f in (lib.or_transform, lib.or_forward, lib.or_backward, lib.or_hyperneat):
                f.restype = ctypes.c_int
            _lib = lib
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _over_genomes(P, threads, call):
    """call(a, b) for contiguous genome slices [a, b) covering [0, P): one
    slice per thread (the C calls release the GIL; genomes are independent
    and the library keeps no global state, so the results are those of one
    call over all of them)."""
    threads = max(1, min(int(threads or 1), P))
    if threads == 1:
        rc = call(0, P)
        assert rc == 0, rc
        return
    from concurrent.futures import ThreadPoolExecutor
    cuts = [P * k // threads for k in range(threads + 1)]
    with ThreadPoolExecutor(threads) as ex:
        for rc in ex.map(lambda k: call(cuts[k], cuts[k + 1]), range(threads)):
            assert rc == 0, rc


def _rows(a, lo, hi):
    """Pointer to rows [lo, hi) of a per-genome array (None stays None)."""
    return None if a is None else _ptr(a[lo:hi])


def _in_rows(x, stride, lo, hi):
    """Pointer to the inputs of genomes [lo, hi) (shared inputs: the same set)."""
    return _ptr(x) if stride == 0 else _ptr(x[lo:hi])


def _f64(a):
    """The oracle reads double arrays; float32 data converts exactly."""
    return np.ascontiguousarray(a, dtype=np.float64)


def _shapes(nodes, conns):
    P, N, k = nodes.shape
    P2, C, k2 = conns.shape
    assert k == 5 and k2 == 4 and P == P2
    return P, N, C


def transform(nodes, conns, I, O, threads=1):
    """(order [P,N] i32, layer [P,N] i32, n_layers [P] i32, status [P] u32)."""
    nodes, conns = _f64(nodes), _f64(conns)
    P, N, C = _shapes(nodes, conns)
    order = np.empty((P, N), np.int32)
    layer = np.empty((P, N), np.int32)
    nl = np.empty(P, np.int32)
    st = np.empty(P, np.uint32)
    lib = _load()
    _over_genomes(P, threads, lambda a, b: lib.or_transform(
        b - a, N, C, I, O, _rows(nodes, a, b), _rows(conns, a, b), _rows(order, a, b),
        _rows(layer, a, b), _rows(nl, a, b), _rows(st, a, b)))
    return order, layer, nl, st


def _inputs(inputs, P, I):
    inputs = _f64(inputs)
    assert inputs.ndim == 3 and inputs.shape[2] == I
    if inputs.shape[0] == 1 and P != 1:
        stride = 0
    else:
        assert inputs.shape[0] == P
        stride = inputs.shape[1] * I
    return inputs, stride, inputs.shape[1]


def forward(nodes, conns, inputs, I, O, with_bound=False, with_values=False, threads=1):
    """outputs [P,S,O] f64 (and bound [P,S,O], values [P,S,N] when asked).
    inputs is [P,S,I] or [1,S,I] (shared by every genome).  `threads` host
    threads evaluate contiguous slices of the genomes."""
    nodes, conns = _f64(nodes), _f64(conns)
    P, N, C = _shapes(nodes, conns)
    inputs, stride, S = _inputs(inputs, P, I)
    out = np.empty((P, S, O), np.float64)
    bnd = np.empty((P, S, O), np.float64) if with_bound else None
    vals = np.empty((P, S, N), np.float64) if with_values else None
    lib = _load()
    _over_genomes(P, threads, lambda a, b: lib.or_forward(
        b - a, N, C, I, O, _rows(nodes, a, b), _rows(conns, a, b), _in_rows(inputs, stride, a, b),
        stride, S, _rows(out, a, b), _rows(bnd, a, b), _rows(vals, a, b)))
    res = [out]
    if with_bound:
        res.append(bnd)
    if with_values:
        res.append(vals)
    return res[0] if len(res) == 1 else tuple(res)


def forward_recurrent(nodes, conns, inputs, I, O, T, with_bound=False, with_status=False,
                      threads=1):
    """Recurrent calculation over T synchronous iterations (reading R11):
    outputs [P,S,O] f64 (and bound [P,S,O], status [P] u32 when asked)."""
    nodes, conns = _f64(nodes), _f64(conns)
    P, N, C = _shapes(nodes, conns)
    inputs, stride, S = _inputs(inputs, P, I)
    out = np.empty((P, S, O), np.float64)
    bnd = np.empty((P, S, O), np.float64) if with_bound else None
    st = np.empty(P, np.uint32) if with_status else None
    lib = _load()
    _over_genomes(P, threads, lambda a, b: lib.or_forward_recurrent(
        b - a, N, C, I, O, _rows(nodes, a, b), _rows(conns, a, b), _in_rows(inputs, stride, a, b),
        stride, S, int(T), _rows(out, a, b), _rows(bnd, a, b), _rows(st, a, b)))
    res = [out]
    if with_bound:
        res.append(bnd)
    if with_status:
        res.append(st)
    return res[0] if len(res) == 1 else tuple(res)


def distance(nodes, conns, I, O, c_disjoint=1.0, c_homologous=0.5):
    """Compatibility distance of every pair (reading R12): dist [P, P] f64."""
    nodes, conns = _f64(nodes), _f64(conns)
    P, N, C = _shapes(nodes, conns)
    out = np.empty((P, P), np.float64)
    rc = _load().or_distance(P, N, C, I, O, _ptr(nodes), _ptr(conns), float(c_disjoint),
                             float(c_homologous), _ptr(out))
    assert rc == 0, rc
    return out


def apply_ops(nodes, conns, ops):
    """Tensorized operations (reading R13) on copies of the population:
    (nodes, conns, op_status [P] u32).  ops is [P, K, 8]."""
    nodes, conns = _f64(nodes).copy(), _f64(conns).copy()
    P, N, C = _shapes(nodes, conns)
    ops = _f64(ops)
    assert ops.ndim == 3 and ops.shape[0] == P and ops.shape[2] == 8
    st = np.empty(P, np.uint32)
    rc = _load().or_apply_ops(P, N, C, _ptr(nodes), _ptr(conns), _ptr(ops), ops.shape[1],
                              _ptr(st))
    assert rc == 0, rc
    return nodes, conns, st


def substrate(weights, inputs, act, with_bound=False):
    """Sandwich substrate (reading R14): weights [P, K, K] (input cell, output
    cell), inputs [P or 1, S, K] -> outputs [P, S, K] f64 (and the fp32 bound)."""
    w = _f64(weights)
    P, K = w.shape[0], w.shape[1]
    assert w.shape == (P, K, K)
    x, stride, S = _inputs(inputs, P, K)
    out = np.empty((P, S, K), np.float64)
    bnd = np.empty((P, S, K), np.float64) if with_bound else None
    rc = _load().or_substrate(P, K, _ptr(w), _ptr(x), stride, S, int(act), _ptr(out), _ptr(bnd))
    assert rc == 0, rc
    return (out, bnd) if with_bound else out


def backward(nodes, conns, inputs, I, O, grad_out, want_inputs=True, threads=1):
    """(grad_w [P,C], grad_b [P,N], grad_r [P,N], grad_in [P,S,I] or None), all f64."""
    nodes, conns = _f64(nodes), _f64(conns)
    P, N, C = _shapes(nodes, conns)
    inputs, stride, S = _inputs(inputs, P, I)
    go = np.ascontiguousarray(grad_out, dtype=np.float64)
    assert go.shape == (P, S, O)
    gw = np.empty((P, C), np.float64)
    gb = np.empty((P, N), np.float64)
    gr = np.empty((P, N), np.float64)
    gi = np.empty((P, S, I), np.float64) if want_inputs else None
    lib = _load()
    _over_genomes(P, threads, lambda a, b: lib.or_backward(
        b - a, N, C, I, O, _rows(nodes, a, b), _rows(conns, a, b), _in_rows(inputs, stride, a, b),
        stride, S, _rows(go, a, b), _rows(gw, a, b), _rows(gb, a, b), _rows(gr, a, b),
        _rows(gi, a, b)))
    return gw, gb, gr, gi


def hyperneat(nodes, conns, grid=32, thresh=0.2, qidx=None, with_raw=False, with_bound=False,
              threads=1):
    """Thresholded substrate weights [P, nq] (nq = grid^4 when qidx is None)."""
    nodes, conns = _f64(nodes), _f64(conns)
    P, N, C = _shapes(nodes, conns)
    if qidx is not None:
        qidx = np.ascontiguousarray(qidx, dtype=np.int64)
        nq = qidx.size
    else:
        nq = grid ** 4
    out = np.empty((P, nq), np.float64)
    raw = np.empty((P, nq), np.float64) if with_raw else None
    bnd = np.empty((P, nq), np.float64) if with_bound else None
    lib = _load()
    _over_genomes(P, threads, lambda a, b: lib.or_hyperneat(
        b - a, N, C, _rows(nodes, a, b), _rows(conns, a, b), grid, thresh, _ptr(qidx),
        nq if qidx is not None else 0, _rows(out, a, b), _rows(raw, a, b), _rows(bnd, a, b)))
    res = [out]
    if with_raw:
        res.append(raw)
    if with_bound:
        res.append(bnd)
    return res[0] if len(res) == 1 else tuple(res)

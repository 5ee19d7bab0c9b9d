"""Comparison rules of the GPU-vs-oracle parity tests.

Outputs (fp32 GPU vs FP64 oracle): an element passes if
    |g - r| <= max(1e-6 + 1e-5 |r|, 2 * bound)
where `bound` is the oracle's first-order bound on the error any fp32
evaluation of that network may make.  Elements inside 2*bound but outside the
1e-6 + 1e-5|r| tolerance are counted as ill-conditioned and reported.
Non-finite oracle values must be matched in class (NaN / +inf / -inf).

Gradients: |g - r| <= 1e-4 * max(|r|, scale) with scale the largest |r| of the
same gradient array of the same genome.
"""
import numpy as np

REL, ABS = 1e-5, 1e-6
GRAD_REL = 1e-4


def compare_outputs(g, r, bound=None, what="outputs"):
    g = np.asarray(g, np.float64)
    r = np.asarray(r, np.float64)
    assert g.shape == r.shape, (g.shape, r.shape)
    fin = np.isfinite(r)
    # non-finite classes
    nf = ~fin
    if nf.any():
        same = (np.isnan(g[nf]) & np.isnan(r[nf])) | (g[nf] == r[nf])
        assert same.all(), f"{what}: non-finite mismatch at {np.argwhere(nf)[~same][:5]}"
    err = np.abs(g - r)
    tol = ABS + REL * np.abs(r)
    lim = tol if bound is None else np.maximum(tol, 2.0 * np.asarray(bound))
    bad = fin & ~(err <= lim)
    if bad.any():
        idx = np.argwhere(bad)[:5]
        raise AssertionError(f"{what}: {bad.sum()} elements outside tolerance, e.g. "
                             + ", ".join(f"{tuple(i)} g={g[tuple(i)]!r} r={r[tuple(i)]!r} "
                                         f"lim={lim[tuple(i)]:.3g}" for i in idx))
    illcond = int((fin & (err > tol)).sum())
    max_err = float(err[fin].max()) if fin.any() else 0.0
    rel = err[fin] / np.maximum(np.abs(r[fin]), 1e-30)
    return dict(max_abs_err=max_err, max_rel_err=float(rel.max()) if rel.size else 0.0,
                ill_conditioned=illcond, n=int(fin.sum()))


def compare_grads(g, r, what="grad"):
    """g, r: [P, ...] arrays; per-genome scale."""
    g = np.asarray(g, np.float64)
    r = np.asarray(r, np.float64)
    assert g.shape == r.shape
    P = r.shape[0]
    rr = r.reshape(P, -1)
    gg = g.reshape(P, -1)
    scale = np.abs(rr).max(axis=1, keepdims=True)
    lim = GRAD_REL * np.maximum(np.abs(rr), scale) + 1e-30
    err = np.abs(gg - rr)
    bad = ~(err <= lim)
    if bad.any():
        idx = np.argwhere(bad)[:5]
        raise AssertionError(f"{what}: {bad.sum()} elements outside tolerance, e.g. "
                             + ", ".join(f"{tuple(i)} g={gg[tuple(i)]!r} r={rr[tuple(i)]!r}"
                                         for i in idx))
    rel = err / np.maximum(scale, 1e-30)
    return dict(max_scaled_err=float(rel.max()) if rel.size else 0.0)

"""The bench's GPU-vs-oracle error report (host logic only): exact results
report zero error, a planted error beyond the tolerance and beyond twice the
bound is counted, non-finite classes must agree."""
import os
import sys

import numpy as np

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402


def test_accuracy_counts_errors_against_tolerance_and_bound():
    r = np.array([1.0, -2.0, 0.5, 0.25, np.nan, np.inf])
    g = r.astype(np.float32).astype(np.float64)
    a = bench.accuracy(g, r, bound=np.zeros_like(r))
    assert a["n"] == 4 and a["max_abs_err"] == 0.0 and a["beyond_tolerance"] == 0
    assert a["beyond_bound"] == 0 and a["nonfinite_mismatch"] == 0
    g2 = g.copy()
    g2[1] += 1e-3                      # beyond 1e-6 + 1e-5 * 2
    g2[4] = 0.0                        # NaN class lost
    a2 = bench.accuracy(g2, r, bound=np.full_like(r, 1e-4))
    assert a2["beyond_tolerance"] == 1 and a2["beyond_bound"] == 1
    assert a2["nonfinite_mismatch"] == 1
    assert abs(a2["max_rel_err"] - 5e-4) < 1e-9
    # inside twice the bound: ill-conditioned, not a failure
    a3 = bench.accuracy(g2[:4], r[:4], bound=np.full(4, 1e-3))
    assert a3["beyond_tolerance"] == 1 and a3["beyond_bound"] == 0


def test_grad_accuracy_is_relative_to_each_genome_largest_gradient():
    r = np.array([[1.0, 1e-6, 0.0], [100.0, 50.0, 1.0]])
    g = r.copy()
    g[0, 1] += 1e-5                    # 1e-5 of genome 0's largest
    g[1, 2] += 1e-1                    # 1e-3 of genome 1's largest
    a = bench.grad_accuracy(g, r)
    assert a["n"] == 6 and a["beyond_1e-4"] == 1
    assert abs(a["max_err_rel_to_genome_max"] - 1e-3) < 1e-12

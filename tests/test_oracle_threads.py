"""The oracle's host-thread slicing changes nothing: every per-genome entry
point gives the bits of one call over the whole population."""
import numpy as np

import oracle
from workloads import population_for, regression_batch


def test_threaded_oracle_calls_equal_one_call():
    nodes, conns, spec = population_for("locomotion", seed=3, P=37)
    x = np.random.default_rng(1).standard_normal((37, 3, spec.I)).astype(np.float32)
    for threads in (2, 5, 64):
        a = oracle.forward(nodes, conns, x, spec.I, spec.O, with_bound=True, with_values=True)
        b = oracle.forward(nodes, conns, x, spec.I, spec.O, with_bound=True, with_values=True,
                           threads=threads)
        for u, v in zip(a, b):
            assert np.array_equal(u, v, equal_nan=True)
        for u, v in zip(oracle.transform(nodes, conns, spec.I, spec.O),
                        oracle.transform(nodes, conns, spec.I, spec.O, threads=threads)):
            assert np.array_equal(u, v)
        u = oracle.forward_recurrent(nodes, conns, x, spec.I, spec.O, 3)
        v = oracle.forward_recurrent(nodes, conns, x, spec.I, spec.O, 3, threads=threads)
        assert np.array_equal(u, v, equal_nan=True)
    nodes, conns, spec = population_for("differentiation", seed=3, P=11)
    xb = regression_batch(0, 16)[0]
    go = np.random.default_rng(2).standard_normal((11, 16, 1))
    for u, v in zip(oracle.backward(nodes, conns, xb, spec.I, spec.O, go),
                    oracle.backward(nodes, conns, xb, spec.I, spec.O, go, threads=4)):
        assert np.array_equal(u, v)
    nodes, conns, spec = population_for("hyperneat", seed=3, P=6)
    q = np.arange(0, 32 ** 4, 4099)
    assert np.array_equal(oracle.hyperneat(nodes, conns, qidx=q),
                          oracle.hyperneat(nodes, conns, qidx=q, threads=3))

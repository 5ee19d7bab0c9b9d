"""The shared-memory bandwidth probe behind the roofline's on-chip peak reads
what it claims to read: every thread's XOR fold matches the fold computed
here from the probe's definition (array contents and read pattern)."""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


def _expected(blocks, iters):
    t = np.arange(512, dtype=np.int64)
    acc = np.zeros(512, dtype=np.uint32)
    mul = np.uint32(0x9E3779B1)
    for it in range(iters):
        for u in range(8):
            idx = (t + 512 * u + it) & 4095
            for c in range(4):
                acc ^= ((4 * idx + c).astype(np.uint32) * mul).astype(np.uint32)
    return np.tile(acc, blocks)


@pytest.mark.parametrize("blocks,iters", [(1, 0), (2, 3), (5, 17)])
def test_probe_reads_every_word_it_counts(blocks, iters):
    from paper_2504_08339_b300.probe import smem_read
    sink = torch.full((blocks * 512,), -1, dtype=torch.int32, device="cuda")
    smem_read(blocks, iters, sink)
    torch.cuda.synchronize()
    got = sink.cpu().numpy().view(np.uint32)
    np.testing.assert_array_equal(got, _expected(blocks, iters))


def test_probe_bandwidth_is_plausible():
    from paper_2504_08339_b300.probe import smem_read_gbs
    r = smem_read_gbs(iters=512, reps=2)
    clk_hz = 2.1e9  # above the part's maximum SM clock
    assert 0 < r["gbs"] < r["sms"] * 128 * clk_hz / 1e9 * 1.05, r

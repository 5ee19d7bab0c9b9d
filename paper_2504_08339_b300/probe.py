"""Shared-memory read bandwidth of the current GPU, measured with the
library's probe kernel (neat_probe_smem_read): the peak of the on-chip term of
the forward/backward roofline."""
from __future__ import annotations

import ctypes

import torch

from . import _lib

THREADS = 512
BYTES_PER_THREAD_ITER = 128  # 8 reads of 16 bytes


def smem_read(blocks: int, iters: int, sink: torch.Tensor, stream=None) -> None:
    """One probe launch (sink: int32 device tensor of blocks * 512)."""
    lib = _lib.load()
    st = stream if stream is not None else torch.cuda.current_stream(sink.device)
    _lib.check(lib.neat_probe_smem_read(blocks, iters, ctypes.c_void_p(sink.data_ptr()),
                                        ctypes.c_void_p(st.cuda_stream)), "probe_smem_read")


def smem_read_gbs(device=None, iters: int = 4096, reps: int = 5) -> dict:
    """Best-of-`reps` shared-memory read bandwidth (GB/s) over 3 CTAs per SM."""
    dev = torch.device("cuda", torch.cuda.current_device() if device is None else device)
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    blocks = 3 * sms
    sink = torch.empty(blocks * THREADS, dtype=torch.int32, device=dev)
    st = torch.cuda.current_stream(dev)
    smem_read(blocks, 64, sink, st)
    best = float("inf")
    for _ in range(reps):
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(st)
        smem_read(blocks, iters, sink, st)
        b.record(st)
        b.synchronize()
        best = min(best, a.elapsed_time(b))
    nbytes = blocks * THREADS * BYTES_PER_THREAD_ITER * iters
    return {"gbs": nbytes / (best * 1e-3) / 1e9, "ms": best, "bytes": nbytes, "blocks": blocks,
            "sms": sms}

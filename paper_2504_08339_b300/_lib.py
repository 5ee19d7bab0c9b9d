"""ctypes binding of libneat.so: the C ABI of include/neat.h under the same
names.  Argument marshalling only; every step runs in the library's kernels.

Importing this module does not build anything.  If the shared library is
missing the import of the package's compute functions fails loudly: there is
no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libneat.so")

(NEAT_OK, NEAT_ERR_ARG, NEAT_ERR_CUDA, NEAT_ERR_WORKSPACE, NEAT_ERR_UNSUPPORTED, NEAT_ERR_STATE,
 NEAT_ERR_TIMEOUT) = (0, -1, -2, -3, -4, -5, -6)
DEV_TIMEOUT, DEV_NO_SCRATCH = 1, 2
# neat_plan_validate bits (NEAT_BAD_*)
BAD_QUEUE, BAD_PACKED, BAD_COMPILED, BAD_BATCHES = 1, 2, 4, 8
G_CYCLE, G_DANGLING_KEY, G_DUP_KEY, G_DUP_EDGE, G_EDGE_INTO_INPUT, G_BAD_ATTR, G_IO_ROW_INVALID = (
    1, 2, 4, 8, 16, 32, 64)

# every symbol include/neat.h declares
SYMBOLS = ("neat_version", "neat_status_string", "neat_last_cuda_error",
           "neat_workspace_bytes", "neat_plan_create",
           "neat_plan_destroy", "neat_plan_set_tuning", "neat_plan_get_tuning",
           "neat_plan_device_errors", "neat_plan_check", "neat_plan_validate", "neat_transform",
           "neat_forward", "neat_forward_plain", "neat_backward", "neat_sum_genomes",
           "neat_hyperneat_query",
           "neat_forward_noalloc", "neat_probe_smem_read", "neat_transform_recurrent",
           "neat_forward_recurrent", "neat_distance_scratch_bytes", "neat_distance",
           "neat_apply_ops", "neat_mutate_transform", "neat_substrate_forward",
           "neat_hyperneat_substrate")


class NeatError(RuntimeError):
    pass


class neat_tuning(ctypes.Structure):
    _fields_ = [("warps_per_cta", ctypes.c_int), ("samples_per_lane", ctypes.c_int),
                ("lvl_threads", ctypes.c_int), ("small_s_max", ctypes.c_int),
                ("lvl_budget_kb", ctypes.c_int),
                ("prune_dead", ctypes.c_int), ("wait_polls", ctypes.c_int),
                ("bwd_global", ctypes.c_int)]


_lock = threading.Lock()
_lib = None


def load(path: str = LIB_PATH):
    """Load libneat.so and declare its signatures (no CUDA call is made)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(path):
            raise NeatError(f"{path} is missing: build it with "
                            "`python -m paper_2504_08339_b300.build` (no CPU fallback exists)")
        lib = ctypes.CDLL(path)
        vp, i32, i64, f32, sz = (ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_float,
                                 ctypes.c_size_t)
        sig = {
            "neat_version": (i32, []),
            "neat_status_string": (ctypes.c_char_p, [i32]),
            "neat_last_cuda_error": (i32, []),
            "neat_workspace_bytes": (sz, [i32, i32, i32, i32, i32]),
            "neat_plan_create": (i32, [ctypes.POINTER(vp), i32, i32, i32, i32, i32, vp, sz]),
            "neat_plan_destroy": (i32, [vp]),
            "neat_plan_set_tuning": (i32, [vp, ctypes.POINTER(neat_tuning)]),
            "neat_plan_get_tuning": (i32, [vp, ctypes.POINTER(neat_tuning)]),
            "neat_plan_device_errors": (i32, [vp, vp, i32, vp]),
            "neat_plan_check": (i32, [vp, vp]),
            "neat_plan_validate": (i32, [vp, vp, vp]),
            "neat_transform": (i32, [vp, vp, vp, vp, vp, vp, vp, vp]),
            "neat_forward": (i32, [vp, vp, i64, i32, vp, vp, vp]),
            "neat_forward_plain": (i32, [vp, vp, i64, i32, vp, vp]),
            "neat_sum_genomes": (i32, [vp, i32, i64, vp, vp]),
            "neat_backward": (i32, [vp, vp, i64, i32, vp, vp, vp, vp, vp, vp, vp]),
            "neat_hyperneat_query": (i32, [vp, i32, f32, vp, vp]),
            "neat_forward_noalloc": (i32, [vp, vp, i32, i32, i32, i32, i32, vp, i64, i32, vp, vp,
                                           vp]),
            "neat_probe_smem_read": (i32, [i32, i32, vp, vp]),
            "neat_transform_recurrent": (i32, [vp, vp, vp, vp, vp]),
            "neat_forward_recurrent": (i32, [vp, vp, i64, i32, i32, vp, vp]),
            "neat_distance_scratch_bytes": (sz, [i32, i32, i32]),
            "neat_apply_ops": (i32, [vp, vp, i32, i32, i32, vp, i32, vp, vp]),
            "neat_substrate_forward": (i32, [vp, i32, i32, vp, i64, i32, i32, vp, vp]),
            "neat_hyperneat_substrate": (i32, [vp, i32, f32, vp, i64, i32, i32, vp, vp, vp]),
            "neat_mutate_transform": (i32, [vp, vp, vp, vp, i32, vp, vp, vp, vp, vp, vp]),
            "neat_distance": (i32, [vp, vp, vp, i32, i32, i32, i32, i32, f32, f32, vp, vp, sz, vp]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


def check(code: int, what: str = "") -> None:
    if code != NEAT_OK:
        lib = load()
        msg = lib.neat_status_string(code).decode()
        if code == NEAT_ERR_CUDA:
            msg += f" (cudaError {lib.neat_last_cuda_error()})"
        raise NeatError(f"{what}: {msg} ({code})")

"""B300-native (sm_103a) population-wide NEAT network evaluation.

The compute path is libneat.so (hand-written CUDA kernels behind the C ABI of
include/neat.h); this package is its thin Python binding:

  _lib     ctypes declarations of the C ABI, same names as the header
  api      Plan (workspace, transform, forward, backward, HyperNEAT query) and a
           torch.autograd.Function over forward/backward
  rollout  CUDA-graph capture of a multi-step rollout
  build    nvcc build of libneat.so in-tree
"""
from ._lib import NeatError, load  # noqa: F401

__all__ = ["NeatError", "load", "Plan", "evaluate", "NeatFunction"]


def __getattr__(name):
    if name in ("Plan", "evaluate", "NeatFunction", "Transformed"):
        from . import api
        return getattr(api, name)
    raise AttributeError(name)

"""CPU checks of the C ABI library: it loads, exports every symbol the header
declares, and its host-only entry points behave (no GPU needed)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2504_08339_b300 import build, _lib
    build.build()
    return _lib.load()


def _declared():
    src = open(os.path.join(ROOT, "include", "neat.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(neat_[a-z_]+)\s*\(", src)))


def test_every_declared_symbol_is_exported(lib):
    from paper_2504_08339_b300 import _lib
    declared = _declared()
    assert len(declared) >= 12
    for name in declared:
        assert hasattr(lib, name), name
    assert sorted(_lib.SYMBOLS) == declared


def test_host_only_entry_points(lib):
    assert lib.neat_version() == 100
    assert lib.neat_status_string(0) == b"ok"
    assert lib.neat_status_string(-3) == b"workspace too small"
    n = lib.neat_workspace_bytes(10000, 128, 512, 27, 8)
    assert n > 10000 * (128 * 16 + 512 * 8) * 2
    assert lib.neat_workspace_bytes(0, 16, 32, 3, 1) > 0
    assert lib.neat_workspace_bytes(-1, 16, 32, 3, 1) == 0
    assert lib.neat_workspace_bytes(1, 3, 32, 3, 1) == 0          # N < I + O
    assert lib.neat_workspace_bytes(1, 1025, 32, 3, 1) == 0       # N over the limit
    assert lib.neat_workspace_bytes(1, 16, 9000, 3, 1) == 0       # C over the limit
    assert lib.neat_workspace_bytes(1, 16, 0, 3, 1) == 0
    # argument errors are returned before any CUDA call
    assert lib.neat_plan_create(None, 1, 16, 32, 3, 1, None, 0) == -1
    h = ctypes.c_void_p()
    assert lib.neat_plan_create(ctypes.byref(h), 1, 3, 32, 3, 1, None, 0) == -4
    assert lib.neat_plan_destroy(None) == -1
    assert lib.neat_transform(None, None, None, None, None, None, None, None) == -1
    assert lib.neat_forward(None, None, 0, 1, None, None, None) == -1


def test_library_is_built_for_sm_103a():
    from paper_2504_08339_b300 import build
    lib = build.build()
    assert "arch=compute_103a,code=sm_103a" in " ".join(build.ARCH)
    assert os.path.getsize(lib) > 0

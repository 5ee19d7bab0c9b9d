"""Host-side choices of the binding that need no GPU: the autograd
function's store-or-recompute rule and the autotuner's candidate sets."""
from types import SimpleNamespace

from paper_2504_08339_b300 import api, autotune


def test_store_rule_is_the_byte_budget():
    plan = SimpleNamespace(P=2048, N=64, C=256, I=2, O=1)
    S = 4096
    need = api.saved_bytes(plan, S)
    assert need == 4 * 2048 * 64 * 4096  # 2 GiB
    assert api.choose_store(plan, S, need)
    assert not api.choose_store(plan, S, need - 1)
    assert api.choose_store(plan, S)  # under the default budget
    assert not api.choose_store(plan, 65536 * 8)  # 32 GiB: above it
    assert api.SAVED_BUDGET_BYTES == 8 << 30


def test_autotune_candidates_cover_both_forms_and_respect_ragged_tiles():
    plan = SimpleNamespace(P=10, N=128, C=512, I=27, O=8)
    small = autotune.candidates(plan, 1)
    assert any("lvl_budget_kb" in c for c in small)
    assert all(c.get("samples_per_lane", 1) == 1 for c in small)  # S < 32 spl
    big = autotune.candidates(plan, 64)
    assert not any("lvl_budget_kb" in c for c in big)
    assert {c["samples_per_lane"] for c in big} == {1, 2}

"""The roofline bookkeeping of bench.py, on CPU: the algorithmic bytes of a
step and the reading of the committed ncu summary."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402
import pytest  # noqa: E402

import bench  # noqa: E402


def test_algorithmic_bytes_of_a_step():
    # two steps of counters: each interference op (R^dag, H P H, R) streams its
    # input and output once, at 8 W_live + B_amp bytes per branch with
    # W_live = ceil((4 nb + 18) / 64) key words
    stats = {"in": 200, "after_rdag": 300, "after_h1": 0, "after_hph": 320, "out": 310, "steps": 2}
    b_alg, b_min = bench.algorithmic_bytes(stats, nb=14, amp_bytes=8)
    entry = 8 * 2 + 8  # nb = 14: 74 bits -> 2 words
    assert b_alg == ((200 + 300) + (300 + 320) + (320 + 310)) * entry / 2
    assert b_min == (200 + 310) * (8 + 8) / 2
    b_alg1, _ = bench.algorithmic_bytes(stats, nb=11, amp_bytes=16)  # 62 bits -> 1 word
    assert b_alg1 == ((200 + 300) + (300 + 320) + (320 + 310)) * (8 + 16) / 2
    # the literal schedule adds the first H as its own op
    stats["after_h1"] = 900
    b_lit, _ = bench.algorithmic_bytes(stats, nb=14, amp_bytes=8)
    assert b_lit == ((200 + 300) + (300 + 900) + (900 + 320) + (320 + 310)) * entry / 2


@pytest.mark.parametrize("attr,variant", [("PROFILE_SLOT", 4), ("PROFILE_POS", 7)])
def test_profiled_traffic_follows_the_kernel_source_hash(tmp_path, monkeypatch, attr, variant):
    text = open(getattr(bench, attr)).read()
    committed = bench.profiled_traffic("fp32", variant)
    if f"`{bench.kernel_hash()}`" in text:
        assert committed is not None and committed > 0
    stale = tmp_path / "stale.md"
    stale.write_text(text.replace("kernel_source_sha256_16: `", "kernel_source_sha256_16: `0"))
    monkeypatch.setattr(bench, attr, str(stale))
    assert bench.profiled_traffic("fp32", variant) is None


def test_kernel_names_follow_the_variant():
    assert bench.kernel_name(7) == "k_walk_pos<float2, s = 16>"
    assert bench.kernel_name(4) == "k_walk_slot<float2, s = 16>"
    assert bench.kernel_name(0).startswith("k_walk<float2, rows")


def test_state_error_over_the_union_of_keys():
    """The bench's per-result error: equal keys give the amplitude differences;
    a key held by one side only counts as amplitude 0 on the other."""
    regs = np.array([[0, 1, 0, 0, 2, 1, 0], [0, 3, 1, 0, 0, 0, 0], [0, 2, 0, 0, 1, 0, 0]], dtype=np.uint64)
    a = np.array([0.5 + 0.5j, -0.25, 0.1j])
    st = bench.state_error((regs, a), (regs[::-1], a[::-1]))
    assert st["max_abs"] == 0.0 and st["keys_equal"] and st["keys"] == 3
    b = a.copy()
    b[1] += 1e-7
    st = bench.state_error((regs, b), (regs[:2], a[:2]))
    assert not st["keys_equal"] and st["one_sided"] == 1
    assert abs(st["one_sided_max_abs"] - 0.1) < 1e-15
    assert abs(st["max_abs"] - 0.1) < 1e-15
    assert abs(st["l2"] - np.hypot(0.1, 1e-7)) < 1e-15

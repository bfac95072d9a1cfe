"""The roofline bookkeeping of bench.py, on CPU: the algorithmic bytes of a
step and the reading of the committed ncu summary."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

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


def test_profiled_traffic_follows_the_kernel_source_hash(tmp_path, monkeypatch):
    text = open(bench.PROFILE).read()
    committed = bench.profiled_traffic("fp32")
    if f"`{bench.kernel_hash()}`" in text:
        assert committed is not None and committed > 0
    stale = tmp_path / "stale.md"
    stale.write_text(text.replace("kernel_source_sha256_16: `", "kernel_source_sha256_16: `0"))
    monkeypatch.setattr(bench, "PROFILE", str(stale))
    assert bench.profiled_traffic("fp32") is None

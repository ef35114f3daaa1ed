"""The autotuner's table (host logic only): nearest-bucket lookup per
workload class, defaults when untuned, JSON round trip."""
from paper_1610_03007_gb300 import autotune


def test_table_lookup_and_roundtrip(tmp_path):
    path = str(tmp_path / "t.json")
    t = autotune.Table(path)
    assert t.get("zipf", 1 << 28) == autotune.DEFAULTS
    t.put("zipf", 1 << 28, {"sort_items": 12, "refine_shape": 2}, 120.0)
    t.put("zipf", 1 << 20, {"sort_items": 8, "refine_shape": 1}, 1.0)
    t.put("dna", 1 << 31, {"sort_items": 16, "refine_shape": 3}, 900.0)
    t.save()
    u = autotune.Table(path)
    assert u.get("zipf", (1 << 28) + 5) == {"sort_items": 12, "refine_shape": 2}
    assert u.get("zipf", 1 << 21) == {"sort_items": 8, "refine_shape": 1}
    assert u.get("dna", 1 << 10) == {"sort_items": 16, "refine_shape": 3}
    assert u.get("markov", 1 << 28) == autotune.DEFAULTS


def test_buckets():
    assert autotune.bucket(1) == 0
    assert autotune.bucket(1 << 28) == 28
    assert autotune.bucket((1 << 28) - 1) == 27


def test_key_width_candidates_fill_whole_digit_passes():
    # batched DNA: 2 bits per character, 12 text-id bits -> 7..3 passes
    assert autotune.key_width_candidates(26, 2) == [22, 18, 14, 10, 6]
    # one text over 8-bit characters: 8 characters fill 64 bits
    assert autotune.key_width_candidates(8, 8) == [7, 6, 5, 4, 3]
    # nothing at or above the maximum, nothing below two characters
    assert all(2 <= c < 4 for c in autotune.key_width_candidates(4, 8))

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

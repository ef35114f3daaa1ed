"""The autotuner's table (host logic only, no GPU): the Python writer and
the library's reader agree on the format and on the nearest-bucket rule,
malformed files are refused, entries are kept per class, and the knobs'
candidate sets."""
import numpy as np
import pytest

from paper_1610_03007_gb300 import autotune


@pytest.fixture()
def gb():
    from paper_1610_03007_gb300 import _build
    _build.build()
    import paper_1610_03007_gb300 as g
    g.load()
    yield g
    # put the library's default table back for the tests that follow
    import os
    g.tuning_load(autotune.DEFAULT_TABLE if os.path.exists(autotune.DEFAULT_TABLE) else None)


def test_table_roundtrip_and_lookup(tmp_path):
    path = str(tmp_path / "t.txt")
    t = autotune.Table(path)
    assert t.get(False, 8, 1 << 28) == autotune.DEFAULTS
    t.put(False, 8, 1 << 28, {"sort_items": 12, "refine_shape": 2}, "zipf")
    t.put(False, 8, 1 << 20, {"sort_items": 8, "refine_shape": 1, "bucket_min": 1 << 20})
    t.put(False, 2, 1 << 31, {"sort_items": 16, "refine_shape": 3, "h0_chars": 28})
    t.put(True, 2, 1 << 30, {"sort_items": 12, "h0_chars": 14})
    t.save()
    u = autotune.Table(path)
    assert u.get(False, 8, (1 << 28) + 5)["sort_items"] == 12
    assert u.get(False, 8, 1 << 21) == {"sort_items": 8, "refine_shape": 1, "h0_chars": 0,
                                        "bucket_min": 1 << 20}
    assert u.get(False, 2, 1 << 10)["h0_chars"] == 28  # nearest bucket of its class
    assert u.get(True, 2, 1 << 31)["h0_chars"] == 14
    assert u.get(True, 8, 1 << 31) == autotune.DEFAULTS   # no entry of that class
    assert u.get(False, 4, 1 << 28) == autotune.DEFAULTS


def test_library_reads_the_written_table(gb, tmp_path):
    path = str(tmp_path / "tuning.txt")
    t = autotune.Table(path)
    t.put(False, 2, 1 << 31, {"sort_items": 12, "refine_shape": 4, "h0_chars": 28,
                              "bucket_min": 0xFFFFFFFF})
    t.put(False, 2, 1 << 16, {"sort_items": 8, "refine_shape": 2, "h0_chars": 0,
                              "bucket_min": 1 << 20})
    t.put(True, 2, 1 << 30, {"sort_items": 16, "refine_shape": 0, "h0_chars": 14,
                             "bucket_min": 0})
    t.save()
    gb.tuning_load(path)
    for batched, bits, n in ((0, 2, 1 << 31), (0, 2, 1 << 25), (0, 2, 1 << 22), (0, 2, 100),
                             (1, 2, 2 * 10**9), (1, 2, 1000), (0, 8, 1 << 28), (1, 8, 5)):
        got, count = gb.tuning_lookup(batched, bits, n)
        assert count == 3
        want = t.get(bool(batched), bits, n) if (batched, bits) in ((0, 2), (1, 2)) else None
        if want is None:
            assert got == {f: 0 for f in autotune.FIELDS}
        else:
            assert got == want, (batched, bits, n)
    # sa_tuning_set adds and removes single entries
    gb.tuning_set(0, 8, 28, {"sort_items": 12, "refine_shape": 1, "h0_chars": 6,
                             "bucket_min": 1 << 24})
    assert gb.tuning_lookup(0, 8, 1 << 27)[0]["h0_chars"] == 6
    gb.tuning_set(0, 8, 28, None)
    assert gb.tuning_lookup(0, 8, 1 << 27) == ({f: 0 for f in autotune.FIELDS}, 3)


def test_library_refuses_malformed_tables(gb, tmp_path):
    gb.tuning_load(None)
    gb.tuning_set(0, 2, 20, {"sort_items": 8, "refine_shape": 1, "h0_chars": 0,
                             "bucket_min": 0})
    for body in ("0 2 20 8 1 0\n", "0 9 20 8 1 0 0\n", "2 2 20 8 1 0 0\n",
                 "0 2 40 8 1 0 0\n", "0 2 20 8 1 0 0 7\n"):
        p = tmp_path / "bad.txt"
        p.write_text("# header\n" + body)
        with pytest.raises(gb.SAError):
            gb.tuning_load(str(p))
        assert gb.tuning_lookup(0, 2, 1 << 20) == ({"sort_items": 8, "refine_shape": 1,
                                                    "h0_chars": 0, "bucket_min": 0}, 1)
    with pytest.raises(gb.SAError):
        gb.tuning_load(str(tmp_path / "missing.txt"))
    with pytest.raises(gb.SAError):
        gb.tuning_set(2, 2, 20, None)
    with pytest.raises(gb.SAError):
        gb.tuning_set(0, 0, 20, None)


def test_committed_table_parses_if_present():
    """The table shipped beside the library is in the library's format."""
    import os
    if not os.path.exists(autotune.DEFAULT_TABLE):
        pytest.skip("no tuning table committed")
    t = autotune.Table()
    assert t.entries
    for (b, bits, lg), p in t.entries.items():
        assert b in (0, 1) and 1 <= bits <= 8 and 0 <= lg <= 31
        assert p["sort_items"] in (0, 8, 12, 16) and 0 <= p["refine_shape"] <= 4


def test_widest_key_is_explicit():
    """The tuner passes the full key width as a number (0 would mean "the
    library's table" to the library)."""
    assert autotune.widest_key(2) == 32 and autotune.widest_key(8) == 8
    assert autotune.widest_key(2, 4096) == 26 and autotune.widest_key(8, 2) == 7
    assert autotune.widest_key(1, 1) == 64


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
    assert np.all(np.diff(autotune.BUCKET_MINS) > 0)

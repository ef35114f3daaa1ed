"""bench.py's reporting, on the host: the roofline arithmetic of its JSON
line and the link between the committed ncu summaries and the kernel
sources they were captured from (a summary counts only while its kernel's
sources are unchanged, so `traffic` is reported for the current kernels)."""
import glob
import os
import re
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def summaries():
    out = []
    for p in sorted(glob.glob(os.path.join(ROOT, "profiles", "ncu_*.md"))):
        m = re.fullmatch(r"ncu_(\w+?)_(markov|zipf)\.md", os.path.basename(p))
        if m:
            out.append(m.groups())
    return out


def test_summaries_exist_for_the_dominant_kernels():
    have = set(summaries())
    assert ("onesweep", "markov") in have   # the 2^31 headline's dominant kernel
    assert ("refine", "zipf") in have       # the 2^28 repeated-Zipf text's


@pytest.mark.parametrize("kernel,workload", summaries())
def test_summary_matches_the_current_sources(kernel, workload):
    """Each summary names the hash of the sources it was captured from; it
    must be today's, and its DRAM bytes per algorithmic byte a plausible
    ratio (re-reads would show as well above 1)."""
    ratio = bench.ncu_traffic(kernel, workload)
    assert ratio is not None, f"profiles/ncu_{kernel}_{workload}.md is stale"
    assert 0.5 < ratio < 2.0


def test_stale_or_unknown_summaries_give_no_traffic(tmp_path, monkeypatch):
    assert bench.ncu_traffic("no_such_kernel", "markov") is None
    assert bench.ncu_traffic("onesweep", "no_such_workload") is None
    # a summary whose hash is not the sources' is ignored
    prof = tmp_path / "profiles"
    prof.mkdir()
    (prof / "ncu_onesweep_markov.md").write_text(
        "source_sha256_16: 0123456789abcdef\ndram_bytes_per_algorithmic_byte: 1.0\n")
    real = bench.kernel_source_hash("onesweep")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "kernel_source_hash", lambda k: real)
    assert bench.ncu_traffic("onesweep", "markov") is None
    (prof / "ncu_onesweep_markov.md").write_text(
        f"source_sha256_16: {real}\ndram_bytes_per_algorithmic_byte: 1.25\n")
    assert bench.ncu_traffic("onesweep", "markov") == 1.25


def test_roofline_of_the_dominant_kernel(monkeypatch):
    """achieved = algorithmic bytes / event time of the kernel with the most
    event time; frac against the peak; traffic = the summary's ratio times
    the bytes of one launch."""
    monkeypatch.setattr(bench, "peaks", lambda: (8000.0, "measured"))
    monkeypatch.setattr(bench, "ncu_traffic", lambda k, w: 1.5 if k == "onesweep" else None)
    kern = {"onesweep": {"ms": 100.0, "launches": 10, "bytes": 400e9},
            "refine": {"ms": 40.0, "launches": 14, "bytes": 20e9},
            "rename": {"ms": 0.0, "launches": 0, "bytes": 0}}
    r = bench._roofline(kern, "markov")
    assert r["kernel"] == "onesweep" and r["bound"] == "hbm" and r["unit"] == "GB/s"
    assert r["achieved"] == pytest.approx(4000.0)
    assert r["frac"] == pytest.approx(0.5)
    assert r["bytes_per_launch"] == pytest.approx(40e9)
    assert r["ms_per_launch"] == pytest.approx(10.0)
    assert r["traffic"] == pytest.approx(60e9)
    kern["refine"]["ms"] = 200.0
    r = bench._roofline(kern, "markov")
    assert r["kernel"] == "refine" and r["traffic"] is None
    assert r["achieved"] == pytest.approx(100.0)


def test_kernel_table_per_step():
    t = bench._kernel_table({"onesweep": {"ms": 30.0, "launches": 9, "bytes": 60e9},
                             "apply": {"ms": 0.0, "launches": 0, "bytes": 0}}, steps=3)
    assert set(t) == {"onesweep"}
    assert t["onesweep"]["ms_per_step"] == pytest.approx(10.0)
    assert t["onesweep"]["launches_per_step"] == pytest.approx(3.0)
    assert t["onesweep"]["gbs"] == pytest.approx(2000.0)

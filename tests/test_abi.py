"""The C-ABI library (no GPU needed): it builds for sm_103a, loads, exports
every entry point include/gbsa.h declares, and rejects bad arguments on
the host before touching a GPU."""
import ctypes
import os
import re

import numpy as np
import pytest

from conftest import ROOT


@pytest.fixture(scope="module")
def lib():
    from paper_1610_03007_gb300 import _build
    _build.build()
    import paper_1610_03007_gb300 as gbsa
    return gbsa.load()


def declared_symbols():
    with open(os.path.join(ROOT, "include", "gbsa.h")) as f:
        text = f.read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(sa_\w+)\s*\(", text, flags=re.M)))


def test_header_declares_the_boundary():
    syms = declared_symbols()
    for s in ("sa_build", "sa_build_batched", "sa_build_ex", "sa_workspace_bytes",
              "sa_status_string", "sa_build_host", "sa_sort_pairs"):
        assert s in syms


def test_every_declared_symbol_is_exported(lib):
    import paper_1610_03007_gb300 as gbsa
    syms = declared_symbols()
    missing = [s for s in syms if not hasattr(lib, s)]
    assert not missing
    assert sorted(gbsa.EXPORTED) == syms


def test_status_strings(lib):
    import paper_1610_03007_gb300 as gbsa
    for code, name in gbsa.STATUS_NAMES.items():
        assert gbsa.status_string(code) == name


def test_host_side_argument_checks(lib):
    # These return before any CUDA call, so they run without a GPU.
    assert lib.sa_build(None, (1 << 31) + 1, None, None) == 2      # too large
    assert lib.sa_build(None, 10, None, None) == 1                 # null pointers
    assert lib.sa_build(None, 0, None, None) == 0                  # empty text: ok
    off = np.array([0, 5, 3], dtype=np.uint64)                     # decreasing
    assert lib.sa_build_batched(None, off.ctypes.data, 2, None, None) == 1
    off = np.array([1, 5], dtype=np.uint64)                        # offsets[0] != 0
    assert lib.sa_build_batched(None, off.ctypes.data, 1, None, None) == 1
    off = np.array([0, (1 << 31) + 1], dtype=np.uint64)
    assert lib.sa_build_batched(None, off.ctypes.data, 1, None, None) == 2
    assert lib.sa_sort_pairs(None, None, 10, 8, 8, None, 0, None) == 1   # empty bit range
    assert lib.sa_sort_pairs(None, None, 10, 0, 65, None, 0, None) == 1
    # BWT: NULL outputs, NULL inputs with n > 0, n above 2^31 (no GPU work)
    assert lib.sa_bwt(None, 0, None, None, None, None) == 1
    assert lib.sa_bwt(None, 5, None, 8, 8, None) == 1
    assert lib.sa_bwt(8, (1 << 31) + 1, 8, 8, 8, None) == 2
    # LCP: NULL arrays with n > 0, n above 2^31, a short or misaligned
    # workspace; n = 0 does nothing (no GPU work in any of these)
    assert lib.sa_lcp(None, 5, None, None, None, 0, None) == 1
    assert lib.sa_lcp(8, (1 << 31) + 1, 8, 8, None, 0, None) == 2
    assert lib.sa_lcp(256, 100, 256, 256, 256, 10, None) == 1
    assert lib.sa_lcp(256, 100, 256, 256, 257, 1 << 20, None) == 1
    assert lib.sa_lcp(None, 0, None, None, None, 0, None) == 0
    assert lib.sa_lcp_workspace_bytes(1000) >= 8000
    # DC3: NULL arrays with n > 0, n above 2^31, n = 0 (no GPU work)
    assert lib.sa_build_dc3(None, 5, None, None, None) == 1
    assert lib.sa_build_dc3(8, (1 << 31) + 1, 8, None, None) == 2
    assert lib.sa_build_dc3(None, 0, None, None, None) == 0
    # DC7: the same argument checks
    assert lib.sa_build_dc7(None, 5, None, None, None) == 1
    assert lib.sa_build_dc7(8, (1 << 31) + 1, 8, None, None) == 2
    assert lib.sa_build_dc7(None, 0, None, None, None) == 0
    # prefix doubling using sorting: the same argument checks
    assert lib.sa_build_pd_sort(None, 5, None, None, 0, None, None) == 1
    assert lib.sa_build_pd_sort(8, (1 << 31) + 1, 8, None, 0, None, None) == 2
    assert lib.sa_build_pd_sort(None, 0, None, None, 0, None, None) == 0


def test_workspace_model(lib):
    # About 67 bytes per character: keys A/B (16), values A/B (8), two
    # active lists (16), the update list (8), ISA (4), group starts, names
    # and head ranks x2 plus parent names (14) and look-back status; plus
    # about 1 MiB whatever n (the position-bucketing counts).
    for n in (1 << 20, 1 << 28, 1 << 31):
        b = lib.sa_workspace_bytes(n)
        assert 66 * n < b < 68 * n + (2 << 20)


def test_multiplier_option_is_checked_on_the_host(lib):
    """sa_options.multiplier outside {0, 2, 3, 4} is refused before any GPU
    work, on the single and the batched entry points; n = 0 with a valid
    multiplier returns at once."""
    import paper_1610_03007_gb300 as gbsa
    for bad in (1, 5, 64):
        opt = gbsa.Options(multiplier=bad)
        assert lib.sa_build_ex(8, 100, 8, None, None, 0, ctypes.byref(opt), None, None) == 1
        off = np.array([0, 100], dtype=np.uint64)
        assert lib.sa_build_batched_ex(8, off.ctypes.data, 1, 8, None, 0, ctypes.byref(opt),
                                       None, None) == 1
    for good in (0, 2, 3, 4):
        opt = gbsa.Options(multiplier=good)
        assert lib.sa_build_ex(None, 0, None, None, None, 0, ctypes.byref(opt), None, None) == 0


def test_initial_keys_option_is_checked_on_the_host(lib):
    """sa_options.initial_keys outside {0, 1, 2} is refused before any GPU
    work; the valid values with n = 0 return at once."""
    import paper_1610_03007_gb300 as gbsa
    for bad in (3, 7, 0xFFFFFFFF):
        opt = gbsa.Options(initial_keys=bad)
        assert lib.sa_build_ex(8, 100, 8, None, None, 0, ctypes.byref(opt), None, None) == 1
    for good in (0, 1, 2):
        opt = gbsa.Options(initial_keys=good)
        assert lib.sa_build_ex(None, 0, None, None, None, 0, ctypes.byref(opt), None, None) == 0


def test_tile_options_are_checked_on_the_host(lib):
    """sort_items outside {0, 8, 12, 16} and refine_shape above 4 are refused
    before any GPU work, by the single and the batched build."""
    import paper_1610_03007_gb300 as gbsa
    off = (ctypes.c_uint64 * 3)(0, 50, 100)
    for kw in ({"sort_items": 7}, {"sort_items": 24}, {"sort_items": 1}, {"refine_shape": 5},
               {"refine_shape": 0xFFFFFFFF}):
        opt = gbsa.Options(**kw)
        assert lib.sa_build_ex(8, 100, 8, None, None, 0, ctypes.byref(opt), None, None) == 1
        assert lib.sa_build_batched_ex(8, off, 2, 8, None, 0, ctypes.byref(opt), None, None) == 1
    for kw in ({"sort_items": 8}, {"sort_items": 12}, {"sort_items": 16}, {"refine_shape": 4}):
        opt = gbsa.Options(**kw)
        assert lib.sa_build_ex(None, 0, None, None, None, 0, ctypes.byref(opt), None, None) == 0


def test_batched_host_build_checks_its_arguments_on_the_host(lib):
    """sa_build_batched_host refuses malformed calls before touching the
    device, and a batch of empty texts returns at once."""
    vp3 = ctypes.c_void_p * 3
    ln = (ctypes.c_uint64 * 3)(0, 0, 0)
    texts, sas = vp3(None, None, None), vp3(None, None, None)
    assert lib.sa_build_batched_host(texts, ln, sas, 0, None) == 1     # count = 0
    assert lib.sa_build_batched_host(None, ln, sas, 3, None) == 1      # NULL arrays
    assert lib.sa_build_batched_host(texts, None, sas, 3, None) == 1
    assert lib.sa_build_batched_host(texts, ln, None, 3, None) == 1
    assert lib.sa_build_batched_host(texts, ln, sas, 3, None) == 0     # all empty
    assert lib.sa_build_batched_host(texts, ln, sas, (1 << 20) + 1, None) == 2
    buf = (ctypes.c_uint8 * 8)()
    out = (ctypes.c_uint32 * 8)()
    ln[1] = 5
    assert lib.sa_build_batched_host(texts, ln, sas, 3, None) == 1     # NULL non-empty text
    texts[1], sas[1] = ctypes.addressof(buf), ctypes.addressof(out)
    ln[2] = (1 << 31) + 1
    assert lib.sa_build_batched_host(texts, ln, sas, 3, None) == 2     # one text too long
    ln[0], ln[2] = 1 << 30, 1 << 30
    texts[0] = texts[2] = ctypes.addressof(buf)
    sas[0] = sas[2] = ctypes.addressof(out)
    assert lib.sa_build_batched_host(texts, ln, sas, 3, None) == 2     # total above 2^31


def test_binding_fails_loudly_without_the_library_or_a_gpu_tensor():
    """No CPU fallback: a missing library and a host tensor both raise."""
    import torch

    import paper_1610_03007_gb300 as gbsa
    with pytest.raises(RuntimeError, match="not built"):
        gbsa.load(os.path.join(ROOT, "no_such_dir", "libgbsa.so"))
    with pytest.raises(TypeError):
        gbsa.sa_build(torch.zeros(16, dtype=torch.uint8))
    with pytest.raises(TypeError):
        gbsa.sa_build_dc7(torch.zeros(16, dtype=torch.uint8))


def test_no_alloc_limit_matches_its_scratch_array(lib):
    """sa_build_noalloc's scratch array is 20 MiB and its text limit 2^18
    bytes: the build workspace at that limit must fit the array (the entry
    point also checks this on every call), and the pool query refuses NULL
    outputs without touching a GPU."""
    assert lib.sa_workspace_bytes(1 << 18) <= 20 << 20
    assert lib.sa_workspace_bytes((1 << 18) + 4096) > lib.sa_workspace_bytes(1 << 18)
    assert lib.sa_build_noalloc(None, (1 << 18) + 1, None, None) == 2
    assert lib.sa_pool_usage(None, None) == 1


def test_binding_refuses_buffers_the_library_could_overrun():
    """The binding checks every caller-provided buffer before a call: output
    arrays of the wrong element size, length or layout, read-only arrays and
    non-CUDA tensors are refused with ValueError, so no kernel or copy can
    run past a buffer."""
    import torch

    import paper_1610_03007_gb300 as gbsa
    text = np.frombuffer(b"mississippi", dtype=np.uint8)
    good = np.empty(text.size, np.uint32)
    assert gbsa._host_out(good, text.size, "out") is good
    bad = [np.empty(text.size, np.uint64), np.empty(text.size - 1, np.uint32),
           np.empty(2 * text.size, np.uint32)[::2]]
    ro = np.empty(text.size, np.uint32)
    ro.flags.writeable = False
    bad.append(ro)
    for b in bad:
        with pytest.raises(ValueError):
            gbsa._host_out(b, text.size, "out")
        with pytest.raises(ValueError):
            gbsa.sa_build_host(text, sa_out=b)
        with pytest.raises(ValueError):
            gbsa.sa_build_batched_host([text], [b])
    with pytest.raises(ValueError):
        gbsa.sa_build_batched_host([text, text], [good])
    with gbsa.Server(budget_bytes=1 << 30, slots=1, simulate_ns_per_byte=1.0) as srv:
        for b in bad:
            with pytest.raises(ValueError):
                srv.submit(text, out=b)
    cpu = torch.zeros(16, dtype=torch.int32)
    with pytest.raises(ValueError):
        gbsa._dev_buf(cpu, "sa_out", torch.device("cuda:0"), 4, 16)
    with pytest.raises(ValueError):
        gbsa._dev_ws(cpu, torch.device("cuda:0"))
    assert gbsa._dev_ws(None, torch.device("cuda:0")) == (None, 0)
    with pytest.raises(ValueError):
        gbsa.sa_sort_pairs(torch.zeros(8, dtype=torch.int64), torch.zeros(8, dtype=torch.int32))

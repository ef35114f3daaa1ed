"""GPU unit tests of the building blocks through the C-ABI: the one-sweep
radix sort (stability, ragged sizes, skipped digits, bit ranges, both
ranking methods), the batched build, and the bounded-wait failure path."""
import numpy as np
import pytest

import gen

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gb():
    import __graft_entry__
    __graft_entry__.build()
    import paper_1610_03007_gb300 as gbsa
    return gbsa


def sort_on_gpu(gb, keys, vals, lo, hi):
    import torch
    k = torch.from_numpy(keys.view(np.int64).copy()).cuda()
    v = torch.from_numpy(vals.view(np.int32).copy()).cuda()
    gb.sa_sort_pairs(k, v, lo, hi)
    torch.cuda.synchronize()
    return k.cpu().numpy().view(np.uint64), v.cpu().numpy().view(np.uint32)


def reference_sort(keys, vals, lo, hi):
    """numpy's stable sort on the selected key bits."""
    span = hi - lo
    mask = np.uint64((1 << span) - 1) if span < 64 else np.uint64(0xFFFFFFFFFFFFFFFF)
    sel = (keys >> np.uint64(lo)) & mask
    order = np.argsort(sel, kind="stable")
    return keys[order], vals[order]


@pytest.mark.parametrize("m", [2, 31, 4095, 4096, 4097, 100003, 1 << 20])
def test_sort_random_keys(gb, m):
    rng = np.random.default_rng(m)
    keys = rng.integers(0, 2**63, m, dtype=np.uint64) * np.uint64(2) + rng.integers(0, 2, m, dtype=np.uint64)
    vals = np.arange(m, dtype=np.uint32)
    gk, gv = sort_on_gpu(gb, keys, vals, 0, 64)
    rk, rv = reference_sort(keys, vals, 0, 64)
    assert np.array_equal(gk, rk) and np.array_equal(gv, rv)


@pytest.mark.parametrize("lo,hi", [(0, 8), (0, 13), (5, 37), (40, 64), (56, 64), (63, 64)])
def test_sort_bit_ranges_are_stable(gb, lo, hi):
    m = 200001
    rng = np.random.default_rng(lo * 100 + hi)
    keys = rng.integers(0, 2**63, m, dtype=np.uint64)
    vals = rng.integers(0, 2**32, m, dtype=np.uint64).astype(np.uint32)
    gk, gv = sort_on_gpu(gb, keys, vals, lo, hi)
    rk, rv = reference_sort(keys, vals, lo, hi)
    assert np.array_equal(gk, rk) and np.array_equal(gv, rv)


@pytest.mark.parametrize("m", [4097, 300007])
def test_sort_mixed_digit_entropy(gb, m):
    """Passes ranked both ways in one sort: the plan ranks a pass with
    match.any when its histogram predicts few distinct digits per warp
    (bits 8-15 Zipf-skewed, bits 24-31 two values, bits 40-47 one value in
    ninety) and with the shared-memory masks otherwise (bits 0-7 and 32-39
    uniform); bits 16-23 are constant (skipped). Stable, element-wise."""
    rng = np.random.default_rng(m + 5)
    u = lambda lo_, hi_: rng.integers(lo_, hi_, m, dtype=np.uint64)
    zipf = np.minimum(rng.zipf(1.3, m), 255).astype(np.uint64)
    rare = np.where(rng.random(m) < 1 / 90, np.uint64(7), np.uint64(3))
    keys = (u(0, 256) | (zipf << np.uint64(8)) | (np.uint64(0x5A) << np.uint64(16))
            | (u(0, 2) << np.uint64(24)) | (u(0, 256) << np.uint64(32)) | (rare << np.uint64(40)))
    vals = np.arange(m, dtype=np.uint32)
    gk, gv = sort_on_gpu(gb, keys, vals, 0, 48)
    rk, rv = reference_sort(keys, vals, 0, 48)
    assert np.array_equal(gk, rk) and np.array_equal(gv, rv)


def test_sort_degenerate_key_sets(gb):
    m = 300000
    vals = np.arange(m, dtype=np.uint32)
    same = np.full(m, 0x1234_5678_9ABC_DEF0, dtype=np.uint64)  # every digit constant
    gk, gv = sort_on_gpu(gb, same, vals, 0, 64)
    assert np.array_equal(gk, same) and np.array_equal(gv, vals)
    rng = np.random.default_rng(3)
    high = rng.integers(0, 256, m, dtype=np.uint64) << np.uint64(56)  # only the top digit varies
    gk, gv = sort_on_gpu(gb, high, vals, 0, 64)
    rk, rv = reference_sort(high, vals, 0, 64)
    assert np.array_equal(gk, rk) and np.array_equal(gv, rv)
    few = rng.integers(0, 3, m, dtype=np.uint64)  # heavy ties: stability matters
    gk, gv = sort_on_gpu(gb, few, vals, 0, 64)
    rk, rv = reference_sort(few, vals, 0, 64)
    assert np.array_equal(gk, rk) and np.array_equal(gv, rv)
    desc = np.arange(m, 0, -1, dtype=np.uint64)
    gk, gv = sort_on_gpu(gb, desc, vals, 0, 64)
    rk, rv = reference_sort(desc, vals, 0, 64)
    assert np.array_equal(gk, rk) and np.array_equal(gv, rv)


def batched_reference(orc, flat, off):
    out = np.empty(flat.size, dtype=np.uint32)
    for k in range(off.size - 1):
        a, b = int(off[k]), int(off[k + 1])
        out[a:b] = orc.pd_sa(flat[a:b])[0]
    return out


def run_batched(gb, flat, off, **opt):
    import torch
    sa = gb.sa_build_batched(torch.from_numpy(flat).cuda(), off, **opt)
    torch.cuda.synchronize()
    return sa.cpu().numpy().view(np.uint32)


def test_batched_small_and_empty_texts(gb, orc):
    texts = [b"", b"a", b"", b"banana", b"\x00\x00\x00", b"ab" * 50, b"", b"x", b"mississippi"]
    flat = np.frombuffer(b"".join(texts), dtype=np.uint8).copy()
    off = np.zeros(len(texts) + 1, dtype=np.uint64)
    off[1:] = np.cumsum([len(t) for t in texts])
    assert np.array_equal(run_batched(gb, flat, off), batched_reference(orc, flat, off))


@pytest.mark.parametrize("count,lo,hi", [(64, 1, 3000), (1000, 1024, 8192), (4096, 16, 4096)])
def test_batched_matches_per_text(gb, orc, count, lo, hi):
    flat, off = gen.batch(count, count, lo, hi)
    got = run_batched(gb, flat, off)
    assert np.array_equal(got, batched_reference(orc, flat, off))


def test_batched_repeats_and_mixed_alphabets(gb, orc):
    parts = [gen.text("zipf_repeats", 1, 70000), gen.text("markov", 2, 50000),
             gen.text("bytes", 3, 4097), gen.text("dna", 4, 1), np.zeros(300, np.uint8)]
    flat = np.concatenate(parts)
    off = np.zeros(len(parts) + 1, dtype=np.uint64)
    off[1:] = np.cumsum([p.size for p in parts])
    assert np.array_equal(run_batched(gb, flat, off), batched_reference(orc, flat, off))


@pytest.mark.parametrize("h0", [2, 7, 13])
def test_batched_key_widths(gb, orc, h0):
    """Fewer characters per initial key than fit (the tuner's key width):
    short keys leave more suffixes tied for the doubling rounds."""
    flat, off = gen.batch(77, 300, 1, 6000)
    parts = [flat, gen.text("zipf_repeats", 5, 9000), np.zeros(40, np.uint8)]
    flat2 = np.concatenate(parts)
    off2 = np.concatenate([off, [off[-1] + 9000, off[-1] + 9040]]).astype(np.uint64)
    assert np.array_equal(run_batched(gb, flat2, off2, h0_chars=h0),
                          batched_reference(orc, flat2, off2))


def test_bounded_wait_expires_and_context_survives(gb, orc):
    """A tile that never publishes makes its successor's bounded look-back
    wait expire: the call returns SA_ERR_TIMEOUT and the next call works."""
    import torch
    t = gen.text("dna", 9, 1 << 20)
    d = torch.from_numpy(t).cuda()
    with pytest.raises(gb.SAError) as e:
        gb.sa_build_ex(d, inject_stall=1, spin_limit=2000)
    assert e.value.status == gb.SA_ERR_TIMEOUT
    sa = gb.sa_build(d)
    torch.cuda.synchronize()
    assert np.array_equal(sa.cpu().numpy().view(np.uint32), orc.pd_sa(t)[0])


def test_argument_errors(gb):
    import torch
    with pytest.raises(TypeError):
        gb.sa_build(torch.zeros(4, dtype=torch.int32, device="cuda"))
    lib = gb.load()
    assert lib.sa_build(None, 5, None, None) == 1
    assert lib.sa_build(None, (1 << 31) + 1, None, None) == 2


def test_workload_4_batched_full_size(gb, orc):
    """4096 uniform-DNA texts, log-uniform lengths in [1 KiB, 4 MiB] (about
    2 GB): every text's SA passes the linear-time checker; 48 sampled texts
    equal the oracle element by element."""
    import torch
    flat, off = gen.batch(4001, 4096, 1 << 10, 4 << 20)
    sa = gb.sa_build_batched(torch.from_numpy(flat).cuda(), off)
    torch.cuda.synchronize()
    s = sa.cpu().numpy().view(np.uint32)
    del sa
    torch.cuda.empty_cache()
    rng = np.random.default_rng(9)
    sample = set(rng.integers(0, 4096, 48).tolist()) | {0, 4095}
    for k in range(4096):
        a, b = int(off[k]), int(off[k + 1])
        if k in sample:
            assert np.array_equal(s[a:b], orc.pd_sa(flat[a:b])[0]), k
        else:
            assert orc.check_sa(flat[a:b], s[a:b])[0] == 0, k

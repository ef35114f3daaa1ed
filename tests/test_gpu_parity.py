"""GPU parity: sa_build (through the C-ABI) against the CPU oracle, bit-exact.

Every input is seeded and synthetic. The oracle runs prefix doubling with
discarding (oracle/oracle.c); the GPU result must equal it element by
element: SA, ISA and, with the same initial prefix length, the names of
every position after every round.
"""
import numpy as np
import pytest

import gen
from conftest import ints, read_golden

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gb():
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_1610_03007_gb300 as gbsa
    assert torch.cuda.is_available()
    return gbsa


def dev_text(t):
    import torch
    a = np.frombuffer(bytes(t), dtype=np.uint8) if isinstance(t, (bytes, bytearray)) else t
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def gpu_sa(gb, t):
    import torch
    sa = gb.sa_build(dev_text(t))
    torch.cuda.synchronize()
    return sa.cpu().numpy().view(np.uint32)


def test_paper_example_1_and_2(gb, orc):
    g = read_golden("ex1_ex2_bdacbdacb.txt")
    t = g["text"].encode()
    assert list(gpu_sa(gb, t)) == ints(g["sa"])
    # Example 2's names after every round, with the paper's 2-character
    # initial names.
    sa, isa, stats, trace = gb.sa_build_ex(dev_text(t), isa=True, h0_chars=2, trace_cap=8,
                                           paper_names=True)
    rows = [list(r) for r in trace[: stats["rounds"]].cpu().numpy()]
    assert rows == [ints(g[f"names_{k}"]) for k in range(3)]
    assert list(isa.cpu().numpy()) == ints(g["names_2"])


def test_paper_example_3(gb):
    g = read_golden("ex3_dbacbacbd.txt")
    assert list(gpu_sa(gb, g["text"].encode())) == ints(g["sa"])
    assert list(gpu_sa(gb, bytes(ints(g["sub_text_bytes"])))) == ints(g["sub_sa"])


def test_degenerate_inputs(gb, orc):
    assert gpu_sa(gb, b"").size == 0
    assert list(gpu_sa(gb, b"x")) == [0]
    for n in list(range(2, 70)) + [4095, 4096, 4097, 10000]:
        for ch in (b"a", b"\x00", b"\xff"):
            t = ch * n
            assert list(gpu_sa(gb, t)) == list(range(n - 1, -1, -1)), (ch, n)
    for m in (1, 2, 33, 1000, 2049):
        t = b"ab" * m
        want = list(range(2 * m - 2, -1, -2)) + list(range(2 * m - 1, 0, -2))
        assert list(gpu_sa(gb, t)) == want
    t = np.random.default_rng(1).permutation(256).astype(np.uint8)
    assert np.array_equal(gpu_sa(gb, t), np.argsort(t))
    # texts ending in runs of the smallest code (the end-of-text rule)
    for tail in (b"\x00\x00", b"\x00" * 40, b"A" * 70):
        t = b"CAGT" * 300 + tail
        assert np.array_equal(gpu_sa(gb, t), orc.pd_sa(t)[0])


def test_bruteforce_short_strings(gb, orc):
    import itertools
    for L in range(1, 11):
        for tup in itertools.product(b"\x00\x01", repeat=L):
            t = bytes(tup)
            assert np.array_equal(gpu_sa(gb, t), orc.pd_sa(t)[0]), t


@pytest.mark.parametrize("recipe", ["dna", "zipf_repeats", "markov", "zipf", "bytes"])
@pytest.mark.parametrize("n", [1, 7, 100, 4095, 4097, 12289, 100003])
def test_random_inputs(gb, orc, recipe, n):
    t = gen.text(recipe, 7 * n + 1, n)
    assert np.array_equal(gpu_sa(gb, t), orc.pd_sa(t)[0])


@pytest.mark.parametrize("recipe,n", [("dna", 1 << 20), ("zipf_repeats", 1 << 20),
                                      ("markov", 1 << 20), ("zipf_repeats", (1 << 21) + 12345)])
def test_every_round_matches_the_oracle(gb, orc, recipe, n):
    """With the paper's naming rule, the names after every round equal the
    oracle's with the same initial prefix length (the key's c0 characters);
    SA and ISA equal at the end."""
    t = gen.text(recipe, 31337, n)
    sa, isa, stats, trace = gb.sa_build_ex(dev_text(t), isa=True, trace_cap=24, paper_names=True)
    c0 = stats["chars_per_key"]
    osa, oisa, orounds, otrace = orc.pd_sa(t, h0=c0, trace_cap=24)
    assert stats["rounds"] == orounds + 1
    g = trace[: stats["rounds"]].cpu().numpy().view(np.uint32)
    for k in range(stats["rounds"]):
        assert np.array_equal(g[k], otrace[k]), f"round {k}"
    assert np.array_equal(sa.cpu().numpy().view(np.uint32), osa)
    assert np.array_equal(isa.cpu().numpy().view(np.uint32), oisa)


def names_agree(gpu_names, oracle_names):
    """The GPU names induce the oracle's groups in the oracle's order, and
    every GPU name lies in its group's SA interval [head, head + size)."""
    o = oracle_names.astype(np.int64)
    g = gpu_names.astype(np.int64)
    order = np.argsort(o, kind="stable")
    os_, gs_ = o[order], g[order]
    same_o = np.diff(os_) == 0
    if not np.array_equal(same_o, np.diff(gs_) == 0):
        return False
    if np.any(np.diff(gs_) < 0):
        return False
    size = np.bincount(o, minlength=o.size)[o]
    return bool(np.all((g >= o) & (g < o + size)))


@pytest.mark.parametrize("recipe,n", [("zipf_repeats", 1 << 20), ("markov", 1 << 20),
                                      ("zipf_repeats", (1 << 21) + 777)])
def test_every_round_default_names_are_valid(gb, orc, recipe, n):
    """With the default interval-retaining names, every round has exactly the
    oracle's groups, in its order, each name inside its group's interval."""
    t = gen.text(recipe, 4242, n)
    sa, isa, stats, trace = gb.sa_build_ex(dev_text(t), isa=True, trace_cap=24)
    c0 = stats["chars_per_key"]
    osa, oisa, orounds, otrace = orc.pd_sa(t, h0=c0, trace_cap=24)
    assert stats["rounds"] == orounds + 1
    g = trace[: stats["rounds"]].cpu().numpy().view(np.uint32)
    for k in range(stats["rounds"]):
        assert names_agree(g[k], otrace[k]), f"round {k}"
    assert np.array_equal(sa.cpu().numpy().view(np.uint32), osa)
    assert np.array_equal(isa.cpu().numpy().view(np.uint32), oisa)


def test_workload_1_full_size(gb, orc):
    """Uniform DNA, n = 2^20, with the library's own parameters (the tuning
    table's key width) and with the full 32-character key, which resolves
    every suffix in round 0."""
    t = gen.text("dna", 1001, 1 << 20)
    want = orc.pd_sa(t)[0]
    sa, _, stats, _ = gb.sa_build_ex(dev_text(t))
    assert stats["bits_per_char"] == 2
    assert np.array_equal(sa.cpu().numpy().view(np.uint32), want)
    sa, _, stats, _ = gb.sa_build_ex(dev_text(t), h0_chars=32)
    assert stats["chars_per_key"] == 32 and stats["rounds"] == 1
    assert np.array_equal(sa.cpu().numpy().view(np.uint32), want)


@pytest.mark.parametrize("recipe", ["zipf_repeats", "markov"])
def test_scaled_workloads_elementwise(gb, orc, recipe):
    t = gen.text(recipe, 2002, 1 << 22)
    assert np.array_equal(gpu_sa(gb, t), orc.pd_sa(t)[0])


def test_bucketed_isa_writes_elementwise(gb, orc):
    """Above 2^22 pending ISA writes the names go through position buckets
    (round 0's survivors and the later rounds' queued updates): SA and ISA
    equal the oracle's at a ragged size where both paths run."""
    n = 5 * (1 << 20) + 77
    t = gen.text("zipf_repeats", 2003, n)
    sa, isa, stats, _ = gb.sa_build_ex(dev_text(t), isa=True, profile=True, bucket_min=1 << 22,
                                       h0_chars=8)
    want_sa, want_isa, _, _ = orc.pd_sa(t)
    assert stats["active"][1] >= 1 << 22
    assert stats["kernels"]["bucket"]["launches"] >= 4
    assert np.array_equal(sa.cpu().numpy().view(np.uint32), want_sa)
    assert np.array_equal(isa.cpu().numpy().view(np.uint32), want_isa)


def test_workload_2_full_size_properties(gb, orc):
    """n = 2^28 repeated Zipf text, in the benchmark's launch configuration:
    the linear-time checker (permutation + adjacent order through the ranks),
    direct comparison of sampled adjacent suffixes, and the oracle's rank of
    sampled suffixes computed one by one."""
    import torch
    n = 1 << 28
    t = gen.text("zipf_repeats", 2001, n)
    d = dev_text(t)
    ws = torch.empty(gb.workspace_bytes(n), dtype=torch.uint8, device="cuda")
    sa, _, stats, _ = gb.sa_build_ex(d, workspace=ws)
    s = sa.cpu().numpy().view(np.uint32)
    del ws, sa, d
    assert stats["rounds"] > 5
    assert orc.check_sa(t, s) == (0, -1)
    rng = np.random.default_rng(5)
    assert orc.check_adjacent(t, s, rng.integers(0, n - 1, 20000)) == 0
    isa_of = {}
    for j in rng.integers(0, n, 3):
        isa_of[int(s[j])] = int(j)
    for i, j in isa_of.items():
        assert orc.suffix_rank(t, i) == j


def test_isa_output(gb):
    t = gen.text("markov", 5, 300000)
    sa, isa, _, _ = gb.sa_build_ex(dev_text(t), isa=True)
    s = sa.cpu().numpy().view(np.uint32)
    r = isa.cpu().numpy().view(np.uint32)
    assert np.array_equal(r[s], np.arange(t.size, dtype=np.uint32))


def test_host_entry_point(gb, orc):
    t = gen.text("zipf_repeats", 77, 500000)
    assert np.array_equal(gb.sa_build_host(t), orc.pd_sa(t)[0])


def test_repeated_builds_reuse_workspace(gb, orc):
    import torch
    ws = torch.empty(gb.workspace_bytes(1 << 18), dtype=torch.uint8, device="cuda")
    for seed in range(3):
        for recipe in ("dna", "zipf_repeats"):
            t = gen.text(recipe, seed, 1 << 18)
            sa, _, _, _ = gb.sa_build_ex(dev_text(t), workspace=ws)
            assert np.array_equal(sa.cpu().numpy().view(np.uint32), orc.pd_sa(t)[0])


@pytest.mark.parametrize("shape", [1, 2, 3, 4])
@pytest.mark.parametrize("recipe", ["zipf_repeats", "markov", "bytes"])
def test_every_refine_tile_shape(gb, orc, shape, recipe):
    """Each refine tile shape (which also moves the small/large group
    threshold) gives the oracle's SA and ISA."""
    t = gen.text(recipe, 90 + shape, (1 << 20) + 3 * shape)
    sa, isa, _, _ = gb.sa_build_ex(dev_text(t), isa=True, refine_shape=shape)
    osa, oisa, _, _ = orc.pd_sa(t)
    assert np.array_equal(sa.cpu().numpy().view(np.uint32), osa)
    assert np.array_equal(isa.cpu().numpy().view(np.uint32), oisa)


@pytest.mark.parametrize("recipe,n", [("zipf_repeats", 300007), ("dna", 1 << 18),
                                      ("bytes", 65537), ("markov", 200003)])
@pytest.mark.parametrize("h0", [1, 3, 5, 12])
def test_key_widths(gb, orc, recipe, n, h0):
    """The tuner's key width: h0 characters per initial key (capped at what
    fits), so more rounds resolve what round 0 would have."""
    t = gen.text(recipe, 911 + h0, n)
    sa, isa, stats, _ = gb.sa_build_ex(dev_text(t), isa=True, h0_chars=h0)
    assert stats["chars_per_key"] <= h0
    want_sa, want_isa, _, _ = orc.pd_sa(t)
    assert np.array_equal(sa.cpu().numpy().view(np.uint32), want_sa)
    assert np.array_equal(isa.cpu().numpy().view(np.uint32), want_isa)


@pytest.mark.parametrize("items", [8, 12, 16])
def test_every_radix_tile_size(gb, orc, items):
    """Each radix-pass tile size gives the oracle's SA (round 0 sorts all n
    keys; repeats force later large-group sorts too)."""
    for recipe, n in (("dna", 200003), ("zipf_repeats", 1 << 20), ("bytes", 77777)):
        t = gen.text(recipe, 500 + items, n)
        sa, _, _, _ = gb.sa_build_ex(dev_text(t), sort_items=items)
        assert np.array_equal(sa.cpu().numpy().view(np.uint32), orc.pd_sa(t)[0])
    t = b"a" * 300000  # one large group every round: the global sort path
    sa, _, _, _ = gb.sa_build_ex(dev_text(t), sort_items=items)
    assert list(sa.cpu().numpy()) == list(range(299999, -1, -1))


def test_workload_3_full_size_complete(gb, orc):
    """n = 2^31 order-3 Markov DNA with 5% copied segments (the largest
    input and the benchmark's headline, about 153 GB on the device), in the
    benchmark's launch configuration (the library's tuned parameters, a
    caller workspace): the whole SA through the linear-time checker of
    Burkhardt and Kaerkkaeinen (a permutation, and every adjacent pair in
    order through the ranks: the SA of Section 2's definition), plus 200000
    sampled adjacent suffixes compared directly and the oracle's rank of one
    suffix computed one by one."""
    import torch
    n = 1 << 31
    t = gen.text("markov", 3001, n)
    d = dev_text(t)
    ws = torch.empty(gb.workspace_bytes(n), dtype=torch.uint8, device="cuda")
    sa, _, stats, _ = gb.sa_build_ex(d, workspace=ws)
    torch.cuda.synchronize()
    del ws
    s = sa.cpu().numpy().view(np.uint32)
    del sa, d
    torch.cuda.empty_cache()
    assert stats["rounds"] > 3
    assert orc.check_sa(t, s) == (0, -1)
    rng = np.random.default_rng(31)
    assert orc.check_adjacent(t, s, rng.integers(0, n - 1, 200000)) == 0
    j = int(rng.integers(0, n))
    assert orc.suffix_rank(t, int(s[j])) == j


@pytest.mark.parametrize("n", [1, 2, 1000, (4 << 20) - 1, 4 << 20, (4 << 20) + 1])
def test_host_build_with_pinned_buffers(gb, orc, n):
    """sa_build_host with both host buffers pinned copies by kernels up to
    4 MiB (their device mapping) and by the copy engine above; with one
    buffer pageable it always takes the copy engine. Every form gives the
    device build's SA, on a text that starts at an odd offset of its
    pinned buffer."""
    import torch
    t = gen.text("markov", 31 + n % 7, n + 3)
    pinned = torch.from_numpy(t).pin_memory()
    out = torch.empty(n, dtype=torch.int32).pin_memory()
    want = gb.sa_build(torch.from_numpy(t[3:3 + n]).cuda()).cpu().numpy().view(np.uint32)
    gb.sa_build_host_ptr(pinned.data_ptr() + 3, n, out.data_ptr())
    assert np.array_equal(out.numpy().view(np.uint32), want)
    pageable = np.empty(n, dtype=np.uint32)
    gb.sa_build_host_ptr(pinned.data_ptr() + 3, n, pageable.ctypes.data)
    assert np.array_equal(pageable, want)
    if n <= 4096:
        assert np.array_equal(want, orc.pd_sa(t[3:3 + n])[0])


@pytest.mark.parametrize("copies", [5, 8, 12, 16])
@pytest.mark.parametrize("alphabet", [4, 200])
def test_groups_of_up_to_sixteen_copies(gb, orc, copies, alphabet):
    """A random block repeated `copies` times (a few substitutions per
    copy) leaves groups of up to `copies` members for several rounds, whose
    refine tiles take the counting path (groups of 5 to 64 members) rather
    than the per-thread path for groups of up to 4. SA and ISA equal the
    oracle's."""
    rng = np.random.default_rng(copies * 1000 + alphabet)
    block = rng.integers(0, alphabet, 20011).astype(np.uint8)
    parts = []
    for c in range(copies):
        b = block.copy()
        hits = rng.integers(0, b.size, 3)
        b[hits] = rng.integers(0, alphabet, 3).astype(np.uint8)
        parts.append(b)
    t = np.concatenate(parts)
    want_sa, want_isa, _, _ = orc.pd_sa(t)
    sa, isa, st, _ = gb.sa_build_ex(dev_text(t), isa=True, refine_shape=1)
    assert np.array_equal(sa.cpu().numpy().view(np.uint32), want_sa)
    assert np.array_equal(isa.cpu().numpy().view(np.uint32), want_isa)
    assert st["rounds"] > 2

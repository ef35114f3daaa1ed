"""GPU parity of the a-fold rounds (Section 2.1, Prefix Quadrupling): with
sa_options.multiplier = 3 or 4 each round ranks the names of i, i + h, ...,
i + (a-1)h. Compared, through the C-ABI, with the oracle's a-fold form
(oracle_pq_sa) on the same seeded inputs: SA and ISA bit for bit, and with
the paper's naming rule the names of every position after every round.
"""
import itertools

import numpy as np
import pytest

import gen
from conftest import ints, read_golden

pytestmark = pytest.mark.gpu

MULTS = (3, 4)


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


def u32(x):
    return x.cpu().numpy().view(np.uint32)


def build(gb, t, a, **kw):
    sa, isa, stats, trace = gb.sa_build_ex(dev_text(t), isa=True, multiplier=a, **kw)
    return u32(sa), u32(isa), stats, trace


@pytest.mark.parametrize("a", MULTS)
def test_paper_example_1(gb, orc, a):
    g = read_golden("ex1_ex2_bdacbdacb.txt")
    t = g["text"].encode()
    sa, isa, stats, trace = build(gb, t, a, h0_chars=2, trace_cap=8, paper_names=True)
    assert list(sa) == ints(g["sa"])
    _, oisa, orounds, otrace = orc.pd_sa(t, h0=2, trace_cap=8, a=a)
    assert stats["rounds"] == orounds + 1
    rows = u32(trace[: stats["rounds"]])
    assert [list(r) for r in rows] == [list(r) for r in otrace]
    assert np.array_equal(isa, oisa)


@pytest.mark.parametrize("a", MULTS)
def test_bruteforce_short_strings(gb, orc, a):
    for L in range(1, 10):
        for tup in itertools.product(b"\x00\x01", repeat=L):
            t = bytes(tup)
            sa, isa, _, _ = build(gb, t, a)
            osa, oisa, _, _ = orc.pd_sa(t, a=a)
            assert np.array_equal(sa, osa), t
            assert np.array_equal(isa, oisa), t


@pytest.mark.parametrize("a", MULTS)
def test_degenerate_inputs(gb, a):
    for n in list(range(2, 40)) + [4095, 4097, 1 << 20]:  # one group of all suffixes
        sa, _, _, _ = build(gb, b"a" * n, a)
        assert np.array_equal(sa, np.arange(n - 1, -1, -1, dtype=np.uint32)), n
    for m in (1, 33, 2049, 300001):
        sa, _, _, _ = build(gb, b"ab" * m, a)
        want = list(range(2 * m - 2, -1, -2)) + list(range(2 * m - 1, 0, -2))
        assert list(sa) == want, m


@pytest.mark.parametrize("a", MULTS)
@pytest.mark.parametrize("recipe", ["dna", "zipf_repeats", "markov", "zipf", "bytes"])
@pytest.mark.parametrize("n", [7, 4097, 100003])
def test_random_inputs(gb, orc, a, recipe, n):
    t = gen.text(recipe, 7 * n + a, n)
    sa, isa, _, _ = build(gb, t, a)
    osa, oisa, _, _ = orc.pd_sa(t, a=a)
    assert np.array_equal(sa, osa)
    assert np.array_equal(isa, oisa)


@pytest.mark.parametrize("a", MULTS)
@pytest.mark.parametrize("recipe,n", [("dna", 1 << 20), ("zipf_repeats", 1 << 20),
                                      ("markov", (1 << 20) + 77)])
def test_every_round_matches_the_oracle(gb, orc, a, recipe, n):
    """Names after every round (paper's naming rule, initial names of c0
    characters) equal the oracle's a-fold rounds; this covers the
    large-group path (two global sorts, tuple-aware rename) on the repeated
    text, whose first round keeps groups larger than a tile."""
    t = gen.text(recipe, 4242 + a, n)
    sa, isa, stats, trace = build(gb, t, a, trace_cap=24, paper_names=True)
    c0 = stats["chars_per_key"]
    osa, oisa, orounds, otrace = orc.pd_sa(t, h0=c0, trace_cap=24, a=a)
    assert stats["rounds"] == orounds + 1
    g = u32(trace[: stats["rounds"]])
    for k in range(stats["rounds"]):
        assert np.array_equal(g[k], otrace[k]), f"round {k}"
    assert np.array_equal(sa, osa)
    assert np.array_equal(isa, oisa)


@pytest.mark.parametrize("a", MULTS)
def test_large_groups_and_shapes(gb, orc, a):
    """A text whose repeats keep groups above every tile size for rounds,
    under every refine shape and the default (retaining) names."""
    rng = np.random.default_rng(5)
    block = rng.integers(0, 4, 3000, dtype=np.uint8)
    t = np.concatenate([np.tile(block, 120), rng.integers(0, 4, 999, dtype=np.uint8)])
    osa, oisa, _, _ = orc.pd_sa(t, a=a)
    for shape in (0, 1, 2, 3, 4):
        sa, isa, stats, _ = build(gb, t, a, refine_shape=shape)
        assert np.array_equal(sa, osa), shape
        assert np.array_equal(isa, oisa), shape


@pytest.mark.parametrize("a", MULTS)
def test_batched(gb, orc, a):
    """Many texts in one build: the later partners never cross into the next
    text (the gap slot's sentinel ends each tuple)."""
    import torch
    rng = np.random.default_rng(77 + a)
    texts = []
    for k in range(40):
        n = int(rng.integers(0, 5000))
        recipe = ("dna", "zipf_repeats", "markov", "bytes")[k % 4]
        t = gen.text(recipe, 1000 + k, n)
        if k % 5 == 0:
            t = np.tile(t[: max(1, n // 50)], 50)[:n] if n else t
        texts.append(t)
    off = np.zeros(len(texts) + 1, dtype=np.uint64)
    off[1:] = np.cumsum([len(x) for x in texts])
    flat = np.concatenate(texts) if int(off[-1]) else np.zeros(0, np.uint8)
    sa = gb.sa_build_batched(torch.from_numpy(flat).cuda(), off, multiplier=a)
    torch.cuda.synchronize()
    got = u32(sa)
    for k, t in enumerate(texts):
        want = orc.pd_sa(t, a=a)[0]
        assert np.array_equal(got[int(off[k]):int(off[k + 1])], want), k


@pytest.mark.parametrize("a", MULTS)
def test_large_text_checked(gb, orc, a):
    """2^26 characters of the repeated-Zipf text: the linear-time checker of
    the oracle (Burkhardt-Kaerkkaeinen) accepts the GPU's SA."""
    t = gen.text("zipf_repeats", 99, 1 << 26)
    sa, _, stats, _ = build(gb, t, a)
    assert orc.check_sa(t, sa)[0] == 0
    d, _, d_stats, _ = build(gb, t, 2)
    assert np.array_equal(sa, d)
    assert stats["rounds"] < d_stats["rounds"]


def test_invalid_multiplier(gb):
    for bad in (1, 5, 64):
        with pytest.raises(RuntimeError):
            build(gb, b"banana", bad)

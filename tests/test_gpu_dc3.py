"""GPU parity of sa_build_dc3 (the skew algorithm, through the C-ABI) with
the oracle's suffix array, and the paper's Example 3 recursion string."""
import itertools

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


def dc3(gb, t, trace=False):
    import torch
    a = np.frombuffer(bytes(t), dtype=np.uint8) if isinstance(t, (bytes, bytearray)) else t
    d = torch.from_numpy(np.ascontiguousarray(a).copy()).cuda()
    r = gb.sa_build_dc3(d, trace=trace)
    torch.cuda.synchronize()
    if trace:
        return r[0].cpu().numpy().view(np.uint32), r[1].cpu().numpy().view(np.uint32)
    return r.cpu().numpy().view(np.uint32)


def test_paper_example_3(gb):
    """SA of dbacbacbd and its recursion string: the paper's names
    1 1 2 0 0 3 (0-based) are 2 2 3 1 1 4 here (1-based)."""
    g = read_golden("ex3_dbacbacbd.txt")
    sa, tr = dc3(gb, g["text"].encode(), trace=True)
    assert list(sa) == ints(g["sa"])
    assert list(tr) == [x + 1 for x in ints(g["sub_text_bytes"])]


def test_degenerate_inputs(gb, orc):
    assert dc3(gb, b"").size == 0
    assert list(dc3(gb, b"x")) == [0]
    for n in list(range(2, 40)) + [255, 256, 257, 1000, 4097]:
        for ch in (b"a", b"\x00", b"\xff"):
            assert list(dc3(gb, ch * n)) == list(range(n - 1, -1, -1)), (ch, n)
    for m in (1, 2, 3, 50, 2049):
        want = list(range(2 * m - 2, -1, -2)) + list(range(2 * m - 1, 0, -2))
        assert list(dc3(gb, b"ab" * m)) == want
    t = np.random.default_rng(2).permutation(256).astype(np.uint8)
    assert np.array_equal(dc3(gb, t), np.argsort(t))


def test_bruteforce_short_strings(gb, orc):
    for L in range(1, 10):
        for tup in itertools.product(b"\x00\x01", repeat=L):
            t = bytes(tup)
            assert np.array_equal(dc3(gb, t), orc.naive_sa(t)), t


@pytest.mark.parametrize("recipe", ["dna", "zipf_repeats", "markov", "bytes", "zipf"])
@pytest.mark.parametrize("n", [3, 100, 4097, 100003, (1 << 20) + 1])
def test_matches_oracle(gb, orc, recipe, n):
    t = gen.text(recipe, 13 * n + 5, n)
    assert np.array_equal(dc3(gb, t), orc.pd_sa(t)[0])


def test_full_size_bench_workload(gb, orc):
    """n = 2^28 repeated Zipf text: the linear-time checker and sampled
    adjacent suffixes compared directly."""
    n = 1 << 28
    t = gen.text("zipf_repeats", 2001, n)
    s = dc3(gb, t)
    assert orc.check_sa(t, s) == (0, -1)
    rng = np.random.default_rng(8)
    assert orc.check_adjacent(t, s, rng.integers(0, n - 1, 20000)) == 0

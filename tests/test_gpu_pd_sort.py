"""GPU parity of sa_build_pd_sort (prefix doubling using sorting, Algorithms
1-3 with Eq. 1's comparator, through the C-ABI) with the oracle: SA bit for
bit, and the names of every position after every naming equal to the
oracle's rounds with 2-character initial names (Example 2's trace)."""
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


def pds(gb, t, trace_cap=0):
    import torch
    a = np.frombuffer(bytes(t), dtype=np.uint8) if isinstance(t, (bytes, bytearray)) else t
    d = torch.from_numpy(np.ascontiguousarray(a).copy()).cuda()
    sa, tr, rounds = gb.sa_build_pd_sort(d, trace_cap=trace_cap)
    torch.cuda.synchronize()
    sa = sa.cpu().numpy().view(np.uint32)
    tr = tr[:rounds].cpu().numpy().view(np.uint32) if tr is not None else None
    return sa, tr, rounds


def test_paper_examples_1_and_2(gb):
    """Ex. 1's SA; Ex. 2's names of every position after each round."""
    g = read_golden("ex1_ex2_bdacbdacb.txt")
    sa, tr, rounds = pds(gb, g["text"].encode(), trace_cap=8)
    assert list(sa) == ints(g["sa"])
    assert rounds == int(g["rounds"]) + 1
    assert [list(r) for r in tr] == [ints(g[f"names_{k}"]) for k in range(rounds)]
    g3 = read_golden("ex3_dbacbacbd.txt")
    assert list(pds(gb, g3["text"].encode())[0]) == ints(g3["sa"])


def test_degenerate_inputs(gb, orc):
    assert pds(gb, b"")[0].size == 0
    assert list(pds(gb, b"x")[0]) == [0]
    for n in list(range(2, 40)) + [255, 256, 257, 4097, 70001]:
        for ch in (b"a", b"\x00", b"\xff"):
            assert list(pds(gb, ch * n)[0]) == list(range(n - 1, -1, -1)), (ch, n)
    for m in (1, 2, 3, 50, 2049):
        want = list(range(2 * m - 2, -1, -2)) + list(range(2 * m - 1, 0, -2))
        assert list(pds(gb, b"ab" * m)[0]) == want
    t = np.random.default_rng(2).permutation(256).astype(np.uint8)
    assert np.array_equal(pds(gb, t)[0], np.argsort(t))


def test_bruteforce_short_strings(gb, orc):
    for L in range(1, 11):
        for tup in itertools.product(b"\x00\x01", repeat=L):
            t = bytes(tup)
            assert np.array_equal(pds(gb, t)[0], orc.naive_sa(t)), t


@pytest.mark.parametrize("recipe", ["dna", "zipf_repeats", "markov", "bytes", "zipf"])
@pytest.mark.parametrize("n", [3, 100, 4097, 100003])
def test_every_naming_matches_the_oracle(gb, orc, recipe, n):
    t = gen.text(recipe, 11 * n + 7, n)
    sa, tr, rounds = pds(gb, t, trace_cap=40)
    osa, _, orounds, otr = orc.pd_sa(t, h0=2, trace_cap=40)
    assert np.array_equal(sa, osa)
    assert rounds == orounds + 1
    for k in range(rounds):
        assert np.array_equal(tr[k], otr[k]), f"naming {k}"


@pytest.mark.parametrize("recipe", ["dna", "zipf_repeats"])
def test_large_inputs(gb, orc, recipe):
    n = (1 << 20) + 5
    t = gen.text(recipe, 5, n)
    assert np.array_equal(pds(gb, t)[0], orc.pd_sa(t)[0])


def test_bench_size_checked(gb, orc):
    """n = 2^26 repeated Zipf text: the linear-time checker."""
    n = 1 << 26
    t = gen.text("zipf_repeats", 2001, n)
    sa = pds(gb, t)[0]
    assert orc.check_sa(t, sa) == (0, -1)

"""GPU parity of sa_build_dc7 (difference cover {0, 1, 3} modulo 7, through
the C-ABI) with the oracle: the suffix array's definition and DC7's first
recursion text (oracle_dc7_names)."""
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


def dc7(gb, t, trace=False):
    import torch
    a = np.frombuffer(bytes(t), dtype=np.uint8) if isinstance(t, (bytes, bytearray)) else t
    d = torch.from_numpy(np.ascontiguousarray(a).copy()).cuda()
    r = gb.sa_build_dc7(d, trace=trace)
    torch.cuda.synchronize()
    if trace:
        return r[0].cpu().numpy().view(np.uint32), r[1].cpu().numpy().view(np.uint32)
    return r.cpu().numpy().view(np.uint32)


def test_paper_examples(gb):
    for name in ("ex1_ex2_bdacbdacb.txt", "ex3_dbacbacbd.txt"):
        g = read_golden(name)
        assert list(dc7(gb, g["text"].encode())) == ints(g["sa"])


def test_recursion_text(gb, orc):
    """The top level's names equal the oracle's (dense ranks of the windows
    by definition), including texts whose names repeat (recursion)."""
    texts = [b"x", b"ab", b"abcdefg", b"abcdefgh", b"a" * 100, b"ab" * 77,
             b"mississippi" * 9]
    for recipe, n in (("zipf_repeats", 5000), ("dna", 4096), ("bytes", 3001),
                      ("zipf_repeats", 100003)):
        texts.append(gen.text(recipe, n + 3, n).tobytes())
    for t in texts:
        sa, tr = dc7(gb, t, trace=True)
        assert np.array_equal(tr, orc.dc7_names(t)), t[:12]
        assert np.array_equal(sa, orc.naive_sa(t) if len(t) < 20000 else orc.pd_sa(t)[0])


def test_degenerate_inputs(gb, orc):
    assert dc7(gb, b"").size == 0
    assert list(dc7(gb, b"x")) == [0]
    for n in list(range(2, 60)) + [255, 256, 257, 1000, 4097, 70001]:
        for ch in (b"a", b"\x00", b"\xff"):
            assert list(dc7(gb, ch * n)) == list(range(n - 1, -1, -1)), (ch, n)
    for m in (1, 2, 3, 7, 50, 2049):
        want = list(range(2 * m - 2, -1, -2)) + list(range(2 * m - 1, 0, -2))
        assert list(dc7(gb, b"ab" * m)) == want
    for period in (3, 7, 13, 14):  # periods that meet the modulus 7 in every way
        t = (bytes(range(1, period + 1)) * 300)[:4000]
        assert np.array_equal(dc7(gb, t), orc.pd_sa(t)[0]), period
    t = np.random.default_rng(2).permutation(256).astype(np.uint8)
    assert np.array_equal(dc7(gb, t), np.argsort(t))


def test_bruteforce_short_strings(gb, orc):
    for L in range(1, 12):
        for tup in itertools.product(b"\x00\x01", repeat=L):
            t = bytes(tup)
            assert np.array_equal(dc7(gb, t), orc.naive_sa(t)), t


@pytest.mark.parametrize("recipe", ["dna", "zipf_repeats", "markov", "bytes", "zipf"])
@pytest.mark.parametrize("n", [3, 100, 4097, 100003, (1 << 20) + 1])
def test_matches_oracle(gb, orc, recipe, n):
    t = gen.text(recipe, 17 * n + 3, n)
    assert np.array_equal(dc7(gb, t), orc.pd_sa(t)[0])


@pytest.mark.parametrize("n", [(7 << 16) + k for k in range(7)])
def test_every_residue_of_n(gb, orc, n):
    """n mod 7 decides which classes end with the all-zero window and which
    class positions lie past their sample: all seven residues."""
    t = gen.text("zipf_repeats", n, n)
    assert np.array_equal(dc7(gb, t), orc.pd_sa(t)[0])


def test_full_size_bench_workload(gb, orc):
    """n = 2^28 repeated Zipf text: the linear-time checker and sampled
    adjacent suffixes compared directly."""
    n = 1 << 28
    t = gen.text("zipf_repeats", 2001, n)
    s = dc7(gb, t)
    assert orc.check_sa(t, s) == (0, -1)
    rng = np.random.default_rng(9)
    assert orc.check_adjacent(t, s, rng.integers(0, n - 1, 20000)) == 0

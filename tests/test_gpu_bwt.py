"""GPU parity of sa_bwt (through the C-ABI) against the oracle's BWT of the
oracle's own suffix array, byte for byte, plus the primary index; the
oracle's inverse transform of the GPU's BWT reproduces the text."""
import numpy as np
import pytest

import gen

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gb():
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_1610_03007_gb300 as gbsa
    assert torch.cuda.is_available()
    return gbsa


def gpu_bwt(gb, t):
    import torch
    a = np.frombuffer(bytes(t), dtype=np.uint8) if isinstance(t, (bytes, bytearray)) else t
    d = torch.from_numpy(np.array(a, dtype=np.uint8, copy=True)).cuda()
    sa = gb.sa_build(d)
    bwt, prim = gb.sa_bwt(d, sa)
    torch.cuda.synchronize()
    return sa.cpu().numpy().view(np.uint32), bwt.cpu().numpy(), prim


def test_textbook_and_degenerate(gb, orc):
    _, b, p = gpu_bwt(gb, b"banana")
    assert bytes(b) == b"annb\x00aa" and p == 4
    _, b, p = gpu_bwt(gb, b"")
    assert list(b) == [0] and p == 0
    _, b, p = gpu_bwt(gb, b"x")
    assert list(b) == [ord("x"), 0] and p == 1
    for t in (b"a" * 100, b"\x00" * 77, b"ab" * 33):
        _, b, p = gpu_bwt(gb, t)
        ob, op = orc.bwt(t, orc.naive_sa(t))
        assert np.array_equal(b, ob) and p == op


@pytest.mark.parametrize("recipe", ["dna", "zipf_repeats", "markov", "bytes"])
@pytest.mark.parametrize("n", [1, 255, 4097, 100003, (1 << 20) + 7])
def test_matches_oracle(gb, orc, recipe, n):
    t = gen.text(recipe, 17 * n + 3, n)
    _, b, p = gpu_bwt(gb, t)
    ob, op = orc.bwt(t, orc.pd_sa(t)[0])
    assert np.array_equal(b, ob) and p == op
    assert np.array_equal(orc.bwt_invert(b, p), t)


def test_full_size_bench_workload(gb, orc):
    """n = 2^28 repeated Zipf text (its SA is checked at full size by the
    parity tests): every one of the 2^28 + 1 rows is the byte before its
    suffix, and the oracle's LF inversion of the BWT gives back the text."""
    n = 1 << 28
    t = gen.text("zipf_repeats", 2001, n)
    sa, b, p = gpu_bwt(gb, t)
    s = sa.astype(np.int64)
    want = np.where(s == 0, 0, t[np.maximum(s - 1, 0)]).astype(np.uint8)
    assert b[0] == t[-1] and np.array_equal(b[1:], want)
    assert p == 1 + int(np.flatnonzero(s == 0)[0])
    assert np.array_equal(orc.bwt_invert(b, p), t)

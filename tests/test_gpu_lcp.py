"""GPU parity of sa_lcp (through the C-ABI) against the oracle's LCP array
(the definition, on the oracle's own suffix array), element by element; at
the benchmark size, sampled entries against the definition computed pair by
pair."""
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


def gpu_lcp(gb, t, **kw):
    import torch
    a = np.frombuffer(bytes(t), dtype=np.uint8) if isinstance(t, (bytes, bytearray)) else t
    d = torch.from_numpy(np.ascontiguousarray(a)).cuda()
    sa = gb.sa_build(d)
    lcp = gb.sa_lcp(d, sa, **kw)
    torch.cuda.synchronize()
    return sa.cpu().numpy().view(np.uint32), lcp.cpu().numpy().view(np.uint32)


def test_textbook_and_closed_forms(gb, orc):
    assert list(gpu_lcp(gb, b"banana")[1]) == [0, 1, 3, 0, 0, 2]
    assert gpu_lcp(gb, b"")[1].size == 0
    assert list(gpu_lcp(gb, b"x")[1]) == [0]
    for n in (2, 3, 255, 256, 257, 5000, 20000):  # a^n: 0, 1, .., n-1 (chunk edges)
        assert list(gpu_lcp(gb, b"a" * n)[1]) == list(range(n)), n
    m = 3000
    want = [2 * k for k in range(m)] + [0] + [2 * k + 1 for k in range(m - 1)]
    assert list(gpu_lcp(gb, b"ab" * m)[1]) == want
    assert not gpu_lcp(gb, bytes(range(256)))[1].any()


@pytest.mark.parametrize("recipe", ["dna", "zipf_repeats", "markov", "bytes", "zipf"])
@pytest.mark.parametrize("n", [2, 255, 4099, 100003, (1 << 20) + 13])
def test_matches_oracle(gb, orc, recipe, n):
    t = gen.text(recipe, 29 * n + 1, n)
    _, lcp = gpu_lcp(gb, t)
    assert np.array_equal(lcp, orc.lcp(t, orc.pd_sa(t)[0]))


def test_unaligned_text_and_caller_workspace(gb, orc):
    """A text starting at an odd address takes the byte-by-byte path."""
    import torch
    t = gen.text("zipf_repeats", 5, 70001)
    buf = torch.zeros(70001 + 1, dtype=torch.uint8, device="cuda")
    buf[1:] = torch.from_numpy(t).cuda()
    d = buf[1:]
    sa = gb.sa_build(d)
    ws = torch.empty(gb.load().sa_lcp_workspace_bytes(t.size), dtype=torch.uint8, device="cuda")
    lcp = gb.sa_lcp(d, sa, workspace=ws)
    torch.cuda.synchronize()
    assert np.array_equal(lcp.cpu().numpy().view(np.uint32), orc.lcp(t, orc.pd_sa(t)[0]))


def test_full_size_bench_workload_sampled(gb, orc):
    """n = 2^28 repeated Zipf text (SA checked at full size by the parity
    tests): 100000 sampled entries against the definition, and the maximum
    entry's pair."""
    n = 1 << 28
    t = gen.text("zipf_repeats", 2001, n)
    sa, lcp = gpu_lcp(gb, t)
    rng = np.random.default_rng(41)
    assert lcp[0] == 0
    for j in rng.integers(1, n, 100000):
        assert lcp[j] == orc.lcp_pair(t, int(sa[j - 1]), int(sa[j])), j
    jm = int(np.argmax(lcp))
    assert lcp[jm] == orc.lcp_pair(t, int(sa[jm - 1]), int(sa[jm]))

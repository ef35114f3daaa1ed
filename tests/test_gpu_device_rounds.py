"""Device-driven rounds (sa_options.device_rounds = 1): the loop of
Algorithm 5 runs as one CUDA graph (a while-node over rounds of persistent
kernels that read their sizes from a device round state, if-nodes for the
large-group sort, its rename and the position bucketing). The SA and ISA
must equal the oracle's element by element, and the rounds -- how many,
and the active suffixes, groups and radix passes of each -- must equal the
host-driven build's."""
import numpy as np
import pytest

import gen

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gb():
    import __graft_entry__
    __graft_entry__.build()
    import paper_1610_03007_gb300 as g
    g.load()
    return g


def dev(t):
    import torch
    return torch.from_numpy(np.ascontiguousarray(np.frombuffer(bytes(t), np.uint8)
                                                 if isinstance(t, bytes) else t)).cuda()


def u32(x):
    return x.cpu().numpy().view(np.uint32)


def both(gb, t, **kw):
    d = dev(t)
    sa_d, isa_d, st_d, _ = gb.sa_build_ex(d, isa=True, device_rounds=1, **kw)
    sa_h, isa_h, st_h, _ = gb.sa_build_ex(d, isa=True, device_rounds=2, **kw)
    assert st_d["rounds"] == st_h["rounds"]
    for key in ("active", "groups", "unique", "passes"):
        assert st_d[key] == st_h[key], key
    return u32(sa_d), u32(isa_d), st_d


@pytest.mark.parametrize("recipe,n", [("zipf_repeats", 1 << 20), ("markov", (1 << 20) + 3),
                                      ("dna", 65537), ("bytes", 4099), ("zipf", 300001),
                                      ("zipf_repeats", 777)])
@pytest.mark.parametrize("h0", [0, 3])
def test_recipes_equal_the_oracle(gb, orc, recipe, n, h0):
    t = gen.text(recipe, 31 + h0, n)
    sa, isa, st = both(gb, t, h0_chars=h0)
    want_sa, want_isa, _, _ = orc.pd_sa(t)
    assert np.array_equal(sa, want_sa)
    assert np.array_equal(isa, want_isa)
    if h0 and recipe in ("zipf_repeats", "markov"):
        assert st["rounds"] > 1  # repeats leave work for the device-driven rounds


@pytest.mark.parametrize("t", [b"a" * 300000, b"ab" * 70001, b"abc" * 40000 + b"ab",
                               bytes(range(256)) * 900])
def test_large_groups_every_round(gb, orc, t):
    """Periodic texts keep groups above the refine window in every round:
    the if-nodes of the large-group sort and rename run each time. The
    128 x 1024 refine tile (a window of 512) is fixed so that the groups of
    hundreds of copies exceed it whatever the tuning table picks."""
    sa, isa, st = both(gb, t, h0_chars=2, refine_shape=1)
    assert max(st["passes"][1:]) > 0
    assert np.array_equal(sa, orc.pd_sa(t)[0])


@pytest.mark.parametrize("bucket_min", [1, 1 << 12, 0xFFFFFFFF])
def test_bucketed_and_direct_isa_writes(gb, orc, bucket_min):
    t = gen.text("zipf_repeats", 88, (1 << 21) + 77)
    sa, isa, _ = both(gb, t, bucket_min=bucket_min, h0_chars=4)
    want_sa, want_isa, _, _ = orc.pd_sa(t)
    assert np.array_equal(sa, want_sa)
    assert np.array_equal(isa, want_isa)


@pytest.mark.parametrize("shape", [1, 2, 3, 4])
def test_every_refine_shape(gb, orc, shape):
    t = gen.text("markov", 90 + shape, (1 << 19) + shape)
    sa, isa, _ = both(gb, t, refine_shape=shape, h0_chars=6)
    want_sa, want_isa, _, _ = orc.pd_sa(t)
    assert np.array_equal(sa, want_sa)
    assert np.array_equal(isa, want_isa)


def test_batched_texts(gb, orc):
    import torch
    rng = np.random.default_rng(5)
    texts = [gen.text(("dna", "zipf_repeats", "markov")[k % 3], 300 + k,
                      int(rng.integers(0, 20000))) for k in range(40)]
    texts[3] = texts[3][:0]
    texts[7] = texts[7][:1]
    flat = np.concatenate(texts)
    off = np.concatenate([[0], np.cumsum([t.size for t in texts])]).astype(np.uint64)
    d = torch.from_numpy(flat).cuda()
    sa_d, st_d = gb.sa_build_batched(d, off, stats=True, device_rounds=1, h0_chars=3)
    sa_h, st_h = gb.sa_build_batched(d, off, stats=True, device_rounds=2, h0_chars=3)
    assert st_d["rounds"] == st_h["rounds"] > 1
    assert st_d["active"] == st_h["active"]
    got = u32(sa_d)
    assert np.array_equal(got, u32(sa_h))
    for k, t in enumerate(texts):
        assert np.array_equal(got[int(off[k]):int(off[k + 1])], orc.pd_sa(t)[0]), k


def test_resolved_in_round_zero_and_tiny(gb, orc):
    """No round after round 0 (nothing to run on the device), and texts of
    one and two characters."""
    for t in (gen.text("dna", 1, 1 << 16), b"x", b"ba", b"aa"):
        sa, _, _, _ = gb.sa_build_ex(dev(t), device_rounds=1)
        assert np.array_equal(u32(sa), orc.pd_sa(t)[0])

"""Round 0's initial keys (Algorithm 1's initial names, c0 characters each)
formed inside the first radix pass (sa_options.initial_keys = 1, where it
applies: one text, 1, 2, 4 or 8 bits per character, c0 * bits a multiple
of 8) against the separate pack (2) and the oracle: SA, ISA and the names
after round 0 (paper names, so the oracle's initial names with the same
number of characters), over texts shorter than a key, the tail positions,
tile edges and every alphabet width; where the fused form does not apply
the option falls back to the pack."""
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
    return torch.from_numpy(np.ascontiguousarray(t)).cuda()


def u32(x):
    return x.cpu().numpy().view(np.uint32)


def alphabet_text(k, n, seed):
    """n characters drawn from k spread-out byte values, with a repeated
    block so that some suffixes stay tied past round 0."""
    rng = np.random.default_rng(seed)
    values = np.array([(3 + 37 * i) % 256 for i in range(k)], dtype=np.uint8)
    t = values[rng.integers(0, k, n)]
    if n > 64:
        blk = t[: n // 4].copy()
        t[n // 2: n // 2 + blk.size] = blk
    return t


def run(gb, t, **kw):
    sa, isa, st, trace = gb.sa_build_ex(dev(t), isa=True, profile=True, **kw)
    return u32(sa), u32(isa), st, trace


@pytest.mark.parametrize("k,bits", [(2, 1), (4, 2), (16, 4), (200, 8)])
@pytest.mark.parametrize("n", [1, 2, 3, 17, 31, 32, 33, 64, 4095, 4096, 4097, 12289, 65573])
def test_fused_keys_equal_the_pack_and_the_oracle(gb, orc, k, bits, n):
    t = alphabet_text(k, n, 1000 * k + n)
    want_sa, want_isa, _, _ = orc.pd_sa(t)
    sa1, isa1, st1, _ = run(gb, t, initial_keys=1)
    sa2, isa2, st2, _ = run(gb, t, initial_keys=2)
    for sa, isa in ((sa1, isa1), (sa2, isa2)):
        assert np.array_equal(sa, want_sa)
        assert np.array_equal(isa, want_isa)
    assert st1["rounds"] == st2["rounds"] and st1["active"] == st2["active"]
    if n == 1:  # answered on the host: no kernel runs
        assert st1["kernels"]["pack"]["launches"] == st2["kernels"]["pack"]["launches"] == 0
        return
    # the pack of the fused form reads the text only (the keys are never written)
    b, c0 = st1["bits_per_char"], st1["chars_per_key"]
    if len(np.unique(t)) > 2 ** (bits - 1):
        assert b == bits
    fused = b >= 1 and 8 % b == 0 and (c0 * b) % 8 == 0
    assert st1["kernels"]["pack"]["bytes"] == (n if fused else 13 * n)
    assert st2["kernels"]["pack"]["bytes"] == 13 * n


@pytest.mark.parametrize("recipe,n,h0", [("dna", 100003, 4), ("dna", 100003, 12), ("dna", 100003, 7),
                                         ("markov", (1 << 20) + 5, 24), ("zipf", 200001, 3),
                                         ("bytes", 70001, 8), ("zipf_repeats", 300007, 0)])
def test_initial_names_equal_the_oracles(gb, orc, recipe, n, h0):
    """The names after round 0 are the oracle's initial names for c0
    characters, with either way of forming the keys (h0 = 7 on DNA gives
    14-bit keys: the fused form does not apply and the pack runs)."""
    t = gen.text(recipe, 90 + n % 13, n)
    _, _, st1, tr1 = run(gb, t, initial_keys=1, h0_chars=h0, paper_names=True, trace_cap=1)
    _, _, st2, tr2 = run(gb, t, initial_keys=2, h0_chars=h0, paper_names=True, trace_cap=1)
    c0 = st1["chars_per_key"]
    _, _, _, otrace = orc.pd_sa(t, h0=c0, trace_cap=1)
    assert np.array_equal(u32(tr1[0]), otrace[0])
    assert np.array_equal(u32(tr2[0]), otrace[0])


@pytest.mark.parametrize("items", [8, 12, 16])
def test_every_tile_size(gb, orc, items):
    t = gen.text("markov", 77, 3 * 4096 * 5 + 11)
    want_sa, want_isa, _, _ = orc.pd_sa(t)
    sa, isa, st, _ = run(gb, t, initial_keys=1, sort_items=items, h0_chars=16)
    assert st["params"]["sort_items"] == items
    assert np.array_equal(sa, want_sa) and np.array_equal(isa, want_isa)

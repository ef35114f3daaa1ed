"""Group order after round 0 (sa_options.group_order): the groups of the
active list in order of their smallest member position (1, the default
when a round follows) or in rank order (2). A round only needs each group
contiguous, so both must give the oracle's SA, ISA and per-round names,
and the same rounds (active suffixes, unique suffixes and groups per
round)."""
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


@pytest.mark.parametrize("recipe,n,h0", [("zipf_repeats", 1 << 20, 0), ("markov", (1 << 20) + 3, 0),
                                         ("markov", 300007, 6), ("dna", 100003, 3),
                                         ("bytes", 65537, 2), ("zipf", 200001, 2)])
def test_both_orders_equal_the_oracle(gb, orc, recipe, n, h0):
    t = gen.text(recipe, 60 + n % 11, n)
    d = dev(t)
    want_sa, want_isa, _, _ = orc.pd_sa(t)
    runs = {}
    for order in (1, 2):
        sa, isa, st, _ = gb.sa_build_ex(d, isa=True, group_order=order, h0_chars=h0)
        assert np.array_equal(u32(sa), want_sa), order
        assert np.array_equal(u32(isa), want_isa), order
        runs[order] = st
    for key in ("rounds", "active", "unique", "groups"):
        assert runs[1][key] == runs[2][key], key


def test_per_round_names_in_position_order(gb, orc):
    """The paper's names after every round (head ranks, 2-character initial
    names) do not depend on the group order."""
    t = gen.text("zipf_repeats", 71, (1 << 18) + 5)
    sa, _, st, trace = gb.sa_build_ex(dev(t), paper_names=True, h0_chars=2, trace_cap=32,
                                      group_order=1)
    _, _, orounds, otrace = orc.pd_sa(t, h0=2, trace_cap=32)
    assert st["rounds"] == orounds + 1
    got = u32(trace[: st["rounds"]])
    assert np.array_equal(got, np.asarray(otrace[: st["rounds"]], dtype=np.uint32))
    assert np.array_equal(u32(sa), orc.pd_sa(t)[0])


def test_batched_texts_in_position_order(gb, orc):
    import torch
    rng = np.random.default_rng(8)
    texts = [gen.text(("zipf_repeats", "markov")[k % 2], 900 + k, int(rng.integers(1, 30000)))
             for k in range(30)]
    flat = np.concatenate(texts)
    off = np.concatenate([[0], np.cumsum([x.size for x in texts])]).astype(np.uint64)
    d = torch.from_numpy(flat).cuda()
    got = u32(gb.sa_build_batched(d, off, group_order=1, h0_chars=4))
    ref = u32(gb.sa_build_batched(d, off, group_order=2, h0_chars=4))
    assert np.array_equal(got, ref)
    for k, x in enumerate(texts):
        assert np.array_equal(got[int(off[k]):int(off[k + 1])], orc.pd_sa(x)[0]), k

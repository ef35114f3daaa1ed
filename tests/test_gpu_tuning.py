"""The autotuner's knobs on the GPU: every value of the discard threshold
gives the oracle's SA and ISA, and a build through the C-ABI with no
options runs with the tuning table's values for its class (reported in
sa_stats) and still gives the oracle's SA."""
import os

import numpy as np
import pytest

import gen
from paper_1610_03007_gb300 import autotune

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gb():
    import __graft_entry__
    __graft_entry__.build()
    import paper_1610_03007_gb300 as g
    g.load()
    yield g
    g.tuning_load(autotune.DEFAULT_TABLE if os.path.exists(autotune.DEFAULT_TABLE) else None)


@pytest.fixture(scope="module")
def orc():
    import oracle
    return oracle.get()


def dev(t):
    import torch
    return torch.from_numpy(np.ascontiguousarray(t)).cuda()


@pytest.mark.parametrize("bucket_min", [1, 1 << 10, 1 << 16, 1 << 22, 0xFFFFFFFF])
@pytest.mark.parametrize("recipe,n", [("zipf_repeats", (1 << 20) + 17), ("markov", 300007)])
def test_every_discard_threshold(gb, orc, bucket_min, recipe, n):
    t = gen.text(recipe, 60 + n % 7, n)
    sa, isa, st, _ = gb.sa_build_ex(dev(t), isa=True, bucket_min=bucket_min, profile=True)
    want_sa, want_isa, _, _ = orc.pd_sa(t)
    assert st["params"]["bucket_min"] == bucket_min
    if bucket_min <= 1 << 16:
        assert st["kernels"]["bucket"]["launches"] > 0
    if bucket_min == 0xFFFFFFFF:
        assert st["kernels"]["bucket"]["launches"] == 0
    assert np.array_equal(sa.cpu().numpy().view(np.uint32), want_sa)
    assert np.array_equal(isa.cpu().numpy().view(np.uint32), want_isa)


def test_a_build_without_options_takes_the_table(gb, orc, tmp_path):
    import ctypes

    import torch
    lib = gb.load()
    path = str(tmp_path / "tuning.txt")
    table = autotune.Table(path)
    table.put(False, 2, 1 << 18, {"sort_items": 12, "refine_shape": 3, "h0_chars": 9,
                                  "bucket_min": 1 << 12})
    table.put(False, 8, 1 << 18, {"sort_items": 8, "refine_shape": 2, "h0_chars": 5,
                                  "bucket_min": 0xFFFFFFFF})
    table.save()
    gb.tuning_load(path)
    for recipe, bits, want in (("markov", 2, table.get(False, 2, 1 << 18)),
                               ("zipf_repeats", 8, table.get(False, 8, 1 << 18))):
        t = gen.text(recipe, 77, (1 << 18) + 5)
        d = dev(t)
        n = t.size
        out = torch.empty(n, dtype=torch.int32, device="cuda")
        st = gb.Stats()
        rc = lib.sa_build_ex(d.data_ptr(), n, out.data_ptr(), None, None, 0, None,
                             ctypes.byref(st), torch.cuda.current_stream().cuda_stream)
        assert rc == 0
        torch.cuda.synchronize()
        p = st.to_dict()["params"]
        assert st.bits_per_char == bits
        assert p == {"sort_items": want["sort_items"], "refine_shape": want["refine_shape"],
                     "h0_chars": want["h0_chars"], "bucket_min": want["bucket_min"],
                     "from_table": True}
        assert np.array_equal(out.cpu().numpy().view(np.uint32), orc.pd_sa(t)[0])
        # the plain entry point takes the same values (and the same SA)
        out2 = torch.empty_like(out)
        assert lib.sa_build(d.data_ptr(), n, out2.data_ptr(),
                            torch.cuda.current_stream().cuda_stream) == 0
        torch.cuda.synchronize()
        assert torch.equal(out, out2)
    # an explicit option overrides the table; an empty table gives the defaults
    t = gen.text("markov", 78, 1 << 18)
    _, _, st, _ = gb.sa_build_ex(dev(t), sort_items=16)
    assert st["params"]["sort_items"] == 16 and st["params"]["refine_shape"] == 3
    gb.tuning_load(None)
    _, _, st, _ = gb.sa_build_ex(dev(t))
    assert st["params"] == {"sort_items": 16, "refine_shape": 1, "h0_chars": 32,
                            "bucket_min": 1 << 22, "from_table": False}

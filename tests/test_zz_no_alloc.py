"""sa_build_noalloc: the allocation-free entry point, for callers that must
not allocate device memory when they build (for example beside an engine
that already reserved the GPU's memory, or on a path that cannot take
cudaMalloc's synchronisation).

Its output must equal the oracle's SA and sa_build's, exactly, on two calls
in a row (the shared scratch array keeps the previous call's contents,
which must not leak into the next result); once every size has run once,
further calls must change neither the device's free memory nor the
library pool's usage; sizes above its 2^18-byte limit must be refused.

Collected last on purpose (file name): if it fails, a run stopping at the
first failure has already run every other test.
"""
import numpy as np
import pytest

import gen

pytestmark = pytest.mark.gpu

MAX_N = 1 << 18


@pytest.fixture(scope="module")
def lib():
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_1610_03007_gb300 as gbsa
    assert torch.cuda.is_available()
    return gbsa.load()


def _cases():
    return [gen.text("zipf_repeats", 11, MAX_N), gen.text("dna", 12, 100003),
            gen.text("markov", 13, 4097), np.frombuffer(b"banana", np.uint8).copy(),
            np.zeros(1000, np.uint8), gen.text("bytes", 14, 1)]


def test_no_alloc_equals_oracle_and_sa_build_on_two_calls_in_a_row(lib):
    import torch

    import oracle
    orc = oracle.get()
    stream = torch.cuda.current_stream().cuda_stream
    for text in _cases():
        d = torch.from_numpy(text).cuda()
        n = text.size
        want = orc.pd_sa(text)[0]
        ref = torch.empty(n, dtype=torch.int32, device="cuda")
        assert lib.sa_build(d.data_ptr(), n, ref.data_ptr(), stream) == 0
        torch.cuda.synchronize()
        assert np.array_equal(ref.cpu().numpy().view(np.uint32), want), f"sa_build n={n}"
        for call in range(2):
            out = torch.full((n,), -1, dtype=torch.int32, device="cuda")
            assert lib.sa_build_noalloc(d.data_ptr(), n, out.data_ptr(), stream) == 0
            torch.cuda.synchronize()
            assert torch.equal(out, ref), f"n={n} call {call}"
            assert np.array_equal(out.cpu().numpy().view(np.uint32), want), f"n={n} call {call}"


def test_no_alloc_allocates_nothing(lib):
    """After one warm-up call per size (lazy module loading may place code
    and the scratch array on the device at first use), further calls of
    every size leave the device's free memory and the library pool's used
    and reserved bytes unchanged."""
    import torch

    import paper_1610_03007_gb300 as gbsa
    stream = torch.cuda.current_stream().cuda_stream
    texts = [torch.from_numpy(t).cuda() for t in _cases()]
    outs = [torch.empty(t.numel(), dtype=torch.int32, device="cuda") for t in texts]
    refs = []
    for d, o in zip(texts, outs):  # warm-up
        assert lib.sa_build_noalloc(d.data_ptr(), d.numel(), o.data_ptr(), stream) == 0
        refs.append(o.clone())
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    pool0 = gbsa.pool_usage()
    for _ in range(3):
        for d, o in zip(texts, outs):
            assert lib.sa_build_noalloc(d.data_ptr(), d.numel(), o.data_ptr(), stream) == 0
        torch.cuda.synchronize()
        assert torch.cuda.mem_get_info()[0] == free0
        assert gbsa.pool_usage() == pool0
    for o, r in zip(outs, refs):
        assert torch.equal(o, r)


def test_no_alloc_refuses_sizes_above_its_limit(lib):
    import torch
    stream = torch.cuda.current_stream().cuda_stream
    d = torch.zeros(MAX_N + 1, dtype=torch.uint8, device="cuda")
    out = torch.empty(MAX_N + 1, dtype=torch.int32, device="cuda")
    assert lib.sa_build_noalloc(d.data_ptr(), MAX_N + 1, out.data_ptr(), stream) == 2
    assert lib.sa_build_noalloc(None, 10, None, stream) == 1
    assert lib.sa_build_noalloc(None, 0, None, stream) == 0

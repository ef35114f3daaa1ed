"""sa_build_noalloc: the allocation-free entry point for callers that must
not allocate device memory when they build (for example beside an engine
that already reserved the GPU's memory, or on a path that cannot take
cudaMalloc's synchronisation). Its output must equal sa_build's exactly, on
two calls in a row (the shared scratch array keeps the previous call's
contents, which must not leak into the next result), and sizes above its
2^18-byte limit must be refused.

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


def test_no_alloc_equals_sa_build_on_two_calls_in_a_row(lib):
    import torch
    stream = torch.cuda.current_stream().cuda_stream
    for text in _cases():
        d = torch.from_numpy(text).cuda()
        n = text.size
        ref = torch.empty(n, dtype=torch.int32, device="cuda")
        assert lib.sa_build(d.data_ptr(), n, ref.data_ptr(), stream) == 0
        for call in range(2):
            out = torch.full((n,), -1, dtype=torch.int32, device="cuda")
            assert lib.sa_build_noalloc(d.data_ptr(), n, out.data_ptr(), stream) == 0
            torch.cuda.synchronize()
            assert torch.equal(out, ref), f"n={n} call {call}"


def test_no_alloc_refuses_sizes_above_its_limit(lib):
    import torch
    stream = torch.cuda.current_stream().cuda_stream
    d = torch.zeros(MAX_N + 1, dtype=torch.uint8, device="cuda")
    out = torch.empty(MAX_N + 1, dtype=torch.int32, device="cuda")
    assert lib.sa_build_noalloc(d.data_ptr(), MAX_N + 1, out.data_ptr(), stream) == 2
    assert lib.sa_build_noalloc(None, 10, None, stream) == 1
    assert lib.sa_build_noalloc(None, 0, None, stream) == 0

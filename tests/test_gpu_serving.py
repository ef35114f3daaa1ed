"""Serving on the GPU: requests of mixed sizes and alphabets submitted
together run concurrently (several builds in flight on their own streams),
and each result is the same as the request built alone and as the oracle's
(tolerance: exactly equal)."""
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


def test_mixed_requests_equal_their_solo_builds(gb, orc):
    _, sizes, kinds = gen.request_stream(77, 40, 1000.0, 1 << 10, 4 << 20)
    texts = [gen.request_text(77, k, int(sizes[k]), int(kinds[k])) for k in range(40)]
    texts.append(gen.text("zipf_repeats", 78, 16 << 20))  # one long-running request
    with gb.Server(budget_bytes=8 << 30, slots=8) as srv:
        tickets = [srv.submit(t) for t in texts]
        results = [srv.wait(t) for t in tickets]
        st = srv.stats()
    assert st["completed"] == len(texts)
    assert st["peak_in_flight"] > 1          # builds overlapped on the device
    assert st["peak_bytes_in_use"] <= 8 << 30
    for t, (sa, info) in zip(texts, results):
        assert info["status"] == 0
        solo = gb.sa_build_host(t)
        assert np.array_equal(sa, solo)
        if t.size <= 400_000:
            assert np.array_equal(sa, orc.pd_sa(t)[0])


def test_budget_smaller_than_the_mix(gb):
    n = 1 << 20
    texts = [gen.text("dna", 300 + k, n) for k in range(6)]
    budget = 2 * int(gb.load().sa_request_footprint(n)) + 4096
    with gb.Server(budget_bytes=budget, slots=6) as srv:
        tickets = [srv.submit(t) for t in texts]
        results = [srv.wait(t) for t in tickets]
        st = srv.stats()
    assert st["peak_in_flight"] <= 2 and st["peak_bytes_in_use"] <= budget
    for t, (sa, _) in zip(texts, results):
        assert np.array_equal(sa, gb.sa_build_host(t))


def small_texts(seed, count):
    """Texts of the serving mix's recipes with the degenerate lengths 0, 1
    and 2 among them."""
    rng = np.random.default_rng(seed)
    recipes = ("dna", "zipf_repeats", "markov", "bytes")
    texts = [gen.text(recipes[k % 4], seed * 1000 + k, int(rng.integers(3, 40_000)))
             for k in range(count)]
    texts[1], texts[5], texts[9] = texts[1][:0], texts[5][:1], texts[9][:2]
    return texts


def pinned_copy(a, dtype=np.uint8):
    import torch
    tdt = torch.uint8 if dtype == np.uint8 else torch.int32
    p = torch.empty(a.size, dtype=tdt, pin_memory=True).numpy().view(dtype)
    p[:] = a
    return p


@pytest.mark.parametrize("pinned", [False, True])
def test_batched_host_build_equals_the_oracle(gb, orc, pinned):
    """sa_build_batched_host over 70 texts (two 64-text copy tables when the
    buffers are pinned and the copies run as kernels; one copy-engine copy
    per text otherwise): every SA is the oracle's."""
    texts = small_texts(11 + pinned, 70)
    if pinned:
        texts = [pinned_copy(t) for t in texts]
        outs = [pinned_copy(np.zeros(t.size, np.uint32), np.uint32) for t in texts]
    else:
        outs = None
    sas = gb.sa_build_batched_host(texts, outs)
    for t, sa in zip(texts, sas):
        assert np.array_equal(sa, orc.pd_sa(t)[0])


def test_batched_host_build_above_the_kernel_copy_limit(gb):
    """Pinned buffers of more than 4 MiB in all take the copy engine."""
    texts = [pinned_copy(gen.text("markov", 40 + k, (2 << 20) + 7 * k)) for k in range(3)]
    sas = gb.sa_build_batched_host(texts)
    for t, sa in zip(texts, sas):
        assert np.array_equal(sa, gb.sa_build_host(t))


def test_queued_small_requests_merge_into_one_build(gb, orc):
    """With one slot busy on a long request, the small requests queued
    behind it run as merged batches (sa_build_batched_host, pinned buffers:
    kernel copies); each result equals the oracle's."""
    texts = [pinned_copy(t) for t in small_texts(21, 30)]
    outs = [pinned_copy(np.zeros(t.size, np.uint32), np.uint32) for t in texts]
    long_text = gen.text("zipf_repeats", 22, 64 << 20)
    with gb.Server(budget_bytes=8 << 30, slots=1, merge_requests=32) as srv:
        first = srv.submit(long_text)
        tickets = [srv.submit(t, o) for t, o in zip(texts, outs)]
        results = [srv.wait(t) for t in tickets]
        srv.wait(first)
        st = srv.stats()
    assert st["completed"] == 31
    assert st["merged"] >= 2 and st["builds"] < 31
    assert max(info["batch"] for _, info in results) > 1
    for t, (sa, info) in zip(texts, results):
        assert info["status"] == 0
        assert np.array_equal(sa, orc.pd_sa(t)[0])

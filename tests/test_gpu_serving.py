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

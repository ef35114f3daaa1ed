"""Serving loop admission logic, on the host: the server in simulate mode
does no GPU work (a request of n bytes "runs" for n * ns_per_byte), so
these run without a GPU and check FIFO admission, the byte budget, the slot
limit, that requests arriving during others' runs are admitted, and which
queued requests a worker merges into one build."""
import time

import numpy as np
import pytest


@pytest.fixture(scope="module")
def gbsa():
    from paper_1610_03007_gb300 import _build
    _build.build()
    import paper_1610_03007_gb300 as g
    g.load()
    return g


def foot(g, n):
    return int(g.load().sa_request_footprint(n))


def run_all(srv, sizes):
    texts = [np.zeros(n, np.uint8) for n in sizes]
    tickets = [srv.submit(t) for t in texts]
    infos = [srv.wait(t)[1] for t in tickets]
    return infos


def test_footprint_model(gbsa):
    for n in (1, 1000, 1 << 20):
        f = foot(gbsa, n)
        assert f >= n + 4 * n + gbsa.workspace_bytes(n)


def test_fifo_order_and_slot_limit(gbsa):
    with gbsa.Server(budget_bytes=1 << 40, slots=3, simulate_ns_per_byte=20.0,
                     merge_requests=1) as srv:
        infos = run_all(srv, [100_000] * 12)
        st = srv.stats()
    starts = [i["start_s"] for i in infos]
    assert starts == sorted(starts)
    assert st["peak_in_flight"] == 3
    assert st["completed"] == 12
    for i in infos:
        assert i["submit_s"] <= i["start_s"] <= i["done_s"]


def test_budget_limits_concurrency(gbsa):
    n = 200_000
    budget = 2 * foot(gbsa, n) + 1000  # room for two requests at a time
    with gbsa.Server(budget_bytes=budget, slots=8, simulate_ns_per_byte=20.0,
                     merge_requests=1) as srv:
        run_all(srv, [n] * 10)
        st = srv.stats()
    assert st["peak_in_flight"] == 2
    assert st["peak_bytes_in_use"] <= budget
    assert st["bytes_in_use"] == 0


def test_head_of_line_waits_for_memory(gbsa):
    small, big = 50_000, 400_000
    budget = foot(gbsa, big) + foot(gbsa, small)
    with gbsa.Server(budget_bytes=budget, slots=8, simulate_ns_per_byte=20.0) as srv:
        infos = run_all(srv, [small, small, big, small])
    # the big request waits until it fits; the small one behind it does not
    # overtake it (strict FIFO)
    assert infos[3]["start_s"] >= infos[2]["start_s"]
    assert infos[2]["start_s"] >= min(infos[0]["done_s"], infos[1]["done_s"])


def test_arrivals_during_runs_are_admitted(gbsa):
    with gbsa.Server(budget_bytes=1 << 40, slots=4, simulate_ns_per_byte=100.0) as srv:
        first = srv.submit(np.zeros(2_000_000, np.uint8))  # runs ~0.2 s
        time.sleep(0.02)
        later = srv.submit(np.zeros(1000, np.uint8))
        _, a = srv.wait(first)
        _, b = srv.wait(later)
    # continuous batching: the later request started and finished while the
    # first was still running
    assert b["start_s"] < a["done_s"]
    assert b["done_s"] < a["done_s"]


def test_refusals(gbsa):
    with gbsa.Server(budget_bytes=foot(gbsa, 1000), slots=2, simulate_ns_per_byte=1.0) as srv:
        with pytest.raises(gbsa.SAError) as e:
            srv.submit(np.zeros(100_000, np.uint8))
        assert e.value.status == 3  # SA_ERR_OOM: footprint above the whole budget
        t = srv.submit(np.zeros(1000, np.uint8))
        srv.wait(t)


def test_finished_requests_are_forgotten(gbsa):
    """A long-running server must not keep every request it ever saw: once
    wait() or a poll() reporting done has handed a result over, the request
    leaves the server's table and its ticket is unknown."""
    import threading
    lib = gbsa.load()
    with gbsa.Server(budget_bytes=1 << 40, slots=4, simulate_ns_per_byte=5.0) as srv:
        for rnd in range(3):
            tickets = [srv.submit(np.zeros(20_000 + 1000 * k, np.uint8)) for k in range(40)]
            assert srv.stats()["tracked"] <= 40
            for t in tickets[:20]:
                srv.wait(t)
            polled = 0
            for t in tickets[20:]:
                while srv.poll(t) is None:
                    time.sleep(0.001)
                polled += 1
            assert polled == 20
            st = srv.stats()
            assert st["tracked"] == 0, st
            assert st["completed"] == 40 * (rnd + 1)
            for t in tickets[:2]:  # collected tickets are unknown now
                assert lib.sa_server_poll(srv._h, t, None) == -1
                assert lib.sa_server_wait(srv._h, t, None) == 1  # SA_ERR_INVALID_ARG
        # several threads waiting on one ticket: each gets the result, the
        # request is freed once, and the table ends empty
        t = srv.submit(np.zeros(400_000, np.uint8))  # runs ~2 ms
        keep = srv._keep.pop(t)
        codes = []

        def waiter():
            codes.append(lib.sa_server_wait(srv._h, t, None))

        th = [threading.Thread(target=waiter) for _ in range(4)]
        for x in th:
            x.start()
        for x in th:
            x.join()
        del keep
        assert codes == [0, 0, 0, 0] or sorted(codes) == [0] * codes.count(0) + [1] * codes.count(1)
        assert 0 in codes
        assert srv.stats()["tracked"] == 0


def test_smaller_requests_get_higher_stream_priority(gbsa):
    """Size classes up to 256 KiB, 2 MiB, 16 MiB and beyond map to the
    highest priority and the next three levels (the simulate-mode range is
    [-5, 0], lower = higher); with size_priority off every request runs at
    priority 0."""
    sizes = [1, 256 << 10, (256 << 10) + 1, 2 << 20, (2 << 20) + 1, 16 << 20, (16 << 20) + 1]
    want = [-5, -5, -4, -4, -3, -3, -2]
    with gbsa.Server(budget_bytes=1 << 40, slots=2, simulate_ns_per_byte=0.001) as srv:
        infos = run_all(srv, sizes)
    assert [i["priority"] for i in infos] == want
    with gbsa.Server(budget_bytes=1 << 40, slots=2, simulate_ns_per_byte=0.001,
                     size_priority=False) as srv:
        infos = run_all(srv, sizes)
    assert all(i["priority"] == 0 for i in infos)


def merged_foot(g, sizes):
    """Device bytes of one batched build of texts of these sizes (text, SA
    and batched workspace)."""
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.uint64)
    N = int(off[-1])
    a256 = lambda x: (x + 255) & ~255
    return a256(N) + a256(4 * N) + int(g.load().sa_batched_workspace_bytes(off.ctypes.data,
                                                                           len(sizes)))


def queue_behind_one(srv, sizes, first=2_000_000):
    """Submits a request that keeps the server's only slot busy (~0.2 s at
    100 ns/byte), then `sizes` behind it; returns the infos of the queued
    ones and of the first."""
    first_t = srv.submit(np.zeros(first, np.uint8))
    while srv.stats()["in_flight"] == 0:
        time.sleep(0.001)
    tickets = [srv.submit(np.zeros(n, np.uint8)) for n in sizes]
    _, a = srv.wait(first_t)
    return [srv.wait(t)[1] for t in tickets], a


def test_merged_build_takes_the_queued_small_requests(gbsa):
    """A worker that takes a small request also takes the small requests
    queued directly behind it: they start and finish together and count as
    one build; the request that ran while they queued ran alone."""
    with gbsa.Server(budget_bytes=1 << 40, slots=1, simulate_ns_per_byte=100.0,
                     merge_requests=32) as srv:
        infos, a = queue_behind_one(srv, [10_000 + k for k in range(10)])
        st = srv.stats()
    assert a["batch"] == 1
    assert [i["batch"] for i in infos] == [10] * 10
    assert len({i["start_s"] for i in infos}) == 1
    assert len({i["done_s"] for i in infos}) == 1
    assert (st["builds"], st["merged"], st["completed"]) == (2, 10, 11)


@pytest.mark.parametrize("limit,want", [(1, [1] * 10), (4, [4] * 8 + [2] * 2),
                                        (0, [1] * 10), (1000, [10] * 10)])
def test_merge_limit(gbsa, limit, want):
    """merge_requests caps a batch (0 and 1 = no merging, the default;
    values above 64 mean 64)."""
    with gbsa.Server(budget_bytes=1 << 40, slots=1, simulate_ns_per_byte=100.0,
                     merge_requests=limit) as srv:
        infos, _ = queue_behind_one(srv, [10_000] * 10)
        st = srv.stats()
    assert [i["batch"] for i in infos] == want
    assert st["builds"] == 1 + len(set((i["start_s"] for i in infos)))


def test_merging_keeps_queue_order(gbsa):
    """A request above 256 KiB is not merged and ends the batch in front of
    it; the small requests behind it wait for it (queue order is kept)."""
    sizes = [1000, 2000, 300_000, 3000, 4000]
    with gbsa.Server(budget_bytes=1 << 40, slots=1, simulate_ns_per_byte=100.0,
                     merge_requests=32) as srv:
        infos, _ = queue_behind_one(srv, sizes)
    assert [i["batch"] for i in infos] == [2, 2, 1, 2, 2]
    starts = [i["start_s"] for i in infos]
    assert starts == sorted(starts)
    assert starts[0] < starts[2] < starts[3]


def test_merged_batch_stays_within_4_mib(gbsa):
    """A batch holds at most 4 MiB of text: 16 requests of 250,000 bytes fit,
    a 17th does not."""
    with gbsa.Server(budget_bytes=1 << 40, slots=1, simulate_ns_per_byte=10.0,
                     merge_requests=64) as srv:
        infos, _ = queue_behind_one(srv, [250_000] * 20, first=20_000_000)
    assert [i["batch"] for i in infos] == [16] * 16 + [4] * 4


def test_merged_batch_fits_the_budget(gbsa):
    """A request joins a batch only while the batch's own footprint (text,
    SA and batched workspace) fits in the budget, and that footprint is what
    the batch holds against it."""
    n = 100_000
    budget = merged_foot(gbsa, [n] * 3)
    assert merged_foot(gbsa, [n] * 4) > budget
    with gbsa.Server(budget_bytes=budget, slots=1, simulate_ns_per_byte=1000.0,
                     merge_requests=32) as srv:
        infos, _ = queue_behind_one(srv, [n] * 10, first=200_000)
        st = srv.stats()
    assert [i["batch"] for i in infos] == [3] * 9 + [1]
    assert st["peak_bytes_in_use"] == budget
    assert st["bytes_in_use"] == 0


def test_idle_workers_take_requests_unmerged(gbsa):
    """While workers are idle, each queued request goes to a worker of its
    own (running on its own stream at once) rather than into a batch."""
    with gbsa.Server(budget_bytes=1 << 40, slots=4, simulate_ns_per_byte=100.0,
                     merge_requests=32) as srv:
        infos = run_all(srv, [10_000] * 3)
        st = srv.stats()
    assert [i["batch"] for i in infos] == [1, 1, 1]
    assert (st["builds"], st["merged"]) == (3, 0)


def test_queue_is_shared_among_the_idle_workers(gbsa):
    """Four workers held idle by the budget (a large request fills it) wake
    together when it ends; each takes its share of the twelve queued small
    requests, a batch of three, instead of one worker taking all twelve."""
    big, n = 2_000_000, 10_000
    budget = foot(gbsa, big) + foot(gbsa, n) - 1  # no small request fits beside it
    assert 4 * merged_foot(gbsa, [n] * 3) <= budget
    with gbsa.Server(budget_bytes=budget, slots=4, simulate_ns_per_byte=100.0,
                     merge_requests=32) as srv:
        infos, a = queue_behind_one(srv, [n] * 12, first=big)
        st = srv.stats()
    assert a["batch"] == 1
    assert [i["batch"] for i in infos] == [3] * 12
    assert len({i["slot"] for i in infos}) == 4
    assert st["builds"] == 5


@pytest.mark.parametrize("seed", range(6))
def test_random_mixes_keep_the_invariants(gbsa, seed):
    """Random sizes (small and large), slots, budgets and merge limits: every
    request completes; starts follow queue order; a batch is a run of
    consecutive requests that started together on one worker, of at most
    merge_requests requests, each at most 256 KiB and 4 MiB in all when
    there are several; the budget is never exceeded and ends unused."""
    rng = np.random.default_rng(seed)
    count = 60
    small = rng.integers(1, 256 << 10, count)
    large = rng.integers((256 << 10) + 1, 3 << 20, count)
    sizes = np.where(rng.random(count) < 0.7, small, large)
    slots = int(rng.integers(1, 7))
    limit = int(rng.choice([1, 2, 5, 32, 64]))
    budget = int(foot(gbsa, int(sizes.max())) * rng.uniform(1.0, 4.0))
    with gbsa.Server(budget_bytes=budget, slots=slots, simulate_ns_per_byte=2.0,
                     merge_requests=limit) as srv:
        tickets = []
        for n in sizes:
            tickets.append(srv.submit(np.zeros(int(n), np.uint8)))
            if rng.random() < 0.2:
                time.sleep(0.002)
        infos = [srv.wait(t)[1] for t in tickets]
        st = srv.stats()
    assert st["completed"] == count and st["bytes_in_use"] == 0 and st["in_flight"] == 0
    assert st["peak_bytes_in_use"] <= budget
    assert all(i["status"] == 0 for i in infos)
    starts = [i["start_s"] for i in infos]
    assert starts == sorted(starts)
    k, builds = 0, 0
    while k < count:
        b = infos[k]["batch"]
        group = infos[k:k + b]
        assert len(group) == b and b <= max(limit, 1)
        assert len({(i["slot"], i["start_s"], i["done_s"], i["batch"]) for i in group}) == 1
        if b > 1:
            assert all(int(sizes[j]) <= 256 << 10 for j in range(k, k + b))
            assert int(sizes[k:k + b].sum()) <= 4 << 20
        k += b
        builds += 1
    assert st["builds"] == builds
    assert st["merged"] == sum(1 for i in infos if i["batch"] > 1)

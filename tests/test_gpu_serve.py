"""The continuously batched server on the serving ring: every deleteMin
result is the same as when the heap's requests run alone, one at a time, and
as the oracle's; requests that arrive while others are on the GPU enter the
ring at once and run beside them."""
import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1906_06504_gb300 import build
    build.build()
    torch.cuda.set_device(0)


from heaputil import to_dev, to_host  # noqa: E402


def alone(reqs, heap_id, cap, k):
    """The heap's accepted requests, in arrival order, one call at a time."""
    from paper_1906_06504_gb300.heap import GHeap
    res = {}
    with GHeap(capacity=cap, k=k) as h:
        for r in sorted([r for r in reqs if r.heap == heap_id and r.error is None],
                        key=lambda r: (r.arrival, r.rid)):
            if r.kind == "ins":
                h.insert(to_dev(np.asarray(r.keys, np.uint32)))
            else:
                out, cnt = h.delete_min(r.n)
                h.sync()
                res[r.rid] = to_host(out, 4)[:int(cnt.item())]
    return res


def check_against_oracle(reqs):
    by_heap = {}
    for r in sorted(reqs, key=lambda r: (r.arrival, r.rid)):
        if r.error is None:
            by_heap.setdefault(r.heap, []).append(r)
    for h, rs in by_heap.items():
        q = oracle.BinaryHeapPQ()
        try:
            for r in rs:
                if r.kind == "ins":
                    q.push(np.asarray(r.keys, np.uint32))
                else:
                    want = q.pop(r.n, dtype=np.uint32)
                    assert np.array_equal(r.result, want), (h, r.rid)
        finally:
            q.close()


def overlapping_pairs(reqs):
    """Pairs of requests that were in the ring at the same time: (same heap,
    different heaps)."""
    done = sorted([r for r in reqs if r.t_submit is not None], key=lambda r: r.t_submit)
    same = diff = 0
    for i, a in enumerate(done):
        for b in done[i + 1:i + 64]:
            if b.t_submit < a.t_done:
                if a.heap == b.heap:
                    same += 1
                else:
                    diff += 1
    return same, diff


@pytest.mark.parametrize("realtime", [False, True])
def test_server_results_equal_alone_and_oracle(realtime):
    from paper_1906_06504_gb300.serve import HeapServer, poisson_requests
    k, n_heaps, cap = 256, 10, 1 << 16
    reqs = poisson_requests(123, 500, n_heaps, rate_per_s=20000.0, max_keys=2048)
    srv = HeapServer([cap] * n_heaps, k=k, arena_keys=1 << 18)
    try:
        srv.run(reqs, realtime=realtime)
        # several requests were in the ring at once; arriving in real time,
        # requests entered it while earlier ones were still on the GPU
        assert srv.stats["max_inflight"] > 1
        if realtime:
            assert srv.stats["submitted_while_busy"] > 0
    finally:
        srv.close()
    assert all(r.t_done is not None and r.error is None for r in reqs)
    check_against_oracle(reqs)
    for hid in range(n_heaps):
        for rid, res in alone(reqs, hid, cap, k).items():
            assert np.array_equal(reqs[rid].result, res), (hid, rid)


def test_requests_overlap_on_the_device_and_stay_exact():
    """A burst on few heaps: many requests of one heap are in the ring at once
    (each heap still takes them in order), and requests of different heaps
    run side by side; every result equals the heap's requests alone."""
    from paper_1906_06504_gb300.serve import HeapServer, poisson_requests
    k, n_heaps, cap = 1024, 4, 1 << 20
    reqs = poisson_requests(77, 2000, n_heaps, rate_per_s=400000.0, max_keys=4096)
    srv = HeapServer([cap] * n_heaps, k=k, arena_keys=1 << 22)
    try:
        srv.preadmit(range(n_heaps))
        srv.run(reqs, realtime=True)
        assert srv.stats["max_inflight"] >= 8, srv.stats
    finally:
        srv.close()
    same, diff = overlapping_pairs(reqs)
    assert same > 0 and diff > 0, (same, diff)
    assert all(r.error is None for r in reqs)
    check_against_oracle(reqs)
    for hid in range(n_heaps):
        for rid, res in alone(reqs, hid, cap, k).items():
            assert np.array_equal(reqs[rid].result, res), (hid, rid)


def test_capacity_is_enforced_on_the_host():
    """An insert that could overflow its heap waits for the deleteMins ahead
    of it to make room; one that cannot fit when nothing of its heap is in
    flight is refused as full, and one larger than the heap at once; refused
    requests never reach the device and the results stay exact."""
    from paper_1906_06504_gb300.serve import HeapServer, Request
    k, cap = 64, 4096
    rng = np.random.default_rng(3)
    keys = lambda n: rng.integers(0, 2**32, n, dtype=np.uint64).astype(np.uint32)
    reqs = [Request(0, 0.0, 0, "ins", keys=keys(cap - 10)),
            Request(1, 0.0, 0, "ins", keys=keys(cap + 1)),      # larger than the heap
            Request(2, 0.0, 0, "del", n=500),
            Request(3, 0.0, 0, "ins", keys=keys(100)),          # waits for request 2
            Request(4, 0.0, 0, "del", n=cap),
            Request(5, 0.0, 1, "ins", keys=keys(300)),
            Request(6, 0.0, 1, "ins", keys=keys(cap - 100)),    # refused: full
            Request(7, 0.0, 1, "del", n=1000)]
    srv = HeapServer([cap, cap], k=k, arena_keys=1 << 16)
    try:
        srv.run(reqs, realtime=False)
        assert srv.stats["refused"] == 2
    finally:
        srv.close()
    assert "capacity" in reqs[1].error and "full" in reqs[6].error
    assert all(r.error is None for r in reqs if r.rid not in (1, 6))
    assert reqs[2].result.size == 500
    assert reqs[4].result.size == cap - 10 - 500 + 100
    assert reqs[7].result.size == 300
    check_against_oracle(reqs)


def test_server_admits_heaps_by_hbm_budget():
    """A budget for about three heaps: heaps whose work is done (empty, idle)
    are evicted so that later heaps can be admitted; results stay exact."""
    from paper_1906_06504_gb300.serve import HeapServer, Request
    k, n_heaps, cap = 128, 9, 1 << 14
    rng = np.random.default_rng(5)
    reqs, rid = [], 0
    for h in range(n_heaps):
        keys = rng.integers(0, 2**32, 3000, dtype=np.uint64).astype(np.uint32)
        t = 0.001 * h
        reqs.append(Request(rid, t, h, "ins", keys=keys)); rid += 1
        reqs.append(Request(rid, t, h, "del", n=1000)); rid += 1
        reqs.append(Request(rid, t, h, "del", n=5000)); rid += 1
    srv = HeapServer([cap] * n_heaps, k=k, arena_keys=1 << 16)
    srv.budget = 3 * srv._bytes(0) + 1
    try:
        srv.run(reqs, realtime=False)
        assert srv.stats["evicted"] >= n_heaps - 3
    finally:
        srv.close()
    check_against_oracle(reqs)
    for r in reqs:
        if r.kind == "del" and r.n == 5000:
            assert r.result.size == 2000

"""The continuously batched server: every deleteMin result is the same as
when the heap's requests run alone, one at a time, and as the oracle's."""
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
    """The heap's requests, in arrival order, one call at a time."""
    from paper_1906_06504_gb300.heap import GHeap
    res = {}
    with GHeap(capacity=cap, k=k) as h:
        for r in sorted([r for r in reqs if r.heap == heap_id], key=lambda r: (r.arrival, r.rid)):
            if r.kind == "ins":
                h.insert(to_dev(np.asarray(r.keys, np.uint32)))
            else:
                out, cnt = h.delete_min(r.n)
                h.sync()
                res[r.rid] = to_host(out, 4)[:int(cnt.item())]
    return res


def check_against_oracle(reqs, n_heaps):
    by_heap = {}
    for r in sorted(reqs, key=lambda r: (r.arrival, r.rid)):
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


@pytest.mark.parametrize("realtime", [False, True])
def test_server_results_equal_alone_and_oracle(realtime):
    from paper_1906_06504_gb300.serve import HeapServer, poisson_requests
    k, n_heaps, cap = 256, 10, 1 << 16
    reqs = poisson_requests(123, 500, n_heaps, rate_per_s=20000.0, max_keys=2048)
    srv = HeapServer([cap] * n_heaps, k=k, max_batch_keys=1 << 18)
    try:
        srv.run(reqs, realtime=realtime)
        assert srv.stats["batches"] < len(reqs)        # requests were batched
    finally:
        srv.close()
    assert all(r.t_done is not None for r in reqs)
    check_against_oracle(reqs, n_heaps)
    for hid in range(n_heaps):
        for rid, res in alone(reqs, hid, cap, k).items():
            assert np.array_equal(reqs[rid].result, res), (hid, rid)


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
    srv = HeapServer([cap] * n_heaps, k=k)
    srv.budget = 3 * srv._bytes(0) + 1
    try:
        srv.run(reqs, realtime=False)
        assert srv.stats["evicted"] >= n_heaps - 3
    finally:
        srv.close()
    check_against_oracle(reqs, n_heaps)
    for r in reqs:
        if r.kind == "del" and r.n == 5000:
            assert r.result.size == 2000

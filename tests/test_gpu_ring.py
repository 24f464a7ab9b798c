"""The serving ring through its C ABI (include/gheap.h heapring_*).

One persistent launch takes the operations the host appends while it runs.
Checked here: results equal the oracle's per-heap replay in submission order
(each heap takes its requests in that order) for 4- and 8-byte keys; the
launch can be stopped and started again any number of times, every published
operation running exactly once; a request that fails on the device reports
its heap's error in its completion status while the other heaps stay exact;
a launch left idle keeps serving.
"""
import time

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


def make(caps, k, key_bytes, **kw):
    from paper_1906_06504_gb300.heap import GHeap, GHeapRing, GHeapSet
    hs = GHeapSet([0] * len(caps), k=k, key_bytes=key_bytes)
    heaps = []
    for i, c in enumerate(caps):
        h = GHeap(c, k=k, key_bytes=key_bytes)
        hs.bind(i, h)
        heaps.append(h)
    ring = GHeapRing(hs, **kw)
    return hs, heaps, ring


def drain(ring, pending, results, timeout=20.0):
    t0 = time.time()
    while pending:
        ids, counts, status = ring.poll()
        if ids.size:
            dels = np.array([pending[i][0] == 2 for i in ids.tolist()])
            outs = ring.take(ids, np.where(dels, counts, 0))
            for i, st, out in zip(ids.tolist(), status.tolist(), outs):
                results[i] = (pending.pop(i), st, out)
        assert time.time() - t0 < timeout, "ring did not complete"


def run_random(ring, n_heaps, key_bytes, rng, n_req, max_keys, results, restart_every=None):
    from paper_1906_06504_gb300.heap import OP_DEL, OP_INS
    dt = np.uint32 if key_bytes == 4 else np.uint64
    pending = {}
    order = []
    i = 0
    while i < n_req:
        m = int(rng.integers(1, 40))
        heaps = rng.integers(0, n_heaps, m).astype(np.uint32)
        kinds = np.where(rng.random(m) < 0.55, OP_INS, OP_DEL).astype(np.uint32)
        sizes = rng.integers(1, max_keys + 1, m).astype(np.uint64)
        keys = [rng.integers(0, np.iinfo(dt).max, int(s), dtype=dt, endpoint=True)
                for s, kd in zip(sizes, kinds) if kd == OP_INS]
        ids = ring.submit(heaps, kinds, sizes, np.concatenate(keys) if keys else None)
        ki = 0
        for j, rid in enumerate(ids.tolist()):
            ks = None
            if kinds[j] == OP_INS:
                ks = keys[ki]
                ki += 1
            pending[rid] = (int(kinds[j]), int(heaps[j]), int(sizes[j]), ks)
            order.append(rid)
        i += ids.size
        if restart_every and (i // restart_every) != ((i - ids.size) // restart_every):
            ring.stop()             # every published operation runs before it ends
            ring.start()
        if len(pending) > 256:
            drain(ring, pending, results)
    drain(ring, pending, results)
    return order


def check(order, results, n_heaps, key_bytes):
    dt = np.uint32 if key_bytes == 4 else np.uint64
    qs = [oracle.BinaryHeapPQ() for _ in range(n_heaps)]
    try:
        for rid in order:
            (kind, h, n, ks), st, out = results[rid]
            assert st == 0, (rid, st)
            if kind == 1:
                qs[h].push(ks)
            else:
                assert np.array_equal(out, qs[h].pop(n, dtype=dt)), rid
    finally:
        for q in qs:
            q.close()


@pytest.mark.parametrize("key_bytes,k", [(4, 256), (8, 128)])
def test_ring_matches_oracle_with_restarts(key_bytes, k):
    n_heaps = 6
    hs, heaps, ring = make([1 << 16] * n_heaps, k, key_bytes, max_requests=512, max_ops=2048,
                           in_keys=1 << 17, out_keys=1 << 17)
    try:
        ring.start()
        results = {}
        order = run_random(ring, n_heaps, key_bytes, np.random.default_rng(5 + key_bytes), 1500,
                           700, results, restart_every=300)
        ring.stop()
        check(order, results, n_heaps, key_bytes)
        assert ring.pending() == 0
    finally:
        ring.close()
        hs.close()
        for h in heaps:
            h.close()


def test_ring_reports_a_device_error_per_request():
    """Heap 0 has room for three nodes and is sent five nodes' worth of keys
    (the host checks nothing here): that insert completes with
    GHEAP_ERR_FULL, and so does the later request on heap 0; heap 1 is
    served exactly."""
    from paper_1906_06504_gb300.heap import ERR_FULL, OP_DEL, OP_INS
    k = 64
    hs, heaps, ring = make([2 * k, 1 << 14], k, 4, max_requests=64, max_ops=256,
                           in_keys=1 << 14, out_keys=1 << 14)
    try:
        ring.start()
        rng = np.random.default_rng(9)
        a = rng.integers(0, 2**32, 5 * k, dtype=np.uint64).astype(np.uint32)
        b = rng.integers(0, 2**32, 1000, dtype=np.uint64).astype(np.uint32)
        ids = ring.submit([0, 1, 0, 1], [OP_INS, OP_INS, OP_DEL, OP_DEL], [5 * k, 1000, 10, 300],
                          np.concatenate([a, b]))
        assert ids.size == 4
        pending = {int(i): (kd,) for i, kd in zip(ids, [1, 1, 2, 2])}
        results = {}
        drain(ring, pending, results)
        ring.stop()
        st = {rid: results[rid][1] for rid in results}
        assert st[int(ids[0])] == ERR_FULL and st[int(ids[2])] == ERR_FULL
        assert st[int(ids[1])] == 0 and st[int(ids[3])] == 0
        assert np.array_equal(results[int(ids[3])][2], np.sort(b)[:300])
    finally:
        ring.close()
        hs.close()
        for h in heaps:
            h.close()


def test_idle_ring_keeps_serving():
    from paper_1906_06504_gb300.heap import OP_DEL, OP_INS
    k = 128
    hs, heaps, ring = make([1 << 12], k, 4, max_requests=16, max_ops=64, in_keys=1 << 13,
                           out_keys=1 << 13)
    try:
        ring.start()
        rng = np.random.default_rng(2)
        for rnd in range(3):
            time.sleep(0.2)              # nothing published meanwhile
            a = rng.integers(0, 2**32, 500, dtype=np.uint64).astype(np.uint32)
            ids = ring.submit([0, 0], [OP_INS, OP_DEL], [500, 500], a)
            pending = {int(ids[0]): (1,), int(ids[1]): (2,)}
            results = {}
            drain(ring, pending, results)
            assert np.array_equal(results[int(ids[1])][2], np.sort(a))
        ring.stop()
    finally:
        ring.close()
        hs.close()
        for h in heaps:
            h.close()

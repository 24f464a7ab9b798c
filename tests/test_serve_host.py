"""Host-side policy of the serving loop on CPU, with the device side faked.

The server forms each batch from the arrived requests -- at most one per
heap, in arrival order, so that every heap sees its requests in FIFO order --
within a request and key budget, and admits a heap on its first request when
the HBM budget allows, evicting heaps that are empty, idle and not waited
for.  These rules decide which requests share a launch; they involve no heap
arithmetic, so they are checked here against a fake heap set.
"""
import collections

import numpy as np
import pytest

from paper_1906_06504_gb300 import serve
from paper_1906_06504_gb300.serve import HeapServer, Request


class FakeHeap:
    closed = 0

    def __init__(self, capacity, k=1024, key_bytes=4):
        self.capacity = capacity

    def close(self):
        FakeHeap.closed += 1


class FakeSet:
    def __init__(self):
        self.bound = {}

    def bind(self, i, heap, stream=None):
        assert i not in self.bound
        self.bound[i] = heap

    def unbind(self, i, stream=None):
        del self.bound[i]


def make_server(capacities, k=4, budget=None, max_keys=64, max_reqs=8):
    """A HeapServer without device buffers: only its host policy is used."""
    s = HeapServer.__new__(HeapServer)
    s.k = k
    s.key_bytes = 4
    s.capacities = list(capacities)
    s.n_heaps = len(capacities)
    s.budget = budget if budget is not None else 1 << 62
    s.used = 0
    s.set = FakeSet()
    s.heaps = [None] * s.n_heaps
    s.size = [0] * s.n_heaps
    s.busy = [0] * s.n_heaps
    s.max_keys = max_keys
    s.max_reqs = max_reqs
    s.stream = None
    s.stats = {"batches": 0, "admitted": 0, "evicted": 0, "ops": 0}
    return s


@pytest.fixture(autouse=True)
def fake_heap(monkeypatch):
    monkeypatch.setattr(serve, "GHeap", FakeHeap)
    FakeHeap.closed = 0


def ins(rid, heap, n):
    return Request(rid, 0.0, heap, "ins", keys=np.zeros(n, np.uint32))


def dele(rid, heap, n):
    return Request(rid, 0.0, heap, "del", n=n)


def test_one_request_per_heap_fifo():
    s = make_server([100] * 3)
    pending = collections.deque([ins(0, 0, 4), ins(1, 0, 4), ins(2, 1, 4), dele(3, 0, 2),
                                 ins(4, 2, 4), ins(5, 1, 4)])
    first = s._select(pending)
    assert [r.rid for r in first] == [0, 2, 4]
    # the rest keep their order; heap 0's requests stay in arrival order
    assert [r.rid for r in pending] == [1, 3, 5]
    second = s._select(pending)
    assert [r.rid for r in second] == [1, 5]
    assert [r.rid for r in pending] == [3]


def test_request_and_key_budgets():
    s = make_server([1000] * 6, max_keys=10, max_reqs=2)
    pending = collections.deque([ins(0, 0, 6), ins(1, 1, 6), ins(2, 2, 3), ins(3, 3, 1)])
    got = s._select(pending)
    # request 1 would pass the key budget (12 > 10); requests are capped at 2
    assert [r.rid for r in got] == [0, 2]
    assert [r.rid for r in pending] == [1, 3]


def test_delete_counts_what_the_heap_can_return():
    s = make_server([1000] * 2, max_keys=8)
    s.size = [3, 100]
    pending = collections.deque([dele(0, 0, 50), dele(1, 1, 5), dele(2, 1, 1)])
    got = s._select(pending)
    # heap 0 can return 3 keys, heap 1 five: 8 keys fit; request 2 waits (FIFO)
    assert [r.rid for r in got] == [0, 1]
    assert [r.rid for r in pending] == [2]


def test_admission_evicts_empty_idle_heaps_only():
    k = 4
    s = make_server([400] * 4, k=k)
    one = s._bytes(0)
    s.budget = 2 * one
    assert s._admit(0, set()) and s._admit(1, set())
    assert s.used == 2 * one and s.stats["admitted"] == 2
    # heap 0 holds keys, heap 1 is empty but busy: nothing can go
    s.size[0] = 5
    s.busy[1] = 1
    assert not s._admit(2, set())
    assert s.heaps[2] is None and s.stats["evicted"] == 0
    # heap 1 idle now, but a pending request waits for it
    s.busy[1] = 0
    assert not s._admit(2, {1})
    # nobody waits: heap 1 is evicted for heap 2
    assert s._admit(2, set())
    assert s.heaps[1] is None and s.heaps[2] is not None
    assert s.stats["evicted"] == 1 and FakeHeap.closed == 1
    assert s.used == 2 * one
    assert set(s.set.bound) == {0, 2}


def test_admission_failure_keeps_the_request_pending():
    s = make_server([400] * 2)
    s.budget = s._bytes(0)
    assert s._admit(0, set())
    s.size[0] = 1
    pending = collections.deque([ins(0, 1, 4), ins(1, 0, 4)])
    got = s._select(pending)
    # heap 1 cannot be admitted (heap 0 is not empty): its request waits,
    # heap 0's request is served
    assert [r.rid for r in got] == [1]
    assert [r.rid for r in pending] == [0]

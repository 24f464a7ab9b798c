"""Host-side policy of the serving loop on CPU, with the device side faked.

The server submits arrived requests to the serving ring as soon as their heap
may take them: per heap in arrival order (so every heap sees its requests in
FIFO order, several in flight at once), holding an insert that could take its
heap past capacity until deleteMins make room, refusing requests no heap or
ring could ever hold, and admitting a heap on its first request when the HBM
budget allows, evicting heaps that are empty, idle and not waited for (with
the ring's launch paused meanwhile).  These rules decide what enters the ring
and when; they involve no heap arithmetic, so they are checked here against
fakes of the heap, the heap set and the ring.
"""
import collections

import numpy as np
import pytest

from paper_1906_06504_gb300 import serve
from paper_1906_06504_gb300.serve import HeapServer, Request


class FakeHeap:
    closed = 0
    code = 0

    def __init__(self, capacity, k=1024, key_bytes=4):
        self.capacity = capacity

    def sync_code(self):
        return FakeHeap.code

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


class FakeRing:
    def __init__(self, keys=1 << 20):
        self.in_keys = self.out_keys = keys
        self.running = False
        self.log = []

    def start(self):
        self.running = True
        self.log.append("start")

    def stop(self):
        self.running = False
        self.log.append("stop")

    def attach(self, i):
        assert not self.running
        self.log.append("attach %d" % i)


def make_server(capacities, k=4, budget=None, arena=1 << 20):
    """A HeapServer without device state: only its host policy is used."""
    s = HeapServer.__new__(HeapServer)
    s.k = k
    s.key_bytes = 4
    s.capacities = list(capacities)
    s.n_heaps = len(capacities)
    s.budget = budget if budget is not None else 1 << 62
    s.used = 0
    s.set = FakeSet()
    s.ring = FakeRing(arena)
    s.heaps = [None] * s.n_heaps
    s.size = [0] * s.n_heaps
    s.busy = [0] * s.n_heaps
    s.stream = None
    s.stats = {"submits": 0, "admitted": 0, "evicted": 0, "requests": 0, "max_inflight": 0,
               "submitted_while_busy": 0, "refused": 0}
    return s


@pytest.fixture(autouse=True)
def fake_heap(monkeypatch):
    monkeypatch.setattr(serve, "GHeap", FakeHeap)
    FakeHeap.closed = 0
    FakeHeap.code = 0


def ins(rid, heap, n):
    return Request(rid, 0.0, heap, "ins", keys=np.zeros(n, np.uint32))


def dele(rid, heap, n):
    return Request(rid, 0.0, heap, "del", n=n)


def test_several_requests_per_heap_in_arrival_order():
    s = make_server([100] * 3)
    pending = collections.deque([ins(0, 0, 4), ins(1, 0, 4), ins(2, 1, 4), dele(3, 0, 2),
                                 ins(4, 2, 4), ins(5, 1, 4)])
    got = s._select(pending, 0.0)
    assert [r.rid for r in got] == [0, 1, 2, 3, 4, 5]
    assert not pending
    assert s.size == [8, 8, 4]


def test_insert_waits_for_room_and_blocks_only_its_heap():
    s = make_server([10, 10])
    s._admit(0, set())
    s._admit(1, set())
    s.size = [8, 0]
    s.busy = [1, 0]           # an earlier request of heap 0 is in flight
    pending = collections.deque([ins(0, 0, 4), dele(1, 0, 3), ins(2, 1, 4), ins(3, 0, 1)])
    got = s._select(pending, 0.0)
    # heap 0's insert could overflow it: it and everything after it on heap 0
    # wait, in order; heap 1 goes on
    assert [r.rid for r in got] == [2]
    assert [r.rid for r in pending] == [0, 1, 3]
    # the deleteMins of heap 0 made room
    s.size[0] = 5
    got = s._select(pending, 0.0)
    assert [r.rid for r in got] == [0, 1, 3]


def test_refusal_reasons():
    s = make_server([10, 1 << 30], arena=64)
    s.budget = s._bytes(0) + 1
    reqs = [ins(0, 0, 11), dele(1, 0, 65), ins(2, 1, 4), ins(3, 0, 10)]
    assert "capacity" in s._refuse_reason(reqs[0])
    assert "arenas" in s._refuse_reason(reqs[1])
    assert "HBM budget" in s._refuse_reason(reqs[2])
    assert s._refuse_reason(reqs[3]) is None
    pending = collections.deque(reqs)
    got = s._select(pending, 0.25)
    assert [r.rid for r in got] == [3]
    for r in reqs[:3]:
        assert r.error and r.t_done == 0.25 and r.result is None


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


def test_admission_pauses_a_running_ring():
    s = make_server([400] * 2)
    s.ring.start()
    assert s._admit(1, set())
    assert s.ring.log == ["start", "stop", "attach 1", "start"]
    assert s.ring.running
    # an admitted heap needs no pause
    assert s._admit(1, set())
    assert s.ring.log[-1] == "start" and len(s.ring.log) == 4


def test_eviction_reports_a_heap_error():
    s = make_server([400] * 2)
    s.budget = s._bytes(0)
    assert s._admit(0, set())
    FakeHeap.code = -4
    from paper_1906_06504_gb300.heap import GHeapError
    with pytest.raises(GHeapError):
        s._admit(1, set())


def test_admission_failure_keeps_the_request_pending():
    s = make_server([400] * 2)
    s.budget = s._bytes(0)
    assert s._admit(0, set())
    s.size[0] = 1
    pending = collections.deque([ins(0, 1, 4), ins(1, 0, 4)])
    got = s._select(pending, 0.0)
    # heap 1 cannot be admitted (heap 0 is not empty): its request waits,
    # heap 0's request is served
    assert [r.rid for r in got] == [1]
    assert [r.rid for r in pending] == [0]


def test_insert_that_cannot_fit_is_refused_when_its_heap_is_idle():
    s = make_server([10, 10])
    s._admit(0, set())
    s.size = [8, 0]
    pending = collections.deque([ins(0, 0, 4), dele(1, 0, 3)])
    got = s._select(pending, 0.5)
    # nothing of heap 0 is in flight: waiting cannot help, and the deleteMin
    # behind the insert must not overtake it -- the insert is refused as full
    assert [r.rid for r in got] == [1]
    assert not pending and s.stats["refused"] == 1


def test_insert_waits_for_a_deletemin_submitted_with_it():
    s = make_server([10])
    s._admit(0, set())
    s.size = [8]
    pending = collections.deque([dele(0, 0, 5), ins(1, 0, 4)])
    got = s._select(pending, 0.0)
    # the deleteMin ahead of it may make room: the insert waits, not refused
    assert [r.rid for r in got] == [0]
    assert [r.rid for r in pending] == [1] and s.stats["refused"] == 0

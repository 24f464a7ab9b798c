"""Continuous batching of insert / deleteMin requests over many heaps.

Requests name a heap and carry either keys to insert or a count of smallest
keys to remove.  They arrive over time.  The server keeps every heap resident
on the device in one heap set and serves them through the set's serving ring
(include/gheap.h heapring_*): one persistent launch runs for the whole
session, and each request that has arrived is appended to the ring as soon as
its heap may take it, so it starts on the device while earlier requests are
still running there -- requests on different heaps run side by side, and
requests on one heap run in their arrival order, several at a time.  The
launch reads the requests and keys from pinned host memory and writes the
results and completion records back there; the host loop only submits, polls
and collects.  A heap is admitted (allocated and bound into the set) on its
first request when the HBM budget allows, evicting heaps that are empty and
idle when the budget is needed (the launch is paused for that).

Requests a heap cannot hold are refused with an error rather than lost: an
insert that could take a heap past its capacity waits while earlier requests
of that heap are in flight (their deleteMins may make room) and is refused as
full when none are; one larger than the whole capacity, or larger than the
ring's key arenas, is refused at once.

All heap arithmetic runs in the CUDA kernels behind the C ABI; this module
only arranges requests, copies keys into and out of the ring, and keeps time.
"""
import collections
import time

import numpy as np

from .heap import GHeap, GHeapRing, GHeapSet, GHeapError, OP_DEL, OP_INS


class Request:
    """One client request.  kind "ins" carries `keys`; kind "del" asks for the
    `n` smallest keys.  After serving: `result` (del: the keys removed,
    ascending), `t_submit` and `t_done` (seconds since the run started, when
    it entered the ring and when its completion was seen), `latency` (from
    arrival) and `error` (None, or why it was refused or failed)."""

    __slots__ = ("rid", "arrival", "heap", "kind", "keys", "n", "result", "t_done", "latency",
                 "t_submit", "error")

    def __init__(self, rid, arrival, heap, kind, keys=None, n=0):
        self.rid = rid
        self.arrival = float(arrival)
        self.heap = int(heap)
        self.kind = kind
        self.keys = keys
        self.n = int(n if kind == "del" else len(keys))
        self.result = None
        self.t_done = None
        self.latency = None
        self.t_submit = None
        self.error = None         # why the request was refused or failed, else None


class HeapServer:
    """Serves requests on `capacities` heaps (keys each) of node capacity k."""

    def __init__(self, capacities, k=1024, key_bytes=4, hbm_budget=None, max_inflight=8192,
                 max_ops=1 << 16, arena_keys=1 << 24, items_per_thread=None, ctas=0,
                 stats=False):
        import torch
        self.torch = torch
        self.k = int(k)
        self.key_bytes = int(key_bytes)
        self.capacities = [int(c) for c in capacities]
        self.n_heaps = len(self.capacities)
        self.budget = hbm_budget if hbm_budget is not None else 1 << 62
        self.used = 0
        self.set = GHeapSet([0] * self.n_heaps, k=k, key_bytes=key_bytes, stats=stats)
        if items_per_thread is not None or ctas:
            self.set.set_launch(ctas=ctas, items_per_thread=items_per_thread or 8)
        self.ring = GHeapRing(self.set, max_requests=max_inflight, max_ops=max_ops,
                              in_keys=arena_keys, out_keys=arena_keys)
        self.heaps = [None] * self.n_heaps       # owning GHeap per admitted heap
        self.size = [0] * self.n_heaps           # keys held: an upper bound
        self.busy = [0] * self.n_heaps           # requests in the ring
        self.np_key = np.uint32 if key_bytes == 4 else np.uint64
        self.stream = torch.cuda.Stream()
        self.stats = {"submits": 0, "admitted": 0, "evicted": 0, "requests": 0,
                      "max_inflight": 0, "submitted_while_busy": 0, "refused": 0}

    # -- heap admission under the HBM budget
    def _bytes(self, h):
        nodes = self.capacities[h] // self.k + 2
        return nodes * self.k * self.key_bytes + nodes * 4 + self.k * self.key_bytes + 512

    def _admit(self, h, pending_heaps):
        if self.heaps[h] is not None:
            return True
        need = self._bytes(h)
        if need > self.budget:
            return False
        was_running = self.ring.running
        if was_running:
            # heap memory is allocated and freed with the launch paused
            self.ring.stop()
        try:
            if self.used + need > self.budget:
                # evict empty, idle heaps that nobody is waiting for
                for g in range(self.n_heaps):
                    if self.used + need <= self.budget:
                        break
                    if (self.heaps[g] is not None and self.size[g] == 0 and self.busy[g] == 0
                            and g not in pending_heaps):
                        code = self.heaps[g].sync_code()
                        if code != 0:
                            raise GHeapError(code, "heap %d before eviction" % g)
                        self.set.unbind(g, stream=self.stream)
                        self.heaps[g].close()
                        self.heaps[g] = None
                        self.used -= self._bytes(g)
                        self.stats["evicted"] += 1
            if self.used + need > self.budget:
                return False
            heap = GHeap(self.capacities[h], k=self.k, key_bytes=self.key_bytes)
            self.set.bind(h, heap, stream=self.stream)
            self.ring.attach(h)
            self.heaps[h] = heap
            self.used += need
            self.stats["admitted"] += 1
            return True
        finally:
            if was_running:
                self.ring.start()

    def preadmit(self, heaps):
        """Admits heaps ahead of their first request (allocation is not free)."""
        for h in heaps:
            if not self._admit(int(h), set()):
                raise RuntimeError("heap %d does not fit the HBM budget" % h)
        self.torch.cuda.synchronize()

    # -- checks that do not depend on the heap's state
    def _refuse_reason(self, r):
        if r.n < 1:
            return "empty request"
        if r.kind == "ins" and r.n > self.capacities[r.heap]:
            return "insert of %d keys exceeds the heap's capacity %d" % (
                r.n, self.capacities[r.heap])
        if r.n > min(self.ring.in_keys, self.ring.out_keys):
            return "request of %d keys exceeds the ring's key arenas (%d)" % (
                r.n, min(self.ring.in_keys, self.ring.out_keys))
        if self._bytes(r.heap) > self.budget:
            return "heap %d alone exceeds the HBM budget" % r.heap
        return None

    def _select(self, pending, now):
        """The requests to submit now: per heap in arrival order, each heap
        stopping at its first request that must wait (an insert that could
        overflow the heap, or a heap that cannot be admitted yet)."""
        taken, blocked, keep = [], set(), collections.deque()
        taken_heaps = set()
        pend_heaps = {r.heap for r in pending}
        while pending:
            r = pending.popleft()
            h = r.heap
            if h in blocked:
                keep.append(r)
                continue
            why = self._refuse_reason(r)
            if why is not None:
                r.error = why
                r.t_done = now
                r.latency = now - r.arrival
                self.stats["refused"] += 1
                continue
            fits = r.kind == "del" or self.size[h] + r.n <= self.capacities[h]
            if not fits and self.busy[h] == 0 and h not in taken_heaps:
                # nothing of this heap is in flight that could make room, and
                # its later requests must not overtake this one: refuse it
                r.error = "heap %d full: %d keys held, insert of %d, capacity %d" % (
                    h, self.size[h], r.n, self.capacities[h])
                r.t_done = now
                r.latency = now - r.arrival
                self.stats["refused"] += 1
                continue
            if not fits or not self._admit(h, pend_heaps):
                blocked.add(h)
                keep.append(r)
                continue
            taken.append(r)
            taken_heaps.add(h)
            if r.kind == "ins":
                self.size[h] += r.n
        pending.extend(keep)
        return taken

    def _submit(self, batch, now, inflight):
        if not batch:
            return 0
        heaps = np.array([r.heap for r in batch], dtype=np.uint32)
        kinds = np.array([OP_INS if r.kind == "ins" else OP_DEL for r in batch], dtype=np.uint32)
        sizes = np.array([r.n for r in batch], dtype=np.uint64)
        ins = [np.asarray(r.keys, dtype=self.np_key) for r in batch if r.kind == "ins"]
        keys = np.concatenate(ins) if ins else None
        ids = self.ring.submit(heaps, kinds, sizes, keys)
        busy_before = len(inflight)
        for r, rid in zip(batch[:ids.size], ids):
            inflight[int(rid)] = r
            r.t_submit = now
            self.busy[r.heap] += 1
        if ids.size and busy_before:
            self.stats["submitted_while_busy"] += int(ids.size)
        self.stats["submits"] += 1
        self.stats["max_inflight"] = max(self.stats["max_inflight"], len(inflight))
        return int(ids.size)

    def _collect(self, inflight, t0):
        ids, counts, status = self.ring.poll()
        if ids.size == 0:
            return 0
        now = time.perf_counter() - t0
        # inserts report their size as the count; only deleteMins return keys
        dels = np.array([inflight[i].kind == "del" for i in ids.tolist()], dtype=bool)
        outs = self.ring.take(ids, np.where(dels, counts, 0))
        for rid, st, out in zip(ids.tolist(), status.tolist(), outs):
            r = inflight.pop(rid)
            self.busy[r.heap] -= 1
            if r.kind == "del":
                r.result = out
                self.size[r.heap] -= out.size
            if st != 0:
                r.error = "device error %d on heap %d" % (st, r.heap)
            r.t_done = now
            r.latency = now - r.arrival
        self.stats["requests"] += int(ids.size)
        return int(ids.size)

    def run(self, requests, realtime=True, native=True):
        """Serves `requests` (arrival times in seconds from the start).  With
        realtime=False every request is treated as already arrived.  With
        native=True, and every heap the requests name admitted up front, the
        host loop runs in native code (heapring_serve) under the same rules;
        else in Python (admitting and evicting heaps as requests come)."""
        reqs = sorted(requests, key=lambda r: (r.arrival, r.rid))
        if native and self._admit_all({r.heap for r in reqs if 0 <= r.heap < self.n_heaps}):
            return self._run_native(reqs, realtime)
        return self._run_python(reqs, realtime)

    def _admit_all(self, heaps):
        for h in sorted(heaps):
            if self.heaps[h] is None and not self._admit(h, heaps):
                return False
        return all(self.heaps[h] is not None for h in heaps)

    def _run_native(self, reqs, realtime):
        n = len(reqs)
        arrival = np.array([r.arrival for r in reqs], dtype=np.float64)
        heaps = np.array([r.heap for r in reqs], dtype=np.uint32)
        kinds = np.array([OP_INS if r.kind == "ins" else OP_DEL for r in reqs], dtype=np.uint32)
        sizes = np.array([r.n for r in reqs], dtype=np.uint64)
        ins = [np.asarray(r.keys, dtype=self.np_key) for r in reqs if r.kind == "ins"]
        keys = np.concatenate(ins) if ins else None
        held = np.array(self.size, dtype=np.uint64)
        self.ring.start()
        try:
            out, counts, t_sub, t_done, status = self.ring.serve(
                arrival, heaps, kinds, sizes, keys, self.capacities, held, realtime)
        finally:
            self.ring.stop()
        self.size = [int(x) for x in held]
        dels = kinds == OP_DEL
        off = np.concatenate([[0], np.cumsum(np.where(dels, sizes, 0))[:-1]]).astype(np.int64)
        for i, r in enumerate(reqs):
            st = int(status[i])
            r.t_submit = float(t_sub[i]) if t_sub[i] >= 0 else None
            r.t_done = float(t_done[i])
            r.latency = r.t_done - r.arrival
            if st != 0 and r.t_submit is not None:
                r.error = "device error %d on heap %d" % (st, r.heap)
            elif st != 0:
                r.error = self._refusal(r, st)
            if r.kind == "del" and st == 0:
                r.result = out[off[i]:off[i] + int(counts[i])]
        # requests in flight when each one entered the ring
        sub = np.sort(t_sub[t_sub >= 0])
        done = np.sort(t_done[t_sub >= 0])
        at = np.searchsorted(sub, sub, side="right") - np.searchsorted(done, sub, side="right")
        self.stats["requests"] += n
        self.stats["refused"] += int(np.count_nonzero(t_sub < 0))
        self.stats["max_inflight"] = max(self.stats["max_inflight"], int(at.max()) if at.size else 0)
        self.stats["submitted_while_busy"] += int(np.count_nonzero(at > 1))
        self.stats["submits"] += 1
        return reqs

    def _refusal(self, r, code):
        """Why the native loop refused request r (its status `code`)."""
        why = self._refuse_reason(r)
        if why is not None:
            return why
        if code == -3:
            return "heap %d full: insert of %d keys, capacity %d" % (
                r.heap, r.n, self.capacities[r.heap])
        return "refused (%d)" % code

    def _run_python(self, reqs, realtime):
        pending = collections.deque()
        inflight = {}
        nxt = 0
        self.ring.start()
        t0 = time.perf_counter()
        try:
            while nxt < len(reqs) or pending or inflight:
                now = time.perf_counter() - t0
                while nxt < len(reqs) and (not realtime or reqs[nxt].arrival <= now):
                    pending.append(reqs[nxt])
                    nxt += 1
                progressed = self._collect(inflight, t0)
                if pending:
                    batch = self._select(pending, now)
                    done = self._submit(batch, now, inflight)
                    for r in reversed(batch[done:]):
                        # the ring was full: these wait at the front, in order
                        if r.kind == "ins":
                            self.size[r.heap] -= r.n
                        pending.appendleft(r)
                    progressed += done
                if progressed:
                    continue
                if pending and not inflight:
                    raise RuntimeError("pending requests cannot be admitted within the HBM "
                                       "budget (no heap is empty and idle)")
                if not inflight and nxt < len(reqs):
                    time.sleep(max(0.0, min(reqs[nxt].arrival - now, 1e-3)))
        finally:
            self.ring.stop()
        code = self.set.sync_code()
        if code != 0:
            raise GHeapError(code, "heap set after serving")
        return reqs

    def close(self):
        if self.ring is not None:
            self.ring.close()
            self.ring = None
        for h in range(self.n_heaps):
            if self.heaps[h] is not None:
                self.set.unbind(h, stream=self.stream)
                self.heaps[h].close()
                self.heaps[h] = None
        self.set.close()


def latency_summary(reqs):
    """p50/p99 latency (arrival to completion seen) of the served requests and
    the keys they moved per second of the run."""
    ok = [r for r in reqs if r.latency is not None and r.error is None]
    lat = np.array([r.latency for r in ok])
    keys = sum(r.n if r.kind == "ins" else (0 if r.result is None else r.result.size) for r in ok)
    span = max(r.t_done for r in reqs) - min(r.arrival for r in reqs)
    return {"requests": len(reqs), "p50_ms": float(np.percentile(lat, 50) * 1e3),
            "p99_ms": float(np.percentile(lat, 99) * 1e3), "keys": int(keys),
            "keys_per_s": float(keys / span) if span > 0 else None}


def poisson_requests(seed, n_requests, n_heaps, rate_per_s, max_keys=4096, ins_frac=0.5,
                     key_bytes=4):
    """Request stream of the serving workload: Poisson arrivals, uniform heap,
    uniform sizes in [1, max_keys], a 50/50 insert/deleteMin mix."""
    from . import inputs
    t = inputs.poisson_arrivals(seed, n_requests, rate_per_s)
    x = inputs.splitmix64(seed + 1, 3 * n_requests)
    heap = (x[:n_requests] % np.uint64(n_heaps)).astype(np.int64)
    size = (x[n_requests:2 * n_requests] % np.uint64(max_keys) + np.uint64(1)).astype(np.int64)
    is_ins = ((x[2 * n_requests:] >> np.uint64(11)).astype(np.float64) /
              float(1 << 53)) < ins_frac
    keys_all = inputs.splitmix64(seed + 2, int(size.sum()))
    if key_bytes == 4:
        keys_all = (keys_all & np.uint64(0xFFFFFFFF)).astype(np.uint32)
    out, off = [], 0
    for i in range(n_requests):
        if is_ins[i]:
            out.append(Request(i, t[i], heap[i], "ins", keys=keys_all[off:off + size[i]]))
        else:
            out.append(Request(i, t[i], heap[i], "del", n=size[i]))
        off += size[i]
    return out

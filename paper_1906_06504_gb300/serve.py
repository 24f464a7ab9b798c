"""Continuously batched serving of insert / deleteMin requests over many heaps.

Requests name a heap and carry either keys to insert or a count of smallest
keys to remove.  They arrive over time; the server keeps every heap resident
on the device and, whenever the GPU can take more work, forms a batch of the
requests that have arrived -- at most one per heap, taken in arrival order, so
that each heap sees its requests in FIFO order -- and launches the whole batch
as one heap-set launch (include/gheap.h heapset_ops_req): requests on
different heaps run concurrently on the device, and up to `depth` batches are
queued on the stream while the host forms the next one.  A heap is admitted
(allocated and bound into the set) on its first request when the HBM budget
allows; a heap that is empty and idle is evicted when the budget is needed.

All heap arithmetic runs in the CUDA kernels behind the C ABI; this module
only arranges requests into operation lists, moves keys between pinned host
buffers and the device, and keeps time.
"""
import collections
import time

import numpy as np

from .heap import GHeap, GHeapSet, OP_DEL, OP_INS, SET_CURSOR, SETOP_DTYPE


class Request:
    """One client request.  kind "ins" carries `keys`; kind "del" asks for the
    `n` smallest keys.  After serving: `result` (del: the keys removed,
    ascending), `t_done` (seconds since the run started) and `latency`."""

    __slots__ = ("rid", "arrival", "heap", "kind", "keys", "n", "result", "t_done", "latency")

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


class _Slot:
    """Pinned host and device buffers of one in-flight batch."""

    def __init__(self, torch, max_ops, max_keys, max_reqs, key_dtype):
        pin = dict(pin_memory=True)
        self.h_ops = torch.empty(max_ops * SETOP_DTYPE.itemsize, dtype=torch.uint8, **pin)
        self.h_in = torch.empty(max_keys, dtype=key_dtype, **pin)
        self.h_out = torch.empty(max_keys, dtype=key_dtype, **pin)
        self.h_base = torch.empty(max_reqs, dtype=torch.int64, **pin)
        self.h_cur = torch.empty(max_reqs, dtype=torch.int64, **pin)
        self.d_ops = torch.empty(max_ops * SETOP_DTYPE.itemsize, dtype=torch.uint8, device="cuda")
        self.d_in = torch.empty(max_keys, dtype=key_dtype, device="cuda")
        self.d_out = torch.empty(max_keys, dtype=key_dtype, device="cuda")
        self.d_base = torch.empty(max_reqs, dtype=torch.int64, device="cuda")
        self.d_cur = torch.empty(max_reqs, dtype=torch.int64, device="cuda")
        self.event = torch.cuda.Event()
        self.batch = None


class HeapServer:
    def __init__(self, capacities, k=1024, key_bytes=4, hbm_budget=None, depth=2,
                 max_batch_keys=1 << 22, max_batch_reqs=4096, items_per_thread=None, ctas=0):
        import torch
        self.torch = torch
        self.k = int(k)
        self.key_bytes = int(key_bytes)
        self.capacities = [int(c) for c in capacities]
        self.n_heaps = len(self.capacities)
        self.budget = hbm_budget if hbm_budget is not None else 1 << 62
        self.used = 0
        self.set = GHeapSet([0] * self.n_heaps, k=k, key_bytes=key_bytes)
        if items_per_thread is not None or ctas:
            self.set.set_launch(ctas=ctas, items_per_thread=items_per_thread or 8)
        self.heaps = [None] * self.n_heaps       # owning GHeap per admitted heap
        self.size = [0] * self.n_heaps           # keys held (host view)
        self.busy = [0] * self.n_heaps           # requests in flight
        key_dtype = torch.int32 if key_bytes == 4 else torch.int64
        self.np_key = np.uint32 if key_bytes == 4 else np.uint64
        max_ops = max_batch_reqs + max_batch_keys // k + 1
        self.max_keys = max_batch_keys
        self.max_reqs = max_batch_reqs
        self.slots = [_Slot(torch, max_ops, max_batch_keys, max_batch_reqs, key_dtype)
                      for _ in range(depth)]
        self.stream = torch.cuda.current_stream()
        self.stats = {"batches": 0, "admitted": 0, "evicted": 0, "ops": 0}

    # -- heap admission under the HBM budget
    def _bytes(self, h):
        nodes = self.capacities[h] // self.k + 2
        return nodes * self.k * self.key_bytes + nodes * 4 + self.k * self.key_bytes + 512

    def _admit(self, h, pending_heaps):
        if self.heaps[h] is not None:
            return True
        need = self._bytes(h)
        if self.used + need > self.budget:
            # evict empty, idle heaps that nobody is waiting for
            for g in range(self.n_heaps):
                if self.used + need <= self.budget:
                    break
                if (self.heaps[g] is not None and self.size[g] == 0 and self.busy[g] == 0
                        and g not in pending_heaps):
                    self.set.unbind(g, stream=self.stream)
                    self.heaps[g].close()
                    self.heaps[g] = None
                    self.used -= self._bytes(g)
                    self.stats["evicted"] += 1
            if self.used + need > self.budget:
                return False
        heap = GHeap(self.capacities[h], k=self.k, key_bytes=self.key_bytes)
        self.set.bind(h, heap, stream=self.stream)
        self.heaps[h] = heap
        self.used += need
        self.stats["admitted"] += 1
        return True

    def preadmit(self, heaps):
        """Admits heaps ahead of their first request (allocation is not free)."""
        for h in heaps:
            if not self._admit(int(h), set()):
                raise RuntimeError("heap %d does not fit the HBM budget" % h)
        self.torch.cuda.synchronize()

    # -- one batch
    def _select(self, pending):
        """At most one request per heap, in arrival order; a heap's later
        requests wait behind its earlier ones."""
        taken, blocked, keep = [], set(), collections.deque()
        keys_in = keys_out = 0
        pend_heaps = {r.heap for r in pending}
        while pending:
            r = pending.popleft()
            h = r.heap
            if r.kind == "ins":
                fits = keys_in + r.n <= self.max_keys
            else:
                fits = keys_out + min(r.n, self.size_hint(h)) <= self.max_keys
            if (h in blocked or len(taken) >= self.max_reqs or not fits
                    or not self._admit(h, pend_heaps)):
                blocked.add(h)
                keep.append(r)
                continue
            blocked.add(h)
            taken.append(r)
            if r.kind == "ins":
                keys_in += r.n
            else:
                keys_out += min(r.n, self.size_hint(h))
        pending.extend(keep)
        return taken

    def size_hint(self, h):
        # keys inserted (in flight included) minus keys whose removal has been
        # reported: an upper bound on what a deleteMin can return
        return max(self.size[h], 0)

    def _launch(self, slot, batch):
        torch = self.torch
        k = self.k
        ops = []
        in_parts = []
        in_off = 0
        out_off = 0
        bases = np.zeros(len(batch), dtype=np.int64)
        for ri, r in enumerate(batch):
            if r.kind == "ins":
                n = r.n
                for j in range(0, n, k):
                    ops.append((r.heap, (OP_INS << 24) | min(k, n - j), in_off + j))
                in_parts.append(np.asarray(r.keys, dtype=self.np_key))
                in_off += n
                self.size[r.heap] += n
            else:
                want = min(r.n, self.size_hint(r.heap))
                bases[ri] = out_off
                for j in range(0, want, k):
                    ops.append((r.heap, (OP_DEL << 24) | SET_CURSOR | min(k, want - j), ri))
                out_off += want
            self.busy[r.heap] += 1
        ops = np.array(ops, dtype=SETOP_DTYPE)
        nb = ops.size * SETOP_DTYPE.itemsize
        slot.h_ops[:nb].numpy()[:] = ops.view(np.uint8)
        if in_off:
            slot.h_in[:in_off].numpy()[:] = np.concatenate(in_parts).view(
                np.int32 if self.key_bytes == 4 else np.int64)
        slot.h_base[:len(batch)].numpy()[:] = bases
        s = self.stream
        slot.d_ops[:nb].copy_(slot.h_ops[:nb], non_blocking=True)
        if in_off:
            slot.d_in[:in_off].copy_(slot.h_in[:in_off], non_blocking=True)
        slot.d_base[:len(batch)].copy_(slot.h_base[:len(batch)], non_blocking=True)
        slot.d_cur[:len(batch)].zero_()
        if ops.size:
            self.set.ops_req(slot.d_ops[:nb], slot.d_in if in_off else None, slot.d_out, None,
                             slot.d_base, slot.d_cur, stream=s)
        if out_off:
            slot.h_out[:out_off].copy_(slot.d_out[:out_off], non_blocking=True)
        slot.h_cur[:len(batch)].copy_(slot.d_cur[:len(batch)], non_blocking=True)
        slot.event.record(s)
        slot.batch = (batch, bases)
        self.stats["batches"] += 1
        self.stats["ops"] += int(ops.size)

    def _finish(self, slot, now):
        batch, bases = slot.batch
        got = slot.h_cur[:len(batch)].numpy()
        out = slot.h_out.numpy().view(self.np_key)
        for ri, r in enumerate(batch):
            self.busy[r.heap] -= 1
            if r.kind == "del":
                c = int(got[ri])
                r.result = out[bases[ri]:bases[ri] + c].copy()
                self.size[r.heap] -= c
            r.t_done = now
            r.latency = now - r.arrival
        slot.batch = None

    def run(self, requests, realtime=True):
        """Serves `requests` (arrival times in seconds from the start).  With
        realtime=False every request is treated as already arrived."""
        reqs = sorted(requests, key=lambda r: (r.arrival, r.rid))
        pending = collections.deque()
        nxt = 0
        free = list(self.slots)
        busy = collections.deque()
        t0 = time.perf_counter()
        while nxt < len(reqs) or pending or busy:
            now = time.perf_counter() - t0
            while nxt < len(reqs) and (not realtime or reqs[nxt].arrival <= now):
                pending.append(reqs[nxt])
                nxt += 1
            while busy and busy[0].event.query():
                slot = busy.popleft()
                self._finish(slot, time.perf_counter() - t0)
                free.append(slot)
            if free and pending:
                batch = self._select(pending)
                if batch:
                    slot = free.pop()
                    self._launch(slot, batch)
                    busy.append(slot)
                    continue
            if busy:
                continue      # poll the oldest batch
            if nxt < len(reqs) and not pending:
                time.sleep(max(0.0, min(reqs[nxt].arrival - now, 1e-3)))
            elif pending and not busy:
                raise RuntimeError("pending requests cannot be admitted within the HBM budget")
        self.set.sync()
        return reqs

    def close(self):
        for h in range(self.n_heaps):
            if self.heaps[h] is not None:
                self.set.unbind(h, stream=self.stream)
                self.heaps[h].close()
                self.heaps[h] = None
        self.set.close()


def latency_summary(reqs):
    lat = np.array([r.latency for r in reqs if r.latency is not None])
    keys = sum(r.n if r.kind == "ins" else (0 if r.result is None else r.result.size) for r in reqs)
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

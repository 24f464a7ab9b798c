"""Python binding of the C ABI in include/gheap.h (argument marshalling only).

Every heap operation runs in the CUDA kernels of libgheap.so; this module
converts torch tensors to device pointers and streams, and error codes to
exceptions.  There is no CPU fallback: without the built library or a CUDA
device the calls raise.
"""
import ctypes
import os

import numpy as np

from . import build as _build

OK = 0
ERR_ARG, ERR_OOM, ERR_FULL, ERR_TIMEOUT, ERR_CUDA, ERR_STATE, ERR_TOO_LARGE = (
    -1, -2, -3, -4, -5, -6, -7)
FLAG_STATS = 1
FLAG_BOTTOM_UP = 2
OP_INS, OP_DEL = 1, 2
SET_CURSOR = 1 << 23

# gheap_op, gheapset_op and gheap_log_entry of include/gheap.h
OP_DTYPE = np.dtype([("kind", "<u4"), ("n", "<u4"), ("offset", "<u8")])
SETOP_DTYPE = np.dtype([("heap", "<u4"), ("kind_n", "<u4"), ("offset", "<u8")])
LOG_DTYPE = np.dtype([("call_id", "<u4"), ("kind_n", "<u4"), ("ref", "<u8")])
STAT_NAMES = ("node_loads", "node_stores", "merges", "merges_skipped", "ins_ops",
              "del_ops", "lock_waits", "root_hold_ns",
              "del_acquire_cyc", "del_root_step_cyc", "del_child_wait_cyc",
              "del_child_load_cyc", "del_merge_cyc", "del_store_release_cyc", "del_levels",
              "ins_acquire_cyc", "ins_sort_cyc", "ins_wait_cyc", "ins_step_cyc", "ins_levels",
              "deliveries", "del_yields", "target_children", "intercepts")

_lib = None


class GHeapError(RuntimeError):
    def __init__(self, code, what=""):
        self.code = code
        msg = lib().heap_strerror(code).decode() if _lib is not None else str(code)
        super().__init__("%s: %s (%d)" % (what, msg, code))


def lib():
    """Loads libgheap.so (built in-tree by build.build())."""
    global _lib
    if _lib is None:
        if not os.path.exists(_build.LIB):
            raise RuntimeError("libgheap.so is not built (run paper_1906_06504_gb300.build.build())")
        L = ctypes.CDLL(_build.LIB)
        vp, u64, u32 = ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint32
        u64p = ctypes.POINTER(ctypes.c_uint64)
        u32p = ctypes.POINTER(ctypes.c_uint32)
        sig = {
            "heap_create": (ctypes.c_int, [ctypes.POINTER(vp), u64, u32, u32, u32, u64]),
            "heap_destroy": (ctypes.c_int, [vp]),
            "heap_set_launch": (ctypes.c_int, [vp, u32, u32]),
            "heap_set_timeout": (ctypes.c_int, [vp, u64]),
            "heap_set_yields": (ctypes.c_int, [vp, u32]),
            "heap_set_stats": (ctypes.c_int, [vp, u32]),
            "sssp_heap": (vp, [vp]),
            "knapsack_heap": (vp, [vp]),
            "heap_insert": (ctypes.c_int, [vp, vp, u64, vp]),
            "heap_delete_min": (ctypes.c_int, [vp, vp, u64, vp, vp]),
            "heap_ops": (ctypes.c_int, [vp, vp, u64, vp, vp, vp, u64, vp]),
            "heap_sync": (ctypes.c_int, [vp]),
            "heap_size": (ctypes.c_int, [vp, u64p]),
            "heap_reset": (ctypes.c_int, [vp, vp]),
            "heap_get_log": (ctypes.c_int, [vp, vp, u64, u64p, u64p]),
            "heap_snapshot": (ctypes.c_int, [vp, vp, u32p, vp, u64p]),
            "heap_geometry": (ctypes.c_int, [vp, u64p, u32p, u32p]),
            "heap_slot_to_node": (u64, [u64]),
            "heap_get_stats": (ctypes.c_int, [vp, u64p, u32]),
            "heap_debug_hold_root": (ctypes.c_int, [vp, vp]),
            "heap_sort_noalloc": (ctypes.c_int, [vp, vp, u64, vp]),
            "heapset_create": (ctypes.c_int, [ctypes.POINTER(vp), u32, u64p, u32, u32, u32, u64]),
            "heapset_destroy": (ctypes.c_int, [vp]),
            "heapset_heap": (vp, [vp, u32]),
            "heapset_set_launch": (ctypes.c_int, [vp, u32, u32]),
            "heapset_set_timeout": (ctypes.c_int, [vp, u64]),
            "heapset_ops": (ctypes.c_int, [vp, vp, u64, vp, vp, vp, vp]),
            "heapset_sync": (ctypes.c_int, [vp]),
            "heapset_get_stats": (ctypes.c_int, [vp, u64p, u32]),
            "heapset_reset": (ctypes.c_int, [vp, vp]),
            "heapset_bind": (ctypes.c_int, [vp, u32, vp, vp]),
            "heapset_unbind": (ctypes.c_int, [vp, u32, vp]),
            "heapset_ops_req": (ctypes.c_int, [vp, vp, u64, vp, vp, vp, vp, vp, vp]),
            "heapset_graph_create": (ctypes.c_int, [vp, vp, u64, vp, vp, vp, ctypes.POINTER(vp)]),
            "heapset_graph_launch": (ctypes.c_int, [vp, vp]),
            "heapset_graph_destroy": (ctypes.c_int, [vp]),
            "heap_insert_dev": (ctypes.c_int, [vp, vp, vp, u64, vp]),
            "heapring_create": (ctypes.c_int, [ctypes.POINTER(vp), vp, u32, u64, u64, u64]),
            "heapring_destroy": (ctypes.c_int, [vp]),
            "heapring_attach": (ctypes.c_int, [vp, u32]),
            "heapring_start": (ctypes.c_int, [vp]),
            "heapring_stop": (ctypes.c_int, [vp]),
            "heapring_submit": (ctypes.c_int, [vp, u32, vp, vp, vp, vp, vp]),
            "heapring_poll": (ctypes.c_int, [vp, vp, vp, vp, u32, u32p]),
            "heapring_take": (ctypes.c_int, [vp, u32, vp, vp, u64, vp]),
            "heapring_pending": (ctypes.c_int, [vp, u64p]),
            "heapring_serve": (ctypes.c_int, [vp, u64, vp, vp, vp, vp, vp, vp, vp, ctypes.c_int,
                                              vp, vp, vp, vp, vp]),
            "heap_strerror": (ctypes.c_char_p, [ctypes.c_int]),
            # gheap_apps.h
            "sssp_create": (ctypes.c_int, [ctypes.POINTER(vp), u32, u64, u32, u32, u64]),
            "sssp_destroy": (ctypes.c_int, [vp]),
            "sssp_set_launch": (ctypes.c_int, [vp, u32, u32]),
            "sssp_run": (ctypes.c_int, [vp, vp, vp, vp, u32, u64, u32, vp, vp, vp]),
            "knapsack_create": (ctypes.c_int, [ctypes.POINTER(vp), u32, u64, u32, u32, u64]),
            "knapsack_destroy": (ctypes.c_int, [vp]),
            "knapsack_set_launch": (ctypes.c_int, [vp, u32, u32]),
            "knapsack_run": (ctypes.c_int, [vp, vp, vp, u32, u32, vp, vp]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _check(rc, what):
    if rc != OK:
        raise GHeapError(rc, what)


def _stream_ptr(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def slot_to_node(j):
    return int(lib().heap_slot_to_node(int(j)))


class GHeap:
    """A generalized concurrent heap in device memory (include/gheap.h)."""

    def __init__(self, capacity, k=1024, key_bytes=4, log_capacity=0, stats=False,
                 bottom_up=False, _handle=None):
        L = lib()
        self._owned = _handle is None
        if _handle is None:
            h = ctypes.c_void_p()
            flags = (FLAG_STATS if stats else 0) | (FLAG_BOTTOM_UP if bottom_up else 0)
            _check(L.heap_create(ctypes.byref(h), int(capacity), int(k), int(key_bytes),
                                 flags, int(log_capacity)), "heap_create")
        else:
            h = ctypes.c_void_p(_handle)
        self._h = h
        mn = ctypes.c_uint64()
        kk = ctypes.c_uint32()
        kb = ctypes.c_uint32()
        _check(L.heap_geometry(h, ctypes.byref(mn), ctypes.byref(kk), ctypes.byref(kb)),
               "heap_geometry")
        self.k = int(kk.value)
        self.key_bytes = int(kb.value)
        self.capacity = int(capacity)
        self.max_nodes = int(mn.value)

    # -- configuration
    def set_launch(self, ctas=0, items_per_thread=4):
        _check(lib().heap_set_launch(self._h, int(ctas), int(items_per_thread)), "heap_set_launch")

    def set_timeout(self, ns):
        _check(lib().heap_set_timeout(self._h, int(ns)), "heap_set_timeout")

    def set_stats(self, on):
        """Device counters on or off for later launches (stats())."""
        _check(lib().heap_set_stats(self._h, 1 if on else 0), "heap_set_stats")

    def set_yields(self, n):
        """Root hand-backs before a DEL marks an in-flight INS target (0 = the
        paper's mark-and-wait protocol)."""
        _check(lib().heap_set_yields(self._h, int(n)), "heap_set_yields")

    def _key_tensor(self, t, what):
        if not t.is_cuda:
            raise ValueError("%s must be a CUDA tensor" % what)
        if t.element_size() != self.key_bytes:
            raise ValueError("%s has %d-byte elements, heap keys are %d bytes"
                             % (what, t.element_size(), self.key_bytes))
        if not t.is_contiguous():
            raise ValueError("%s must be contiguous" % what)

    # -- operations
    def insert(self, keys, stream=None):
        self._key_tensor(keys, "keys")
        _check(lib().heap_insert(self._h, ctypes.c_void_p(keys.data_ptr()), keys.numel(),
                                 _stream_ptr(stream)), "heap_insert")

    def insert_dev(self, keys, count, stream=None):
        """Inserts the first min(count[0], keys.numel()) keys; `count` is a
        1-element int64 CUDA tensor read when the work runs."""
        self._key_tensor(keys, "keys")
        if not count.is_cuda or count.element_size() != 8:
            raise ValueError("count must be a 1-element int64 CUDA tensor")
        _check(lib().heap_insert_dev(self._h, ctypes.c_void_p(keys.data_ptr()),
                                     ctypes.c_void_p(count.data_ptr()), keys.numel(),
                                     _stream_ptr(stream)), "heap_insert_dev")

    def delete_min(self, n, out=None, count=None, stream=None):
        """Deletes up to n smallest keys into `out` (allocated if None).

        Returns (out, count) with count a 1-element int64 CUDA tensor.
        """
        import torch
        if out is None:
            dt = torch.int32 if self.key_bytes == 4 else torch.int64
            out = torch.empty(int(n), dtype=dt, device="cuda")
        self._key_tensor(out, "out")
        if out.numel() < n:
            raise ValueError("out holds %d keys < n=%d" % (out.numel(), n))
        if count is None:
            count = torch.empty(1, dtype=torch.int64, device="cuda")
        _check(lib().heap_delete_min(self._h, ctypes.c_void_p(out.data_ptr()), int(n),
                                     ctypes.c_void_p(count.data_ptr()), _stream_ptr(stream)),
               "heap_delete_min")
        return out, count

    def ops(self, ops_dev, in_keys, out_keys, counts=None, max_insert_keys=None, stream=None):
        """Runs a device array of gheap_op (viewed as a uint8/int64 tensor)."""
        n_ops = ops_dev.numel() * ops_dev.element_size() // OP_DTYPE.itemsize
        if in_keys is not None:
            self._key_tensor(in_keys, "in_keys")
        if out_keys is not None:
            self._key_tensor(out_keys, "out_keys")
        if max_insert_keys is None:
            max_insert_keys = in_keys.numel() if in_keys is not None else 0
        _check(lib().heap_ops(self._h, ctypes.c_void_p(ops_dev.data_ptr()), n_ops,
                              ctypes.c_void_p(in_keys.data_ptr() if in_keys is not None else 0),
                              ctypes.c_void_p(out_keys.data_ptr() if out_keys is not None else 0),
                              ctypes.c_void_p(counts.data_ptr() if counts is not None else 0),
                              int(max_insert_keys), _stream_ptr(stream)), "heap_ops")

    def sync(self):
        _check(lib().heap_sync(self._h), "heap_sync")

    def sync_code(self):
        return int(lib().heap_sync(self._h))

    def size(self):
        v = ctypes.c_uint64()
        _check(lib().heap_size(self._h, ctypes.byref(v)), "heap_size")
        return int(v.value)

    def reset(self, stream=None):
        _check(lib().heap_reset(self._h, _stream_ptr(stream)), "heap_reset")

    def log(self):
        """The linearization record as a numpy structured array (LOG_DTYPE)."""
        L = lib()
        total = ctypes.c_uint64()
        got = ctypes.c_uint64()
        _check(L.heap_get_log(self._h, None, 0, ctypes.byref(got), ctypes.byref(total)),
               "heap_get_log")
        buf = np.zeros(int(total.value), dtype=LOG_DTYPE)
        if total.value:
            _check(L.heap_get_log(self._h, ctypes.c_void_p(buf.ctypes.data), buf.size,
                                  ctypes.byref(got), ctypes.byref(total)), "heap_get_log")
        return buf[:int(got.value)], int(total.value)

    def snapshot(self):
        """(keys[slots, k], state[slots], buffer[k], (m, s, seq))."""
        dt = np.uint32 if self.key_bytes == 4 else np.uint64
        slots = self.max_nodes + 1
        keys = np.zeros((slots, self.k), dtype=dt)
        st = np.zeros(slots, dtype=np.uint32)
        buf = np.zeros(self.k, dtype=dt)
        hdr = (ctypes.c_uint64 * 3)()
        _check(lib().heap_snapshot(self._h, ctypes.c_void_p(keys.ctypes.data),
                                   st.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32)),
                                   ctypes.c_void_p(buf.ctypes.data), hdr), "heap_snapshot")
        return keys, st, buf, (int(hdr[0]), int(hdr[1]), int(hdr[2]))

    def stats(self):
        out = (ctypes.c_uint64 * len(STAT_NAMES))()
        _check(lib().heap_get_stats(self._h, out, len(STAT_NAMES)), "heap_get_stats")
        return dict(zip(STAT_NAMES, [int(x) for x in out]))

    def debug_hold_root(self, stream=None):
        _check(lib().heap_debug_hold_root(self._h, _stream_ptr(stream)), "heap_debug_hold_root")

    def close(self):
        if getattr(self, "_h", None):
            if self._owned:
                lib().heap_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


class GHeapSet:
    """Many independent heaps driven by one persistent launch (include/gheap.h
    heap sets).  `heaps[i]` is a non-owning GHeap view of heap i."""

    def __init__(self, capacities, k=1024, key_bytes=4, log_capacity=0, stats=False,
                 bottom_up=False):
        L = lib()
        caps = (ctypes.c_uint64 * len(capacities))(*[int(c) for c in capacities])
        h = ctypes.c_void_p()
        _check(L.heapset_create(ctypes.byref(h), len(capacities), caps, int(k), int(key_bytes),
                                (FLAG_STATS if stats else 0) | (FLAG_BOTTOM_UP if bottom_up else 0),
                                int(log_capacity)), "heapset_create")
        self._s = h
        self.k = int(k)
        self.key_bytes = int(key_bytes)
        self.heaps = [GHeap(c, _handle=L.heapset_heap(h, i)) if c else None
                      for i, c in enumerate(capacities)]

    def bind(self, i, heap, stream=None):
        """Put a GHeap (same k and key width, kept by the caller) in empty slot i."""
        _check(lib().heapset_bind(self._s, int(i), heap._h, _stream_ptr(stream)), "heapset_bind")
        self.heaps[i] = GHeap(heap.capacity, _handle=heap._h.value)

    def unbind(self, i, stream=None):
        _check(lib().heapset_unbind(self._s, int(i), _stream_ptr(stream)), "heapset_unbind")
        if self.heaps[i] is not None:
            self.heaps[i]._h = None
        self.heaps[i] = None

    def set_launch(self, ctas=0, items_per_thread=8):
        _check(lib().heapset_set_launch(self._s, int(ctas), int(items_per_thread)),
               "heapset_set_launch")

    def stats(self):
        """The set's counters (needs stats=True), as GHeap.stats."""
        out = (ctypes.c_uint64 * len(STAT_NAMES))()
        _check(lib().heapset_get_stats(self._s, out, len(STAT_NAMES)), "heapset_get_stats")
        return dict(zip(STAT_NAMES, [int(x) for x in out]))

    def set_timeout(self, ns):
        _check(lib().heapset_set_timeout(self._s, int(ns)), "heapset_set_timeout")

    def _ptrs(self, ops_dev, in_keys, out_keys, counts):
        n_ops = ops_dev.numel() * ops_dev.element_size() // SETOP_DTYPE.itemsize
        return (n_ops, ctypes.c_void_p(ops_dev.data_ptr()),
                ctypes.c_void_p(in_keys.data_ptr() if in_keys is not None else 0),
                ctypes.c_void_p(out_keys.data_ptr() if out_keys is not None else 0),
                ctypes.c_void_p(counts.data_ptr() if counts is not None else 0))

    def ops(self, ops_dev, in_keys, out_keys, counts=None, stream=None):
        n_ops, o, i, ou, c = self._ptrs(ops_dev, in_keys, out_keys, counts)
        _check(lib().heapset_ops(self._s, o, n_ops, i, ou, c, _stream_ptr(stream)), "heapset_ops")

    def ops_req(self, ops_dev, in_keys, out_keys, counts, req_base, req_cursor, stream=None):
        """ops() with per-request cursors for SET_CURSOR DELs (uint64 tensors)."""
        n_ops, o, i, ou, c = self._ptrs(ops_dev, in_keys, out_keys, counts)
        _check(lib().heapset_ops_req(self._s, o, n_ops, i, ou, c,
                                     ctypes.c_void_p(req_base.data_ptr()),
                                     ctypes.c_void_p(req_cursor.data_ptr()),
                                     _stream_ptr(stream)), "heapset_ops_req")

    def graph(self, ops_dev, in_keys, out_keys, counts=None):
        """A captured CUDA graph of ops(); launch() replays it."""
        n_ops, o, i, ou, c = self._ptrs(ops_dev, in_keys, out_keys, counts)
        g = ctypes.c_void_p()
        _check(lib().heapset_graph_create(self._s, o, n_ops, i, ou, c, ctypes.byref(g)),
               "heapset_graph_create")
        return SetGraph(g, (ops_dev, in_keys, out_keys, counts))

    def sync(self):
        _check(lib().heapset_sync(self._s), "heapset_sync")

    def sync_code(self):
        return int(lib().heapset_sync(self._s))

    def reset(self, stream=None):
        _check(lib().heapset_reset(self._s, _stream_ptr(stream)), "heapset_reset")

    def close(self):
        if getattr(self, "_s", None):
            for h in self.heaps:
                if h is not None:
                    h._h = None
            lib().heapset_destroy(self._s)
            self._s = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


class SetGraph:
    def __init__(self, g, keep):
        self._g = g
        self._keep = keep   # the captured arrays must outlive the graph

    def launch(self, stream=None):
        _check(lib().heapset_graph_launch(self._g, _stream_ptr(stream)), "heapset_graph_launch")

    def close(self):
        if getattr(self, "_g", None):
            lib().heapset_graph_destroy(self._g)
            self._g = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class GHeapRing:
    """The serving ring of include/gheap.h over a GHeapSet: one persistent
    launch takes insert/deleteMin requests from pinned host memory while the
    host keeps submitting them (argument marshalling only)."""

    def __init__(self, hset, max_requests=4096, max_ops=1 << 15, in_keys=1 << 24,
                 out_keys=1 << 24):
        r = ctypes.c_void_p()
        _check(lib().heapring_create(ctypes.byref(r), hset._s, int(max_requests), int(max_ops),
                                     int(in_keys), int(out_keys)), "heapring_create")
        self._r = r
        self.set = hset
        self.key_dtype = np.uint32 if hset.key_bytes == 4 else np.uint64
        self.max_requests = int(max_requests)
        self.in_keys = int(in_keys)
        self.out_keys = int(out_keys)
        self._ids = np.zeros(self.max_requests, dtype=np.uint64)
        self._cnt = np.zeros(self.max_requests, dtype=np.uint64)
        self._st = np.zeros(self.max_requests, dtype=np.int32)
        self.running = False

    def start(self):
        _check(lib().heapring_start(self._r), "heapring_start")
        self.running = True

    def stop(self):
        self.running = False
        _check(lib().heapring_stop(self._r), "heapring_stop")

    def attach(self, i):
        _check(lib().heapring_attach(self._r, int(i)), "heapring_attach")

    def submit(self, heaps, kinds, sizes, keys=None):
        """Appends requests (uint32 heaps, uint32 kinds OP_INS/OP_DEL, uint64
        sizes; keys: the inserts' keys back to back).  Returns the ids of the
        requests accepted, a prefix of the ones given."""
        heaps = np.ascontiguousarray(heaps, dtype=np.uint32)
        kinds = np.ascontiguousarray(kinds, dtype=np.uint32)
        sizes = np.ascontiguousarray(sizes, dtype=np.uint64)
        ids = np.zeros(heaps.size, dtype=np.uint64)
        kp = None
        if keys is not None and len(keys):
            keys = np.ascontiguousarray(keys, dtype=self.key_dtype)
            kp = ctypes.c_void_p(keys.ctypes.data)
        rc = lib().heapring_submit(self._r, heaps.size, ctypes.c_void_p(heaps.ctypes.data),
                                   ctypes.c_void_p(kinds.ctypes.data),
                                   ctypes.c_void_p(sizes.ctypes.data), kp,
                                   ctypes.c_void_p(ids.ctypes.data))
        if rc < 0:
            raise GHeapError(rc, "heapring_submit")
        return ids[:rc]

    def poll(self):
        """(ids, counts, status) of the requests completed since the last poll."""
        n = ctypes.c_uint32()
        _check(lib().heapring_poll(self._r, ctypes.c_void_p(self._ids.ctypes.data),
                                   ctypes.c_void_p(self._cnt.ctypes.data),
                                   ctypes.c_void_p(self._st.ctypes.data), self.max_requests,
                                   ctypes.byref(n)), "heapring_poll")
        c = int(n.value)
        return self._ids[:c].copy(), self._cnt[:c].copy(), self._st[:c].copy()

    def take(self, ids, counts):
        """Takes completed requests `ids` (with the counts poll reported):
        returns one array per request (its deleteMin keys; empty for an
        insert), views into one buffer, and frees the requests."""
        ids = np.ascontiguousarray(ids, dtype=np.uint64)
        counts = np.asarray(counts, dtype=np.uint64)
        total = int(counts.sum())
        out = np.empty(total, dtype=self.key_dtype)
        got = np.zeros(ids.size, dtype=np.uint64)
        _check(lib().heapring_take(self._r, ids.size, ctypes.c_void_p(ids.ctypes.data),
                                   ctypes.c_void_p(out.ctypes.data), total,
                                   ctypes.c_void_p(got.ctypes.data)), "heapring_take")
        return np.split(out, np.cumsum(got)[:-1].astype(np.int64))

    def pending(self):
        v = ctypes.c_uint64()
        _check(lib().heapring_pending(self._r, ctypes.byref(v)), "heapring_pending")
        return int(v.value)

    def serve(self, arrival, heaps, kinds, sizes, keys, capacities, held, realtime=True):
        """A whole session in the native host loop (heapring_serve).  Returns
        (out keys back to back, out_counts, t_submit, t_done, status); `held`
        (uint64 per heap) is updated in place."""
        n = len(sizes)
        arrival = np.ascontiguousarray(arrival, dtype=np.float64)
        heaps = np.ascontiguousarray(heaps, dtype=np.uint32)
        kinds = np.ascontiguousarray(kinds, dtype=np.uint32)
        sizes = np.ascontiguousarray(sizes, dtype=np.uint64)
        keys = np.ascontiguousarray(keys if keys is not None else np.zeros(1, self.key_dtype),
                                    dtype=self.key_dtype)
        capacities = np.ascontiguousarray(capacities, dtype=np.uint64)
        assert held.dtype == np.uint64 and held.flags["C_CONTIGUOUS"]
        out = np.empty(max(1, int(sizes[kinds == 2].sum())), dtype=self.key_dtype)
        counts = np.zeros(n, dtype=np.uint64)
        t_sub = np.zeros(n, dtype=np.float64)
        t_done = np.zeros(n, dtype=np.float64)
        status = np.zeros(n, dtype=np.int32)
        ptr = lambda a: ctypes.c_void_p(a.ctypes.data)
        _check(lib().heapring_serve(self._r, n, ptr(arrival), ptr(heaps), ptr(kinds), ptr(sizes),
                                    ptr(keys), ptr(capacities), ptr(held), 1 if realtime else 0,
                                    ptr(out), ptr(counts), ptr(t_sub), ptr(t_done), ptr(status)),
               "heapring_serve")
        return out, counts, t_sub, t_done, status

    def close(self):
        if getattr(self, "_r", None):
            lib().heapring_destroy(self._r)
            self._r = None
            self.running = False

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

"""Python binding of include/gheap_apps.h: applications of the heap
(Section 5.7), argument marshalling only.  The work runs in libgheap.so."""
import ctypes

import numpy as np

from .heap import GHeap, _check, _stream_ptr, lib

SSSP_STATS_DTYPE = np.dtype([("iterations", "<u8"), ("keys_deleted", "<u8"), ("visited", "<u8"),
                             ("edges", "<u8"), ("keys_inserted", "<u8")])
KNAPSACK_STATS_DTYPE = np.dtype([(name, "<u8") for name in (
    "best", "iterations", "keys_deleted", "explored", "pruned", "keys_inserted", "nodes",
    "gc_runs", "gc_dropped")])


class SSSP:
    """Single-source shortest paths with the heap as the priority queue of
    active vertices (Section 5.7.1); keys are (distance << 32 | vertex)."""

    def __init__(self, n_vertices, n_edges, k=1024, batch=16384, heap_capacity=0):
        h = ctypes.c_void_p()
        _check(lib().sssp_create(ctypes.byref(h), int(n_vertices), int(n_edges), int(k),
                                 int(batch), int(heap_capacity)), "sssp_create")
        self._h = h
        self.n_vertices = int(n_vertices)
        self.n_edges = int(n_edges)
        self.k = int(k)
        self.batch = int(batch)

    def set_launch(self, ctas=0, items_per_thread=8):
        _check(lib().sssp_set_launch(self._h, int(ctas), int(items_per_thread)), "sssp_set_launch")

    def heap(self):
        """The context's heap, not owned (for its counters)."""
        return GHeap(0, _handle=lib().sssp_heap(self._h))

    def run(self, rowptr, col, w, source=0, dist=None, stream=None):
        """Distances from `source` over the CSR graph (CUDA tensors: rowptr
        int64[n+1], col and w int32[E]).  Returns (dist int32[n] CUDA
        tensor, stats dict); UINT32_MAX (-1 as int32) marks unreachable."""
        import torch
        n = rowptr.numel() - 1
        e = col.numel()
        for t, name, size in ((rowptr, "rowptr", 8), (col, "col", 4), (w, "w", 4)):
            if not t.is_cuda or not t.is_contiguous() or t.element_size() != size:
                raise ValueError("%s must be a contiguous CUDA tensor of %d-byte elements" % (name, size))
        if w.numel() != e:
            raise ValueError("col and w differ in length")
        if dist is None:
            dist = torch.empty(n, dtype=torch.int32, device=rowptr.device)
        st = np.zeros(1, dtype=SSSP_STATS_DTYPE)
        _check(lib().sssp_run(self._h, ctypes.c_void_p(rowptr.data_ptr()),
                              ctypes.c_void_p(col.data_ptr() if e else 0),
                              ctypes.c_void_p(w.data_ptr() if e else 0), n, e, int(source),
                              ctypes.c_void_p(dist.data_ptr()),
                              ctypes.c_void_p(st.ctypes.data), _stream_ptr(stream)), "sssp_run")
        return dist, {name: int(st[name][0]) for name in SSSP_STATS_DTYPE.names}

    def close(self):
        if self._h is not None:
            lib().sssp_destroy(self._h)
            self._h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Knapsack:
    """0/1 knapsack by best-first branch and bound with the heap as the queue
    of open nodes (Section 5.7.2)."""

    def __init__(self, max_items, max_nodes=0, k=1024, batch=16384, gc_threshold=0):
        h = ctypes.c_void_p()
        _check(lib().knapsack_create(ctypes.byref(h), int(max_items), int(max_nodes), int(k),
                                     int(batch), int(gc_threshold)), "knapsack_create")
        self._h = h
        self.max_items = int(max_items)

    def set_launch(self, ctas=0, items_per_thread=8):
        _check(lib().knapsack_set_launch(self._h, int(ctas), int(items_per_thread)),
               "knapsack_set_launch")

    def heap(self):
        """The context's heap, not owned (for its counters)."""
        return GHeap(0, _handle=lib().knapsack_heap(self._h))

    def run(self, w, v, capacity, stream=None):
        """w, v: int32 CUDA tensors (uint32 bit patterns) of the items.
        Returns the stats dict; stats["best"] is the optimum value."""
        for t, name in ((w, "w"), (v, "v")):
            if not t.is_cuda or not t.is_contiguous() or t.element_size() != 4:
                raise ValueError("%s must be a contiguous CUDA tensor of 4-byte elements" % name)
        if w.numel() != v.numel():
            raise ValueError("w and v differ in length")
        st = np.zeros(1, dtype=KNAPSACK_STATS_DTYPE)
        _check(lib().knapsack_run(self._h, ctypes.c_void_p(w.data_ptr()), ctypes.c_void_p(v.data_ptr()),
                                  w.numel(), int(capacity), ctypes.c_void_p(st.ctypes.data),
                                  _stream_ptr(stream)), "knapsack_run")
        return {name: int(st[name][0]) for name in KNAPSACK_STATS_DTYPE.names}

    def close(self):
        if self._h is not None:
            lib().knapsack_destroy(self._h)
            self._h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

"""CPU oracle for the generalized concurrent heap (arXiv 1906.06504).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package; the product path in
``paper_1906_06504_gb300`` never does, and this package never imports it.

Contents
--------
* ``BinaryHeapPQ`` -- the textbook array binary heap of Section 2.1 (in
  ``heap_oracle.c``).  By linearizability (Section 3.3.3, Theorem 1) every DEL
  of the concurrent heap returns the k smallest keys present at its root hold,
  so replaying the recorded root-hold order through this queue fixes every DEL
  output exactly (``replay``).
* ``merge_and_sort`` -- MergeAndSort by its definition (Section 3.2.1).
* ``check_properties`` -- Properties 1-3 of Section 3.1 on a heap snapshot.
* ``dijkstra`` / ``knapsack_dp`` -- textbook solvers for the Section 5.7
  applications.
* ``stl_insert_delete`` -- the paper's sequential CPU baseline (Table 1):
  the C++ standard library's ``std::priority_queue`` (``stl_pq.cpp``), timed
  beside the GPU heap; not part of the oracle's checks.
* ``genheap.GeneralizedHeapModel`` -- a slow sequential model of the
  generalized heap's INS/DEL steps (Sections 3.1-3.3.2, 4.3), for node-level
  parity of a single-CTA GPU run.

The C and C++ parts are built with gcc/g++ -O3 on first use (or by
``build()``).
"""
import ctypes
import os
import subprocess
import threading

import numpy as np

_DIR = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_DIR, "heap_oracle.c")
_SO = os.path.join(_DIR, "liboracle.so")
_STL_SRC = os.path.join(_DIR, "stl_pq.cpp")
_STL_SO = os.path.join(_DIR, "libstlpq.so")
_lock = threading.Lock()
_lib = None
_stl = None


def _compile(cmd, src, so, force):
    if (not force and os.path.exists(so)
            and os.path.getmtime(so) >= os.path.getmtime(src)):
        return so
    tmp = so + ".%d.tmp" % os.getpid()
    subprocess.check_call(cmd + ["-shared", "-fPIC", "-o", tmp, src])
    os.replace(tmp, so)
    return so


def build(force=False):
    """Compile heap_oracle.c into liboracle.so (gcc -O3) and the standard
    library priority-queue baseline stl_pq.cpp into libstlpq.so (g++ -O3),
    next to them."""
    _compile(["g++", "-O3", "-std=c++17"], _STL_SRC, _STL_SO, force)
    return _compile(["gcc", "-O3", "-std=c11"], _SRC, _SO, force)


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_SO)
            u64p = ctypes.POINTER(ctypes.c_uint64)
            u32p = ctypes.POINTER(ctypes.c_uint32)
            L.orc_pq_new.restype = ctypes.c_void_p
            L.orc_pq_new.argtypes = [ctypes.c_size_t]
            L.orc_pq_free.argtypes = [ctypes.c_void_p]
            L.orc_pq_size.restype = ctypes.c_size_t
            L.orc_pq_size.argtypes = [ctypes.c_void_p]
            L.orc_pq_push.restype = ctypes.c_int
            L.orc_pq_push.argtypes = [ctypes.c_void_p, u64p, ctypes.c_size_t]
            L.orc_pq_pop.restype = ctypes.c_size_t
            L.orc_pq_pop.argtypes = [ctypes.c_void_p, u64p, ctypes.c_size_t]
            L.orc_pq_push_u32.restype = ctypes.c_int
            L.orc_pq_push_u32.argtypes = [ctypes.c_void_p, u32p, ctypes.c_size_t]
            L.orc_pq_pop_u32.restype = ctypes.c_size_t
            L.orc_pq_pop_u32.argtypes = [ctypes.c_void_p, u32p, ctypes.c_size_t]
            L.orc_merge_and_sort.restype = ctypes.c_int
            L.orc_merge_and_sort.argtypes = [u64p, ctypes.c_size_t, u64p,
                                             ctypes.c_size_t, ctypes.c_size_t,
                                             u64p, u64p]
            L.orc_check_properties.restype = ctypes.c_int
            L.orc_check_properties.argtypes = [
                u64p, ctypes.POINTER(ctypes.c_uint8), ctypes.c_size_t,
                ctypes.c_size_t, u64p, ctypes.c_size_t,
                ctypes.POINTER(ctypes.c_size_t)]
            L.orc_dijkstra.restype = ctypes.c_int
            L.orc_dijkstra.argtypes = [ctypes.c_uint32, u64p, u32p, u32p,
                                       ctypes.c_uint32, u32p]
            L.orc_knapsack_dp.restype = ctypes.c_uint64
            L.orc_knapsack_dp.argtypes = [ctypes.c_uint32, u32p, u32p,
                                          ctypes.c_uint64]
            _lib = L
    return _lib


def stl_insert_delete(keys):
    """The paper's sequential CPU baseline (Table 1, std::priority_queue):
    pushes every uint32 key, then pops them all.  Returns (sorted output,
    seconds spent in the pushes and pops)."""
    global _stl
    with _lock:
        if _stl is None:
            build()
            L = ctypes.CDLL(_STL_SO)
            L.stl_insert_delete_u32.restype = ctypes.c_double
            L.stl_insert_delete_u32.argtypes = [ctypes.POINTER(ctypes.c_uint32), ctypes.c_size_t,
                                                ctypes.POINTER(ctypes.c_uint32)]
            _stl = L
    keys = np.ascontiguousarray(keys, dtype=np.uint32)
    out = np.empty_like(keys)
    dt = _stl.stl_insert_delete_u32(_p(keys, ctypes.c_uint32), keys.size,
                                    _p(out, ctypes.c_uint32))
    if dt < 0:
        raise MemoryError("std::priority_queue storage allocation failed")
    return out, float(dt)


def _p(arr, ctype):
    return arr.ctypes.data_as(ctypes.POINTER(ctype))


class BinaryHeapPQ:
    """Sequential min-priority queue: the textbook binary heap (Section 2.1)."""

    def __init__(self, cap_hint=1024):
        self._L = lib()
        self._q = self._L.orc_pq_new(int(cap_hint))
        if not self._q:
            raise MemoryError("oracle queue allocation failed")

    def push(self, keys):
        keys = np.ascontiguousarray(keys)
        if keys.dtype == np.uint32:
            rc = self._L.orc_pq_push_u32(self._q, _p(keys, ctypes.c_uint32),
                                         keys.size)
        else:
            keys = np.ascontiguousarray(keys, dtype=np.uint64)
            rc = self._L.orc_pq_push(self._q, _p(keys, ctypes.c_uint64),
                                     keys.size)
        if rc != 0:
            raise MemoryError("oracle queue growth failed")

    def pop(self, n, dtype=np.uint64):
        """Pops min(n, size) keys, ascending."""
        out = np.empty(int(n), dtype=dtype)
        if dtype == np.uint32:
            c = self._L.orc_pq_pop_u32(self._q, _p(out, ctypes.c_uint32), int(n))
        else:
            c = self._L.orc_pq_pop(self._q, _p(out, ctypes.c_uint64), int(n))
        return out[:c]

    def __len__(self):
        return int(self._L.orc_pq_size(self._q))

    def close(self):
        if self._q:
            self._L.orc_pq_free(self._q)
            self._q = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def merge_and_sort(a, b, k_small=None):
    """MergeAndSort (Section 3.2.1) by definition: returns (small, large)."""
    a = np.ascontiguousarray(a, dtype=np.uint64)
    b = np.ascontiguousarray(b, dtype=np.uint64)
    if k_small is None:
        k_small = a.size
    small = np.empty(k_small, dtype=np.uint64)
    large = np.empty(a.size + b.size - k_small, dtype=np.uint64)
    rc = lib().orc_merge_and_sort(_p(a, ctypes.c_uint64), a.size,
                                  _p(b, ctypes.c_uint64), b.size, k_small,
                                  _p(small, ctypes.c_uint64),
                                  _p(large, ctypes.c_uint64))
    if rc != 0:
        raise ValueError("merge_and_sort: bad sizes")
    return small, large


PROPERTY_NAMES = {0: "ok", 1: "Property 1", 2: "Property 2", 3: "Property 3",
                  4: "structure"}


def check_properties(nodes, present, k, buf):
    """Properties 1-3 (Section 3.1) on a snapshot.

    nodes: array of shape (n_slots, k) (row i = node i; row 0 unused);
    present: bool array of n_slots; buf: the partial buffer's keys.
    Returns (code, node) with code 0 when all hold (see heap_oracle.c).
    """
    nodes = np.ascontiguousarray(nodes, dtype=np.uint64).reshape(-1)
    pres = np.ascontiguousarray(present, dtype=np.uint8)
    buf = np.ascontiguousarray(buf, dtype=np.uint64)
    if buf.size == 0:
        buf = np.zeros(1, dtype=np.uint64)
        s = 0
    else:
        s = buf.size
    where = ctypes.c_size_t(0)
    code = lib().orc_check_properties(_p(nodes, ctypes.c_uint64),
                                      _p(pres, ctypes.c_uint8), pres.size,
                                      int(k), _p(buf, ctypes.c_uint64), s,
                                      ctypes.byref(where))
    return int(code), int(where.value)


def dijkstra(rowptr, col, w, src=0):
    """Textbook Dijkstra; UINT32_MAX marks unreachable vertices."""
    rowptr = np.ascontiguousarray(rowptr, dtype=np.uint64)
    col = np.ascontiguousarray(col, dtype=np.uint32)
    w = np.ascontiguousarray(w, dtype=np.uint32)
    n = rowptr.size - 1
    dist = np.empty(n, dtype=np.uint32)
    if col.size == 0:
        col = np.zeros(1, dtype=np.uint32)
        w = np.zeros(1, dtype=np.uint32)
    rc = lib().orc_dijkstra(n, _p(rowptr, ctypes.c_uint64),
                            _p(col, ctypes.c_uint32), _p(w, ctypes.c_uint32),
                            int(src), _p(dist, ctypes.c_uint32))
    if rc != 0:
        raise MemoryError("dijkstra allocation failed")
    return dist


def knapsack_dp(w, v, cap):
    """Textbook 0/1 knapsack DP optimum."""
    w = np.ascontiguousarray(w, dtype=np.uint32)
    v = np.ascontiguousarray(v, dtype=np.uint32)
    r = lib().orc_knapsack_dp(w.size, _p(w, ctypes.c_uint32),
                              _p(v, ctypes.c_uint32), int(cap))
    if r == 2**64 - 1:
        raise MemoryError("knapsack_dp allocation failed")
    return int(r)


def replay(ops, dtype=np.uint32):
    """Replays operations in their linearization order.

    ops: iterable of ("ins", keys) or ("del", n).  Returns the list of DEL
    outputs (each the min(n, size) smallest keys at that point, ascending),
    in the order given.
    """
    q = BinaryHeapPQ()
    outs = []
    try:
        for kind, arg in ops:
            if kind == "ins":
                q.push(np.asarray(arg, dtype=dtype))
            elif kind == "del":
                outs.append(q.pop(int(arg), dtype=dtype))
            else:
                raise ValueError("unknown op kind %r" % (kind,))
    finally:
        q.close()
    return outs

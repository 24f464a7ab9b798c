"""Seeded synthetic inputs for the generalized heap workloads.

This module holds only input generation: a counter-based splitmix64 stream and
the shapes of the workloads (key distributions, graphs, knapsack instances,
heap sizes, request arrivals).  It holds none of the heap's arithmetic, and it
is the one module that both the CUDA path's callers and the CPU oracle's
callers use, so that both sides see identical inputs.

splitmix64 follows its published definition (Steele, Lea and Flood, "Fast
splittable pseudorandom number generators", OOPSLA 2014; the reference C code
by S. Vigna): state_i = seed + i * 0x9e3779b97f4a7c15 (i = 1, 2, ...), output =
mix(state_i) with the two xor-shift-multiply rounds below.

Workload shapes stand in for the paper's (Section 5): raw heap traffic of
32-bit keys (uniform, ascending, descending; Section 5.2), a 2-D grid and an
R-MAT graph for SSSP (Section 5.7.1; the paper's real graphs are not
available), and strongly correlated 0/1 knapsack instances (Section 5.7.2;
the paper's generated sets are not available).
"""
import numpy as np

GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

SEED_BASE = 0x1906065040


def config_seed(n):
    """Seed of workload configuration n (1-based)."""
    return SEED_BASE + int(n)


def splitmix64(seed, n, start=0):
    """Outputs start+1 .. start+n of the splitmix64 stream seeded with `seed`."""
    with np.errstate(over="ignore"):
        i = np.arange(start + 1, start + n + 1, dtype=np.uint64)
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + i * GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform_u32(seed, n):
    """n uniform 32-bit keys: the low 32 bits of the stream."""
    return (splitmix64(seed, n) & np.uint64(0xFFFFFFFF)).astype(np.uint32)


def keys_u32(seed, n, dist="uniform"):
    """Raw-heap key streams of Section 5.2: uniform, ascending or descending.

    ascending/descending hold the same multiset as uniform, ordered.
    """
    k = uniform_u32(seed, n)
    if dist == "uniform":
        return k
    if dist == "ascending":
        return np.sort(k)
    if dist == "descending":
        return np.sort(k)[::-1].copy()
    raise ValueError("unknown distribution %r" % (dist,))


def uniform_range(seed, n, lo, hi):
    """n integers uniform in [lo, hi] (modulo reduction of the stream)."""
    span = np.uint64(hi - lo + 1)
    return (splitmix64(seed, n) % span + np.uint64(lo)).astype(np.uint32)


def grid_graph(side, seed, wlo=1, whi=100):
    """side x side 4-neighbour grid, undirected, one weight per edge.

    Returns CSR (rowptr u64[n+1], col u32[E], w u32[E]), edges of each vertex
    in the order up, left, right, down.
    """
    n = side * side
    # horizontal edge (r, c)-(r, c+1) has id r*(side-1)+c; vertical edge
    # (r, c)-(r+1, c) has id H + r*side + c
    H = side * (side - 1)
    V = (side - 1) * side
    wts = uniform_range(seed, H + V, wlo, whi)
    rows, cols, ws = [], [], []
    r, c = np.divmod(np.arange(n, dtype=np.int64), side)
    v = np.arange(n, dtype=np.int64)
    for dr, dc in ((-1, 0), (0, -1), (0, 1), (1, 0)):
        rr, cc = r + dr, c + dc
        ok = (rr >= 0) & (rr < side) & (cc >= 0) & (cc < side)
        if dr == 0:
            cmin = np.minimum(c, cc)
            eid = r * (side - 1) + cmin
        else:
            rmin = np.minimum(r, rr)
            eid = H + rmin * side + c
        rows.append(v[ok])
        cols.append((rr * side + cc)[ok])
        ws.append(wts[eid[ok]])
    return _to_csr(n, np.concatenate(rows), np.concatenate(cols),
                   np.concatenate(ws))


def rmat_graph(scale, edge_factor, seed, a=0.57, b=0.19, c=0.19, wlo=1,
               whi=1000):
    """Directed R-MAT graph with 2^scale vertices and edge_factor*2^scale
    edges (self-loops and multi-edges kept), weights uniform in [wlo, whi].
    """
    n = 1 << scale
    m = edge_factor * n
    u = np.zeros(m, dtype=np.int64)
    v = np.zeros(m, dtype=np.int64)
    ab, abc = a + b, a + b + c
    for bit in range(scale):
        x = splitmix64(seed, m, start=bit * m)
        p = (x >> np.uint64(11)).astype(np.float64) * (1.0 / (1 << 53))
        down = p >= ab                 # quadrants c or d: source bit set
        right = ((p >= a) & (p < ab)) | (p >= abc)   # quadrants b or d
        u |= down.astype(np.int64) << bit
        v |= right.astype(np.int64) << bit
    w = uniform_range(seed ^ 0x5DEECE66D, m, wlo, whi)
    return _to_csr(n, u, v, w)


def _to_csr(n, src, dst, w):
    order = np.argsort(src, kind="stable")
    src, dst, w = src[order], dst[order], w[order]
    rowptr = np.zeros(n + 1, dtype=np.uint64)
    np.cumsum(np.bincount(src, minlength=n), out=rowptr[1:])
    return rowptr, dst.astype(np.uint32), w.astype(np.uint32)


def knapsack_instance(n, seed, wlo=1, whi=1000, extra=100):
    """Strongly correlated 0/1 knapsack: w ~ U[wlo, whi], v = w + extra,
    capacity = floor(sum(w) / 2)."""
    w = uniform_range(seed, n, wlo, whi)
    v = (w.astype(np.uint64) + extra).astype(np.uint32)
    cap = int(w.astype(np.uint64).sum()) // 2
    return w, v, cap


def loguniform_sizes(seed, n, lo_log2, hi_log2):
    """n sizes 2^U(lo_log2, hi_log2), rounded to integers."""
    x = splitmix64(seed, n)
    u = (x >> np.uint64(11)).astype(np.float64) * (1.0 / (1 << 53))
    return np.rint(np.exp2(lo_log2 + u * (hi_log2 - lo_log2))).astype(np.int64)


def poisson_arrivals(seed, n, rate_per_s):
    """n arrival times (seconds) of a Poisson process with the given rate."""
    x = splitmix64(seed, n)
    u = ((x >> np.uint64(11)).astype(np.float64) + 0.5) * (1.0 / (1 << 53))
    return np.cumsum(-np.log(u) / rate_per_s)


def set_phase_ops(sizes, k, kind, base_offsets=None):
    """Operation list of one phase over many heaps: heap h gets ceil(sizes[h]/k)
    ops of `kind` (1 = INS, 2 = DEL) over its own slice [base_offsets[h],
    base_offsets[h] + sizes[h]) of the launch's key array, the last one partial.
    Ops are interleaved round-robin across heaps so that every heap has work
    from the start.  Returns a structured array (heap, kind_n, offset)."""
    sizes = np.asarray(sizes, dtype=np.int64)
    if base_offsets is None:
        base_offsets = np.concatenate([[0], np.cumsum(sizes)[:-1]])
    counts = -(-sizes // k)
    heap = np.repeat(np.arange(sizes.size, dtype=np.int64), counts)
    j = np.arange(heap.size) - np.repeat(np.cumsum(counts) - counts, counts)
    n = np.minimum(k, sizes[heap] - j * k)
    order = np.lexsort((heap, j))      # round j of every heap, then j + 1, ...
    ops = np.zeros(heap.size, dtype=[("heap", "<u4"), ("kind_n", "<u4"), ("offset", "<u8")])
    ops["heap"] = heap[order]
    ops["kind_n"] = (int(kind) << 24) | n[order]
    ops["offset"] = (np.asarray(base_offsets)[heap] + j * k)[order]
    return ops


def mixed_pairs(n_prefill, n_pairs, k, seed_off=0):
    """The mixed workload of Section 5.5 (ins-del pairs) in the shape of the
    raw-heap configuration: `n_prefill` uniform keys to insert first, then an
    operation list alternating INS and DEL of k keys each, INS j taking keys
    [j*k, (j+1)*k) of its own uniform stream and DEL j writing to output
    offset j*k.  Returns (prefill keys, stream keys, ops) with ops a
    structured array (kind u32, n u32, offset u64), kind 1 = INS, 2 = DEL."""
    pre = keys_u32(config_seed(2) + 100 + seed_off, n_prefill)
    stream = keys_u32(config_seed(2) + 200 + seed_off, n_pairs * k)
    ops = np.zeros(2 * n_pairs, dtype=[("kind", "<u4"), ("n", "<u4"), ("offset", "<u8")])
    ops["kind"][0::2] = 1
    ops["kind"][1::2] = 2
    ops["n"] = k
    ops["offset"][0::2] = np.arange(n_pairs, dtype=np.uint64) * k
    ops["offset"][1::2] = np.arange(n_pairs, dtype=np.uint64) * k
    return pre, stream, ops

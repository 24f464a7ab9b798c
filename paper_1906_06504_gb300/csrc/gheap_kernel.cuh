// gheap_kernel.cuh -- device side of the GB300 generalized concurrent heap.
//
// The TD-INS/TD-DEL heap of arXiv 1906.06504 (Chen et al.):
//   * a heap of nodes that each hold k ascending keys (Section 3.1,
//     Properties 1-3), stored as one flat array, plus a partial buffer of at
//     most k-1 keys guarded by the root lock (Section 3.3.2);
//   * INS walks from the root to a target node, doing a MergeAndSort with
//     every node on the path and carrying the k largest keys down
//     (Section 3.2.2, top-down INS);
//   * DEL returns the root batch, refills the root from the last node and
//     sifts down with two MergeAndSorts per level (Section 3.2.1);
//   * every node has a multi-state lock word (AVAIL / INUSE / TARGET /
//     MARKED, Section 3.3.2) taken with atomicCAS in parent-before-child
//     order (Section 3.3.1), and a DEL whose last node is an in-flight INS
//     target marks it and receives that INS's keys (Section 3.3.2);
//   * one thread block runs one operation (Section 4); merges use the
//     merge-path partition (Section 4.2), batch sorting a block bitonic
//     sort (Section 4.1), and node pairs whose key ranges do not overlap are
//     kept or swapped without merging (Section 4.3).
//
// GB300 specifics.  The root is the serial point of every operation
// (Section 3.3.3), so the kernel is built to shorten each lock hold rather
// than to stream bytes:
//   * the root lock, the node count m and the buffer size s share one 64-bit
//     word: acquiring the root returns the header, releasing it publishes
//     the new header;
//   * node batches move global -> shared with cp.async (16-byte, L2 only),
//     issued as soon as the node is locked and overlapped with other work;
//   * the lock of the next node on a path is tried with a single CAS while
//     the current level's MergeAndSort runs, and the two children of a DEL
//     are locked by two warps at once;
//   * persistent thread blocks pull operations from a device counter;
//   * every wait is bounded by %globaltimer and reports a sticky error.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "gheap.h"

namespace gh {

// Node lock states.  EMPTY: the slot holds no node.  AVAIL: occupied,
// unlocked.  INUSE: locked.  TARGET: allocated to an INS that has not
// arrived yet.  MARKED: a TARGET claimed by a DEL that wants its keys.
// DELIVERED: the INS wrote its keys for the DEL that marked the slot.
enum : uint32_t {
    ST_EMPTY = 0, ST_AVAIL = 1, ST_INUSE = 2, ST_TARGET = 3, ST_MARKED = 4,
    ST_DELIVERED = 5
};
constexpr uint32_t ST_GAVE_UP = ~0u;

enum : uint32_t { MODE_INSERT = 0, MODE_DELETE = 1, MODE_OPS = 2 };

enum : uint32_t { E_NONE = 0, E_TIMEOUT = 1, E_FULL = 2, E_STATE = 3 };

// Counters kept when the heap is created with GHEAP_FLAG_STATS.  The *_CYC
// entries are SM cycles seen by thread 0 of the operating block, per phase.
enum : uint32_t {
    STAT_LOADS = 0, STAT_STORES = 1, STAT_MERGES = 2, STAT_SKIPS = 3,
    STAT_INS = 4, STAT_DEL = 5, STAT_WAITS = 6, STAT_ROOT_NS = 7,
    STAT_DEL_ACQ_CYC = 8,       // waiting for the root lock
    STAT_DEL_ROOT_CYC = 9,      // root step before the children: loads, last node, refill
    STAT_DEL_WAIT_CYC = 10,     // waiting for child locks (all levels)
    STAT_DEL_LOAD_CYC = 11,     // loading children (all levels)
    STAT_DEL_MERGE_CYC = 12,    // MergeAndSorts (all levels)
    STAT_DEL_REL_CYC = 13,      // node stores and lock releases (all levels)
    STAT_DEL_LEVELS = 14,       // sift levels visited
    STAT_INS_ACQ_CYC = 15,      // waiting for the root lock
    STAT_INS_SORT_CYC = 16,     // staging and sorting the batch
    STAT_INS_WAIT_CYC = 17,     // waiting for node locks below the root
    STAT_INS_STEP_CYC = 18,     // level steps: merge, store, release, next load
    STAT_INS_LEVELS = 19,       // levels visited
    N_STATS = 20
};

// The thread that takes node locks beside thread 0 (lane 0 of warp 1; every
// launch has at least two warps).
constexpr uint32_t T2 = 32;

// Root word: bits 0-31 m (full nodes), bits 32-47 s (partial-buffer keys),
// a nonzero top byte = held.
constexpr unsigned long long ROOT_HELD = 1ull << 56;
__host__ __device__ __forceinline__ uint32_t rw_m(unsigned long long v) { return (uint32_t)v; }
__host__ __device__ __forceinline__ uint32_t rw_s(unsigned long long v)
{
    return (uint32_t)(v >> 32) & 0xFFFFu;
}
__host__ __device__ __forceinline__ unsigned long long rw_make(uint32_t m, uint32_t s)
{
    return (unsigned long long)m | ((unsigned long long)s << 32);
}

// Heap header: the root word (waiters spin on it), the linearization counter
// (touched only by the root holder) and the sticky error, each on its own
// 128-byte line.
struct __align__(128) Hdr {
    unsigned long long root;
    uint32_t _p0[30];
    unsigned long long seq;
    uint32_t _p1[30];
    uint32_t err;
    uint32_t _p2[31];
};

// Per-launch work distribution, zeroed before every launch.
struct __align__(16) Ctl {
    unsigned long long next_op;
    unsigned long long delivered;   // MODE_DELETE: keys handed out (root-guarded)
    uint32_t drained;               // MODE_DELETE: heap ran empty
    uint32_t _pad;
};

template <typename K>
struct Params {
    K *keys;                  // (max_nodes + 1) * k keys, slot j at j*k
    uint32_t *state;          // max_nodes + 1 lock words, by slot
    K *buf;                   // partial buffer, k keys
    Hdr *hdr;
    Ctl *ctl;
    gheap_log_entry *log;
    unsigned long long log_cap;
    unsigned long long *stats;   // N_STATS counters or nullptr
    uint32_t k;
    uint32_t max_nodes;
    unsigned long long timeout_ns;
    uint32_t mode;
    uint32_t call_id;
    const K *in;                 // MODE_INSERT / MODE_OPS input keys
    K *out;                      // MODE_DELETE / MODE_OPS output keys
    unsigned long long n;        // MODE_INSERT: keys; MODE_DELETE: keys wanted
    const gheap_op *ops;         // MODE_OPS
    unsigned long long n_ops;
    uint32_t *out_counts;        // MODE_OPS, may be nullptr
    unsigned long long *out_total;  // MODE_DELETE, may be nullptr
};

// Block-shared scalars that carry the lock threads' decisions to the block.
struct Shared {
    unsigned long long op;
    unsigned long long seq;
    unsigned long long out_off;
    unsigned long long t_root;
    uint32_t m, s, take;
    int stop;
    int abort;
    uint32_t lk0, lk1;     // lock results of thread 0 / thread T2
    int deliver;
    unsigned long long cnt[N_STATS];
};

// ---------------------------------------------------------------------------
// memory-model helpers
// ---------------------------------------------------------------------------

__device__ __forceinline__ unsigned long long gtimer()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ uint32_t ld_relaxed(const uint32_t *p)
{
    uint32_t v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ unsigned long long ld_relaxed64(const unsigned long long *p)
{
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ uint32_t cas_acquire(uint32_t *p, uint32_t cmp, uint32_t val)
{
    uint32_t old;
    asm volatile("atom.acquire.gpu.global.cas.b32 %0, [%1], %2, %3;"
                 : "=r"(old) : "l"(p), "r"(cmp), "r"(val) : "memory");
    return old;
}

__device__ __forceinline__ unsigned long long cas_acquire64(unsigned long long *p,
                                                            unsigned long long cmp,
                                                            unsigned long long val)
{
    unsigned long long old;
    asm volatile("atom.acquire.gpu.global.cas.b64 %0, [%1], %2, %3;"
                 : "=l"(old) : "l"(p), "l"(cmp), "l"(val) : "memory");
    return old;
}

__device__ __forceinline__ void st_release(uint32_t *p, uint32_t v)
{
    asm volatile("st.release.gpu.global.u32 [%0], %1;" :: "l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ void st_release64(unsigned long long *p, unsigned long long v)
{
    asm volatile("st.release.gpu.global.u64 [%0], %1;" :: "l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ void st_relaxed(uint32_t *p, uint32_t v)
{
    asm volatile("st.relaxed.gpu.global.u32 [%0], %1;" :: "l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ void prefetch_l2(const void *p)
{
    asm volatile("prefetch.global.L2 [%0];" :: "l"(p));
}

// Publishes `v` on lock word `w` for the whole block.  The barrier orders
// every thread's earlier writes before thread 0's st.release.gpu, and a
// release is cumulative over the writes its thread has observed, so a block
// that acquires `w` sees all of them (the same barrier + single release-store
// hand-off that split-K GEMM epilogues use between thread blocks).
__device__ __forceinline__ void block_release(uint32_t *w, uint32_t v)
{
    __syncthreads();
    if (threadIdx.x == 0) st_release(w, v);
}

template <typename K>
__device__ __forceinline__ void release_root(const Params<K> &p, uint32_t m, uint32_t s)
{
    __syncthreads();
    if (threadIdx.x == 0) st_release64(&p.hdr->root, rw_make(m, s));
}

template <typename K>
__device__ __forceinline__ K kmax() { return ~K(0); }

__device__ __forceinline__ uint32_t level_of(uint32_t x) { return 31u - __clz(x); }

// Tree position of storage slot j (and its inverse): the bit-reversal
// permutation inside the slot's level (Section 4.3).
__device__ __forceinline__ uint32_t slot_node(uint32_t j)
{
    uint32_t d = level_of(j);
    if (d == 0) return j;
    uint32_t o = j - (1u << d);
    return (1u << d) + (__brev(o) >> (32u - d));
}

__device__ __forceinline__ void stat_add(Shared &sh, uint32_t i, unsigned long long v)
{
    atomicAdd(&sh.cnt[i], v);
}

// Phase timer of thread 0: adds the cycles since `t` to counter i, restarts.
__device__ __forceinline__ void lap(Shared &sh, uint32_t i, long long &t)
{
    if (threadIdx.x == 0) {
        const long long now = clock64();
        atomicAdd(&sh.cnt[i], (unsigned long long)(now - t));
        t = now;
    }
}

// ---------------------------------------------------------------------------
// bounded waits (single thread)
// ---------------------------------------------------------------------------

template <typename K>
__device__ __forceinline__ bool keep_waiting(const Params<K> &p, unsigned long long &t0,
                                             uint32_t &it)
{
    ++it;
    if ((it & 7u) == 0) {
        if (ld_relaxed(&p.hdr->err) != E_NONE) return false;
        unsigned long long now = gtimer();
        if (t0 == 0) {
            t0 = now;
        } else if (now - t0 > p.timeout_ns) {
            atomicCAS(&p.hdr->err, E_NONE, E_TIMEOUT);
            return false;
        }
    }
    if (it > 2) __nanosleep(it < 256 ? 32 : 128);
    return true;
}

template <typename K>
__device__ __forceinline__ void set_err(const Params<K> &p, uint32_t e)
{
    atomicCAS(&p.hdr->err, E_NONE, e);
}

// Root lock (also guards the partial buffer and the header).  Returns false
// when the wait gave up; `word` receives the header (m, s).
template <typename K>
__device__ bool lock_root(const Params<K> &p, Shared &sh, unsigned long long &word)
{
    unsigned long long *w = &p.hdr->root;
    unsigned long long t0 = 0;
    uint32_t it = 0;
    for (;;) {
        unsigned long long v = ld_relaxed64(w);
        if ((v >> 56) == 0) {
            unsigned long long old = cas_acquire64(w, v, v | ROOT_HELD);
            if (old == v) {
                if (it) stat_add(sh, STAT_WAITS, 1);
                word = v;
                return true;
            }
        }
        if (!keep_waiting(p, t0, it)) return false;
    }
}

// One attempt AVAIL -> INUSE; returns the state observed (ST_AVAIL means
// acquired).
__device__ __forceinline__ uint32_t try_lock(uint32_t *w)
{
    return cas_acquire(w, ST_AVAIL, ST_INUSE);
}

// AVAIL -> INUSE, waiting while another block holds the node; `first` is the
// result of an earlier try.  Returns ST_AVAIL when acquired, the observed
// state when the slot holds no lockable node (EMPTY, TARGET, MARKED,
// DELIVERED), or ST_GAVE_UP.
template <typename K>
__device__ uint32_t lock_node(const Params<K> &p, Shared &sh, uint32_t *w, uint32_t first)
{
    uint32_t v = first;
    if (v != ST_INUSE) return v;
    unsigned long long t0 = 0;
    uint32_t it = 0;
    stat_add(sh, STAT_WAITS, 1);
    for (;;) {
        if (!keep_waiting(p, t0, it)) return ST_GAVE_UP;
        v = ld_relaxed(w);
        if (v == ST_AVAIL) v = try_lock(w);
        if (v != ST_INUSE) return v;
    }
}

// An INS arriving at its target: TARGET -> INUSE.  Returns ST_TARGET (claimed)
// or ST_MARKED (a DEL wants the keys); anything else is a protocol error.
__device__ __forceinline__ uint32_t claim_target(uint32_t *w)
{
    return atomicCAS(w, ST_TARGET, ST_INUSE);
}

// DEL takes the last node, `first` being an earlier try: lock it if it is a
// stored node; if it is the target of an INS still in flight, mark it and wait
// until that INS delivers its keys there (Section 3.3.2, INS/DEL cooperation).
// The caller holds the root and no other lock.
template <typename K>
__device__ bool take_last(const Params<K> &p, Shared &sh, uint32_t *w, uint32_t first)
{
    unsigned long long t0 = 0;
    uint32_t it = 0;
    uint32_t v = first;
    for (;;) {
        if (v == ST_AVAIL) {
            return true;   // `first` was a successful try
        } else if (v == ST_TARGET) {
            if (atomicCAS(w, ST_TARGET, ST_MARKED) == ST_TARGET) {
                stat_add(sh, STAT_WAITS, 1);
                for (;;) {
                    v = ld_relaxed(w);
                    if (v == ST_DELIVERED) {
                        __threadfence();
                        return true;
                    }
                    if (v != ST_MARKED) {
                        set_err(p, E_STATE);
                        return false;
                    }
                    if (!keep_waiting(p, t0, it)) return false;
                }
            }
        } else if (v != ST_INUSE) {
            set_err(p, E_STATE);
            return false;
        }
        if (!keep_waiting(p, t0, it)) return false;
        v = ld_relaxed(w);
        if (v == ST_AVAIL) {
            v = try_lock(w);
            if (v == ST_AVAIL) return true;
        }
    }
}

// ---------------------------------------------------------------------------
// block-wide data movement
// ---------------------------------------------------------------------------

__device__ __forceinline__ void cp_async16(void *smem, const void *gmem)
{
    unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" :: "r"(s), "l"(gmem) : "memory");
}

__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }

// Waits for this thread's async copies, then for the block.
__device__ __forceinline__ void cp_async_join()
{
    asm volatile("cp.async.wait_all;" ::: "memory");
    __syncthreads();
}

// global (L2) -> shared, asynchronous when aligned (complete with
// cp_async_join); small or unaligned batches are copied synchronously.
template <typename K>
__device__ __forceinline__ void g2s_async(K *dst, const K *src, uint32_t n)
{
    const uint32_t bytes = n * (uint32_t)sizeof(K);
    if (((reinterpret_cast<uintptr_t>(src) | reinterpret_cast<uintptr_t>(dst)) & 15u) == 0 &&
        (bytes & 15u) == 0) {
        const char *s = reinterpret_cast<const char *>(src);
        char *d = reinterpret_cast<char *>(dst);
        for (uint32_t i = threadIdx.x; i < bytes / 16u; i += blockDim.x)
            cp_async16(d + 16u * i, s + 16u * i);
    } else {
        for (uint32_t i = threadIdx.x; i < n; i += blockDim.x) dst[i] = __ldcg(src + i);
    }
}

// shared -> global (L2)
template <typename K>
__device__ __forceinline__ void s2g(K *dst, const K *src, uint32_t n)
{
    const uint32_t bytes = n * (uint32_t)sizeof(K);
    if (((reinterpret_cast<uintptr_t>(src) | reinterpret_cast<uintptr_t>(dst)) & 15u) == 0 &&
        (bytes & 15u) == 0) {
        const uint4 *s4 = reinterpret_cast<const uint4 *>(src);
        uint4 *d4 = reinterpret_cast<uint4 *>(dst);
        for (uint32_t i = threadIdx.x; i < bytes / 16u; i += blockDim.x) __stcg(d4 + i, s4[i]);
    } else {
        for (uint32_t i = threadIdx.x; i < n; i += blockDim.x) __stcg(dst + i, src[i]);
    }
}

// Block bitonic sort of a[0..k), k a power of two, ascending (Section 4.1).
template <typename K>
__device__ void block_sort(K *a, uint32_t k)
{
    for (uint32_t size = 2; size <= k; size <<= 1) {
        for (uint32_t stride = size >> 1; stride > 0; stride >>= 1) {
            for (uint32_t i = threadIdx.x; i < (k >> 1); i += blockDim.x) {
                uint32_t lo = 2 * i - (i & (stride - 1));
                uint32_t hi = lo + stride;
                bool asc = (lo & size) == 0;
                K x = a[lo], y = a[hi];
                if ((x > y) == asc) {
                    a[lo] = y;
                    a[hi] = x;
                }
            }
            __syncthreads();
        }
    }
}

// MergeAndSort of two ascending runs in shared memory (Section 3.2.1) by the
// merge-path partition (Section 4.2): output position q < split goes to
// dlo[q], the rest to dhi[q - split].  Thread t produces outputs
// [t*IPT, t*IPT + IPT); na + nb must not exceed IPT * blockDim.x.  The
// destinations may alias the sources.  Ends with a barrier.
template <typename K, int IPT>
__device__ __forceinline__ void merge_split(const K *a, uint32_t na, const K *b, uint32_t nb,
                                            K *dlo, uint32_t split, K *dhi)
{
    const uint32_t total = na + nb;
    const uint32_t start = threadIdx.x * IPT;
    K v[IPT];
    if (na == 0 || nb == 0) {
        // one run is empty: the merge is a copy of the other
        const K *src = na ? a : b;
        if (start < total) {
#pragma unroll
            for (int q = 0; q < IPT; ++q)
                if (start + q < total) v[q] = src[start + q];
        }
    } else if (start < total) {
        uint32_t lo = start > nb ? start - nb : 0u;
        uint32_t hi = start < na ? start : na;
        while (lo < hi) {
            uint32_t mid = (lo + hi) >> 1;
            if (a[mid] <= b[start - 1 - mid]) lo = mid + 1;
            else hi = mid;
        }
        uint32_t i = lo, j = start - lo;
#pragma unroll
        for (int q = 0; q < IPT; ++q) {
            if (start + q < total) {
                bool ta = (j >= nb) || (i < na && a[i] <= b[j]);
                v[q] = ta ? a[i] : b[j];
                i += ta;
                j += !ta;
            }
        }
    }
    __syncthreads();
    if (start < total) {
#pragma unroll
        for (int q = 0; q < IPT; ++q) {
            uint32_t pos = start + q;
            if (pos < total) {
                if (pos < split) dlo[pos] = v[q];
                else dhi[pos - split] = v[q];
            }
        }
    }
    __syncthreads();
}

// MergeAndSort of two full ascending runs a[0..k), b[0..k) (Section 3.2.1) as
// a bitonic merge (a followed by b reversed is bitonic): one compare stage
// across the halves leaves the k smallest in dlo and the k largest in dhi,
// each a bitonic run; each half is then sorted by its own half-cleaner
// stages -- strides of 32*IPT keys and more in shared memory, smaller ones
// in registers via warp shuffles.  Needs blockDim.x * IPT == 2k and k >=
// 32 * IPT; destinations may alias the sources.  Ends with a barrier.
template <typename K, int IPT>
__device__ __forceinline__ void merge_full(const K *a, const K *b, K *dlo, K *dhi, uint32_t k)
{
    const uint32_t T = blockDim.x, tid = threadIdx.x;
    K lo_v[IPT / 2], hi_v[IPT / 2];
#pragma unroll
    for (int r = 0; r < IPT / 2; ++r) {
        const uint32_t i = tid + r * T;
        const K x = a[i], y = b[k - 1 - i];
        lo_v[r] = x < y ? x : y;
        hi_v[r] = x < y ? y : x;
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < IPT / 2; ++r) {
        const uint32_t i = tid + r * T;
        dlo[i] = lo_v[r];
        dhi[i] = hi_v[r];
    }
    __syncthreads();
    const uint32_t half = T >> 1;
    const uint32_t u = tid < half ? tid : tid - half;
    K *d = tid < half ? dlo : dhi;
    for (uint32_t st = k >> 1; st >= 32u * IPT; st >>= 1) {
#pragma unroll
        for (int r = 0; r < IPT / 2; ++r) {
            const uint32_t j = u + r * half;
            const uint32_t l = 2 * j - (j & (st - 1)), h = l + st;
            const K x = d[l], y = d[h];
            if (y < x) {
                d[l] = y;
                d[h] = x;
            }
        }
        __syncthreads();
    }
    K v[IPT];
#pragma unroll
    for (int q = 0; q < IPT; ++q) v[q] = d[u * IPT + q];
    const uint32_t lane = tid & 31u;
#pragma unroll
    for (uint32_t lm = 16; lm >= 1; lm >>= 1) {
        if (lm * IPT <= (k >> 1)) {
            const bool upper = (lane & lm) != 0;
#pragma unroll
            for (int q = 0; q < IPT; ++q) {
                const K o = __shfl_xor_sync(0xffffffffu, v[q], lm);
                v[q] = upper ? (o < v[q] ? v[q] : o) : (o < v[q] ? o : v[q]);
            }
        }
    }
#pragma unroll
    for (int st = IPT / 2; st >= 1; st >>= 1) {
#pragma unroll
        for (int q = 0; q < IPT; ++q) {
            if ((q & st) == 0) {
                const K x = v[q], y = v[q + st];
                v[q] = x < y ? x : y;
                v[q + st] = x < y ? y : x;
            }
        }
    }
#pragma unroll
    for (int q = 0; q < IPT; ++q) d[u * IPT + q] = v[q];
    __syncthreads();
}

// MergeAndSort of two full k-runs into (k smallest -> dlo, k largest -> dhi):
// the bitonic form when the block shape allows it, else merge path.
template <typename K, int IPT>
__device__ __forceinline__ void merge_kk(const K *a, const K *b, K *dlo, K *dhi, uint32_t k)
{
    if (blockDim.x * IPT == 2 * k && k >= 32u * IPT) merge_full<K, IPT>(a, b, dlo, dhi, k);
    else merge_split<K, IPT>(a, k, b, k, dlo, k, dhi);
}

// Takes a ticket under the root lock and records the operation in the
// linearization record (thread 0).
template <typename K>
__device__ __forceinline__ void take_ticket(const Params<K> &p, Shared &sh, uint32_t kind,
                                            uint32_t n, unsigned long long ref)
{
    unsigned long long seq = __ldcg(&p.hdr->seq);
    __stcg(&p.hdr->seq, seq + 1);
    sh.seq = seq;
    if (seq < p.log_cap) {
        gheap_log_entry e;
        e.call_id = p.call_id;
        e.kind_n = (kind << 24) | n;
        e.ref = ref;
        p.log[seq] = e;
    }
}

// ---------------------------------------------------------------------------
// INS (Section 3.2.2 top-down INS, Section 3.3.2 partial buffer)
// ---------------------------------------------------------------------------

// The batch a[0..n) is sorted (a[n..k) hold the key maximum).  Returns false
// when the operation had to give up (the block must stop).
template <typename K, int IPT>
__device__ bool ins_op(const Params<K> &p, Shared &sh, K *a, K *b, K *c, uint32_t n,
                       unsigned long long ref)
{
    const uint32_t k = p.k;
    const uint32_t tid = threadIdx.x;
    long long tp = clock64();
    if (tid == 0) {
        unsigned long long w = 0;
        sh.abort = !lock_root(p, sh, w);
        if (!sh.abort) {
            sh.t_root = gtimer();
            sh.m = rw_m(w);
            sh.s = rw_s(w);
            take_ticket(p, sh, GHEAP_OP_INS, n, ref);
        }
    }
    lap(sh, STAT_INS_ACQ_CYC, tp);
    __syncthreads();
    if (sh.abort) return false;
    const uint32_t m = sh.m;
    uint32_t s = sh.s;
    K *root = p.keys + (size_t)k;

    if (n < k) {
        // partial batch: merge into the partial buffer
        const bool fits = n + s < k;
        g2s_async(c, p.buf, s);
        if (fits && m >= 1) g2s_async(b, root, k);
        cp_async_commit();
        cp_async_join();
        if (fits) {
            merge_split<K, IPT>(a, n, c, s, c, n + s, c);
            if (m >= 1) {
                // Property 3: the root keeps the k smallest of root + buffer
                merge_split<K, IPT>(b, k, c, n + s, b, k, c);
                s2g(root, b, k);
                if (tid == 0) {
                    stat_add(sh, STAT_LOADS, 1);
                    stat_add(sh, STAT_STORES, 1);
                    stat_add(sh, STAT_MERGES, 1);
                }
            }
            s2g(p.buf, c, n + s);
            if (tid == 0) stat_add(sh, STAT_ROOT_NS, gtimer() - sh.t_root);
            release_root(p, m, n + s);
            return true;
        }
        // the k smallest of batch + buffer go down as a full batch
        merge_split<K, IPT>(a, n, c, s, a, k, c);
        s = n + s - k;
        s2g(p.buf, c, s);
    } else if (m == 0 && s > 0) {
        // the batch becomes the root: keep Property 3 with the buffer
        g2s_async(c, p.buf, s);
        cp_async_commit();
        cp_async_join();
        merge_split<K, IPT>(a, k, c, s, a, k, c);
        s2g(p.buf, c, s);
    }

    if (m == 0) {
        s2g(root, a, k);
        if (tid == 0) {
            stat_add(sh, STAT_STORES, 1);
            stat_add(sh, STAT_ROOT_NS, gtimer() - sh.t_root);
        }
        release_root(p, 1u, s);
        return true;
    }

    // full top-down INS to the next target slot
    const uint32_t tslot = m + 1;
    if (tslot > p.max_nodes) {
        if (tid == 0) set_err(p, E_FULL);
        return false;
    }
    const uint32_t tnode = slot_node(tslot);
    const uint32_t depth = level_of(tnode);
    // the thread that later claims the target also marks it (program order)
    if (tid == T2) st_relaxed(&p.state[tslot], ST_TARGET);

    // root data, and a first try on the level-1 node of the path
    g2s_async(b, root, k);
    cp_async_commit();
    if (tid == T2) {
        const uint32_t n1 = tnode >> (depth - 1);
        uint32_t *w1 = &p.state[slot_node(n1)];
        sh.lk1 = (n1 == tnode) ? claim_target(w1) : try_lock(w1);
    }
    cp_async_join();

    K *cur_keys = root;
    uint32_t *cur_w = nullptr;   // nullptr = the root word
    for (uint32_t lvl = 0;; ++lvl) {
        const uint32_t nxt = tnode >> (depth - lvl - 1);
        const uint32_t nslot = slot_node(nxt);
        uint32_t *nw = &p.state[nslot];
        K *nkeys = p.keys + (size_t)nslot * k;
        const bool at_target = (nxt == tnode);
        // finish taking the next node (hand-over-hand: we hold the current one)
        if (tid == T2) {
            uint32_t v = sh.lk1;
            if (at_target) {
                sh.deliver = (v == ST_MARKED);
                if (v != ST_TARGET && v != ST_MARKED) {
                    set_err(p, E_STATE);
                    sh.abort = 1;
                }
            } else if (v != ST_AVAIL) {
                v = lock_node(p, sh, nw, v);
                if (v != ST_AVAIL) {
                    if (v != ST_GAVE_UP) set_err(p, E_STATE);
                    sh.abort = 1;
                }
            }
        }
        __syncthreads();
        lap(sh, STAT_INS_WAIT_CYC, tp);
        if (tid == 0) stat_add(sh, STAT_INS_LEVELS, 1);
        if (sh.abort) return false;
        uint32_t next_try = ST_EMPTY;
        if (!at_target) {
            g2s_async(c, nkeys, k);
            cp_async_commit();
            // try the node after next while this level merges
            if (tid == T2) {
                const uint32_t n2 = tnode >> (depth - lvl - 2);
                uint32_t *w2 = &p.state[slot_node(n2)];
                next_try = (n2 == tnode) ? claim_target(w2) : try_lock(w2);
            }
        }
        // MergeAndSort(node, batch): the node keeps the k smallest, the k
        // largest are carried on (Section 3.2.2); disjoint ranges are kept or
        // swapped without merging (Section 4.3).
        {
            const K bmax = b[k - 1], bmin = b[0], amax = a[k - 1], amin = a[0];
            if (bmax <= amin) {
                if (tid == 0) stat_add(sh, STAT_SKIPS, 1);
            } else if (amax <= bmin) {
                s2g(cur_keys, a, k);
                K *t = a; a = b; b = t;
                if (tid == 0) { stat_add(sh, STAT_SKIPS, 1); stat_add(sh, STAT_STORES, 1); }
            } else {
                merge_kk<K, IPT>(b, a, b, a, k);
                s2g(cur_keys, b, k);
                if (tid == 0) { stat_add(sh, STAT_MERGES, 1); stat_add(sh, STAT_STORES, 1); }
            }
            if (tid == 0) stat_add(sh, STAT_LOADS, 1);
        }
        if (cur_w == nullptr) {
            if (tid == 0) stat_add(sh, STAT_ROOT_NS, gtimer() - sh.t_root);
            release_root(p, tslot, s);
        } else {
            block_release(cur_w, ST_AVAIL);
        }
        if (at_target) {
            s2g(nkeys, a, k);
            if (tid == 0) stat_add(sh, STAT_STORES, 1);
            block_release(nw, sh.deliver ? ST_DELIVERED : ST_AVAIL);
            return true;
        }
        if (tid == T2) sh.lk1 = next_try;
        cp_async_join();
        lap(sh, STAT_INS_STEP_CYC, tp);
        K *t = b; b = c; c = t;
        cur_keys = nkeys;
        cur_w = nw;
    }
}

// ---------------------------------------------------------------------------
// DEL (Section 3.2.1, partial buffer of Section 3.3.2)
// ---------------------------------------------------------------------------

// Children of `node` that exist in storage: slot numbers, or 0.
__device__ __forceinline__ void child_slots(uint32_t node, uint32_t max_nodes, uint32_t &sl,
                                            uint32_t &sr)
{
    const uint32_t l = 2 * node;
    sl = sr = 0;
    if (level_of(l) <= level_of(max_nodes)) {
        uint32_t a = slot_node(l), b = slot_node(l + 1);
        sl = a <= max_nodes ? a : 0;
        sr = b <= max_nodes ? b : 0;
    }
}

// Deletes up to `want` keys.  MODE_DELETE takes its output offset and count
// from the launch's running total under the root lock; MODE_OPS writes to
// `out_off`.  Returns false when the block must stop.
template <typename K, int IPT>
__device__ bool del_op(const Params<K> &p, Shared &sh, K *A, K *B, K *C, K *D,
                       uint32_t want, unsigned long long out_off, unsigned long long ref,
                       uint32_t *count_out)
{
    const uint32_t k = p.k;
    const uint32_t tid = threadIdx.x;
    long long tp = clock64();
    if (tid == 0) {
        unsigned long long w = 0;
        sh.abort = !lock_root(p, sh, w);
        lap(sh, STAT_DEL_ACQ_CYC, tp);
        if (!sh.abort) {
            sh.t_root = gtimer();
            const uint32_t m = rw_m(w), s = rw_s(w);
            sh.m = m;
            sh.s = s;
            if (p.mode == MODE_DELETE) {
                unsigned long long done = p.ctl->delivered;
                unsigned long long rem = p.n > done ? p.n - done : 0ull;
                want = rem < want ? (uint32_t)rem : want;
                out_off = done;
            }
            const uint32_t avail = m >= 1 ? k : s;
            const uint32_t take = want < avail ? want : avail;
            sh.take = take;
            sh.out_off = out_off;
            if (p.mode == MODE_DELETE) {
                p.ctl->delivered = out_off + take;
                if (p.out_total) *p.out_total = out_off + take;
                if (take == 0 || out_off + take >= p.n) p.ctl->drained = 1u;
            }
            if (count_out) *count_out = take;
            take_ticket(p, sh, GHEAP_OP_DEL, take, p.mode == MODE_DELETE ? out_off : ref);
        }
    }
    __syncthreads();
    if (sh.abort) return false;
    const uint32_t m = sh.m, s = sh.s;
    const uint32_t take = sh.take;
    out_off = sh.out_off;
    K *root = p.keys + (size_t)k;

    if (m == 0) {
        // no full node: serve from the partial buffer (Section 3.3.2)
        g2s_async(C, p.buf, s);
        cp_async_commit();
        cp_async_join();
        s2g(p.out + out_off, C, take);
        s2g(p.buf, C + take, s - take);
        if (tid == 0) stat_add(sh, STAT_ROOT_NS, gtimer() - sh.t_root);
        release_root(p, 0u, s - take);
        return true;
    }

    // the root refill needs the last node when the buffer cannot supply take
    const bool need_last = s < take && m >= 2;
    g2s_async(B, root, k);
    g2s_async(C, p.buf, s);
    cp_async_commit();
    if (need_last && tid == T2) sh.lk1 = try_lock(&p.state[m]);
    cp_async_join();
    s2g(p.out + out_off, B, take);
    if (tid == 0) stat_add(sh, STAT_LOADS, 1);
    uint32_t nm = m, ns;
    if (s >= take) {
        // refill the root from the partial buffer
        merge_split<K, IPT>(B + take, k - take, C, s, B, k, C);
        ns = s - take;
        s2g(p.buf, C, ns);
    } else {
        const uint32_t tn = k - take + s;
        merge_split<K, IPT>(B + take, k - take, C, s, C, tn, C);
        if (m == 1) {
            // the root was the last full node
            s2g(p.buf, C, tn);
            if (tid == 0) stat_add(sh, STAT_ROOT_NS, gtimer() - sh.t_root);
            release_root(p, 0u, tn);
            return true;
        }
        // refill the root from the last node (slot m)
        uint32_t *lw = &p.state[m];
        if (tid == T2) {
            if (take_last(p, sh, lw, sh.lk1)) {
                // nobody may lock or target slot m until the root is released
                st_relaxed(lw, ST_EMPTY);
            } else {
                sh.abort = 1;
            }
        } else if (tid >= 64 && tid < 96 && m >= 3) {
            // the next DEL's last node: warm L2 (one 128-byte line a thread)
            const char *nxt = reinterpret_cast<const char *>(p.keys + (size_t)(m - 1) * k);
            for (uint32_t off = (tid - 64) * 128u; off < k * sizeof(K); off += 32 * 128u)
                prefetch_l2(nxt + off);
        }
        __syncthreads();
        if (sh.abort) return false;
        if (tn == 0) {
            // nothing left of the root or the buffer: the last node is the root
            g2s_async(B, p.keys + (size_t)m * k, k);
            cp_async_commit();
            cp_async_join();
        } else {
            g2s_async(A, p.keys + (size_t)m * k, k);
            cp_async_commit();
            cp_async_join();
            merge_split<K, IPT>(C, tn, A, k, B, k, C);
        }
        if (tid == 0) stat_add(sh, STAT_LOADS, 1);
        ns = tn;
        nm = m - 1;
        s2g(p.buf, C, ns);
    }

    // sift down from the root; B holds the current node's keys
    uint32_t node = 1;
    K *cur_keys = root;
    uint32_t *cur_w = nullptr;       // nullptr = the root word
    uint32_t tried0 = 0, tried1 = 0; // earlier tries on the children
    bool pre = false;
    lap(sh, STAT_DEL_ROOT_CYC, tp);
    for (;;) {
        uint32_t sl, sr;
        child_slots(node, p.max_nodes, sl, sr);
        // lock both children at once (thread 0: left, thread T2: right)
        if (tid == 0) {
            uint32_t v = sl ? (pre ? tried0 : try_lock(&p.state[sl])) : ST_EMPTY;
            if (sl) v = lock_node(p, sh, &p.state[sl], v);
            sh.lk0 = v;
        } else if (tid == T2) {
            uint32_t v = sr ? (pre ? tried1 : try_lock(&p.state[sr])) : ST_EMPTY;
            if (sr) v = lock_node(p, sh, &p.state[sr], v);
            sh.lk1 = v;
        }
        __syncthreads();
        lap(sh, STAT_DEL_WAIT_CYC, tp);
        if (tid == 0) stat_add(sh, STAT_DEL_LEVELS, 1);
        if (sh.lk0 == ST_GAVE_UP || sh.lk1 == ST_GAVE_UP) return false;
        const bool pl = sh.lk0 == ST_AVAIL, pr = sh.lk1 == ST_AVAIL;
        if (!pl && !pr) break;
        K *lk = p.keys + (size_t)sl * k;
        K *rk = p.keys + (size_t)sr * k;
        if (pl) g2s_async(C, lk, k);
        if (pr) g2s_async(D, rk, k);
        cp_async_commit();
        cp_async_join();
        lap(sh, STAT_DEL_LOAD_CYC, tp);
        if (tid == 0) stat_add(sh, STAT_LOADS, (unsigned long long)(pl + pr));
        const K cmax = B[k - 1];
        if (pl != pr) {
            // one child present (the other is absent or an INS target)
            K *X = pl ? C : D;
            uint32_t *xw = &p.state[pl ? sl : sr];
            if (cmax <= X[0]) {
                block_release(xw, ST_AVAIL);
                break;
            }
            const uint32_t x = pl ? 2 * node : 2 * node + 1;
            uint32_t gl, gr;
            child_slots(x, p.max_nodes, gl, gr);
            uint32_t t_try0 = ST_EMPTY, t_try1 = ST_EMPTY;
            if (tid == 0 && gl) t_try0 = try_lock(&p.state[gl]);
            if (tid == T2 && gr) t_try1 = try_lock(&p.state[gr]);
            merge_kk<K, IPT>(B, X, B, X, k);
            lap(sh, STAT_DEL_MERGE_CYC, tp);
            s2g(cur_keys, B, k);
            if (tid == 0) {
                stat_add(sh, STAT_MERGES, 1);
                stat_add(sh, STAT_STORES, 1);
            }
            if (cur_w == nullptr) {
                if (tid == 0) stat_add(sh, STAT_ROOT_NS, gtimer() - sh.t_root);
                release_root(p, nm, ns);
            } else {
                block_release(cur_w, ST_AVAIL);
            }
            lap(sh, STAT_DEL_REL_CYC, tp);
            tried0 = t_try0;
            tried1 = t_try1;
            pre = true;
            node = x;
            cur_keys = pl ? lk : rk;
            cur_w = xw;
            K *t = B; B = X;
            if (pl) C = t; else D = t;
            continue;
        }
        // both children present
        if (cmax <= C[0] && cmax <= D[0]) {
            // early stop (Section 4.3)
            if (tid == 0) st_release(&p.state[sl], ST_AVAIL);
            if (tid == T2) st_release(&p.state[sr], ST_AVAIL);
            break;
        }
        // MergeAndSort(l, r): the k largest go to the child whose maximum
        // was larger (the right child on a tie), the k smallest to the other
        const bool big_l = C[k - 1] > D[k - 1];
        const uint32_t smn = big_l ? 2 * node + 1 : 2 * node;
        uint32_t gl, gr;
        child_slots(smn, p.max_nodes, gl, gr);
        uint32_t t_try0 = ST_EMPTY, t_try1 = ST_EMPTY;
        if (tid == 0 && gl) t_try0 = try_lock(&p.state[gl]);
        if (tid == T2 && gr) t_try1 = try_lock(&p.state[gr]);
        K *S, *L;               // smem of the small and large halves
        bool l_changed, r_changed;
        if (C[k - 1] <= D[0]) {
            S = C; L = D;
            l_changed = r_changed = big_l;   // false here: nothing moves
        } else if (D[k - 1] <= C[0]) {
            S = D; L = C;
            l_changed = r_changed = !big_l;
        } else {
            merge_kk<K, IPT>(C, D, C, D, k);
            S = C; L = D;
            l_changed = r_changed = true;
            if (tid == 0) stat_add(sh, STAT_MERGES, 1);
        }
        lap(sh, STAT_DEL_MERGE_CYC, tp);
        if (!l_changed && tid == 0) stat_add(sh, STAT_SKIPS, 1);
        K *big_keys = big_l ? lk : rk;
        uint32_t *big_w = &p.state[big_l ? sl : sr];
        K *sm_keys = big_l ? rk : lk;
        uint32_t *sm_w = &p.state[big_l ? sr : sl];
        const bool big_changed = big_l ? l_changed : r_changed;
        const bool sm_changed = big_l ? r_changed : l_changed;
        if (big_changed) {
            s2g(big_keys, L, k);
            if (tid == 0) stat_add(sh, STAT_STORES, 1);
        }
        block_release(big_w, ST_AVAIL);
        lap(sh, STAT_DEL_REL_CYC, tp);
        if (cmax <= S[0]) {
            if (sm_changed) {
                s2g(sm_keys, S, k);
                if (tid == 0) stat_add(sh, STAT_STORES, 1);
            }
            // give back the grandchildren taken by the tries
            if (tid == 0 && t_try0 == ST_AVAIL) st_release(&p.state[gl], ST_AVAIL);
            if (tid == T2 && t_try1 == ST_AVAIL) st_release(&p.state[gr], ST_AVAIL);
            block_release(sm_w, ST_AVAIL);
            break;
        }
        // MergeAndSort(cur, small child): cur keeps the k smallest
        merge_kk<K, IPT>(B, S, B, S, k);
        lap(sh, STAT_DEL_MERGE_CYC, tp);
        s2g(cur_keys, B, k);
        if (tid == 0) {
            stat_add(sh, STAT_MERGES, 1);
            stat_add(sh, STAT_STORES, 1);
        }
        if (cur_w == nullptr) {
            if (tid == 0) stat_add(sh, STAT_ROOT_NS, gtimer() - sh.t_root);
            release_root(p, nm, ns);
        } else {
            block_release(cur_w, ST_AVAIL);
        }
        lap(sh, STAT_DEL_REL_CYC, tp);
        tried0 = t_try0;
        tried1 = t_try1;
        pre = true;
        node = smn;
        cur_keys = sm_keys;
        cur_w = sm_w;
        K *oldB = B;
        B = S;
        if (S == C) C = oldB; else D = oldB;
    }
    // last node of the walk: write it and release it
    s2g(cur_keys, B, k);
    if (tid == 0) stat_add(sh, STAT_STORES, 1);
    if (cur_w == nullptr) {
        if (tid == 0) stat_add(sh, STAT_ROOT_NS, gtimer() - sh.t_root);
        release_root(p, nm, ns);
    } else {
        block_release(cur_w, ST_AVAIL);
    }
    (void)A;
    return true;
}

// ---------------------------------------------------------------------------
// persistent kernel
// ---------------------------------------------------------------------------

template <typename K, int IPT>
__global__ void __launch_bounds__(512, 1) heap_kernel(Params<K> p)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ Shared sh;
    const uint32_t k = p.k;
    K *A = reinterpret_cast<K *>(smem_raw);
    K *B = A + k;
    K *C = B + k;
    K *D = C + k;
    if (threadIdx.x < N_STATS) sh.cnt[threadIdx.x] = 0;

    unsigned long long n_ops;
    if (p.mode == MODE_OPS) n_ops = p.n_ops;
    else n_ops = (p.n + k - 1) / k;

    for (;;) {
        if (threadIdx.x == 0) {
            unsigned long long op = atomicAdd(&p.ctl->next_op, 1ull);
            sh.op = op;
            int stop = op >= n_ops || ld_relaxed(&p.hdr->err) != E_NONE;
            if (!stop && p.mode == MODE_DELETE && ld_relaxed(&p.ctl->drained)) stop = 1;
            sh.stop = stop;
            sh.abort = 0;
        }
        __syncthreads();
        if (sh.stop) break;
        const unsigned long long op = sh.op;
        bool ok;
        uint32_t kind, n;
        unsigned long long off;
        if (p.mode == MODE_INSERT) {
            kind = GHEAP_OP_INS;
            off = op * k;
            n = (uint32_t)min((unsigned long long)k, p.n - off);
        } else if (p.mode == MODE_DELETE) {
            kind = GHEAP_OP_DEL;
            n = k;
            off = 0;
        } else {
            gheap_op d = p.ops[op];
            kind = d.kind;
            n = d.n;
            off = d.offset;
        }
        if (kind == GHEAP_OP_INS) {
            // stage and sort the batch before taking the root (Section 4.1)
            long long ts = clock64();
            const K *src = p.in + off;
            if (n < k) {
                for (uint32_t i = threadIdx.x; i < k; i += blockDim.x)
                    A[i] = i < n ? __ldcg(src + i) : kmax<K>();
                __syncthreads();
            } else {
                g2s_async(A, src, k);
                cp_async_commit();
                cp_async_join();
            }
            block_sort(A, k);
            lap(sh, STAT_INS_SORT_CYC, ts);
            ok = ins_op<K, IPT>(p, sh, A, B, C, n, p.mode == MODE_OPS ? op : off);
            if (threadIdx.x == 0) {
                stat_add(sh, STAT_INS, 1);
                if (p.mode == MODE_OPS && p.out_counts) p.out_counts[op] = n;
            }
        } else {
            ok = del_op<K, IPT>(p, sh, A, B, C, D, n, off, op,
                                p.mode == MODE_OPS && p.out_counts ? p.out_counts + op : nullptr);
            if (threadIdx.x == 0) stat_add(sh, STAT_DEL, 1);
        }
        if (!ok) break;
        __syncthreads();
    }
    __syncthreads();
    if (p.stats && threadIdx.x < N_STATS && sh.cnt[threadIdx.x])
        atomicAdd(p.stats + threadIdx.x, sh.cnt[threadIdx.x]);
}

}  // namespace gh

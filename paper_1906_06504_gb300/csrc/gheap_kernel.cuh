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
// GB300 specifics: thread blocks are persistent and pull operations from a
// device counter; node batches move between L2/HBM and shared memory with
// 16-byte L1-bypassing accesses; lock words are acquired with
// atom.acquire.gpu and released with st.release.gpu after a block-wide
// fence; every wait is bounded by %globaltimer and reports a sticky error
// instead of hanging.
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

enum : uint32_t { MODE_INSERT = 0, MODE_DELETE = 1, MODE_OPS = 2 };

enum : uint32_t { E_NONE = 0, E_TIMEOUT = 1, E_FULL = 2, E_STATE = 3 };

enum : uint32_t {
    STAT_LOADS = 0, STAT_STORES = 1, STAT_MERGES = 2, STAT_SKIPS = 3,
    STAT_INS = 4, STAT_DEL = 5, STAT_WAITS = 6, STAT_ROOT_NS = 7, N_STATS = 8
};

// Heap header.  The root lock sits on its own 128-byte line (waiters spin
// on it); m, s and seq are guarded by the root lock; err is the sticky
// device error that every wait polls.
struct __align__(128) Hdr {
    uint32_t root_lock;
    uint32_t _p0[31];
    uint32_t m;                 // allocated nodes (slots 1..m)
    uint32_t s;                 // keys in the partial buffer
    unsigned long long seq;     // operations linearized so far
    uint32_t _p1[28];
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

// Block-shared scalars that carry thread 0's decisions to the block.
struct Shared {
    unsigned long long op;
    unsigned long long seq;
    unsigned long long out_off;
    uint32_t m, s, take;
    int stop;
    int abort;
    int pl, pr;
    int deliver;
    unsigned long long t_root;
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

__device__ __forceinline__ uint32_t cas_acquire(uint32_t *p, uint32_t cmp, uint32_t val)
{
    uint32_t old;
    asm volatile("atom.acquire.gpu.global.cas.b32 %0, [%1], %2, %3;"
                 : "=r"(old) : "l"(p), "r"(cmp), "r"(val) : "memory");
    return old;
}

__device__ __forceinline__ void st_release(uint32_t *p, uint32_t v)
{
    asm volatile("st.release.gpu.global.u32 [%0], %1;" :: "l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ void st_relaxed(uint32_t *p, uint32_t v)
{
    asm volatile("st.relaxed.gpu.global.u32 [%0], %1;" :: "l"(p), "r"(v) : "memory");
}

// Release a lock word on behalf of the whole block: every thread's global
// writes are made visible at GPU scope before thread 0 publishes `v`.
__device__ __forceinline__ void block_release(uint32_t *w, uint32_t v)
{
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) st_release(w, v);
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

// ---------------------------------------------------------------------------
// bounded waits (thread 0 only)
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
    if (it > 4) __nanosleep(it < 64 ? 20 : 200);
    return true;
}

template <typename K>
__device__ __forceinline__ void set_err(const Params<K> &p, uint32_t e)
{
    atomicCAS(&p.hdr->err, E_NONE, e);
}

// Root lock (also guards the partial buffer and the header).
template <typename K>
__device__ bool lock_root(const Params<K> &p, Shared &sh)
{
    uint32_t *w = &p.hdr->root_lock;
    unsigned long long t0 = 0;
    uint32_t it = 0;
    for (;;) {
        if (ld_relaxed(w) == 0u && cas_acquire(w, 0u, 1u) == 0u) {
            if (it) sh.cnt[STAT_WAITS]++;
            return true;
        }
        if (!keep_waiting(p, t0, it)) return false;
    }
}

// AVAIL -> INUSE, waiting while another block holds the node.  Returns
// ST_AVAIL when acquired, the observed state when the slot holds no
// lockable node (EMPTY, TARGET, MARKED, DELIVERED), or ~0u when the wait
// gave up.
template <typename K>
__device__ uint32_t lock_node(const Params<K> &p, Shared &sh, uint32_t *w)
{
    unsigned long long t0 = 0;
    uint32_t it = 0;
    for (;;) {
        uint32_t v = ld_relaxed(w);
        if (v == ST_AVAIL) {
            v = cas_acquire(w, ST_AVAIL, ST_INUSE);
            if (v == ST_AVAIL) {
                if (it) sh.cnt[STAT_WAITS]++;
                return ST_AVAIL;
            }
        }
        if (v != ST_INUSE && v != ST_AVAIL) return v;
        if (!keep_waiting(p, t0, it)) return ~0u;
    }
}

// DEL takes the last node: lock it if it is a stored node; if it is the
// target of an INS still in flight, mark it and wait until that INS
// delivers its keys there (Section 3.3.2, INS/DEL cooperation).
template <typename K>
__device__ bool take_last(const Params<K> &p, Shared &sh, uint32_t *w)
{
    unsigned long long t0 = 0;
    uint32_t it = 0;
    for (;;) {
        uint32_t v = ld_relaxed(w);
        if (v == ST_AVAIL) {
            if (cas_acquire(w, ST_AVAIL, ST_INUSE) == ST_AVAIL) return true;
        } else if (v == ST_TARGET) {
            if (atomicCAS(w, ST_TARGET, ST_MARKED) == ST_TARGET) {
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
    }
}

// ---------------------------------------------------------------------------
// block-wide data movement
// ---------------------------------------------------------------------------

// global (L2, bypassing L1) -> shared
template <typename K>
__device__ __forceinline__ void g2s(K *dst, const K *src, uint32_t n)
{
    const uint32_t bytes = n * (uint32_t)sizeof(K);
    if (((reinterpret_cast<uintptr_t>(src) | reinterpret_cast<uintptr_t>(dst)) & 15u) == 0 &&
        (bytes & 15u) == 0) {
        const uint4 *s4 = reinterpret_cast<const uint4 *>(src);
        uint4 *d4 = reinterpret_cast<uint4 *>(dst);
        for (uint32_t i = threadIdx.x; i < bytes / 16u; i += blockDim.x) d4[i] = __ldcg(s4 + i);
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
    if (start < total) {
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
    if (threadIdx.x == 0) {
        sh.abort = !lock_root(p, sh);
        if (!sh.abort) {
            sh.t_root = gtimer();
            uint4 h = __ldcg(reinterpret_cast<const uint4 *>(&p.hdr->m));
            sh.m = h.x;
            sh.s = h.y;
            sh.seq = (unsigned long long)h.z | ((unsigned long long)h.w << 32);
            if (sh.seq < p.log_cap) {
                gheap_log_entry e;
                e.call_id = p.call_id;
                e.kind_n = (GHEAP_OP_INS << 24) | n;
                e.ref = ref;
                p.log[sh.seq] = e;
            }
        }
    }
    __syncthreads();
    if (sh.abort) return false;
    uint32_t m = sh.m, s = sh.s;
    K *root = p.keys + (size_t)k;

    if (n < k) {
        // partial batch: merge into the partial buffer
        g2s(c, p.buf, s);
        __syncthreads();
        if (n + s < k) {
            merge_split<K, IPT>(a, n, c, s, c, n + s, c);
            if (m >= 1) {
                // Property 3: the root keeps the k smallest of root + buffer
                g2s(b, root, k);
                __syncthreads();
                merge_split<K, IPT>(b, k, c, n + s, b, k, c);
                s2g(root, b, k);
                if (threadIdx.x == 0) {
                    sh.cnt[STAT_LOADS]++;
                    sh.cnt[STAT_STORES]++;
                    sh.cnt[STAT_MERGES]++;
                }
            }
            s2g(p.buf, c, n + s);
            if (threadIdx.x == 0) {
                uint4 h = make_uint4(m, n + s, (uint32_t)(sh.seq + 1), (uint32_t)((sh.seq + 1) >> 32));
                __stcg(reinterpret_cast<uint4 *>(&p.hdr->m), h);
            }
            block_release(&p.hdr->root_lock, 0u);
            return true;
        }
        // the k smallest of batch + buffer go down as a full batch
        merge_split<K, IPT>(a, n, c, s, a, k, c);
        s = n + s - k;
        s2g(p.buf, c, s);
    } else if (m == 0 && s > 0) {
        // the batch becomes the root: keep Property 3 with the buffer
        g2s(c, p.buf, s);
        __syncthreads();
        merge_split<K, IPT>(a, k, c, s, a, k, c);
        s2g(p.buf, c, s);
    }

    if (m == 0) {
        s2g(root, a, k);
        if (threadIdx.x == 0) {
            sh.cnt[STAT_STORES]++;
            uint4 h = make_uint4(1u, s, (uint32_t)(sh.seq + 1), (uint32_t)((sh.seq + 1) >> 32));
            __stcg(reinterpret_cast<uint4 *>(&p.hdr->m), h);
        }
        block_release(&p.hdr->root_lock, 0u);
        return true;
    }

    // full top-down INS to the next target slot
    const uint32_t tslot = m + 1;
    if (tslot > p.max_nodes) {
        if (threadIdx.x == 0) set_err(p, E_FULL);
        return false;
    }
    if (threadIdx.x == 0) {
        st_relaxed(&p.state[tslot], ST_TARGET);
        uint4 h = make_uint4(tslot, s, (uint32_t)(sh.seq + 1), (uint32_t)((sh.seq + 1) >> 32));
        __stcg(reinterpret_cast<uint4 *>(&p.hdr->m), h);
    }
    const uint32_t tnode = slot_node(tslot);
    const uint32_t depth = level_of(tnode);

    uint32_t *cur_w = &p.hdr->root_lock;
    uint32_t cur_free = 0u;
    K *cur_keys = root;
    uint32_t node = 1;
    for (uint32_t lvl = 0;; ++lvl) {
        // MergeAndSort(node, batch): the node keeps the k smallest, the k
        // largest are carried on (Section 3.2.2); disjoint ranges are kept or
        // swapped without merging (Section 4.3).
        g2s(b, cur_keys, k);
        __syncthreads();
        {
            K bmax = b[k - 1], bmin = b[0], amax = a[k - 1], amin = a[0];
            if (bmax <= amin) {
                if (threadIdx.x == 0) sh.cnt[STAT_SKIPS]++;
            } else if (amax <= bmin) {
                s2g(cur_keys, a, k);
                K *t = a; a = b; b = t;
                if (threadIdx.x == 0) { sh.cnt[STAT_SKIPS]++; sh.cnt[STAT_STORES]++; }
            } else {
                merge_split<K, IPT>(b, k, a, k, b, k, a);
                s2g(cur_keys, b, k);
                if (threadIdx.x == 0) { sh.cnt[STAT_MERGES]++; sh.cnt[STAT_STORES]++; }
            }
            if (threadIdx.x == 0) sh.cnt[STAT_LOADS]++;
        }
        // next node on the root-to-target path
        const uint32_t nxt = tnode >> (depth - lvl - 1);
        const uint32_t nslot = slot_node(nxt);
        uint32_t *nw = &p.state[nslot];
        if (nxt == tnode) {
            if (threadIdx.x == 0) {
                uint32_t old = atomicCAS(nw, ST_TARGET, ST_INUSE);
                sh.deliver = (old == ST_MARKED);
                if (old != ST_TARGET && old != ST_MARKED) {
                    set_err(p, E_STATE);
                    sh.abort = 1;
                }
            }
            __syncthreads();
            if (sh.abort) return false;
            if (lvl == 0 && threadIdx.x == 0) {
                sh.cnt[STAT_ROOT_NS] += (gtimer() - sh.t_root);
            }
            block_release(cur_w, cur_free);
            s2g(p.keys + (size_t)nslot * k, a, k);
            if (threadIdx.x == 0) sh.cnt[STAT_STORES]++;
            block_release(nw, sh.deliver ? ST_DELIVERED : ST_AVAIL);
            return true;
        }
        if (threadIdx.x == 0) {
            uint32_t r = lock_node(p, sh, nw);
            if (r != ST_AVAIL) {
                if (r != ~0u) set_err(p, E_STATE);
                sh.abort = 1;
            }
        }
        __syncthreads();
        if (sh.abort) return false;
        if (lvl == 0 && threadIdx.x == 0) {
            sh.cnt[STAT_ROOT_NS] += (gtimer() - sh.t_root);
        }
        block_release(cur_w, cur_free);
        cur_w = nw;
        cur_free = ST_AVAIL;
        cur_keys = p.keys + (size_t)nslot * k;
        node = nxt;
    }
}

// ---------------------------------------------------------------------------
// DEL (Section 3.2.1, partial buffer of Section 3.3.2)
// ---------------------------------------------------------------------------

// Deletes up to `want` keys.  MODE_DELETE takes its output offset and count
// from the launch's running total under the root lock; MODE_OPS writes to
// `out_off`.  Returns false when the block must stop.
template <typename K, int IPT>
__device__ bool del_op(const Params<K> &p, Shared &sh, K *A, K *B, K *C, K *D,
                       uint32_t want, unsigned long long out_off, unsigned long long ref,
                       uint32_t *count_out)
{
    const uint32_t k = p.k;
    if (threadIdx.x == 0) {
        sh.abort = !lock_root(p, sh);
        if (!sh.abort) {
            sh.t_root = gtimer();
            uint4 h = __ldcg(reinterpret_cast<const uint4 *>(&p.hdr->m));
            sh.m = h.x;
            sh.s = h.y;
            sh.seq = (unsigned long long)h.z | ((unsigned long long)h.w << 32);
            if (p.mode == MODE_DELETE) {
                unsigned long long done = p.ctl->delivered;
                unsigned long long rem = p.n > done ? p.n - done : 0ull;
                want = rem < want ? (uint32_t)rem : want;
                out_off = done;
            }
            uint32_t avail = sh.m >= 1 ? k : sh.s;
            uint32_t take = want < avail ? want : avail;
            sh.take = take;
            sh.out_off = out_off;
            if (p.mode == MODE_DELETE) {
                p.ctl->delivered = out_off + take;
                if (p.out_total) *p.out_total = out_off + take;
                if (take == 0 || out_off + take >= p.n) p.ctl->drained = 1u;
            }
            if (count_out) *count_out = take;
            if (sh.seq < p.log_cap) {
                gheap_log_entry e;
                e.call_id = p.call_id;
                e.kind_n = (GHEAP_OP_DEL << 24) | take;
                e.ref = p.mode == MODE_DELETE ? out_off : ref;
                p.log[sh.seq] = e;
            }
        }
    }
    __syncthreads();
    if (sh.abort) return false;
    uint32_t m = sh.m, s = sh.s;
    const uint32_t take = sh.take;
    out_off = sh.out_off;
    K *root = p.keys + (size_t)k;
    const unsigned long long nseq = sh.seq + 1;

    if (m == 0) {
        // no full node: serve from the partial buffer (Section 3.3.2)
        g2s(C, p.buf, s);
        __syncthreads();
        s2g(p.out + out_off, C, take);
        s2g(p.buf, C + take, s - take);
        if (threadIdx.x == 0) {
            uint4 h = make_uint4(0u, s - take, (uint32_t)nseq, (uint32_t)(nseq >> 32));
            __stcg(reinterpret_cast<uint4 *>(&p.hdr->m), h);
        }
        block_release(&p.hdr->root_lock, 0u);
        return true;
    }

    g2s(B, root, k);
    g2s(C, p.buf, s);
    __syncthreads();
    s2g(p.out + out_off, B, take);
    if (threadIdx.x == 0) sh.cnt[STAT_LOADS]++;
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
            if (threadIdx.x == 0) {
                uint4 h = make_uint4(0u, tn, (uint32_t)nseq, (uint32_t)(nseq >> 32));
                __stcg(reinterpret_cast<uint4 *>(&p.hdr->m), h);
            }
            block_release(&p.hdr->root_lock, 0u);
            return true;
        }
        // refill the root from the last node (slot m)
        uint32_t *lw = &p.state[m];
        if (threadIdx.x == 0) sh.abort = !take_last(p, sh, lw);
        __syncthreads();
        if (sh.abort) return false;
        g2s(D, p.keys + (size_t)m * k, k);
        __syncthreads();
        if (threadIdx.x == 0) {
            st_relaxed(lw, ST_EMPTY);
            sh.cnt[STAT_LOADS]++;
        }
        merge_split<K, IPT>(C, tn, D, k, B, k, C);
        ns = tn;
        nm = m - 1;
        s2g(p.buf, C, ns);
    }
    if (threadIdx.x == 0) {
        uint4 h = make_uint4(nm, ns, (uint32_t)nseq, (uint32_t)(nseq >> 32));
        __stcg(reinterpret_cast<uint4 *>(&p.hdr->m), h);
    }

    // sift down from the root; B holds the current node's keys
    uint32_t node = 1;
    K *cur_keys = root;
    uint32_t *cur_w = &p.hdr->root_lock;
    uint32_t cur_free = 0u;
    const uint32_t top_level = level_of(p.max_nodes);
    for (;;) {
        const uint32_t l = 2 * node, r = l + 1;
        const bool in_range = level_of(l) <= top_level;
        const uint32_t sl = in_range ? slot_node(l) : 0u;
        const uint32_t sr = in_range ? slot_node(r) : 0u;
        if (threadIdx.x == 0) {
            uint32_t rl = ST_EMPTY, rr = ST_EMPTY;
            if (in_range && sl <= p.max_nodes) rl = lock_node(p, sh, &p.state[sl]);
            if (rl != ~0u && in_range && sr <= p.max_nodes) rr = lock_node(p, sh, &p.state[sr]);
            sh.abort = (rl == ~0u || rr == ~0u);
            sh.pl = (rl == ST_AVAIL);
            sh.pr = (rr == ST_AVAIL);
        }
        __syncthreads();
        if (sh.abort) return false;
        const int pl = sh.pl, pr = sh.pr;
        if (!pl && !pr) break;
        K *lk = p.keys + (size_t)sl * k;
        K *rk = p.keys + (size_t)sr * k;
        if (pl) g2s(C, lk, k);
        if (pr) g2s(D, rk, k);
        __syncthreads();
        if (threadIdx.x == 0) sh.cnt[STAT_LOADS] += pl + pr;
        const K cmax = B[k - 1];
        if (pl != pr) {
            // one child present (the other is absent or an INS target)
            K *X = pl ? C : D;
            K *xk = pl ? lk : rk;
            uint32_t *xw = &p.state[pl ? sl : sr];
            if (cmax <= X[0]) {
                block_release(xw, ST_AVAIL);
                break;
            }
            merge_split<K, IPT>(B, k, X, k, B, k, X);
            s2g(cur_keys, B, k);
            if (threadIdx.x == 0) {
                sh.cnt[STAT_MERGES]++;
                sh.cnt[STAT_STORES]++;
                if (node == 1) sh.cnt[STAT_ROOT_NS] += (gtimer() - sh.t_root);
            }
            block_release(cur_w, cur_free);
            node = pl ? l : r;
            cur_keys = xk;
            cur_w = xw;
            cur_free = ST_AVAIL;
            K *t = B; B = X; X = t;
            if (pl) C = t; else D = t;
            continue;
        }
        // both children present
        if (cmax <= C[0] && cmax <= D[0]) {
            // early stop (Section 4.3)
            if (threadIdx.x == 0) st_release(&p.state[sl], ST_AVAIL);
            if (threadIdx.x == 0) st_release(&p.state[sr], ST_AVAIL);
            break;
        }
        // MergeAndSort(l, r): the k largest go to the child whose maximum
        // was larger (the right child on a tie), the k smallest to the other
        const bool big_l = C[k - 1] > D[k - 1];
        K *S, *L;               // smem of the small and large halves
        bool l_changed, r_changed;
        if (C[k - 1] <= D[0]) {
            S = C; L = D;
            l_changed = big_l;        // big_l is false here: no change
            r_changed = big_l;
        } else if (D[k - 1] <= C[0]) {
            S = D; L = C;
            l_changed = !big_l;
            r_changed = !big_l;
        } else {
            merge_split<K, IPT>(C, k, D, k, C, k, D);
            S = C; L = D;
            l_changed = true;
            r_changed = true;
            if (threadIdx.x == 0) sh.cnt[STAT_MERGES]++;
        }
        if (!l_changed && threadIdx.x == 0) sh.cnt[STAT_SKIPS]++;
        K *big_keys = big_l ? lk : rk;
        uint32_t *big_w = &p.state[big_l ? sl : sr];
        K *sm_keys = big_l ? rk : lk;
        uint32_t *sm_w = &p.state[big_l ? sr : sl];
        const bool big_changed = big_l ? l_changed : r_changed;
        const bool sm_changed = big_l ? r_changed : l_changed;
        if (big_changed) {
            s2g(big_keys, L, k);
            if (threadIdx.x == 0) sh.cnt[STAT_STORES]++;
        }
        block_release(big_w, ST_AVAIL);
        if (cmax <= S[0]) {
            if (sm_changed) {
                s2g(sm_keys, S, k);
                if (threadIdx.x == 0) sh.cnt[STAT_STORES]++;
            }
            block_release(sm_w, ST_AVAIL);
            break;
        }
        // MergeAndSort(cur, small child): cur keeps the k smallest
        merge_split<K, IPT>(B, k, S, k, B, k, S);
        s2g(cur_keys, B, k);
        if (threadIdx.x == 0) {
            sh.cnt[STAT_MERGES]++;
            sh.cnt[STAT_STORES]++;
            if (node == 1) sh.cnt[STAT_ROOT_NS] += (gtimer() - sh.t_root);
        }
        block_release(cur_w, cur_free);
        node = big_l ? r : l;
        cur_keys = sm_keys;
        cur_w = sm_w;
        cur_free = ST_AVAIL;
        // rotate buffers: S becomes the current node
        K *oldB = B;
        B = S;
        if (S == C) { C = oldB; } else { D = oldB; }
        (void)A;
    }
    // final node of the walk: write it and release it
    s2g(cur_keys, B, k);
    if (threadIdx.x == 0) {
        sh.cnt[STAT_STORES]++;
        if (node == 1) sh.cnt[STAT_ROOT_NS] += (gtimer() - sh.t_root);
    }
    block_release(cur_w, cur_free);
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
            const K *src = p.in + off;
            if (n < k) {
                for (uint32_t i = threadIdx.x; i < k; i += blockDim.x)
                    A[i] = i < n ? __ldcg(src + i) : kmax<K>();
            } else {
                g2s(A, src, k);
            }
            __syncthreads();
            block_sort(A, k);
            ok = ins_op<K, IPT>(p, sh, A, B, C, n, p.mode == MODE_OPS ? op : off);
            if (threadIdx.x == 0) {
                sh.cnt[STAT_INS]++;
                if (p.mode == MODE_OPS && p.out_counts) p.out_counts[op] = n;
            }
        } else {
            ok = del_op<K, IPT>(p, sh, A, B, C, D, n, off, op,
                                p.mode == MODE_OPS && p.out_counts ? p.out_counts + op : nullptr);
            if (threadIdx.x == 0) sh.cnt[STAT_DEL]++;
        }
        if (!ok) break;
        __syncthreads();
    }
    __syncthreads();
    if (p.stats && threadIdx.x < N_STATS && sh.cnt[threadIdx.x])
        atomicAdd(p.stats + threadIdx.x, sh.cnt[threadIdx.x]);
}

}  // namespace gh

// gheap_kernel.cuh -- device side of the GB300 generalized concurrent heap.
//
// The TD-INS/TD-DEL and BU-INS/TD-DEL heaps of arXiv 1906.06504 (Chen et al.):
//   * a heap of nodes that each hold k ascending keys (Section 3.1,
//     Properties 1-3), stored as one flat array, plus a partial buffer of at
//     most k-1 keys guarded by the root lock (Section 3.3.2);
//   * top-down INS walks from the root to a target node, doing a
//     MergeAndSort with every node on the path and carrying the k largest
//     keys down (Section 3.2.2); bottom-up INS stores its batch at the target
//     and rises, merging with each parent until the parent is no larger
//     (Sections 3.2.2, 3.3.4; insert-only launches);
//   * DEL returns the root batch, refills the root from the last node and
//     sifts down with two MergeAndSorts per level (Section 3.2.1);
//   * every node has a multi-state lock word (AVAIL / INUSE / TARGET /
//     MARKED / DELIVERED, and INSHOLD for a rising batch; Sections 3.3.2,
//     3.3.4) taken with atomicCAS in parent-before-child order (Section
//     3.3.1), and a DEL whose last node is an in-flight INS target marks it
//     and receives that INS's keys (Section 3.3.2);
//   * one thread block runs one operation (Section 4); merges are block-wide
//     (Section 4.2), batch sorting is a block bitonic sort (Section 4.1), and
//     node pairs whose key ranges do not overlap are kept or swapped without
//     merging (Section 4.3).
//
// GB300 organisation.  The root lock is the serial point of every operation
// (Section 3.3.3) and each level of a walk waits on its predecessor's
// release, so the kernel is built to shorten lock holds:
//   * a block is nmt() "merge threads" plus a control warp and a release
//     warp.  The control warp takes every lock (an acquire stalls only that
//     warp; it polls as one converged warp) and issues the cp.async copies of
//     the nodes it has locked -- for the next level while the merge threads
//     still work on this one.  Merge threads synchronise among themselves on
//     named barrier 1; merge threads and control warp meet on barrier 0 only
//     where data or lock results change hands.  A DEL's node is released as
//     soon as its keys are stored: the release warp takes the fence and the
//     lock-word stores off the merge threads' path;
//   * the root lock is a FIFO ticket lock whose turn shares one 64-bit word
//     with the node count m and the buffer size s: the block whose ticket
//     comes up reads (m, s) with the same acquire-load, and one store
//     releases; full bottom-up batches reserve their target with an atomic
//     add on m, without the lock;
//   * MergeAndSort of two full nodes is a bitonic merge (shared-memory stages
//     for wide strides, warp shuffles and registers for the rest), or a
//     bitonic split and a sort of only the half that must be stored first;
//   * delete-only launches run a kernel specialisation without the insert,
//     list and heap-set paths;
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
    ST_DELIVERED = 5, ST_INSHOLD = 6
};
// INSHOLD (bottom-up insert, Section 3.3.4): the node holds the keys of an
// insert still on its way up, released while that insert waits for the
// parent.  The word is ST_INSHOLD | owner << 8, owner naming the insert.
__host__ __device__ __forceinline__ uint32_t inshold(uint32_t owner)
{
    return ST_INSHOLD | (owner << 8);
}
constexpr uint32_t ST_GAVE_UP = ~0u;
// How often a DEL hands the root back rather than wait, holding it, for an
// INS still on its way to the last node (the default of Params::del_yields).
// 0, the paper's protocol -- mark the target at once and wait for delivery --
// is the default: the marked INS delivers at the level it is on (ins_op), so
// the wait is one level step, and queueing again cost more (config-2 mixed
// run 1.32 s with 64 hand-backs against 0.91 s).
constexpr uint32_t DEL_YIELDS = 0;
constexpr uint32_t NO_TRY = ~1u;     // "no earlier lock attempt"

enum : uint32_t { MODE_INSERT = 0, MODE_DELETE = 1, MODE_OPS = 2, MODE_SET = 3, MODE_RING = 4 };

// MODE_RING: the serving form.  One persistent launch takes its operations
// from a ring that the host appends to while the launch runs; the ring, the
// request tables, the input keys and the output keys live in pinned host
// memory, which the GPU reads and writes directly (NVLink-C2C on a Grace
// host).  An operation names its heap, its request slot and its root ticket:
// the host numbers each heap's operations in ring order, so every heap takes
// its requests in arrival order however the blocks pick them up.
struct __align__(16) RingOp {
    uint32_t heap;
    uint32_t kind_n;              // as gheapset_op (DELs use the request cursor)
    unsigned long long offset;    // INS: key position in the input arena; DEL: request slot
    unsigned long long ticket;    // this heap's root ticket for the operation
    uint32_t req;                 // request slot
    uint32_t _pad;
};
// Completion record of a request slot, written by the block that finishes the
// request's last operation: count and status first, then seq (release).
struct __align__(16) RingDone {
    unsigned long long seq;       // request sequence number + 1 once complete
    unsigned long long count;     // DEL: keys written; INS: 0
    uint32_t status;              // 0, or the device error that hit an operation
    uint32_t _pad[3];
};

enum : uint32_t { E_NONE = 0, E_TIMEOUT = 1, E_FULL = 2, E_STATE = 3 };

// Counters kept when the heap is created with GHEAP_FLAG_STATS.  The *_CYC
// entries are SM cycles of one observer thread per phase.
enum : uint32_t {
    STAT_LOADS = 0, STAT_STORES = 1, STAT_MERGES = 2, STAT_SKIPS = 3,
    STAT_INS = 4, STAT_DEL = 5, STAT_WAITS = 6, STAT_ROOT_NS = 7,
    STAT_DEL_ACQ_CYC = 8,       // waiting for the root lock
    STAT_DEL_ROOT_CYC = 9,      // root step: loads, last node, children, refill
    STAT_DEL_WAIT_CYC = 10,     // control warp: child locks and copies
    STAT_DEL_LOAD_CYC = 11,     // (unused)
    STAT_DEL_MERGE_CYC = 12,    // merge threads: MergeAndSorts and stores
    STAT_DEL_REL_CYC = 13,      // control warp: lock releases
    STAT_DEL_LEVELS = 14,       // sift levels visited
    STAT_INS_ACQ_CYC = 15,      // waiting for the root lock
    STAT_INS_SORT_CYC = 16,     // staging and sorting the batch
    STAT_INS_WAIT_CYC = 17,     // control warp: node locks and copies
    STAT_INS_STEP_CYC = 18,     // merge threads: level steps
    STAT_INS_LEVELS = 19,       // levels visited
    STAT_DELIVERIES = 20,       // DELs that received a marked target's keys (Section 3.3.2)
    STAT_DEL_YIELDS = 21,       // DELs that handed the root back to let an INS land first
    STAT_TARGET_CHILDREN = 22,  // children a DEL found reserved by an INS in flight (absent)
    STAT_INTERCEPTS = 23,       // INSs that delivered to a marked target before reaching it
    N_STATS = 24
};

// Root word: bits 0-29 m (full nodes), bits 30-41 s (partial-buffer keys),
// bits 42-63 the turn of the root's ticket lock.  The lock holder stores
// (m, s, turn + 1) in one release, so the next ticket learns that it holds
// the root and reads (m, s) with the same load.
constexpr uint32_t RW_TURN_BITS = 22;
constexpr unsigned long long RW_TURN_MASK = (1ull << RW_TURN_BITS) - 1;
__host__ __device__ __forceinline__ uint32_t rw_m(unsigned long long v)
{
    return (uint32_t)v & ((1u << 30) - 1u);
}
__host__ __device__ __forceinline__ uint32_t rw_s(unsigned long long v)
{
    return (uint32_t)(v >> 30) & 0xFFFu;
}
__host__ __device__ __forceinline__ uint32_t rw_turn(unsigned long long v)
{
    return (uint32_t)(v >> 42);
}
__host__ __device__ __forceinline__ unsigned long long rw_make(uint32_t m, uint32_t s, uint32_t turn)
{
    return (unsigned long long)m | ((unsigned long long)s << 30) |
           ((unsigned long long)(turn & RW_TURN_MASK) << 42);
}

// Heap header.  The root lock is a ticket lock: an operation draws a ticket
// from `next` and waits until the root word's turn equals it (modulo 2^22,
// far more than the blocks that can wait at once); waiters poll the root
// word only, so a release wakes exactly one of them, in arrival order.  The
// ticket dispenser, the linearization counter (touched only by the root
// holder) and the sticky error each have a 128-byte line.
struct __align__(128) Hdr {
    unsigned long long root;
    uint32_t _p0[30];
    unsigned long long seq;
    uint32_t _p1[30];
    uint32_t err;
    uint32_t _p2[31];
    unsigned long long next;
    uint32_t _p3[30];
};

// Per-launch work distribution.  Zero when a launch starts: zeroed when the
// heap is created or reset, and put back to zero by the last block to leave
// each launch (so no memset precedes a launch).
struct __align__(16) Ctl {
    unsigned long long next_op;
    unsigned long long delivered;   // MODE_DELETE: keys handed out (root-guarded)
    uint32_t drained;               // MODE_DELETE: heap ran empty
    uint32_t exited;                // blocks of this launch that have finished
};

// The device arrays of one heap.
template <typename K>
struct HeapView {
    K *keys;                  // (max_nodes + 1) * k keys, slot j at j*k
    uint32_t *state;          // max_nodes + 1 lock words, by slot
    K *buf;                   // partial buffer, k keys
    Hdr *hdr;
    gheap_log_entry *log;
    unsigned long long log_cap;
    uint32_t max_nodes;
    uint32_t _pad;
};

// Node keys and lock word of storage slot s.
template <typename K>
__device__ __forceinline__ K *node_keys(const HeapView<K> &H, uint32_t s, uint32_t k)
{
    return H.keys + (size_t)s * k;
}

template <typename K>
__device__ __forceinline__ uint32_t *node_state(const HeapView<K> &H, uint32_t s)
{
    return H.state + s;
}

template <typename K>
struct Params {
    HeapView<K> h;
    Ctl *ctl;
    unsigned long long *stats;   // N_STATS counters or nullptr
    uint32_t k;
    uint32_t mode;
    uint32_t call_id;
    uint32_t bu;                 // MODE_INSERT: bottom-up inserts (Section 3.3.4)
    unsigned long long timeout_ns;
    uint32_t del_yields;         // hand-backs allowed before a DEL marks an in-flight target
    uint32_t _pad0;
    const K *in;                 // MODE_INSERT / MODE_OPS input keys
    K *out;                      // MODE_DELETE / MODE_OPS output keys
    unsigned long long n;        // MODE_INSERT: keys; MODE_DELETE: keys wanted
    const gheap_op *ops;         // MODE_OPS
    unsigned long long n_ops;
    uint32_t *out_counts;        // MODE_OPS / MODE_SET, may be nullptr
    unsigned long long *out_total;  // MODE_DELETE, may be nullptr
    const HeapView<K> *table;    // MODE_SET: one view per heap
    const gheapset_op *sops;     // MODE_SET operations
    uint32_t n_heaps;            // MODE_SET
    const unsigned long long *req_base;   // MODE_SET cursor DELs: output base
    unsigned long long *req_cursor;       //   and running count, per request
    const unsigned long long *n_dev;      // MODE_INSERT: key count in device memory
    const uint32_t *set_bu;      // MODE_SET: nonzero = the list has no DEL, insert bottom-up
    // MODE_RING (host memory unless marked device)
    const RingOp *ring_ops;      // the op ring, ring_cap entries (a power of two)
    unsigned long long ring_cap;
    unsigned long long ring_base; // ring position of this launch's first operation
    const unsigned long long *ring_tail;   // positions published by the host
    const uint32_t *ring_stop;   // nonzero: leave once every published op is taken
    const uint32_t *ring_req_ops;          // operations per request slot
    const unsigned long long *ring_req_seq; // request sequence number per slot
    RingDone *ring_done;         // completion records per slot
    uint32_t *ring_ops_done;     // device: operations finished per slot
    uint32_t *ring_status;       // device: error bits per slot
    uint32_t *ring_err;          // device: the ring's own error (a wait gave up)
    unsigned long long ring_idle_ns;       // bound on a wait for new operations
};

// A hand-off to the release warp: behind one fence, up to two lock words set
// to AVAIL and the root word set to `root_v`.  `stop` ends the release warp.
struct RelReq {
    uint32_t *w0;
    uint32_t *w1;
    unsigned long long *root_w;
    unsigned long long root_v;
    unsigned long long t_root;    // root acquisition time (root hold statistic)
    uint32_t stop;
};
constexpr uint32_t N_REQ = 4;     // request ring

// Block-shared scalars that carry decisions between the control warp and the
// merge threads (always across a block barrier).
struct Shared {
    unsigned long long op;
    unsigned long long seq;
    unsigned long long out_off;
    unsigned long long t_root;
    uint32_t m, s, take, tslot;
    uint32_t turn;            // root ticket held by this block
    uint32_t use_fixed;       // MODE_RING: the root ticket is fixed_ticket
    unsigned long long fixed_ticket;
    int lockfree;             // bottom-up INS: target reserved without the root lock
    int stop;
    int abort;
    int deliver;
    int halt;                 // DEL: the sift ends after MergeAndSort(l, r)
    int swap;                 // DEL: MergeAndSort(cur, small child) is a swap
    uint32_t lk[2][2];        // lock results, double-buffered by level
    // delete-only launches: the mbarriers of the root step's TMA fetches
    // (level 1, the last node), the fetches issued on each and seen landed
    unsigned long long l1_mbar, last_mbar;
    uint32_t l1_arms, l1_seen, last_arms, last_seen;
    // release ring: posted by merge thread 0, taken in order by the release
    // warp (`rq_read`: requests taken, their slots free again)
    RelReq rq[N_REQ];
    uint32_t rq_posted, rq_read;
    uint32_t stats_on;        // the launch counts statistics
    unsigned long long cnt[N_STATS];
    // launches other than delete-only: the mbarrier of the TMA fetches of
    // the nodes below the root step, fetches issued on it and seen landed
    unsigned long long kid_mbar;
    uint32_t kid_arms, kid_seen;
    // top-down INS, the control warp's decision for a level (0 go on, 1 hand
    // the keys over to the target a DEL marked, 2 give up), by level parity:
    // the merge threads read a level's word after its barrier, and the next
    // word the control warp writes (at the top of the next level, before
    // any barrier) is the other one
    int ilvl[2];
};

// ---------------------------------------------------------------------------
// block roles and barriers
// ---------------------------------------------------------------------------

// Merge threads are threadIdx.x < nmt(); then the control warp (locks and
// loads); the last warp is the release warp (the fences and lock releases
// handed over by the merge threads, one lane).  The release warp takes part
// in no barrier but the one at kernel start.
__device__ __forceinline__ uint32_t nmt() { return blockDim.x - 64u; }
__device__ __forceinline__ bool is_rel() { return threadIdx.x >= blockDim.x - 32u; }
__device__ __forceinline__ bool is_ctrl() { return threadIdx.x >= blockDim.x - 64u; }
__device__ __forceinline__ uint32_t clane() { return threadIdx.x - (blockDim.x - 64u); }

// Merge threads and control warp (named barrier 0).
__device__ __forceinline__ void bar_all()
{
    asm volatile("bar.sync 0, %0;" :: "r"(blockDim.x - 32u) : "memory");
}

// Merge threads only (named barrier 1).
__device__ __forceinline__ void bar_mg()
{
    asm volatile("bar.sync 1, %0;" :: "r"(blockDim.x - 64u) : "memory");
}

// Merge threads only, with an OR of `v` over them (named barrier 1): the
// same result in every merge thread.
__device__ __forceinline__ bool bar_mg_or(bool v)
{
    uint32_t r;
    asm volatile("{\n\t.reg .pred p, q;\n\t"
                 "setp.ne.u32 p, %1, 0;\n\t"
                 "bar.red.or.pred q, 1, %2, p;\n\t"
                 "selp.u32 %0, 1, 0, q;\n\t}"
                 : "=r"(r) : "r"((uint32_t)v), "r"(blockDim.x - 64u) : "memory");
    return r != 0;
}

// Every thread of the block, release warp included (named barrier 2).
__device__ __forceinline__ void bar_block()
{
    asm volatile("bar.sync 2, %0;" :: "r"(blockDim.x) : "memory");
}

__device__ __forceinline__ uint32_t ld_acquire_cta(const uint32_t *p)
{
    uint32_t v;
    asm volatile("ld.acquire.cta.shared.u32 %0, [%1];"
                 : "=r"(v) : "r"((unsigned)__cvta_generic_to_shared(p)) : "memory");
    return v;
}

__device__ __forceinline__ void st_release_cta(uint32_t *p, uint32_t v)
{
    asm volatile("st.release.cta.shared.u32 [%0], %1;"
                 :: "r"((unsigned)__cvta_generic_to_shared(p)), "r"(v) : "memory");
}

// ---------------------------------------------------------------------------
// memory-model helpers
// ---------------------------------------------------------------------------

// mbarrier and TMA bulk copies (global -> shared, completion counted in
// bytes on the mbarrier).  Addresses 16-byte aligned, sizes multiples of 16.
__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(unsigned long long *b, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(smem_u32(b)), "r"(count)
                 : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(unsigned long long *b, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;"
                 :: "r"(smem_u32(b)), "r"(bytes) : "memory");
}

// One test (suspending for at most a hardware-bounded time) that the phase
// of parity `par` has completed.
__device__ __forceinline__ bool mbar_try_wait(unsigned long long *b, uint32_t par)
{
    uint32_t ok;
    asm volatile("{\n\t.reg .pred q;\n\t"
                 "mbarrier.try_wait.parity.shared::cta.b64 q, [%1], %2;\n\t"
                 "selp.u32 %0, 1, 0, q;\n\t}"
                 : "=r"(ok) : "r"(smem_u32(b)), "r"(par) : "memory");
    return ok != 0;
}

__device__ __forceinline__ void tma_load_1d(void *dst, const void *src, uint32_t bytes,
                                            unsigned long long *b)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes "
                 "[%0], [%1], %2, [%3];"
                 :: "r"(smem_u32(dst)), "l"(src), "r"(bytes), "r"(smem_u32(b)) : "memory");
}

// Orders this thread's generic-proxy accesses of global memory (the lock
// acquisitions, and what they made visible) with its later async-proxy ones
// (the TMA reads of the nodes).  The shared buffers need none: their last
// readers finished before a barrier that precedes the copy.
__device__ __forceinline__ void fence_proxy_async_global()
{
    asm volatile("fence.proxy.async.global;" ::: "memory");
}


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

__device__ __forceinline__ unsigned long long ld_acquire64(const unsigned long long *p)
{
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
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

__device__ __forceinline__ void st_release64(unsigned long long *p, unsigned long long v)
{
    asm volatile("st.release.gpu.global.u64 [%0], %1;" :: "l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ void st_relaxed(uint32_t *p, uint32_t v)
{
    asm volatile("st.relaxed.gpu.global.u32 [%0], %1;" :: "l"(p), "r"(v) : "memory");
}


// Releases (a st.release.gpu, or a fence.acq_rel.gpu and relaxed stores) are
// issued by one thread after a block barrier that follows the merge threads'
// stores -- control lane 0 or merge thread 0, or in deleteMin the release
// warp after a shared-memory release / acquire hand-over from merge thread 0:
// the barrier orders those stores before the release, and a release is
// cumulative over the writes its thread has observed, so a block that
// acquires the word sees all of them (the barrier + single release-store
// hand-off used between thread blocks by split-K GEMM epilogues).
// Release for launches in which full bottom-up batches reserve their target
// slots without the lock (an atomic add on m): the holder adds its own
// changes of m and s and the turn increment in one atomic, so that the
// concurrent reservations are kept.  Fields cannot carry into each other:
// m < 2^30 and 0 <= s + ds < 2^12 throughout.
template <typename K>
__device__ __forceinline__ void release_root_delta(const HeapView<K> &H, int dm, int ds)
{
    const unsigned long long d = (unsigned long long)(long long)dm +
                                 (unsigned long long)(long long)ds * (1ull << 30) +
                                 (1ull << 42);
    asm volatile("red.release.gpu.global.add.u64 [%0], %1;" :: "l"(&H.hdr->root), "l"(d)
                 : "memory");
}

template <typename K>
__device__ __forceinline__ void release_root_word(const HeapView<K> &H, const Shared &sh,
                                                  uint32_t m, uint32_t s)
{
    // the release orders every write the block made before its barrier ahead
    // of the hand-over to the next ticket
    st_release64(&H.hdr->root, rw_make(m, s, sh.turn + 1));
}
__device__ __forceinline__ void fence_acq_rel()
{
    asm volatile("fence.acq_rel.gpu;" ::: "memory");
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

// Children of tree node `node` that exist in storage: slot numbers, or 0.
__device__ __forceinline__ void child_slots(uint32_t node, uint32_t max_nodes, uint32_t &sl,
                                            uint32_t &sr)
{
    const uint32_t l = 2 * node;
    sl = sr = 0;
    if (level_of(l) <= level_of(max_nodes)) {
        const uint32_t a = slot_node(l), b = slot_node(l + 1);
        sl = a <= max_nodes ? a : 0;
        sr = b <= max_nodes ? b : 0;
    }
}

// Statistics are counted only when the launch asks for them (the shared
// 64-bit atomics cost a few hundred cycles on the paths they sit on).
__device__ __forceinline__ void stat_add(Shared &sh, uint32_t i, unsigned long long v)
{
    if (sh.stats_on) atomicAdd(&sh.cnt[i], v);
}

// Phase timer of one observer thread: adds the cycles since `t`, restarts.
__device__ __forceinline__ void lap(Shared &sh, uint32_t i, long long &t)
{
    if (!sh.stats_on) return;
    const long long now = clock64();
    atomicAdd(&sh.cnt[i], (unsigned long long)(now - t));
    t = now;
}

// Root hold statistic: time since the root was taken (sh.t_root).
__device__ __forceinline__ void stat_root(Shared &sh)
{
    if (sh.stats_on) atomicAdd(&sh.cnt[STAT_ROOT_NS], gtimer() - sh.t_root);
}

// DEL: hands back the current node (the root word at the root) and `pend`, a
// child kept locked since the level above, after a barrier that follows the
// block's stores to both.  Two words behind one fence (fence + strong
// stores is a release pattern for each).
template <typename K>
__device__ __forceinline__ void release_step(const HeapView<K> &H, Shared &sh, uint32_t *cur_w,
                                             uint32_t *pend, uint32_t m, uint32_t s)
{
    if (cur_w == nullptr) {
        stat_root(sh);
        release_root_word(H, sh, m, s);
        if (pend) st_release(pend, ST_AVAIL);
    } else if (pend) {
        fence_acq_rel();
        st_relaxed(cur_w, ST_AVAIL);
        st_relaxed(pend, ST_AVAIL);
    } else {
        st_release(cur_w, ST_AVAIL);
    }
}

__device__ __forceinline__ void st_relaxed64(unsigned long long *p, unsigned long long v)
{
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" :: "l"(p), "l"(v) : "memory");
}

// Spins until the shared counter *w reaches v (modulo 2^32), at most
// `timeout_ns`, with short sleeps between the polls (the release warp's first
// request after a long idle time is a root release: a longer sleep there
// measured 3% slower on a deleteMin-all).  False: gave up.
__device__ __forceinline__ bool spin_until(const uint32_t *w, uint32_t v,
                                           unsigned long long timeout_ns)
{
    unsigned long long t0 = 0;
    for (uint32_t it = 1; (int)(ld_acquire_cta(w) - v) < 0; ++it) {
        if ((it & 63u) == 0) {
            const unsigned long long now = gtimer();
            if (t0 == 0) t0 = now;
            else if (now - t0 > timeout_ns) return false;
        }
        __nanosleep(32);
    }
    return true;
}

// The release warp (its lane 0; the other lanes leave).  Takes the requests
// in order and, behind one fence per request, sets the named lock words to
// AVAIL and the root word to its new value.  The keys those releases publish
// were stored by the merge threads before the barrier that preceded the
// post; the post and the take are a release / acquire pair in shared
// memory, so the fence is cumulative over those stores.  Returns at a stop
// request, or after a long idle time (a safety bound, at least 20 s: the other
// warps' waits are all bounded and their last request is a stop), setting
// rel_exited.
template <typename K>
__device__ void release_loop(const Params<K> &p, Shared &sh, uint32_t *rel_exited)
{
    if ((threadIdx.x & 31u) != 0) return;
    unsigned long long idle_max =
        8ull * p.timeout_ns > 20000000000ull ? 8ull * p.timeout_ns : 20000000000ull;
    // a serving launch may wait that long for its next operation
    if (p.mode == MODE_RING && idle_max < p.ring_idle_ns + 10000000000ull)
        idle_max = p.ring_idle_ns + 10000000000ull;
    for (uint32_t next = 0;; ++next) {
        if (!spin_until(&sh.rq_posted, next + 1, idle_max)) break;
        const RelReq r = sh.rq[next % N_REQ];
        st_release_cta(&sh.rq_read, next + 1);
        if (r.stop) break;
        long long tr = clock64();
        fence_acq_rel();
        if (r.root_w) st_relaxed64(r.root_w, r.root_v);
        if (r.w0) st_relaxed(r.w0, ST_AVAIL);
        if (r.w1) st_relaxed(r.w1, ST_AVAIL);
        lap(sh, STAT_DEL_REL_CYC, tr);
        if (r.root_w && sh.stats_on) atomicAdd(&sh.cnt[STAT_ROOT_NS], gtimer() - r.t_root);
    }
    st_release_cta(rel_exited, 1u);
}

// ---------------------------------------------------------------------------
// bounded waits (single control lane)
// ---------------------------------------------------------------------------

// Counts one more poll of a wait; every 8th checks the sticky error and the
// time bound.  False: give up.
template <typename K>
__device__ __forceinline__ bool wait_ok(const Params<K> &p, const HeapView<K> &H,
                                        unsigned long long &t0, uint32_t &it)
{
    ++it;
    if ((it & 7u) == 0) {
        if (ld_relaxed(&H.hdr->err) != E_NONE) return false;
        unsigned long long now = gtimer();
        if (t0 == 0) {
            t0 = now;
        } else if (now - t0 > p.timeout_ns) {
            atomicCAS(&H.hdr->err, E_NONE, E_TIMEOUT);
            return false;
        }
    }
    return true;
}

template <typename K>
__device__ __forceinline__ bool keep_waiting(const Params<K> &p, const HeapView<K> &H,
                                             unsigned long long &t0, uint32_t &it)
{
    ++it;
    if ((it & 7u) == 0) {
        if (ld_relaxed(&H.hdr->err) != E_NONE) return false;
        unsigned long long now = gtimer();
        if (t0 == 0) {
            t0 = now;
        } else if (now - t0 > p.timeout_ns) {
            atomicCAS(&H.hdr->err, E_NONE, E_TIMEOUT);
            return false;
        }
    }
    if (it > 2) __nanosleep(it < 256 ? 32 : 128);
    return true;
}

template <typename K>
__device__ __forceinline__ void set_err(const HeapView<K> &H, uint32_t e)
{
    atomicCAS(&H.hdr->err, E_NONE, e);
}

// A TMA fetch of n held nodes (slots s0, s1) into a, b, completing on the
// mbarrier `mb` (arms: fetches issued on it).  One thread, after the locks.
template <typename K>
__device__ __forceinline__ void tma_fetch(const HeapView<K> &H, uint32_t k, uint32_t n,
                                          uint32_t s0, K *a, uint32_t s1, K *b,
                                          unsigned long long *mb, uint32_t &arms)
{
    const uint32_t bytes = k * (uint32_t)sizeof(K);
    fence_proxy_async_global();
    mbar_arrive_expect_tx(mb, n * bytes);
    tma_load_1d(a, node_keys(H, s0, k), bytes, mb);
    if (n > 1) tma_load_1d(b, node_keys(H, s1, k), bytes, mb);
    ++arms;
}

// Waits (bounded by the heap's timeout) until the last fetch issued on `mb`
// has landed.  False: gave up (the heap's sticky error is set).
template <typename K>
__device__ bool tma_land(const Params<K> &p, const HeapView<K> &H, unsigned long long *mb,
                         uint32_t arms, uint32_t &seen)
{
    if (seen == arms) return true;
    const uint32_t par = (arms - 1u) & 1u;
    unsigned long long t0 = 0;
    uint32_t it = 0;
    while (!mbar_try_wait(mb, par)) {
        if (!wait_ok(p, H, t0, it)) return false;
    }
    seen = arms;
    return true;
}

// Merge thread 0 (the only writer of rq_posted), after a barrier that follows
// the shared-memory writes of the request's sources: queues `r` for the
// release warp, waiting (bounded) for a free slot.  A wait that gives up has
// set the heap's sticky error; the request is dropped.
template <typename K>
__device__ void post_rel(const Params<K> &p, const HeapView<K> &H, Shared &sh, const RelReq &r)
{
    const uint32_t idx = sh.rq_posted;
    unsigned long long t0 = 0;
    uint32_t it = 0;
    while (idx - ld_acquire_cta(&sh.rq_read) >= N_REQ)
        if (!keep_waiting(p, H, t0, it)) return;
    sh.rq[idx % N_REQ] = r;
    st_release_cta(&sh.rq_posted, idx + 1);
}

// DEL and top-down INS, merge thread 0 after the barrier that follows the
// merge threads' stores of the node's keys (and of any larger child's keys
// since the last post): the node (the root word at the root: m, s and the
// next turn) and `pend` are released by the release warp.
template <typename K>
__device__ void post_step(const Params<K> &p, const HeapView<K> &H, Shared &sh,
                          uint32_t *cur_w, uint32_t *pend, uint32_t m, uint32_t s)
{
    RelReq r = {};
    r.w1 = pend;
    if (cur_w == nullptr) {
        r.root_w = &H.hdr->root;
        r.root_v = rw_make(m, s, sh.turn + 1);
        r.t_root = sh.t_root;
    } else {
        r.w0 = cur_w;
    }
    post_rel(p, H, sh, r);
}

// Root lock (also guards the partial buffer and the header).  Returns false
// when the wait gave up; `word` receives the header (m, s).
template <typename K>
__device__ bool lock_root(const Params<K> &p, const HeapView<K> &H, Shared &sh,
                          unsigned long long &word)
{
    unsigned long long t0 = 0;
    uint32_t it = 0;
    // a ring operation's ticket was drawn by the host, in the heap's request
    // order; the dispenser is advanced past it so that later launches go on
    const uint32_t ticket =
        sh.use_fixed ? (uint32_t)(sh.fixed_ticket & RW_TURN_MASK)
                     : (uint32_t)(atomicAdd(&H.hdr->next, 1ull) & RW_TURN_MASK);
    for (;;) {
        const unsigned long long v = ld_acquire64(&H.hdr->root);
        const uint32_t ahead = (ticket - rw_turn(v)) & (uint32_t)RW_TURN_MASK;
        if (ahead == 0) {
            if (it) stat_add(sh, STAT_WAITS, 1);
            sh.turn = ticket;
            word = v;
            if (sh.use_fixed)
                asm volatile("red.relaxed.gpu.global.max.u64 [%0], %1;"
                             :: "l"(&H.hdr->next), "l"(sh.fixed_ticket + 1ull) : "memory");
            return true;
        }
        if (!wait_ok(p, H, t0, it)) return false;
        // the head of the queue polls fast; the others sleep about as long as
        // the holds ahead of them
        __nanosleep(ahead <= 1 ? 32u : (ahead < 16 ? 256u * ahead : 4096u));
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
__device__ uint32_t lock_node(const Params<K> &p, const HeapView<K> &H, Shared &sh,
                              uint32_t *w, uint32_t first)
{
    uint32_t v = first;
    if (v != ST_INUSE) return v;
    unsigned long long t0 = 0;
    uint32_t it = 0;
    stat_add(sh, STAT_WAITS, 1);
    for (;;) {
        if (!keep_waiting(p, H, t0, it)) return ST_GAVE_UP;
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
// While it waits for a delivery the caller holds the root and no node lock.
template <typename K>
__device__ bool take_last(const Params<K> &p, const HeapView<K> &H, Shared &sh, uint32_t *w,
                          uint32_t first)
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
                        stat_add(sh, STAT_DELIVERIES, 1);
                        return true;
                    }
                    if (v != ST_MARKED) {
                        set_err(H, E_STATE);
                        return false;
                    }
                    if (!keep_waiting(p, H, t0, it)) return false;
                }
            }
        } else if (v != ST_INUSE) {
            set_err(H, E_STATE);
            return false;
        }
        if (!keep_waiting(p, H, t0, it)) return false;
        v = ld_relaxed(w);
        if (v == ST_AVAIL) {
            v = try_lock(w);
            if (v == ST_AVAIL) return true;
        }
    }
}

// ---------------------------------------------------------------------------
// data movement
// ---------------------------------------------------------------------------

__device__ __forceinline__ void cp_async16(void *smem, const void *gmem)
{
    unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" :: "r"(s), "l"(gmem) : "memory");
}

__device__ __forceinline__ void cp_async_commit()
{
    asm volatile("cp.async.commit_group;" ::: "memory");
}

__device__ __forceinline__ void cp_async_wait()
{
    asm volatile("cp.async.wait_all;" ::: "memory");
}

// global (L2) -> shared by `nthr` threads with index `t`; cp.async when
// aligned (complete with cp_async_wait and a barrier), else synchronous.
template <typename K>
__device__ __forceinline__ void g2s(K *dst, const K *src, uint32_t n, uint32_t t, uint32_t nthr)
{
    const uint32_t bytes = n * (uint32_t)sizeof(K);
    if (((reinterpret_cast<uintptr_t>(src) | reinterpret_cast<uintptr_t>(dst)) & 15u) == 0 &&
        (bytes & 15u) == 0) {
        const char *s = reinterpret_cast<const char *>(src);
        char *d = reinterpret_cast<char *>(dst);
        for (uint32_t i = t; i < bytes / 16u; i += nthr) cp_async16(d + 16u * i, s + 16u * i);
    } else {
        for (uint32_t i = t; i < n; i += nthr) dst[i] = __ldcg(src + i);
    }
}

// shared -> global (L2) by the merge threads.
template <typename K>
__device__ __forceinline__ void s2g(K *dst, const K *src, uint32_t n)
{
    const uint32_t t = threadIdx.x, nthr = nmt();
    const uint32_t bytes = n * (uint32_t)sizeof(K);
    if (((reinterpret_cast<uintptr_t>(src) | reinterpret_cast<uintptr_t>(dst)) & 15u) == 0 &&
        (bytes & 15u) == 0) {
        const uint4 *s4 = reinterpret_cast<const uint4 *>(src);
        uint4 *d4 = reinterpret_cast<uint4 *>(dst);
        for (uint32_t i = t; i < bytes / 16u; i += nthr) __stcg(d4 + i, s4[i]);
    } else {
        for (uint32_t i = t; i < n; i += nthr) __stcg(dst + i, src[i]);
    }
}

// MergeAndSort of two ascending runs in shared memory (Section 3.2.1) by the
// merge-path partition (Section 4.2), merge threads only: output position
// q < split goes to dlo[q], the rest to dhi[q - split].  Thread t produces
// outputs [t*IPT, t*IPT + IPT); na + nb must not exceed IPT * nmt().  The
// destinations may alias the sources.  Ends with bar_mg.
template <typename K, int IPT>
__device__ __noinline__ void merge_split(const K *a, uint32_t na, const K *b, uint32_t nb,
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
    bar_mg();
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
    bar_mg();
}

// N contiguous keys between shared memory and registers with the widest
// aligned vector accesses (16 or 8 bytes), so that a warp touching
// consecutive runs stays free of bank conflicts.  `p` must be aligned to the
// run's size when that is 8 or 16 bytes or a multiple of 16.
template <typename K, int N>
__device__ __forceinline__ void ld_run(const K *p, K (&v)[N])
{
    constexpr int B = (int)sizeof(K) * N;
    if constexpr (B % 16 == 0) {
        constexpr int PER = 16 / (int)sizeof(K);
#pragma unroll
        for (int c = 0; c < N / PER; ++c) {
            union { uint4 u; K k[PER]; } t;
            t.u = reinterpret_cast<const uint4 *>(p)[c];
#pragma unroll
            for (int e = 0; e < PER; ++e) v[c * PER + e] = t.k[e];
        }
    } else if constexpr (B == 8) {
        union { uint2 u; K k[N]; } t;
        t.u = *reinterpret_cast<const uint2 *>(p);
#pragma unroll
        for (int e = 0; e < N; ++e) v[e] = t.k[e];
    } else {
#pragma unroll
        for (int e = 0; e < N; ++e) v[e] = p[e];
    }
}

// Block bitonic sort of a[0..k) (Section 4.1) with every merge thread
// holding E consecutive keys in registers: strides below E are exchanged in
// registers, strides below 32·E between lanes with warp shuffles, and only
// the wider ones pass through shared memory (6 of the 55 stages at k = 1024,
// E = 4).  nmt()·E is a power of two >= k; when it exceeds k (one warp, small
// k) the missing keys count as the key maximum and are never written back.
template <typename K, int E>
__device__ __noinline__ void block_sort_reg(K *a, uint32_t k)
{
    const uint32_t T = nmt(), tid = threadIdx.x;
    const uint32_t n = T * E;
    const uint32_t base = tid * E;
    K v[E];
#pragma unroll
    for (int q = 0; q < E; ++q) v[q] = base + q < k ? a[base + q] : kmax<K>();
    for (uint32_t size = 2; size <= n; size <<= 1) {
        for (uint32_t s = size >> 1; s > 0; s >>= 1) {
            if (s >= 32u * E) {
                // shared-memory stage (n == k here: T > 32)
#pragma unroll
                for (int q = 0; q < E; ++q) a[base + q] = v[q];
                bar_mg();
                for (uint32_t pr = tid; pr < (n >> 1); pr += T) {
                    const uint32_t lo = 2 * pr - (pr & (s - 1)), hi = lo + s;
                    const bool asc = (lo & size) == 0;
                    const K x = a[lo], y = a[hi];
                    if ((x > y) == asc) {
                        a[lo] = y;
                        a[hi] = x;
                    }
                }
                bar_mg();
#pragma unroll
                for (int q = 0; q < E; ++q) v[q] = a[base + q];
            } else if (s >= (uint32_t)E) {
                // partner in lane (lane ^ s/E), same register
                const uint32_t ls = s / E;
#pragma unroll
                for (int q = 0; q < E; ++q) {
                    const uint32_t i = base + q;
                    const K o = __shfl_xor_sync(0xffffffffu, v[q], ls);
                    const bool keep_min = ((i & s) == 0) == ((i & size) == 0);
                    v[q] = keep_min ? (o < v[q] ? o : v[q]) : (o < v[q] ? v[q] : o);
                }
            } else {
#pragma unroll
                for (int st = E / 2; st >= 1; st >>= 1) {
                    if ((uint32_t)st != s) continue;
#pragma unroll
                    for (int q = 0; q < E; ++q) {
                        if ((q & st) == 0) {
                            const bool asc = ((base + q) & size) == 0;
                            const K x = v[q], y = v[q + st];
                            if ((x > y) == asc) {
                                v[q] = y;
                                v[q + st] = x;
                            }
                        }
                    }
                }
            }
        }
    }
    bar_mg();
#pragma unroll
    for (int q = 0; q < E; ++q)
        if (base + q < k) a[base + q] = v[q];
    bar_mg();
}

// ld_run / st_run of a run wider than 16 bytes per thread, with the 16-byte
// chunks taken in a per-thread rotated order: thread t starts at chunk
// (t >> (3 - log2 C)) mod C, so that the 8 threads of a quarter warp cover
// 8 distinct groups of 4 banks (without the rotation, runs of 32 bytes give
// a 2-way and runs of 64 bytes a 4-way bank conflict).  The merge uses it
// for 32-byte runs, where the rotation is a swap of two registers.
template <typename K, int N>
__device__ __forceinline__ void ld_run_rot(const K *p, K (&v)[N])
{
    constexpr int C = (int)sizeof(K) * N / 16;          // chunks per thread
    constexpr int PER = 16 / (int)sizeof(K);
    static_assert(C == 2 || C == 4 || C == 8, "run of 2, 4 or 8 chunks");
    constexpr int SH = C == 2 ? 2 : (C == 4 ? 1 : 0);
    const int r = (int)(threadIdx.x >> SH) & (C - 1);
    uint4 t[C];
#pragma unroll
    for (int i = 0; i < C; ++i) t[i] = reinterpret_cast<const uint4 *>(p)[(i + r) & (C - 1)];
#pragma unroll
    for (int j = 0; j < C; ++j) {
        // chunk j was loaded by instruction (j - r) mod C
        uint4 x = t[0];
#pragma unroll
        for (int i = 1; i < C; ++i)
            if (((j - r) & (C - 1)) == i) x = t[i];
        union { uint4 u; K k[PER]; } q;
        q.u = x;
#pragma unroll
        for (int e = 0; e < PER; ++e) v[j * PER + e] = q.k[e];
    }
}

template <typename K, int N>
__device__ __forceinline__ void st_run_rot(K *p, const K (&v)[N])
{
    constexpr int C = (int)sizeof(K) * N / 16;
    constexpr int PER = 16 / (int)sizeof(K);
    static_assert(C == 2 || C == 4 || C == 8, "run of 2, 4 or 8 chunks");
    constexpr int SH = C == 2 ? 2 : (C == 4 ? 1 : 0);
    const int r = (int)(threadIdx.x >> SH) & (C - 1);
    uint4 t[C];
#pragma unroll
    for (int j = 0; j < C; ++j) {
        union { uint4 u; K k[PER]; } q;
#pragma unroll
        for (int e = 0; e < PER; ++e) q.k[e] = v[j * PER + e];
        t[j] = q.u;
    }
#pragma unroll
    for (int i = 0; i < C; ++i) {
        // instruction i stores chunk (i + r) mod C
        uint4 x = t[0];
#pragma unroll
        for (int j = 1; j < C; ++j)
            if (((i + r) & (C - 1)) == j) x = t[j];
        reinterpret_cast<uint4 *>(p)[(i + r) & (C - 1)] = x;
    }
}

template <typename K, int N>
__device__ __forceinline__ void st_run(K *p, const K (&v)[N])
{
    constexpr int B = (int)sizeof(K) * N;
    if constexpr (B % 16 == 0) {
        constexpr int PER = 16 / (int)sizeof(K);
#pragma unroll
        for (int c = 0; c < N / PER; ++c) {
            union { uint4 u; K k[PER]; } t;
#pragma unroll
            for (int e = 0; e < PER; ++e) t.k[e] = v[c * PER + e];
            reinterpret_cast<uint4 *>(p)[c] = t.u;
        }
    } else if constexpr (B == 8) {
        union { uint2 u; K k[N]; } t;
#pragma unroll
        for (int e = 0; e < N; ++e) t.k[e] = v[e];
        *reinterpret_cast<uint2 *>(p) = t.u;
    } else {
#pragma unroll
        for (int e = 0; e < N; ++e) p[e] = v[e];
    }
}

// MergeAndSort of two full ascending runs a[0..k), b[0..k) (Section 3.2.1) as
// a bitonic merge (a followed by b reversed is bitonic): one compare stage
// across the halves leaves the k smallest in dlo and the k largest in dhi,
// each a bitonic run; each half is then sorted by its own half-cleaner
// stages -- strides of 32*IPT keys and more in shared memory, smaller ones
// in registers via warp shuffles.  Every thread moves contiguous runs of
// IPT/2 or IPT keys with vector accesses.  Merge threads only; needs
// nmt()*IPT == 2k and k >= 32*IPT; destinations may alias the sources.  Ends
// with bar_mg.
template <typename K, int IPT>
__device__ __noinline__ void merge_full(const K *a, const K *b, K *dlo, K *dhi, uint32_t k)
{
    constexpr int H2 = IPT / 2;
    const uint32_t T = nmt(), tid = threadIdx.x;
    {
        // pairs (a[i], b[k-1-i]) for i in [tid*H2, tid*H2 + H2)
        const uint32_t i0 = tid * H2;
        K x[H2], yr[H2], lo[H2], hi[H2];
        ld_run<K, H2>(a + i0, x);
        ld_run<K, H2>(b + (k - i0 - H2), yr);
#pragma unroll
        for (int e = 0; e < H2; ++e) {
            const K y = yr[H2 - 1 - e];
            lo[e] = x[e] < y ? x[e] : y;
            hi[e] = x[e] < y ? y : x[e];
        }
        bar_mg();
        st_run<K, H2>(dlo + i0, lo);
        st_run<K, H2>(dhi + i0, hi);
        bar_mg();
    }
    (void)T;
    const uint32_t half = nmt() >> 1;
    const uint32_t u = tid < half ? tid : tid - half;
    K *d = tid < half ? dlo : dhi;
    for (uint32_t st = k >> 1; st >= 32u * IPT; st >>= 1) {
        // half-cleaner: thread u takes H2 adjacent pairs (l, l + st)
        const uint32_t j = u * H2;
        const uint32_t l = 2 * j - (j & (st - 1)), h = l + st;
        K x[H2], y[H2];
        ld_run<K, H2>(d + l, x);
        ld_run<K, H2>(d + h, y);
#pragma unroll
        for (int e = 0; e < H2; ++e) {
            const K mn = x[e] < y[e] ? x[e] : y[e];
            const K mx = x[e] < y[e] ? y[e] : x[e];
            x[e] = mn;
            y[e] = mx;
        }
        st_run<K, H2>(d + l, x);
        st_run<K, H2>(d + h, y);
        bar_mg();
    }
    K v[IPT];
    if constexpr (sizeof(K) * IPT == 32) ld_run_rot<K, IPT>(d + u * IPT, v);
    else ld_run<K, IPT>(d + u * IPT, v);
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
    if constexpr (sizeof(K) * IPT == 32) st_run_rot<K, IPT>(d + u * IPT, v);
    else st_run<K, IPT>(d + u * IPT, v);
    bar_mg();
}

// MergeAndSort of two full k-runs into (k smallest -> dlo, k largest -> dhi):
// the bitonic form when the block shape allows it, else merge path.
template <typename K, int IPT>
__device__ __forceinline__ void merge_kk(const K *a, const K *b, K *dlo, K *dhi, uint32_t k)
{
    if (nmt() * IPT == 2 * k && k >= 32u * IPT) merge_full<K, IPT>(a, b, dlo, dhi, k);
    else merge_split<K, IPT>(a, k, b, k, dlo, k, dhi);
}

// Contiguous keys between shared memory and registers: the rotated form for
// 32-byte runs, the plain one otherwise.
template <typename K, int N>
__device__ __forceinline__ void ld_keys(const K *p, K (&v)[N])
{
    if constexpr (sizeof(K) * N == 32) ld_run_rot<K, N>(p, v);
    else ld_run<K, N>(p, v);
}

template <typename K, int N>
__device__ __forceinline__ void st_keys(K *p, const K (&v)[N])
{
    if constexpr (sizeof(K) * N == 32) st_run_rot<K, N>(p, v);
    else st_run<K, N>(p, v);
}

// First stage of MergeAndSort of two ascending k-runs (Section 3.2.1) in
// bitonic form: lo[i] = min(a[i], b[k-1-i]) are the k smallest keys and
// hi[i] the k largest, each a bitonic run still to be sorted.  Every merge
// thread takes E pairs: needs nmt()*E == k.  The destinations may alias the
// sources.  Ends with bar_mg.
template <typename K, int E>
__device__ __forceinline__ void bitonic_split(const K *a, const K *b, K *lo, K *hi, uint32_t k)
{
    const uint32_t i0 = threadIdx.x * E;
    K x[E], yr[E], l[E], h[E];
    ld_keys<K, E>(a + i0, x);
    ld_keys<K, E>(b + (k - i0 - E), yr);
#pragma unroll
    for (int e = 0; e < E; ++e) {
        const K y = yr[E - 1 - e];
        l[e] = x[e] < y ? x[e] : y;
        h[e] = x[e] < y ? y : x[e];
    }
    bar_mg();
    st_keys<K, E>(lo + i0, l);
    st_keys<K, E>(hi + i0, h);
    bar_mg();
}

// Sorts the bitonic run d[0..k) ascending with all merge threads, each
// holding E consecutive keys: half-cleaner strides of 32*E keys and more in
// shared memory (E/2 pairs per thread), smaller ones between lanes (warp
// shuffles) and within registers.  Needs nmt()*E == k, E >= 2 and k >= 64*E.
// Ends with bar_mg.
template <typename K, int E>
__device__ __noinline__ void sort_bitonic(K *d, uint32_t k)
{
    constexpr int P = E / 2;
    const uint32_t u = threadIdx.x;
    for (uint32_t st = k >> 1; st >= 32u * E; st >>= 1) {
        const uint32_t j = u * P;
        const uint32_t l = 2 * j - (j & (st - 1)), h = l + st;
        K x[P], y[P];
        ld_run<K, P>(d + l, x);
        ld_run<K, P>(d + h, y);
#pragma unroll
        for (int e = 0; e < P; ++e) {
            const K mn = x[e] < y[e] ? x[e] : y[e];
            const K mx = x[e] < y[e] ? y[e] : x[e];
            x[e] = mn;
            y[e] = mx;
        }
        st_run<K, P>(d + l, x);
        st_run<K, P>(d + h, y);
        bar_mg();
    }
    K v[E];
    ld_keys<K, E>(d + u * E, v);
    const uint32_t lane = u & 31u;
#pragma unroll
    for (uint32_t lm = 16; lm >= 1; lm >>= 1) {
        const bool upper = (lane & lm) != 0;
#pragma unroll
        for (int q = 0; q < E; ++q) {
            const K o = __shfl_xor_sync(0xffffffffu, v[q], lm);
            v[q] = upper ? (o < v[q] ? v[q] : o) : (o < v[q] ? o : v[q]);
        }
    }
#pragma unroll
    for (int st = E / 2; st >= 1; st >>= 1) {
#pragma unroll
        for (int q = 0; q < E; ++q) {
            if ((q & st) == 0) {
                const K x = v[q], y = v[q + st];
                v[q] = x < y ? x : y;
                v[q + st] = x < y ? y : x;
            }
        }
    }
    st_keys<K, E>(d + u * E, v);
    bar_mg();
}

// ---- transposed form of the split and sort (4-byte keys, 2 or 4 per thread)
//
// The bitonic run of k = 2^n keys is held in two layouts.  Layout A gives a
// thread E keys k/E apart -- register bits are key-index bits n-1..n-R
// (R = log2 E), lane bits the next 5, warp bits the lowest wb = n-R-5 -- so
// that the first R+5 stages run in registers and shuffles.  One pass through
// shared memory turns it into layout B (E consecutive keys per thread: the
// warp bits on top), where the last wb stages run the same way.  Between the
// split and the sort the run is kept at swizzled positions (bits 5-9 folded
// into bits 0-4), so that the split's stores, layout A's single-key accesses
// and layout B's vector loads each spread over all 32 banks.

template <typename K, int E>
struct Transposed { static constexpr bool value = sizeof(K) == 4 && (E == 2 || E == 4); };

__device__ __forceinline__ uint32_t swz(uint32_t i) { return i ^ ((i >> 5) & 31u); }

template <typename K, int E>
__device__ __forceinline__ void ld_vec(const K *p, K (&v)[E])
{
    if constexpr (E == 4) {
        const uint4 u = *reinterpret_cast<const uint4 *>(p);
        v[0] = (K)u.x; v[1] = (K)u.y; v[2] = (K)u.z; v[3] = (K)u.w;
    } else {
        const uint2 u = *reinterpret_cast<const uint2 *>(p);
        v[0] = (K)u.x; v[1] = (K)u.y;
    }
}

template <typename K, int E>
__device__ __forceinline__ void st_vec(K *p, const K (&v)[E])
{
    if constexpr (E == 4) {
        *reinterpret_cast<uint4 *>(p) = make_uint4((uint32_t)v[0], (uint32_t)v[1],
                                                   (uint32_t)v[2], (uint32_t)v[3]);
    } else {
        *reinterpret_cast<uint2 *>(p) = make_uint2((uint32_t)v[0], (uint32_t)v[1]);
    }
}

// v[q] <- v[q ^ xm], xm < E.
template <typename K, int E>
__device__ __forceinline__ void xperm(K (&v)[E], uint32_t xm)
{
    if (xm & 1u) {
#pragma unroll
        for (int q = 0; q < E; q += 2) {
            const K t = v[q]; v[q] = v[q + 1]; v[q + 1] = t;
        }
    }
    if constexpr (E == 4) {
        if (xm & 2u) {
            K t = v[0]; v[0] = v[2]; v[2] = t;
            t = v[1]; v[1] = v[3]; v[3] = t;
        }
    }
}

// bitonic_split with the halves stored at swizzled positions, for
// sort_bitonic_t.  Same contract otherwise.
template <typename K, int E>
__device__ __forceinline__ void bitonic_split_t(const K *a, const K *b, K *lo, K *hi, uint32_t k)
{
    const uint32_t i0 = threadIdx.x * E;
    K x[E], yr[E], l[E], h[E];
    ld_vec<K, E>(a + i0, x);
    ld_vec<K, E>(b + (k - i0 - E), yr);
#pragma unroll
    for (int e = 0; e < E; ++e) {
        const K y = yr[E - 1 - e];
        l[e] = x[e] < y ? x[e] : y;
        h[e] = x[e] < y ? y : x[e];
    }
    const uint32_t s = (i0 >> 5) & 31u;
    const uint32_t cb = i0 ^ (s & ~(uint32_t)(E - 1));
    xperm<K, E>(l, s & (E - 1));
    xperm<K, E>(h, s & (E - 1));
    bar_mg();
    st_vec<K, E>(lo + cb, l);
    st_vec<K, E>(hi + cb, h);
    bar_mg();
}

// sort_bitonic of a run left at swizzled positions by bitonic_split_t; the
// sorted run is stored in plain order.  Needs nmt()*E == k, 32 <= nmt() <= 512.
// Ends with bar_mg.
template <typename K, int E>
__device__ __noinline__ void sort_bitonic_t(K *d, uint32_t k)
{
    constexpr uint32_t R = E == 4 ? 2u : 1u;
    const uint32_t n = 31u - __clz(k);
    const uint32_t wb = n - R - 5u;
    const uint32_t lane = threadIdx.x & 31u, w = threadIdx.x >> 5;
    const uint32_t a0 = (lane << wb) | w;
    K v[E];
#pragma unroll
    for (int q = 0; q < E; ++q) v[q] = d[swz(((uint32_t)q << (n - R)) | a0)];
    // layout A: strides k/2 .. k/E between registers, then k/(2E) .. 2^wb
    // between lanes
#pragma unroll
    for (int st = E / 2; st >= 1; st >>= 1) {
#pragma unroll
        for (int q = 0; q < E; ++q) {
            if ((q & st) == 0) {
                const K x = v[q], y = v[q + st];
                v[q] = x < y ? x : y;
                v[q + st] = x < y ? y : x;
            }
        }
    }
#pragma unroll
    for (uint32_t lm = 16; lm >= 1; lm >>= 1) {
        const bool upper = (lane & lm) != 0;
#pragma unroll
        for (int q = 0; q < E; ++q) {
            const K o = __shfl_xor_sync(0xffffffffu, v[q], lm);
            v[q] = upper ? (o < v[q] ? v[q] : o) : (o < v[q] ? o : v[q]);
        }
    }
    // every thread rewrites the positions it read
#pragma unroll
    for (int q = 0; q < E; ++q) d[swz(((uint32_t)q << (n - R)) | a0)] = v[q];
    bar_mg();
    // layout B: strides 2^(wb-1) .. E between lanes, then within registers
    const uint32_t b0 = (w << (R + 5u)) | (lane << R);
    const uint32_t x = (b0 >> 5) & 31u;
    ld_vec<K, E>(d + (b0 ^ (x & ~(uint32_t)(E - 1))), v);
    xperm<K, E>(v, x & (E - 1));
    for (uint32_t pos = wb; pos > R; --pos) {
        const uint32_t lm = 1u << (pos - 1u - R);
        const bool upper = (lane & lm) != 0;
#pragma unroll
        for (int q = 0; q < E; ++q) {
            const K o = __shfl_xor_sync(0xffffffffu, v[q], lm);
            v[q] = upper ? (o < v[q] ? v[q] : o) : (o < v[q] ? o : v[q]);
        }
    }
#pragma unroll
    for (int st = E / 2; st >= 1; st >>= 1) {
        if ((uint32_t)st < (1u << wb)) {
#pragma unroll
            for (int q = 0; q < E; ++q) {
                if ((q & st) == 0) {
                    const K x0 = v[q], y = v[q + st];
                    v[q] = x0 < y ? x0 : y;
                    v[q + st] = x0 < y ? y : x0;
                }
            }
        }
    }
    bar_mg();   // every layout-B load is done before the plain stores
    st_vec<K, E>(d + b0, v);
    bar_mg();
}

// The split and sort in the form the key type allows.
template <typename K, int E>
__device__ __forceinline__ void split_run(const K *a, const K *b, K *lo, K *hi, uint32_t k)
{
    if constexpr (Transposed<K, E>::value) bitonic_split_t<K, E>(a, b, lo, hi, k);
    else bitonic_split<K, E>(a, b, lo, hi, k);
}

template <typename K, int E>
__device__ __forceinline__ void sort_run(K *d, uint32_t k)
{
    if constexpr (Transposed<K, E>::value) sort_bitonic_t<K, E>(d, k);
    else sort_bitonic<K, E>(d, k);
}

// Takes a ticket under the root lock and records the operation in the
// linearization record (root holder only).
template <typename K>
__device__ __forceinline__ void take_ticket(const Params<K> &p, const HeapView<K> &H, Shared &sh,
                                            uint32_t kind, uint32_t n, unsigned long long ref)
{
    // no record kept: no number to draw (it would cost a round trip to L2
    // inside the root hold)
    if (H.log_cap == 0) {
        sh.seq = 0;
        return;
    }
    // atomic: a bottom-up insert takes its number under its last lock, which
    // need not be the root's
    const unsigned long long seq = atomicAdd(&H.hdr->seq, 1ull);
    sh.seq = seq;
    if (seq < H.log_cap) {
        gheap_log_entry e;
        e.call_id = p.call_id;
        e.kind_n = (kind << 24) | n;
        e.ref = ref;
        H.log[seq] = e;
    }
}

// ---------------------------------------------------------------------------
// INS (Section 3.2.2 top-down INS, Section 3.3.2 partial buffer)
// ---------------------------------------------------------------------------

template <typename K, int IPT>
__device__ bool bu_rise(const Params<K> &p, const HeapView<K> &H, Shared &sh, K *base,
                        uint32_t tslot, bool locked, int ds, uint32_t n, unsigned long long ref);

// The batch PB(0)[0..n) is sorted (PB(0)[n..k) hold the key maximum) and the
// block has met on a barrier since.  Buffers: 0 = the carried batch, 1 and 2
// = the current and the next node, 3 = the partial buffer.  Returns false
// when the operation had to give up (the block must stop).  BU: a full batch
// is placed at its target and rises (bottom-up INS, Section 3.2.2) instead
// of walking down from the root; the root step and the partial buffer are
// the same.
template <typename K, int IPT, bool BU>
__device__ bool ins_op(const Params<K> &p, const HeapView<K> &H, Shared &sh, K *base,
                       uint32_t n, unsigned long long ref)
{
    const uint32_t k = p.k;
    const bool ctrl = is_ctrl();
    const uint32_t lane = clane();
    K *const A = base;                        // carry
    K *const Bq = base + 3 * (size_t)k;       // partial buffer
    K *root = H.keys + (size_t)k;
    long long tp = clock64();

    // take the root; for a full batch that goes down, mark the target, copy
    // the root and try the first node of the path
    if (ctrl) {
        if (lane == 0) {
            sh.tslot = 0;
            sh.lockfree = 0;
            if (BU && n == k && rw_m(ld_relaxed64(&H.hdr->root)) >= 1) {
                // a full bottom-up batch touches neither the root nor the
                // buffer: it reserves its target with an atomic add on m and
                // never takes the root lock here (m only grows during an
                // insert launch, and no DEL runs in one)
                const unsigned long long old = atomicAdd(&H.hdr->root, 1ull);
                const uint32_t slot = rw_m(old) + 1;
                sh.m = rw_m(old);
                sh.s = rw_s(old);
                sh.lockfree = 1;
                if (slot > H.max_nodes) {
                    set_err(H, E_FULL);
                    sh.abort = 1;
                } else {
                    sh.tslot = slot;
                    st_relaxed(&H.state[slot], ST_INUSE);
                }
            } else {
                unsigned long long w = 0;
                sh.abort = !lock_root(p, H, sh, w);
                lap(sh, STAT_INS_ACQ_CYC, tp);
                if (!sh.abort) {
                    if (sh.stats_on) sh.t_root = gtimer();
                    const uint32_t m = rw_m(w), s = rw_s(w);
                    sh.m = m;
                    sh.s = s;
                    const bool full = n == k || n + s >= k;
                    // a bottom-up batch that leaves the root level is
                    // linearized under its last lock instead
                    if (!(BU && full && m >= 1)) take_ticket(p, H, sh, GHEAP_OP_INS, n, ref);
                    if (full && m >= 1) {
                        // bottom-up: the slot comes from the same atomic add
                        // as the unlocked reservations
                        const uint32_t slot =
                            BU ? rw_m(atomicAdd(&H.hdr->root, 1ull)) + 1 : m + 1;
                        if (slot > H.max_nodes) {
                            set_err(H, E_FULL);
                            sh.abort = 1;
                        } else {
                            sh.tslot = slot;
                            st_relaxed(&H.state[slot], BU ? ST_INUSE : ST_TARGET);
                        }
                    }
                }
            }
        }
        __syncwarp();
        const uint32_t tslot = sh.tslot;
        if (!BU && tslot) {
            g2s(base + (size_t)k, root, k, lane, 32u);   // root -> buffer 1
            cp_async_commit();
            if (lane == 0) {
                const uint32_t tnode = slot_node(tslot);
                const uint32_t n1 = tnode >> (level_of(tnode) - 1);
                uint32_t *w1 = &H.state[slot_node(n1)];
                sh.lk[0][0] = (n1 == tnode) ? claim_target(w1) : try_lock(w1);
            }
            cp_async_wait();
        }
    }
    bar_all();
    if (sh.abort) return false;
    const uint32_t m = sh.m;
    uint32_t s = sh.s;

    if (!sh.tslot) {
        // the batch stays at the root level: the partial buffer and/or a new
        // root (no full node existed)
        const bool fits = n < k && n + s < k;
        if (!ctrl) {
            if (n < k) {
                g2s(Bq, H.buf, s, threadIdx.x, nmt());
                if (fits && m >= 1) g2s(base + (size_t)k, root, k, threadIdx.x, nmt());
                cp_async_commit();
                cp_async_wait();
                bar_mg();
                if (fits) {
                    merge_split<K, IPT>(A, n, Bq, s, Bq, n + s, Bq);
                    if (m >= 1) {
                        // Property 3: the root keeps the k smallest of root + buffer
                        K *R = base + (size_t)k;
                        merge_split<K, IPT>(R, k, Bq, n + s, R, k, Bq);
                        s2g(root, R, k);
                        if (threadIdx.x == 0) {
                            stat_add(sh, STAT_LOADS, 1);
                            stat_add(sh, STAT_STORES, 1);
                            stat_add(sh, STAT_MERGES, 1);
                        }
                    }
                    s2g(H.buf, Bq, n + s);
                } else {
                    // the k smallest of batch + buffer become the root (m == 0)
                    merge_split<K, IPT>(A, n, Bq, s, A, k, Bq);
                    s2g(H.buf, Bq, n + s - k);
                }
            } else if (s > 0) {
                // a full batch becomes the root: keep Property 3 with the buffer
                g2s(Bq, H.buf, s, threadIdx.x, nmt());
                cp_async_commit();
                cp_async_wait();
                bar_mg();
                merge_split<K, IPT>(A, k, Bq, s, A, k, Bq);
                s2g(H.buf, Bq, s);
            }
            if (!fits) {
                s2g(root, A, k);
                if (threadIdx.x == 0) stat_add(sh, STAT_STORES, 1);
            }
        }
        bar_all();
        if (ctrl && lane == 0) {
            stat_root(sh);
            if (BU) {
                if (fits) release_root_delta(H, 0, (int)n);
                else release_root_delta(H, 1, (n < k ? (int)(n + s - k) : (int)s) - (int)s);
            } else {
                if (fits) release_root_word(H, sh, m, n + s);
                else release_root_word(H, sh, 1u, n < k ? n + s - k : s);
            }
        }
        return true;
    }

    // full top-down INS to slot tslot
    const uint32_t tslot = sh.tslot;
    const uint32_t tnode = slot_node(tslot);
    const uint32_t depth = level_of(tnode);
    if (n < k) {
        // overflow of the partial buffer: the k smallest go down
        if (!ctrl) {
            g2s(Bq, H.buf, s, threadIdx.x, nmt());
            cp_async_commit();
            cp_async_wait();
            bar_mg();
            merge_split<K, IPT>(A, n, Bq, s, A, k, Bq);
            s2g(H.buf, Bq, n + s - k);
        }
        s = n + s - k;
    }
    if (BU) return bu_rise<K, IPT>(p, H, sh, base, tslot, !sh.lockfree, (int)s - (int)sh.s, n, ref);

    uint32_t ib = 1, ic = 2;       // current node, next node
    // nodes of a multiple of 16 bytes move by TMA (aligned buffers and nodes)
    const bool tma_ok = (k * (uint32_t)sizeof(K)) % 16u == 0;
    K *cur_keys = root;
    uint32_t *cur_w = nullptr;     // nullptr = the root word
    uint32_t par = 0;
    bool icpt_held = false;        // control lane 0: the next node was locked by the last try
    for (uint32_t lvl = 0;; ++lvl) {
        const uint32_t nxt = tnode >> (depth - lvl - 1);
        const uint32_t nslot = slot_node(nxt);
        uint32_t *nw = &H.state[nslot];
        K *nkeys = H.keys + (size_t)nslot * k;
        const bool at_target = nxt == tnode;
        K *b = base + (size_t)ib * k;
        K *c = base + (size_t)ic * k;
        if (ctrl) {
            // finish taking the next node (hand-over-hand: the current one is
            // held); below the root also copy it now and try the one after
            long long tw = clock64();
            if (lane == 0) {
                uint32_t v = sh.lk[par][0];
                // a DEL that needs this insert's target as its refill has
                // marked it and waits: the keys carried after this level go
                // to it at once instead of down the rest of the path (an
                // insert-only launch has no DEL: no look at the target)
                int dec = (p.mode != MODE_INSERT && lvl > 0 && !at_target &&
                           ld_relaxed(&H.state[tslot]) == ST_MARKED) ? 1 : 0;
                icpt_held = dec == 1 && v == ST_AVAIL;
                if (at_target) {
                    sh.deliver = (v == ST_MARKED);
                    if (v != ST_TARGET && v != ST_MARKED) {
                        set_err(H, E_STATE);
                        dec = 2;
                    }
                } else if (dec == 1) {
                    // the next node is not taken (only given back if the last
                    // level's try took it)
                } else if (v != ST_AVAIL) {
                    v = lock_node(p, H, sh, nw, v);
                    if (v != ST_AVAIL) {
                        if (v != ST_GAVE_UP) set_err(H, E_STATE);
                        dec = 2;
                    }
                }
                sh.ilvl[par] = dec;
            }
            __syncwarp();
            if (lvl > 0 && !at_target && sh.ilvl[par] == 0) {
                if (tma_ok) {
                    // the node by TMA (one lane), the next one tried meanwhile
                    if (lane == 0) {
                        tma_fetch(H, k, 1u, nslot, c, 0u, c, &sh.kid_mbar, sh.kid_arms);
                        const uint32_t n2 = tnode >> (depth - lvl - 2);
                        uint32_t *w2 = &H.state[slot_node(n2)];
                        sh.lk[par ^ 1][0] = (n2 == tnode) ? claim_target(w2) : try_lock(w2);
                        if (!tma_land(p, H, &sh.kid_mbar, sh.kid_arms, sh.kid_seen))
                            sh.ilvl[par] = 2;
                    }
                } else {
                    g2s(c, nkeys, k, lane, 32u);
                    cp_async_commit();
                    if (lane == 0) {
                        const uint32_t n2 = tnode >> (depth - lvl - 2);
                        uint32_t *w2 = &H.state[slot_node(n2)];
                        sh.lk[par ^ 1][0] = (n2 == tnode) ? claim_target(w2) : try_lock(w2);
                    }
                    cp_async_wait();
                }
            }
            if (lane == 0) {
                lap(sh, STAT_INS_WAIT_CYC, tw);
                stat_add(sh, STAT_INS_LEVELS, 1);
            }
        } else {
            // MergeAndSort(node, batch): the node keeps the k smallest, the k
            // largest are carried on (Section 3.2.2); disjoint ranges are
            // kept or swapped without merging (Section 4.3)
            long long tm = clock64();
            const K bmax = b[k - 1], bmin = b[0], amax = A[k - 1], amin = A[0];
            bar_mg();
            if (bmax <= amin) {
                if (threadIdx.x == 0) stat_add(sh, STAT_SKIPS, 1);
            } else if (amax <= bmin) {
                // the node takes the batch; the old node keys are carried on
                s2g(cur_keys, A, k);
                bar_mg();
                for (uint32_t i = threadIdx.x; i < k; i += nmt()) A[i] = b[i];
                bar_mg();
                if (threadIdx.x == 0) {
                    stat_add(sh, STAT_SKIPS, 1);
                    stat_add(sh, STAT_STORES, 1);
                }
            } else {
                merge_kk<K, IPT>(b, A, b, A, k);
                s2g(cur_keys, b, k);
                if (threadIdx.x == 0) {
                    stat_add(sh, STAT_MERGES, 1);
                    stat_add(sh, STAT_STORES, 1);
                }
            }
            if (threadIdx.x == 0) {
                stat_add(sh, STAT_LOADS, 1);
                lap(sh, STAT_INS_STEP_CYC, tm);
            }
        }
        bar_all();
        const int dec = sh.ilvl[par];
        if (dec == 2) return false;
        // the root word and the level-1 node are released at once by the
        // control warp (the next operation waits for them); a node further
        // down goes back through the release warp, so that the control warp
        // takes the next node without the fence
        if (lvl <= 1) {
            if (ctrl && lane == 0) {
                if (cur_w == nullptr) {
                    stat_root(sh);
                    release_root_word(H, sh, tslot, s);
                } else {
                    st_release(cur_w, ST_AVAIL);
                }
            }
        } else if (threadIdx.x == 0) {
            post_step(p, H, sh, cur_w, nullptr, 0u, 0u);
        }
        if (dec == 1) {
            // deliver the carried keys to the marked target (Section 3.3.2's
            // hand-off, one level step after the mark instead of at the end
            // of the path): the nodes below were not touched
            if (!ctrl) {
                s2g(H.keys + (size_t)tslot * k, A, k);
                if (threadIdx.x == 0) stat_add(sh, STAT_STORES, 1);
            }
            bar_all();
            if (ctrl && lane == 0) {
                if (icpt_held) st_release(nw, ST_AVAIL);
                st_release(&H.state[tslot], ST_DELIVERED);
                stat_add(sh, STAT_INTERCEPTS, 1);
            }
            return true;
        }
        if (at_target) {
            if (!ctrl) {
                s2g(nkeys, A, k);
                if (threadIdx.x == 0) stat_add(sh, STAT_STORES, 1);
            }
            bar_all();
            if (ctrl && lane == 0) st_release(nw, sh.deliver ? ST_DELIVERED : ST_AVAIL);
            return true;
        }
        if (lvl == 0) {
            // the root is released: now copy the level-1 node and try level 2
            if (ctrl) {
                if (tma_ok) {
                    if (lane == 0) {
                        tma_fetch(H, k, 1u, nslot, c, 0u, c, &sh.kid_mbar, sh.kid_arms);
                        const uint32_t n2 = tnode >> (depth - 2);
                        uint32_t *w2 = &H.state[slot_node(n2)];
                        sh.lk[par ^ 1][0] = (n2 == tnode) ? claim_target(w2) : try_lock(w2);
                        if (!tma_land(p, H, &sh.kid_mbar, sh.kid_arms, sh.kid_seen)) sh.abort = 1;
                    }
                    __syncwarp();
                } else {
                    g2s(c, nkeys, k, lane, 32u);
                    cp_async_commit();
                    if (lane == 0) {
                        const uint32_t n2 = tnode >> (depth - 2);
                        uint32_t *w2 = &H.state[slot_node(n2)];
                        sh.lk[par ^ 1][0] = (n2 == tnode) ? claim_target(w2) : try_lock(w2);
                    }
                    cp_async_wait();
                }
            }
            bar_all();
            if (sh.abort) return false;
        }
        const uint32_t t = ib; ib = ic; ic = t;
        cur_keys = nkeys;
        cur_w = nw;
        par ^= 1;
    }
}

// Bottom-up INS (Sections 3.2.2 and 3.3.4) of a full batch A = PB(0) whose
// target slot `tslot` is reserved (state INUSE, held by this block).  When
// the reservation took the root lock (`locked`: a partial batch that
// overflowed the buffer, or the heap's first node), the root is released
// first, publishing the buffer-size change `ds`; a full batch on a non-empty
// heap reserved its slot without the lock.  The batch is stored at the
// target, and then, level by level: lock the parent (waiting while it is in
// use or holds another insert's batch), take the own node back from
// INSHOLD, stop when parent max <= batch min (early stop, Section 4.3), else
// MergeAndSort(parent, batch): the parent keeps the k smallest, which rise
// on, and the node keeps the k largest.  Between levels the node is
// released as INSHOLD; the operation is linearized under its last lock (the
// early-stop pair or the root).  Locks are only ever requested while
// holding nothing but the own INSHOLD node, which no other operation takes,
// so the upward walk cannot deadlock with the top-down locking of other
// inserts.  This path runs in insert-only launches: a DEL never meets an
// INSHOLD node, and m only grows.
template <typename K, int IPT>
__device__ bool bu_rise(const Params<K> &p, const HeapView<K> &H, Shared &sh, K *base,
                        uint32_t tslot, bool locked, int ds, uint32_t n, unsigned long long ref)
{
    const uint32_t k = p.k;
    const bool ctrl = is_ctrl();
    const uint32_t lane = clane();
    K *const A = base;                        // the rising batch
    K *const P = base + (size_t)k;            // the parent's keys
    const uint32_t me = inshold((uint32_t)(sh.op & 0xFFFFFFull));

    // publish the buffer and release the root (when the reservation took
    // it), store the batch at the target and hand the target over as INSHOLD
    bar_all();
    if (ctrl && lane == 0 && locked) {
        stat_root(sh);
        release_root_delta(H, 0, ds);
    }
    if (!ctrl) {
        s2g(H.keys + (size_t)tslot * k, A, k);
        if (threadIdx.x == 0) stat_add(sh, STAT_STORES, 1);
    }
    bar_all();
    if (ctrl && lane == 0) st_release(&H.state[tslot], me);

    uint32_t cslot = tslot, cnode = slot_node(tslot);
    for (;;) {
        const uint32_t pnode = cnode >> 1;
        const bool proot = pnode == 1;
        const uint32_t pslot = slot_node(pnode);     // the map is its own inverse
        K *pkeys = H.keys + (size_t)pslot * k;
        uint32_t *pw = &H.state[pslot];
        if (ctrl) {
            long long tw = clock64();
            if (lane == 0) {
                if (proot) {
                    unsigned long long w = 0;
                    sh.abort = !lock_root(p, H, sh, w);
                    sh.m = rw_m(w);
                    sh.s = rw_s(w);
                    if (sh.stats_on) sh.t_root = gtimer();
                } else {
                    unsigned long long t0 = 0;
                    uint32_t it = 0;
                    for (;;) {
                        const uint32_t v = ld_relaxed(pw);
                        if (v == ST_AVAIL && try_lock(pw) == ST_AVAIL) break;
                        if (v != ST_AVAIL && v != ST_INUSE && (v & 0xFFu) != ST_INSHOLD) {
                            set_err(H, E_STATE);
                            sh.abort = 1;
                            break;
                        }
                        if (!keep_waiting(p, H, t0, it)) {
                            sh.abort = 1;
                            break;
                        }
                    }
                    if (it) stat_add(sh, STAT_WAITS, 1);
                }
                if (!sh.abort && atomicCAS(&H.state[cslot], me, ST_INUSE) != me) {
                    set_err(H, E_STATE);
                    sh.abort = 1;
                }
                lap(sh, STAT_INS_WAIT_CYC, tw);
                stat_add(sh, STAT_INS_LEVELS, 1);
            }
            __syncwarp();
            if (!sh.abort) {
                g2s(P, pkeys, k, lane, 32u);
                cp_async_commit();
                cp_async_wait();
            }
        }
        bar_all();
        if (sh.abort) return false;
        if (!ctrl) {
            long long tm = clock64();
            const K pmax = P[k - 1], amin = A[0];
            bar_mg();
            if (pmax <= amin) {
                if (threadIdx.x == 0) {
                    sh.halt = 1;
                    stat_add(sh, STAT_SKIPS, 1);
                }
            } else {
                // MergeAndSort(parent, batch): the k smallest rise with the
                // parent, the k largest stay in the node
                merge_kk<K, IPT>(P, A, A, P, k);
                s2g(H.keys + (size_t)cslot * k, P, k);
                s2g(pkeys, A, k);
                if (threadIdx.x == 0) {
                    sh.halt = 0;
                    stat_add(sh, STAT_MERGES, 1);
                    stat_add(sh, STAT_STORES, 2);
                }
            }
            if (threadIdx.x == 0) {
                stat_add(sh, STAT_LOADS, 1);
                lap(sh, STAT_INS_STEP_CYC, tm);
            }
        }
        bar_all();
        const bool done = sh.halt || proot;
        if (ctrl && lane == 0) {
            if (done) take_ticket(p, H, sh, GHEAP_OP_INS, n, ref);
            st_release(&H.state[cslot], ST_AVAIL);
            if (proot) {
                stat_root(sh);
                release_root_delta(H, 0, 0);
            } else {
                st_release(pw, done ? ST_AVAIL : me);
            }
        }
        if (done) {
            bar_all();
            if (threadIdx.x == 0) sh.halt = 0;
            return true;
        }
        cslot = pslot;
        cnode = pnode;
    }
}

// ---------------------------------------------------------------------------
// DEL (Section 3.2.1, partial buffer of Section 3.3.2)
// ---------------------------------------------------------------------------

// Control warp: lock the children (slots sl, sr; 0 = none) of a held node --
// lane 0 the left, lane 1 the right, waiting as needed (`first0/1` are earlier
// tries or NO_TRY) -- and copy the present ones into dl / dr.  Results go to
// lk[0..1].  Returns with the copies complete.  The warp waits as one (a vote
// per poll, each poll a compare-and-swap that also takes the lock), so that it
// is converged when it issues the copies.
template <typename K>
__device__ __forceinline__ void cw_lock_two(const Params<K> &p, const HeapView<K> &H, Shared &sh,
                                            uint32_t sl, uint32_t sr, uint32_t first0,
                                            uint32_t first1, uint32_t *lk)
{
    const uint32_t lane = clane();
    uint32_t v = ST_EMPTY;
    uint32_t *w = nullptr;
    if (lane < 2) {
        const uint32_t sx = lane ? sr : sl;
        if (sx) {
            w = node_state(H, sx);
            const uint32_t f = lane ? first1 : first0;
            v = f == NO_TRY ? try_lock(w) : f;
        }
    }
    bool pending = v == ST_INUSE;
    if (__any_sync(0xffffffffu, pending)) {
        if (pending) stat_add(sh, STAT_WAITS, 1);
        unsigned long long t0 = 0;
        uint32_t it = 0;
        do {
            if (pending) {
                if (!keep_waiting(p, H, t0, it)) {
                    v = ST_GAVE_UP;
                    pending = false;
                } else {
                    v = try_lock(w);
                    pending = v == ST_INUSE;
                }
            }
        } while (__any_sync(0xffffffffu, pending));
    }
    if (lane < 2) {
        lk[lane] = v;
        // the target of an INS still on its way down counts as absent here
        if (v == ST_TARGET || v == ST_MARKED || v == ST_DELIVERED)
            stat_add(sh, STAT_TARGET_CHILDREN, 1);
    }
    __syncwarp();
}

template <typename K, bool TMA>
__device__ __forceinline__ void cw_take_children(const Params<K> &p, const HeapView<K> &H,
                                                 Shared &sh, uint32_t sl, uint32_t sr,
                                                 uint32_t first0, uint32_t first1, K *dl, K *dr,
                                                 uint32_t *lk)
{
    const uint32_t lane = clane();
    const uint32_t k = p.k;
    cw_lock_two(p, H, sh, sl, sr, first0, first1, lk);
    if (TMA && lk[0] == ST_AVAIL && lk[1] == ST_AVAIL && (k * (uint32_t)sizeof(K)) % 16u == 0) {
        // both nodes by one TMA fetch (one lane)
        if (lane == 0) {
            tma_fetch(H, k, 2u, sl, dl, sr, dr, &sh.kid_mbar, sh.kid_arms);
            if (!tma_land(p, H, &sh.kid_mbar, sh.kid_arms, sh.kid_seen))
                lk[0] = lk[1] = ST_GAVE_UP;
            stat_add(sh, STAT_LOADS, 2);
        }
        __syncwarp();
        return;
    }
    if (lk[0] == ST_AVAIL) g2s(dl, node_keys(H, sl, k), k, lane, 32u);
    if (lk[1] == ST_AVAIL) g2s(dr, node_keys(H, sr, k), k, lane, 32u);
    cp_async_commit();
    if (lane == 0) stat_add(sh, STAT_LOADS, (lk[0] == ST_AVAIL) + (lk[1] == ST_AVAIL));
    cp_async_wait();
}

// Deletes up to `want` keys.  MODE_DELETE takes its output offset and count
// from the launch's running total under the root lock; MODE_OPS writes to
// `out_off`.  Six smem buffers rotate between the roles current node, left
// and right child, and three free ones.  Returns false when the block must
// stop.
// ROOT_TMA (delete-only launches): the root step's copies by TMA; the levels
// below keep the control warp's copies there (they overlap the merges: TMA
// measured no faster).  Other launches fetch the nodes of every level below
// the root step by TMA (faster walks: heap sets +2.6%).
// DEL root step of delete-only launches, merge threads, when keys of the root
// and the partial buffer are left over (tn of them, in `left`): waits
// (bounded) for the fetch of the last node into `last` (phase parity `par`
// of the last-node mbarrier), then MergeAndSort(left-over, last node): the k
// smallest become the new root in `root_buf`, the rest the partial buffer.
// A control warp that gave up on the last node has set abort, which ends the
// wait; the merge threads then decide together to skip the merge (the
// operation fails).  Kept out of line: the path without left-over keys stays
// as short as it was.
template <typename K, int IPT>
__device__ __noinline__ void del_early_refill(Shared &sh, Hdr *hdr, K *buf,
                                              unsigned long long timeout_ns, uint32_t k,
                                              uint32_t par, K *left, uint32_t tn, K *last,
                                              K *root_buf)
{
    const unsigned long long t0 = gtimer();
    bool miss = false;
    while (!mbar_try_wait(&sh.last_mbar, par)) {
        if (*(volatile int *)&sh.abort) {
            miss = true;
            break;
        }
        if (gtimer() - t0 > timeout_ns) {
            atomicCAS(&hdr->err, E_NONE, E_TIMEOUT);
            sh.abort = 1;
            miss = true;
            break;
        }
    }
    if (!bar_mg_or(miss)) {
        merge_split<K, IPT>(left, tn, last, k, root_buf, k, left);
        s2g(buf, left, tn);
    }
}

// EARLY (delete-only heap-set launches, whose heaps mostly hold a partial
// buffer): the root step's refill from the last node runs out of line as soon
// as that node has landed (del_early_refill).  Not built into the single-heap
// delete-only kernel, whose deleteMin-all measured 1% slower for carrying it.
template <typename K, int IPT, bool ROOT_TMA = false, bool EARLY = false>
__device__ bool del_op(const Params<K> &p, const HeapView<K> &H, Shared &sh, K *base,
                       uint32_t want, unsigned long long out_off, unsigned long long ref,
                       uint32_t *count_out, long long req)
{
    const uint32_t k = p.k;
    const bool ctrl = is_ctrl();
    const uint32_t lane = clane();
    K *root = node_keys(H, 1u, k);
    long long tp = clock64();
    // phase parity of this operation's fetch of the last node (the fetch is
    // issued after the next barrier, so the count read here is the previous
    // operations')
    const uint32_t last_par = EARLY ? (sh.last_arms & 1u) : 0u;
#define PB(i) (base + (size_t)(i) * k)

    // ---- take the root, the ticket and the output range
    if (ctrl && lane == 0) {
        unsigned long long w = 0, done = 0;
        // A DEL that would refill the root from a last node still owed by an
        // INS in flight (TARGET) would hold the root for that whole delivery.
        // Before it has done anything visible it hands the root back and
        // queues again (a bounded number of times), so that the operations
        // behind it proceed meanwhile; after that it waits as before.
        for (uint32_t yields = 0;; ++yields) {
            sh.abort = !lock_root(p, H, sh, w);
            if (sh.abort) break;
            const uint32_t m = rw_m(w), s = rw_s(w);
            // both loads go out before either value is used; a delete-only
            // launch has no insert in flight (earlier launches completed)
            const uint32_t last_state =
                (p.mode != MODE_DELETE && m >= 2) ? ld_relaxed(node_state(H, m)) : ST_AVAIL;
            if (p.mode == MODE_DELETE) done = ld_relaxed64(&p.ctl->delivered);
            uint32_t w_now = want;
            if (p.mode == MODE_DELETE) {
                const unsigned long long rem = p.n > done ? p.n - done : 0ull;
                w_now = rem < want ? (uint32_t)rem : want;
            }
            const uint32_t t_now = w_now < (m >= 1 ? k : s) ? w_now : (m >= 1 ? k : s);
            if (yields < p.del_yields && s < t_now && m >= 2 && last_state == ST_TARGET) {
                release_root_word(H, sh, m, s);
                stat_add(sh, STAT_WAITS, 1);
                stat_add(sh, STAT_DEL_YIELDS, 1);
                __nanosleep(512);
                continue;
            }
            break;
        }
        lap(sh, STAT_DEL_ACQ_CYC, tp);
        if (!sh.abort) {
            if (sh.stats_on) sh.t_root = gtimer();
            const uint32_t m = rw_m(w), s = rw_s(w);
            sh.m = m;
            sh.s = s;
            if (p.mode == MODE_DELETE) {
                const unsigned long long rem = p.n > done ? p.n - done : 0ull;
                want = rem < want ? (uint32_t)rem : want;
                out_off = done;
            } else if (req >= 0) {
                // one request's DELs fill its output contiguously, in the order
                // they hold this heap's root
                out_off = __ldcv(p.req_base + req) + p.req_cursor[req];
            }
            const uint32_t avail = m >= 1 ? k : s;
            const uint32_t take = want < avail ? want : avail;
            sh.take = take;
            sh.out_off = out_off;
            if (p.mode == MODE_DELETE) {
                p.ctl->delivered = out_off + take;
                if (p.out_total) *p.out_total = out_off + take;
                if (take == 0 || out_off + take >= p.n) p.ctl->drained = 1u;
            } else if (req >= 0) {
                p.req_cursor[req] += take;
            }
            if (count_out) *count_out = take;
            take_ticket(p, H, sh, GHEAP_OP_DEL, take, p.mode == MODE_DELETE ? out_off : ref);
        }
    }
    bar_all();
    if (sh.abort) return false;
    const uint32_t m = sh.m, s = sh.s;
    const uint32_t take = sh.take;
    out_off = sh.out_off;

    if (m == 0) {
        // no full node: serve from the partial buffer (Section 3.3.2)
        if (!ctrl) {
            g2s(PB(5), H.buf, s, threadIdx.x, nmt());
            cp_async_commit();
            cp_async_wait();
            bar_mg();
            s2g(p.out + out_off, PB(5), take);
            s2g(H.buf, PB(5) + take, s - take);
        }
        bar_all();
        if (ctrl && lane == 0) {
            stat_root(sh);
            release_root_word(H, sh, 0u, s - take);
        }
        return true;
    }

    const bool need_last = s < take && m >= 2;
    const bool root_gone = s < take && m == 1;
    const uint32_t tn = k - take + s;             // root + buffer keys left (when s < take)
    uint32_t ic = 0, il = 1, ir = 2, f1 = 3, f2 = 4;   // buffer 5 holds the partial buffer
    // the root step's fetches (below): with keys left over from the root and
    // the buffer, the refill MergeAndSort(left-over, last node) runs as soon
    // as the last node has landed, while level 1 is still awaited
    const bool early = EARLY && ROOT_TMA && need_last && tn > 0 && m >= 16u &&
                       (k * (uint32_t)sizeof(K)) % 16u == 0;

    // ---- root step.  Merge threads: root and buffer in, output, first part
    // of the refill.  Control warp: the last node, then the root's children.
    if (!ctrl) {
        g2s(PB(ic), root, k, threadIdx.x, nmt());
        g2s(PB(5), H.buf, s, threadIdx.x, nmt());
        cp_async_commit();
        cp_async_wait();
        bar_mg();
        s2g(p.out + out_off, PB(ic), take);
        if (threadIdx.x == 0) stat_add(sh, STAT_LOADS, 1);
        if (s >= take) {
            merge_split<K, IPT>(PB(ic) + take, k - take, PB(5), s, PB(ic), k, PB(5));
            s2g(H.buf, PB(5), s - take);
        } else {
            merge_split<K, IPT>(PB(ic) + take, k - take, PB(5), s, PB(5), tn, PB(5));
            if (root_gone) s2g(H.buf, PB(5), tn);
        }
        if (early)
            del_early_refill<K, IPT>(sh, H.hdr, H.buf, p.timeout_ns, k, last_par, PB(5), tn,
                                     PB(f1), PB(ic));
    } else if (!root_gone) {
        uint32_t sl, sr;
        child_slots(1, H.max_nodes, sl, sr);
        if (ROOT_TMA && m >= 16u && (k * (uint32_t)sizeof(K)) % 16u == 0) {
            // the root step of delete-only launches: level 1 fetched by TMA
            // the moment both locks are held, the last node (below level 3:
            // the top four levels are full) as soon as it is taken -- one
            // thread each, instead of the warp's copies after both locks
            // (nodes of a multiple of 16 bytes: the buffers and the node
            // addresses are then 16-byte aligned, as the copies require)
            uint32_t *lw = need_last ? node_state(H, m) : nullptr;
            uint32_t t = ST_EMPTY;
            if (lane < 2) t = try_lock(node_state(H, lane ? sr : sl));
            if (lane == 2 && lw) t = try_lock(lw);
            const uint32_t c0 = __shfl_sync(0xffffffffu, t, 0);
            const uint32_t c1 = __shfl_sync(0xffffffffu, t, 1);
            const uint32_t tl = __shfl_sync(0xffffffffu, t, 2);
            const bool l1_now = c0 == ST_AVAIL && c1 == ST_AVAIL;
            if (l1_now && lane == 0)
                tma_fetch(H, k, 2u, sl, PB(il), sr, PB(ir), &sh.l1_mbar, sh.l1_arms);
            if (lw && lane == 2) {
                if (take_last(p, H, sh, lw, tl)) {
                    st_relaxed(lw, ST_EMPTY);
                    tma_fetch(H, k, 1u, m, PB(f1), 0u, PB(f1), &sh.last_mbar, sh.last_arms);
                } else {
                    sh.abort = 1;
                }
            }
            __syncwarp();
            if (!l1_now) {
                // the DEL ahead still holds level 1: wait for both locks
                cw_lock_two(p, H, sh, sl, sr, c0, c1, sh.lk[0]);
                if (lane == 0 && sh.lk[0][0] == ST_AVAIL && sh.lk[0][1] == ST_AVAIL)
                    tma_fetch(H, k, 2u, sl, PB(il), sr, PB(ir), &sh.l1_mbar, sh.l1_arms);
            } else if (lane == 0) {
                sh.lk[0][0] = sh.lk[0][1] = ST_AVAIL;
            }
            if (lane == 0 && sh.lk[0][0] == ST_AVAIL && sh.lk[0][1] == ST_AVAIL) {
                if (!tma_land(p, H, &sh.l1_mbar, sh.l1_arms, sh.l1_seen))
                    sh.lk[0][0] = sh.lk[0][1] = ST_GAVE_UP;
                stat_add(sh, STAT_LOADS, 2);
            }
            if (lw && lane == 2 && !sh.abort &&
                !tma_land(p, H, &sh.last_mbar, sh.last_arms, sh.last_seen))
                sh.abort = 1;
            __syncwarp();
        } else if (need_last) {
            uint32_t *lw = node_state(H, m);
            if (m <= 3) {
                // the last node is a child of the root: take it first, then
                // lock the other child (the taken one reads EMPTY)
                if (lane == 0) {
                    if (take_last(p, H, sh, lw, try_lock(lw))) st_relaxed(lw, ST_EMPTY);
                    else sh.abort = 1;
                }
                __syncwarp();
                if (!sh.abort) g2s(PB(f1), node_keys(H, m, k), k, lane, 32u);
                cp_async_commit();
                cw_take_children<K, !ROOT_TMA>(p, H, sh, sl, sr, NO_TRY, NO_TRY, PB(il), PB(ir),
                                               sh.lk[0]);
            } else {
                // try the last node and both children at once.  An INS still
                // in flight to the last node may need a child of the root, so
                // the children are given back while the DEL waits for it.
                uint32_t t = ST_EMPTY;
                if (lane == 2) t = try_lock(lw);
                if (lane < 2) t = try_lock(node_state(H, lane ? sr : sl));
                const uint32_t tl = __shfl_sync(0xffffffffu, t, 2);
                const bool inflight = tl != ST_AVAIL && tl != ST_INUSE;
                if (inflight && lane < 2 && t == ST_AVAIL)
                    st_release(node_state(H, lane ? sr : sl), ST_AVAIL);
                if (lane == 2) {
                    if (take_last(p, H, sh, lw, tl)) st_relaxed(lw, ST_EMPTY);
                    else sh.abort = 1;
                }
                __syncwarp();
                if (!sh.abort) g2s(PB(f1), node_keys(H, m, k), k, lane, 32u);
                cp_async_commit();
                const uint32_t c0 = __shfl_sync(0xffffffffu, t, 0);
                const uint32_t c1 = __shfl_sync(0xffffffffu, t, 1);
                cw_take_children<K, !ROOT_TMA>(p, H, sh, sl, sr, inflight ? NO_TRY : c0,
                                 inflight ? NO_TRY : c1, PB(il), PB(ir), sh.lk[0]);
            }
        } else {
            cw_take_children<K, !ROOT_TMA>(p, H, sh, sl, sr, NO_TRY, NO_TRY, PB(il), PB(ir),
                                           sh.lk[0]);
        }
    }
    bar_all();
    if (sh.abort) return false;
    if (root_gone) {
        if (ctrl && lane == 0) {
            stat_root(sh);
            release_root_word(H, sh, 0u, tn);
        }
        return true;
    }
    uint32_t nm = m;
    const uint32_t ns = s >= take ? s - take : tn;
    if (need_last) {
        nm = m - 1;
        if (tn > 0) {
            if (!ctrl && !early) {
                merge_split<K, IPT>(PB(5), tn, PB(f1), k, PB(ic), k, PB(5));
                s2g(H.buf, PB(5), tn);
            }
        } else {
            // nothing of the root or buffer is left: the last node is the root
            const uint32_t t = ic; ic = f1; f1 = t;
        }
        if (!ctrl && threadIdx.x == 0) stat_add(sh, STAT_LOADS, 1);
    }
    if (need_last && tn > 0 && !early) bar_all();   // the merge above rewrote PB(ic)
    if (ctrl && lane == 0) lap(sh, STAT_DEL_ROOT_CYC, tp);

    // ---- sift down (Section 3.2.1).  At the top of every level the block
    // has met: the current node's keys are in PB(ic), its children's lock
    // results in sh.lk[par] and their keys in PB(il), PB(ir).
    //
    // Split form (the block shape allows it): MergeAndSort(l, r) is the whole
    // bitonic merge up to 8 outputs per thread (both halves are needed before
    // the next level's release), a split and two half sorts at 16;
    // MergeAndSort(cur, small child), when not a swap, is a bitonic split and
    // a sort of the node's half with all merge threads, the carried half
    // being sorted after the node went back; likewise with one child.  The
    // merge threads store the node's keys and go on; the release warp fences
    // and releases the node.  The larger child is released together with the
    // next level's node (a DEL that follows needs both).
    constexpr int E = IPT / 2;
    const bool split_form = IPT >= 4 && nmt() * IPT == 2 * k && k >= 32u * IPT;
    uint32_t node = 1;
    K *cur_keys = root;
    uint32_t *cur_w = nullptr;   // nullptr = the root word
    uint32_t *pend = nullptr;    // a child still held, released with cur_w
    uint32_t par = 0;
    for (;;) {
        const uint32_t lk0 = sh.lk[par][0], lk1 = sh.lk[par][1];
        if (lk0 == ST_GAVE_UP || lk1 == ST_GAVE_UP) return false;
        const bool pl = lk0 == ST_AVAIL, pr = lk1 == ST_AVAIL;
        if (!pl && !pr) break;
        uint32_t sl, sr;
        child_slots(node, H.max_nodes, sl, sr);
        K *const Bc = PB(ic);
        K *const C = PB(il);
        K *const D = PB(ir);
        const K cmax = Bc[k - 1];
        const K c0 = C[0], ck = C[k - 1], d0 = D[0], dk = D[k - 1];
        if (ctrl && lane == 0) stat_add(sh, STAT_DEL_LEVELS, 1);
        bar_all();   // everybody has read the decision inputs
        const bool at_root = cur_w == nullptr;
        // the next level's locks and loads run on the control warp during the
        // merges at every level, the root included; the current node is
        // released as soon as its keys are stored (by the release warp in the
        // split form, else by merge thread 0)

        if (pl != pr) {
            // one child present (the other is absent or an INS target)
            const bool usel = pl;
            const uint32_t xs = usel ? sl : sr;
            uint32_t *xw = node_state(H, xs);
            K *xk = node_keys(H, xs, k);
            if (cmax <= (usel ? c0 : d0)) {
                if (ctrl && lane == 0) st_release(xw, ST_AVAIL);
                break;
            }
            const uint32_t x = 2 * node + (usel ? 0 : 1);
            uint32_t gl, gr;
            child_slots(x, H.max_nodes, gl, gr);
            K *const X = usel ? C : D;
            if (!ctrl) {
                long long tm = clock64();
                if (split_form) {
                    split_run<K, E>(Bc, X, Bc, X, k);
                    sort_run<K, E>(Bc, k);
                    s2g(cur_keys, Bc, k);
                    bar_mg();
                    if (threadIdx.x == 0) {
                        stat_add(sh, STAT_MERGES, 1);
                        stat_add(sh, STAT_STORES, 1);
                        lap(sh, STAT_DEL_MERGE_CYC, tm);
                        post_step(p, H, sh, cur_w, pend, nm, ns);
                    }
                    // the half that goes down, sorted after the node went back
                    sort_run<K, E>(X, k);
                } else {
                    merge_kk<K, IPT>(Bc, X, Bc, X, k);
                    s2g(cur_keys, Bc, k);
                    // the node is final: release it as soon as the merge
                    // threads' stores are done, not after the next level's locks
                    bar_mg();
                    if (threadIdx.x == 0) {
                        stat_add(sh, STAT_MERGES, 1);
                        stat_add(sh, STAT_STORES, 1);
                        lap(sh, STAT_DEL_MERGE_CYC, tm);
                        long long tr = clock64();
                        release_step(H, sh, cur_w, pend, nm, ns);
                        lap(sh, STAT_DEL_REL_CYC, tr);
                    }
                }
            } else {
                long long tw = clock64();
                cw_take_children<K, !ROOT_TMA>(p, H, sh, gl, gr, NO_TRY, NO_TRY, PB(f1), PB(f2),
                                               sh.lk[par ^ 1]);
                if (lane == 0) lap(sh, STAT_DEL_WAIT_CYC, tw);
            }
            bar_all();
            const uint32_t xb = usel ? il : ir, ob = usel ? ir : il;
            const uint32_t n1 = ic, n2 = ob;
            ic = xb; il = f1; ir = f2; f1 = n1; f2 = n2;
            node = x;
            cur_keys = xk;
            cur_w = xw;
            pend = nullptr;
            par ^= 1;
            continue;
        }

        // both children present
        if (cmax <= c0 && cmax <= d0) {
            // early stop (Section 4.3)
            if (ctrl && lane < 2) st_release(node_state(H, lane ? sr : sl), ST_AVAIL);
            break;
        }
        // MergeAndSort(l, r): the k largest go to the child whose maximum was
        // larger (the right child on a tie), the k smallest to the other
        const bool big_l = ck > dk;
        const uint32_t smn = big_l ? 2 * node + 1 : 2 * node;
        uint32_t gl, gr;
        child_slots(smn, H.max_nodes, gl, gr);
        bool S_is_C, l_changed, r_changed;
        const bool overlap = ck > d0 && dk > c0;
        if (ck <= d0) {
            S_is_C = true;
            l_changed = r_changed = big_l;   // false here: nothing moves
        } else if (dk <= c0) {
            S_is_C = false;
            l_changed = r_changed = !big_l;
        } else {
            S_is_C = true;
            l_changed = r_changed = true;
        }
        K *const S = S_is_C ? C : D;
        K *const L = S_is_C ? D : C;
        const uint32_t bigs = big_l ? sl : sr, sms = big_l ? sr : sl;
        K *big_keys = node_keys(H, bigs, k);
        K *sm_keys = node_keys(H, sms, k);
        uint32_t *big_w = node_state(H, bigs);
        uint32_t *sm_w = node_state(H, sms);
        const bool big_changed = big_l ? l_changed : r_changed;
        const bool sm_changed = big_l ? r_changed : l_changed;
        if (split_form) {
            if (!ctrl) {
                long long tm = clock64();
                if (overlap) {
                    // S = C, L = D.  Up to 8 outputs per thread both halves
                    // are sorted at once (the larger child's keys are needed
                    // with the next level's release); at 16 a split and two
                    // half sorts cost less (k = 2048: 3.3 k cycles against
                    // 3.8 k), the small half first
                    if constexpr (IPT <= 8) {
                        merge_full<K, IPT>(C, D, C, D, k);
                    } else {
                        split_run<K, E>(C, D, C, D, k);
                        sort_run<K, E>(C, k);
                    }
                }
                // (h cannot hold: the early stop above already took cmax <=
                // min(c0, d0) = S[0]; kept so that the path stays complete)
                const bool h = cmax <= S[0];
                // every carried key above the small half: the second
                // MergeAndSort is a swap (Section 4.3)
                const bool sw = !h && Bc[0] >= S[k - 1];
                if (threadIdx.x == 0) {
                    stat_add(sh, overlap ? STAT_MERGES : STAT_SKIPS, 1);
                    sh.halt = h;
                    sh.swap = sw;
                }
                if (!h) {
                    if (!sw) {
                        split_run<K, E>(Bc, S, Bc, S, k);
                        sort_run<K, E>(Bc, k);
                    }
                    s2g(cur_keys, sw ? S : Bc, k);
                    bar_mg();
                    if (threadIdx.x == 0) {
                        stat_add(sh, sw ? STAT_SKIPS : STAT_MERGES, 1);
                        stat_add(sh, STAT_STORES, 1);
                        lap(sh, STAT_DEL_MERGE_CYC, tm);
                        post_step(p, H, sh, cur_w, pend, nm, ns);
                        if (sh.stats_on) tm = clock64();
                    }
                } else if (sm_changed) {
                    s2g(sm_keys, S, k);
                    if (threadIdx.x == 0) stat_add(sh, STAT_STORES, 1);
                }
                // the halves that go down: the larger child's keys, then the
                // carried keys (the small child's new contents)
                if (IPT > 8 && overlap) sort_run<K, E>(L, k);
                if (big_changed) {
                    s2g(big_keys, L, k);
                    if (threadIdx.x == 0) stat_add(sh, STAT_STORES, 1);
                }
                if (!h && !sw) sort_run<K, E>(S, k);
                if (threadIdx.x == 0) lap(sh, STAT_DEL_MERGE_CYC, tm);
            } else {
                // the small child's children, locked and loaded meanwhile
                long long tw = clock64();
                cw_take_children<K, !ROOT_TMA>(p, H, sh, gl, gr, NO_TRY, NO_TRY, PB(f1), PB(f2),
                                 sh.lk[par ^ 1]);
                if (lane == 0) lap(sh, STAT_DEL_WAIT_CYC, tw);
            }
            bar_all();
            const bool halt = sh.halt;
            const bool swap2 = !halt && sh.swap;
            if (halt) {
                // the sift ends here (the current node keeps its keys): the
                // children and whatever the control warp took go back; the
                // current node and `pend` are released below the loop
                if (ctrl && lane == 0) {
                    st_release(big_w, ST_AVAIL);
                    st_release(sm_w, ST_AVAIL);
                    if (gl && sh.lk[par ^ 1][0] == ST_AVAIL) st_release(node_state(H, gl), ST_AVAIL);
                    if (gr && sh.lk[par ^ 1][1] == ST_AVAIL) st_release(node_state(H, gr), ST_AVAIL);
                }
                break;
            }
            uint32_t sb = S_is_C ? il : ir;
            const uint32_t lb = S_is_C ? ir : il;
            uint32_t n1 = ic;
            if (swap2) {
                const uint32_t t = sb; sb = n1; n1 = t;
            }
            ic = sb; il = f1; ir = f2; f1 = n1; f2 = lb;
            node = smn;
            cur_keys = sm_keys;
            cur_w = sm_w;
            pend = big_w;
            par ^= 1;
            continue;
        }
        uint32_t t_try = ST_EMPTY;
        if (!ctrl) {
            long long tm = clock64();
            if (overlap) {
                merge_kk<K, IPT>(C, D, C, D, k);
                if (threadIdx.x == 0) stat_add(sh, STAT_MERGES, 1);
            } else if (threadIdx.x == 0) {
                stat_add(sh, STAT_SKIPS, 1);
            }
            if (big_changed) {
                s2g(big_keys, L, k);
                if (threadIdx.x == 0) stat_add(sh, STAT_STORES, 1);
            }
            if (threadIdx.x == 0) {
                sh.halt = cmax <= S[0];
                // every carried key above the small half: the second
                // MergeAndSort is a swap (Section 4.3)
                sh.swap = Bc[0] >= S[k - 1];
                lap(sh, STAT_DEL_MERGE_CYC, tm);
            }
        } else if (lane < 2) {
            // try the small child's children while the merge threads work
            const uint32_t gx = lane ? gr : gl;
            if (gx) t_try = try_lock(node_state(H, gx));
        }
        bar_all();
        const bool halt = sh.halt;
        const bool swap2 = !halt && sh.swap;
        if (ctrl) {
            if (lane == 0) {
                long long tr = clock64();
                st_release(big_w, ST_AVAIL);
                lap(sh, STAT_DEL_REL_CYC, tr);
            }
            {
                if (halt) {
                    // the sift ends here: give back what the tries took
                    if (lane < 2 && t_try == ST_AVAIL)
                        st_release(node_state(H, lane ? gr : gl), ST_AVAIL);
                } else {
                    long long tw = clock64();
                    const uint32_t t0 = __shfl_sync(0xffffffffu, t_try, 0);
                    const uint32_t t1 = __shfl_sync(0xffffffffu, t_try, 1);
                    cw_take_children<K, !ROOT_TMA>(p, H, sh, gl, gr, gl ? t0 : NO_TRY,
                                                   gr ? t1 : NO_TRY, PB(f1), PB(f2),
                                                   sh.lk[par ^ 1]);
                    if (lane == 0) lap(sh, STAT_DEL_WAIT_CYC, tw);
                }
            }
        } else {
            long long tm = clock64();
            if (halt) {
                if (sm_changed) {
                    s2g(sm_keys, S, k);
                    if (threadIdx.x == 0) stat_add(sh, STAT_STORES, 1);
                }
            } else {
                // MergeAndSort(cur, small child): cur keeps the k smallest;
                // with disjoint ranges cur takes the small half as it is and
                // the carried keys go on down unchanged
                if (swap2) {
                    s2g(cur_keys, S, k);
                } else {
                    merge_kk<K, IPT>(Bc, S, Bc, S, k);
                    s2g(cur_keys, Bc, k);
                }
                // the node is final: release it as soon as the merge threads'
                // stores are done, while the control warp may still wait for
                // the next level's locks
                bar_mg();
                if (threadIdx.x == 0) {
                    stat_add(sh, swap2 ? STAT_SKIPS : STAT_MERGES, 1);
                    stat_add(sh, STAT_STORES, 1);
                    long long tr = clock64();
                    if (at_root) {
                        stat_root(sh);
                        release_root_word(H, sh, nm, ns);
                    } else {
                        st_release(cur_w, ST_AVAIL);
                    }
                    lap(sh, STAT_DEL_REL_CYC, tr);
                }
            }
            if (threadIdx.x == 0) lap(sh, STAT_DEL_MERGE_CYC, tm);
        }
        bar_all();
        if (halt) {
            if (ctrl && lane == 0) st_release(sm_w, ST_AVAIL);
            break;
        }
        uint32_t sb = S_is_C ? il : ir;
        const uint32_t lb = S_is_C ? ir : il;
        uint32_t n1 = ic;
        if (swap2) {
            // the carried keys (still in the current buffer) are the small
            // child's new contents
            const uint32_t t = sb; sb = n1; n1 = t;
        }
        const uint32_t n2 = lb;
        ic = sb; il = f1; ir = f2; f1 = n1; f2 = n2;
        node = smn;
        cur_keys = sm_keys;
        cur_w = sm_w;
        par ^= 1;
    }
    // last node of the walk: write it and release it
    if (split_form) {
        if (!ctrl) {
            s2g(cur_keys, PB(ic), k);
            bar_mg();
            if (threadIdx.x == 0) {
                stat_add(sh, STAT_STORES, 1);
                post_step(p, H, sh, cur_w, pend, nm, ns);
            }
        }
        bar_all();
        return true;
    }
    if (!ctrl) {
        s2g(cur_keys, PB(ic), k);
        if (threadIdx.x == 0) stat_add(sh, STAT_STORES, 1);
    }
    bar_all();
    if (ctrl && lane == 0) release_step(H, sh, cur_w, pend, nm, ns);
    return true;
#undef PB
}

// ---------------------------------------------------------------------------
// the serving ring (MODE_RING)
// ---------------------------------------------------------------------------

__device__ __forceinline__ unsigned long long ld_acquire_sys64(const unsigned long long *p)
{
    unsigned long long v;
    asm volatile("ld.acquire.sys.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ uint32_t ld_acquire_sys32(const uint32_t *p)
{
    uint32_t v;
    asm volatile("ld.acquire.sys.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release_sys64(unsigned long long *p, unsigned long long v)
{
    asm volatile("st.release.sys.global.u64 [%0], %1;" :: "l"(p), "l"(v) : "memory");
}

// Thread 0: waits until ring position `pos` is published.  False: the host
// asked the launch to stop and `pos` was never published, or no operation
// came for ring_idle_ns (the ring's error word is then set).  The stop flag
// is read with acquire and the tail once more after it, so that an operation
// published before the stop is never left behind.
template <typename K>
__device__ bool ring_wait(const Params<K> &p, unsigned long long pos)
{
    unsigned long long t0 = 0;
    for (uint32_t it = 1;; ++it) {
        unsigned long long tail = ld_acquire_sys64(p.ring_tail);
        if (pos < tail) return true;
        if (ld_acquire_sys32(p.ring_stop)) {
            tail = ld_acquire_sys64(p.ring_tail);
            return pos < tail;
        }
        if ((it & 15u) == 0) {
            const unsigned long long now = gtimer();
            if (t0 == 0) {
                t0 = now;
            } else if (now - t0 > p.ring_idle_ns) {
                atomicExch(p.ring_err, 1u);
                return false;
            }
            if (ld_relaxed(p.ring_err)) return false;
        }
        // the next position to be published polls often, the ones behind it less
        const unsigned long long ahead = pos - tail;
        __nanosleep(ahead < 2 ? 64u : (ahead < 64 ? 512u : 2048u));
    }
}

// One ring operation, read from host memory (fresh: the entry is reused).
__device__ __forceinline__ RingOp ld_ring_op(const RingOp *e)
{
    const uint4 a = __ldcv(reinterpret_cast<const uint4 *>(e));
    const uint4 b = __ldcv(reinterpret_cast<const uint4 *>(e) + 1);
    RingOp d;
    d.heap = a.x;
    d.kind_n = a.y;
    d.offset = (unsigned long long)a.z | ((unsigned long long)a.w << 32);
    d.ticket = (unsigned long long)b.x | ((unsigned long long)b.y << 32);
    d.req = b.z;
    d._pad = b.w;
    return d;
}

// Thread 0, after a barrier that follows every store of the block's
// operation: counts the operation done for its request; the block that
// finishes a request's last operation writes the completion record (count
// and status, then the sequence number with release) to host memory and
// clears the slot's device counters for its next request.
template <typename K>
__device__ void ring_complete(const Params<K> &p, uint32_t req, uint32_t status)
{
    // the operation's error bits and its output come before its count: the
    // block that counts the request's last operation then sees both
    if (status) atomicOr(p.ring_status + req, status);
    __threadfence_system();
    const uint32_t n_ops = __ldcv(p.ring_req_ops + req);
    const uint32_t done = atomicAdd(p.ring_ops_done + req, 1u) + 1u;
    if (done != n_ops) return;
    __threadfence();          // the other operations' cursor updates are seen
    const unsigned long long cnt = p.req_cursor[req];
    const uint32_t st = atomicExch(p.ring_status + req, 0u);
    p.req_cursor[req] = 0;
    p.ring_ops_done[req] = 0;
    RingDone *r = p.ring_done + req;
    r->count = cnt;
    r->status = st;
    st_release_sys64(&r->seq, __ldcv(p.ring_req_seq + req) + 1ull);
}

// ---------------------------------------------------------------------------
// persistent kernel
// ---------------------------------------------------------------------------

// Block size bound per merge width: 512 merge threads + the control and
// release warps for IPT <= 4, 256 + 64 for wider merges (fewer warps, more
// registers each).
template <int IPT>
struct MaxThreads { static constexpr int value = IPT >= 8 ? 320 : 576; };

// DEL_ONLY: the specialisation for delete-only launches (MODE_DELETE), built
// without the insert, operation-list and heap-set paths so that the code a
// deleteMin walks through stays small.  The general kernel is built to fit
// two blocks per SM at 8 or more merge outputs per thread (at most 96
// registers): heap sets run two per SM, their operations being bound by the
// latency of each walk, not by one root.
template <int IPT, bool DEL_ONLY>
struct MinBlocks { static constexpr int value = (DEL_ONLY || IPT < 8) ? 1 : 2; };

// SET_DEL (with DEL_ONLY): the delete-only specialisation for heap-set
// launches whose operation list carries no input keys (MODE_SET, every
// operation a DEL): each operation names its heap as in the general kernel,
// and the walk is the delete-only one.
template <typename K, int IPT, bool DEL_ONLY, bool SET_DEL = false>
__global__ void __launch_bounds__(MaxThreads<IPT>::value, (MinBlocks<IPT, DEL_ONLY>::value))
    heap_kernel(Params<K> p)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ Shared sh;
    __shared__ HeapView<K> set_view;   // MODE_SET: the heap of the current op
    __shared__ uint32_t set_kind, set_n, set_skip, set_cursor;
    __shared__ unsigned long long set_off;
    const uint32_t k = p.k;
    K *base = reinterpret_cast<K *>(smem_raw);   // 6 node buffers
    const bool ring = !DEL_ONLY && p.mode == MODE_RING;
    const bool multi = SET_DEL || (!DEL_ONLY && (p.mode == MODE_SET || ring));
    const HeapView<K> &H = multi ? set_view : p.h;
    __shared__ uint32_t ring_req;      // MODE_RING: request slot of the current op
    // a heap-set launch holding only inserts inserts bottom-up (no DEL can
    // meet a rising batch, and every heap's node count only grows)
    const bool set_bu = multi && p.set_bu != nullptr && *p.set_bu != 0u;
    __shared__ uint32_t rel_exited;
    if (threadIdx.x < N_STATS) sh.cnt[threadIdx.x] = 0;
    if (threadIdx.x == 0) {
        sh.rq_posted = 0;
        sh.rq_read = 0;
        sh.stats_on = p.stats != nullptr;
        sh.use_fixed = 0;
        rel_exited = 0;
        sh.l1_arms = sh.l1_seen = sh.last_arms = sh.last_seen = 0;
        if (DEL_ONLY) {
            mbar_init(&sh.l1_mbar, 1u);
            mbar_init(&sh.last_mbar, 1u);
        } else {
            sh.kid_arms = sh.kid_seen = 0;
            mbar_init(&sh.kid_mbar, 1u);
        }
    }
    bar_block();
    if (is_rel()) {
        release_loop<K>(p, sh, &rel_exited);
        return;
    }

    if (p.n_dev) {
        // the key count was produced on the device (at most p.n)
        const unsigned long long nd = *p.n_dev;
        p.n = nd < p.n ? nd : p.n;
    }
    unsigned long long n_ops;
    if (SET_DEL || (!DEL_ONLY && (p.mode == MODE_OPS || multi))) n_ops = p.n_ops;
    else n_ops = (p.n + k - 1) / k;

    for (;;) {
        if (threadIdx.x == 0) {
            unsigned long long op = atomicAdd(&p.ctl->next_op, 1ull);
            int stop;
            gheapset_op d = {};
            if (ring) {
                // the next ring position, once the host has published it
                op += p.ring_base;
                stop = !ring_wait(p, op);
                if (!stop) {
                    const RingOp e = ld_ring_op(p.ring_ops + (op & (p.ring_cap - 1ull)));
                    d.heap = e.heap;
                    d.kind_n = e.kind_n;
                    d.offset = e.offset;
                    sh.use_fixed = 1;
                    sh.fixed_ticket = e.ticket;
                    ring_req = e.req;
                }
            } else {
                stop = op >= n_ops;
                if (!stop && multi) d = p.sops[op];
            }
            sh.op = op;
            if (!stop && multi) {
                // the op names its heap; a heap with a sticky error skips it
                const uint32_t hid = d.heap < p.n_heaps ? d.heap : 0u;
                set_view = p.table[hid];
                set_kind = d.kind_n >> 24;
                set_cursor = (d.kind_n >> 23) & 1u;
                set_n = d.kind_n & 0x7FFFFFu;
                set_off = d.offset;
                // ops on a missing heap, an empty slot or a heap with a sticky
                // error are skipped; a malformed op is its heap's sticky error
                set_skip = d.heap >= p.n_heaps || set_view.hdr == nullptr;
                if (!set_skip) {
                    // (a delete-only launch has no input keys for an INS)
                    const bool bad = set_n > k || (set_cursor && (set_kind != GHEAP_OP_DEL ||
                                                                  p.req_cursor == nullptr)) ||
                                     (SET_DEL && set_kind != GHEAP_OP_DEL);
                    if (bad) set_err(set_view, E_STATE);
                    set_skip = bad || ld_relaxed(&set_view.hdr->err) != E_NONE;
                }
            } else if (!stop) {
                stop = ld_relaxed(&H.hdr->err) != E_NONE;
                if (!stop && p.mode == MODE_DELETE && ld_relaxed(&p.ctl->drained)) stop = 1;
            }
            sh.stop = stop;
            sh.abort = 0;
            sh.halt = 0;
        }
        bar_all();
        if (sh.stop) break;
        const unsigned long long op = sh.op;
        bool ok;
        uint32_t kind, n;
        unsigned long long off;
        if (DEL_ONLY && !SET_DEL) {
            kind = GHEAP_OP_DEL;
            n = k;
            off = 0;
        } else if (!DEL_ONLY && p.mode == MODE_INSERT) {
            kind = GHEAP_OP_INS;
            off = op * k;
            n = (uint32_t)min((unsigned long long)k, p.n - off);
        } else if (!DEL_ONLY && p.mode == MODE_DELETE) {
            kind = GHEAP_OP_DEL;
            n = k;
            off = 0;
        } else if (multi) {
            if (set_skip) {
                if (threadIdx.x == 0 && p.out_counts) p.out_counts[op] = 0;
                if (ring && threadIdx.x == 0) {
                    const uint32_t e = set_view.hdr ? ld_relaxed(&set_view.hdr->err) : E_STATE;
                    ring_complete(p, ring_req, 1u << (e ? e : E_STATE));
                }
                bar_all();
                continue;
            }
            kind = set_kind;
            n = set_n;
            off = set_off;
        } else {
            gheap_op d = p.ops[op];
            kind = d.kind;
            n = d.n;
            off = d.offset;
        }
        const bool listed = !DEL_ONLY && (p.mode == MODE_OPS || multi);
        if constexpr (DEL_ONLY) {
            if constexpr (SET_DEL)
                ok = del_op<K, IPT, true, true>(p, H, sh, base, n, off, op,
                                                p.out_counts ? p.out_counts + op : nullptr,
                                                set_cursor ? (long long)off : -1ll);
            else
                ok = del_op<K, IPT, true>(p, H, sh, base, n, off, op, nullptr, -1ll);
            if (threadIdx.x == 0) stat_add(sh, STAT_DEL, 1);
        } else if (kind == GHEAP_OP_INS) {
            // stage and sort the batch before taking the root (Section 4.1)
            if (!is_ctrl()) {
                long long ts = clock64();
                const K *src = p.in + off;
                if (ring) {
                    // host memory that the next requests reuse: read it fresh
                    for (uint32_t i = threadIdx.x; i < k; i += nmt())
                        base[i] = i < n ? __ldcv(src + i) : kmax<K>();
                } else if (n < k) {
                    for (uint32_t i = threadIdx.x; i < k; i += nmt())
                        base[i] = i < n ? __ldcg(src + i) : kmax<K>();
                } else {
                    g2s(base, src, k, threadIdx.x, nmt());
                    cp_async_commit();
                    cp_async_wait();
                }
                bar_mg();
                block_sort_reg<K, IPT / 2>(base, k);
                if (threadIdx.x == 0) lap(sh, STAT_INS_SORT_CYC, ts);
            }
            bar_all();
            ok = ((p.bu && p.mode == MODE_INSERT) || set_bu)
                     ? ins_op<K, IPT, true>(p, H, sh, base, n, listed ? op : off)
                     : ins_op<K, IPT, false>(p, H, sh, base, n, listed ? op : off);
            if (threadIdx.x == 0) {
                stat_add(sh, STAT_INS, 1);
                if (listed && p.out_counts) p.out_counts[op] = ok ? n : 0u;
            }
        } else {
            ok = del_op<K, IPT>(p, H, sh, base, n, off, op,
                                listed && p.out_counts ? p.out_counts + op : nullptr,
                                multi && set_cursor ? (long long)off : -1ll);
            if (threadIdx.x == 0) stat_add(sh, STAT_DEL, 1);
        }
        // one heap giving up ends a single-heap launch; in a set the other
        // heaps go on (the failed heap's later ops are skipped)
        if (!ok && !multi) break;
        bar_all();
        if (ring && threadIdx.x == 0) {
            uint32_t st = 0;
            if (!ok) {
                const uint32_t e = ld_relaxed(&H.hdr->err);
                st = 1u << (e ? e : E_STATE);
            }
            ring_complete(p, ring_req, st);
        }
    }
    bar_all();
    if (threadIdx.x == 0) {
        // the release warp ends after every request before the stop; its
        // statistics are in place once it has said so (waits of at least a
        // second: the release warp drains its ring within microseconds)
        const unsigned long long tmo =
            8ull * p.timeout_ns > 1000000000ull ? 8ull * p.timeout_ns : 1000000000ull;
        if (spin_until(&sh.rq_read, sh.rq_posted - (N_REQ - 1), tmo)) {
            RelReq r = {};
            r.stop = 1;
            sh.rq[sh.rq_posted % N_REQ] = r;
            st_release_cta(&sh.rq_posted, sh.rq_posted + 1);
        }
        spin_until(&rel_exited, 1u, tmo);
        if (DEL_ONLY) {
            // no fetch may still be landing in this block's shared memory
            // when it leaves (one that was given up on: bounded again)
            const unsigned long long t0 = gtimer();
            if (sh.l1_seen != sh.l1_arms)
                while (!mbar_try_wait(&sh.l1_mbar, (sh.l1_arms - 1u) & 1u) &&
                       gtimer() - t0 < 1000000000ull) {
                }
            if (sh.last_seen != sh.last_arms)
                while (!mbar_try_wait(&sh.last_mbar, (sh.last_arms - 1u) & 1u) &&
                       gtimer() - t0 < 2000000000ull) {
                }
        } else if (sh.kid_seen != sh.kid_arms) {
            const unsigned long long t0 = gtimer();
            while (!mbar_try_wait(&sh.kid_mbar, (sh.kid_arms - 1u) & 1u) &&
                   gtimer() - t0 < 1000000000ull) {
            }
        }
    }
    bar_all();
    if (p.stats && threadIdx.x < N_STATS && sh.cnt[threadIdx.x])
        atomicAdd(p.stats + threadIdx.x, sh.cnt[threadIdx.x]);
    if (threadIdx.x == 0) {
        // every block reads the control block only before it counts itself
        // out; the last one leaves it zero for the next launch
        __threadfence();
        if (atomicAdd(&p.ctl->exited, 1u) == gridDim.x - 1) {
            // MODE_DELETE: the call's count is the launch's running total
            // (also when an error stopped every operation)
            if (p.mode == MODE_DELETE && p.out_total) *p.out_total = p.ctl->delivered;
            p.ctl->next_op = 0;
            p.ctl->delivered = 0;
            p.ctl->drained = 0;
            p.ctl->exited = 0;
            __threadfence();
        }
    }
}

}  // namespace gh

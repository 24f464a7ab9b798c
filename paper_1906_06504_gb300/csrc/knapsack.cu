// knapsack.cu -- 0/1 knapsack by best-first branch and bound on the
// concurrent heap (arXiv 1906.06504, Section 5.7.2), written against the
// public C ABI of gheap.h.
//
// A search node decides items 0..i-1 of the items sorted by value/weight
// descending and records (i, profit P, weight W) in a node pool.  Its upper
// bound is the linear-relaxation (Dantzig) bound: P plus every following item
// up to the first that no longer fits, plus the fitting fraction of that item,
// floored; the whole items alone are a feasible solution (a lower bound).
// Heap keys are ((sum of values - bound) << 32 | node id), so the min-heap
// hands out the node of largest bound first.  One iteration:
//   heap_delete_min(batch)  ->  ks_expand  ->  heap_insert_dev
// ks_expand drops popped nodes whose bound no longer beats the incumbent,
// branches the others on item i (take it if it fits, skip it), raises the
// incumbent with every leaf and every child's greedy solution (atomicMax),
// and inserts the children whose bound beats the incumbent.  As soon as the
// smallest popped key's bound does not beat the incumbent, no key left in
// the heap can, and the search is over.  Optionally, when the heap holds
// more than a threshold of keys, a filter pass (the paper's garbage
// collection) deletes all of them and re-inserts only those whose bound
// still beats the incumbent.
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include <new>

#include "app_loop.cuh"
#include "gheap_apps.h"

namespace {

constexpr int RT = 256;
constexpr unsigned FULL = 0xffffffffu;
constexpr uint32_t MAX_ITEMS = 4096;
constexpr int PREP_T = 1024;

// Device counters and the instance summary of one run.
struct Ctr {
    unsigned long long popped;      // keys the iteration's deleteMin returned
    unsigned long long front[2];    // insert-buffer fill, by iteration parity
    unsigned long long live;        // keys in the heap after the iteration
    unsigned long long status;      // 1: empty deleteMin from a non-empty heap,
                                    // 2: node pool exhausted, 3: count underflow
    unsigned long long done;        // blocks of ks_expand finished
    unsigned long long finished;    // the best bound left cannot beat the incumbent
    unsigned long long best;        // incumbent: the best total value found
    unsigned long long nodes;       // node records allocated
    unsigned long long iters, explored, pruned, inserted, deleted;
    unsigned long long gc_popped, gc_kept, gc_runs, gc_dropped;
    unsigned long long n, capacity, umax;   // instance: items, knapsack capacity, sum of values
};

// Sorted instance: weights, values and their prefix sums (n + 1 entries).
struct Items {
    const uint32_t *w;
    const uint32_t *v;
    const unsigned long long *pw;
    const unsigned long long *pv;
};

// Item j precedes item i in value/weight-descending order; weightless items
// come first; equal ratios keep the input order.  Exact in 64-bit products.
__device__ __forceinline__ bool precedes(uint32_t wj, uint32_t vj, uint32_t j, uint32_t wi, uint32_t vi,
                                         uint32_t i)
{
    if (wj == 0 || wi == 0) {
        if (wj == 0 && wi == 0) return j < i;
        return wj == 0;
    }
    const unsigned long long a = (unsigned long long)vj * wi, b = (unsigned long long)vi * wj;
    return a != b ? a > b : j < i;
}

// One block: ranks the items, writes them sorted with prefix sums, and sets
// up the root node, the incumbent and the first insert.
__global__ void __launch_bounds__(PREP_T) ks_prepare(const uint32_t *w_in, const uint32_t *v_in,
                                                     uint32_t n, uint32_t capacity, uint32_t *sw,
                                                     uint32_t *sv, unsigned long long *pw,
                                                     unsigned long long *pv, uint4 *pool,
                                                     unsigned long long *front, Ctr *c)
{
    for (uint32_t i = threadIdx.x; i < n; i += blockDim.x) {
        const uint32_t wi = w_in[i], vi = v_in[i];
        uint32_t r = 0;
        for (uint32_t j = 0; j < n; j++) r += precedes(w_in[j], v_in[j], j, wi, vi, i);
        sw[r] = wi;
        sv[r] = vi;
    }
    __syncthreads();
    if (threadIdx.x != 0) return;
    unsigned long long a = 0, b = 0;
    pw[0] = 0;
    pv[0] = 0;
    for (uint32_t i = 0; i < n; i++) {
        a += sw[i];
        b += sv[i];
        pw[i + 1] = a;
        pv[i + 1] = b;
    }
    c->n = n;
    c->capacity = capacity;
    c->umax = b;
    // root: nothing decided; its greedy solution is the first incumbent
    uint32_t lo = 0, hi = n;                        // largest t with pw[t] <= capacity
    while (lo < hi) {
        const uint32_t mid = (lo + hi + 1) >> 1;
        if (pw[mid] <= capacity) lo = mid;
        else hi = mid - 1;
    }
    unsigned long long ub = pv[lo];
    c->best = ub;
    if (lo < n) ub += ((unsigned long long)capacity - pw[lo]) * sv[lo] / sw[lo];
    pool[0] = make_uint4(0u, 0u, 0u, 0u);
    front[0] = (b - ub) << 32;                      // node 0
    c->nodes = 1;
    c->live = 1;
}

// Bound of the node (i, P, W): *g = P + the items i.. up to the first that no
// longer fits; the return value adds the floored fraction of that item.
__device__ __forceinline__ unsigned long long bound(const Items &it, uint32_t n, unsigned long long cap,
                                                    uint32_t i, unsigned long long P,
                                                    unsigned long long W, unsigned long long *g)
{
    const unsigned long long rem = cap - W;
    const unsigned long long base = __ldg(it.pw + i);
    uint32_t lo = i, hi = n;                        // largest t with pw[t] - pw[i] <= rem
    while (lo < hi) {
        const uint32_t mid = (lo + hi + 1) >> 1;
        if (__ldg(it.pw + mid) - base <= rem) lo = mid;
        else hi = mid - 1;
    }
    const unsigned long long whole = P + __ldg(it.pv + lo) - __ldg(it.pv + i);
    *g = whole;
    if (lo == n) return whole;
    const unsigned long long left = rem - (__ldg(it.pw + lo) - base);
    return whole + left * __ldg(it.v + lo) / __ldg(it.w + lo);
}

__device__ __forceinline__ unsigned long long warp_sum(unsigned long long x)
{
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(FULL, x, o);
    return x;
}

// Allocates node records and insert slots for the lanes with `push` set and
// writes them; the whole warp calls it.
__device__ __forceinline__ void push_child(bool push, uint32_t i1, unsigned long long P,
                                           unsigned long long W, unsigned long long ub,
                                           unsigned long long umax, Ctr *c, uint32_t par,
                                           unsigned long long *front, uint4 *pool,
                                           unsigned long long max_nodes)
{
    const unsigned mask = __ballot_sync(FULL, push);
    if (mask == 0) return;
    const int lane = threadIdx.x & 31;
    const int leader = __ffs(mask) - 1;
    unsigned long long id0 = 0, pos0 = 0;
    if (lane == leader) {
        id0 = atomicAdd(&c->nodes, (unsigned long long)__popc(mask));
        pos0 = atomicAdd(&c->front[par], (unsigned long long)__popc(mask));
    }
    id0 = __shfl_sync(FULL, id0, leader);
    pos0 = __shfl_sync(FULL, pos0, leader);
    if (!push) return;
    const unsigned rank = __popc(mask & ((1u << lane) - 1u));
    const unsigned long long id = id0 + rank;
    unsigned long long key;
    if (id < max_nodes) {
        pool[id] = make_uint4(i1, (uint32_t)P, (uint32_t)W, 0u);
        key = ((umax - ub) << 32) | id;
    } else {
        atomicCAS(&c->status, 0ull, 2ull);
        key = 0xFFFFFFFFull;                        // an id no node has
    }
    front[pos0 + rank] = key;
}

__global__ void __launch_bounds__(RT) ks_expand(Items it, const unsigned long long *popped, Ctr *c,
                                                uint32_t par, unsigned long long *front, uint4 *pool,
                                                unsigned long long max_nodes,
                                                unsigned long long *ring, uint32_t slot)
{
    __shared__ bool last;
    const unsigned long long np = c->popped;
    const uint32_t n = (uint32_t)c->n;
    const unsigned long long cap = c->capacity, umax = c->umax;
    const bool finished = *(volatile unsigned long long *)&c->finished != 0;
    unsigned long long explored = 0, pruned = 0, ins = 0;
    if (!finished && blockIdx.x == 0 && threadIdx.x == 0 && np > 0) {
        // popped[0] is the heap's smallest key: the largest bound left
        if (umax - (popped[0] >> 32) <= *(volatile unsigned long long *)&c->best) c->finished = 1;
    }
    for (unsigned long long b = (unsigned long long)blockIdx.x * RT; !finished && b < np;
         b += (unsigned long long)gridDim.x * RT) {
        const unsigned long long idx = b + threadIdx.x;
        bool live = false;
        uint4 nd = make_uint4(0u, 0u, 0u, 0u);
        if (idx < np) {
            const unsigned long long key = popped[idx];
            const unsigned long long id = key & 0xFFFFFFFFull;
            const unsigned long long ub = umax - (key >> 32);
            if (id < max_nodes && ub > *(volatile unsigned long long *)&c->best) {
                nd = pool[id];
                live = true;
                explored++;
            } else {
                pruned++;
            }
        }
        const uint32_t i = nd.x, i1 = nd.x + 1;
        const unsigned long long P = nd.y, W = nd.z;
        // child 1 takes item i, child 0 skips it
        for (int take = 1; take >= 0; take--) {
            bool push = false;
            unsigned long long cp = P, cw = W, ub = 0;
            if (live) {
                if (take) {
                    cw = W + __ldg(it.w + i);
                    cp = P + __ldg(it.v + i);
                }
                if (!take || cw <= cap) {
                    if (i1 == n) {
                        if (cp > *(volatile unsigned long long *)&c->best) atomicMax(&c->best, cp);
                    } else {
                        unsigned long long g;
                        ub = bound(it, n, cap, i1, cp, cw, &g);
                        if (g > *(volatile unsigned long long *)&c->best) atomicMax(&c->best, g);
                        push = ub > *(volatile unsigned long long *)&c->best;
                    }
                }
            }
            push_child(push, i1, cp, cw, ub, umax, c, par, front, pool, max_nodes);
            ins += push;
        }
    }
    explored = warp_sum(explored);
    pruned = warp_sum(pruned);
    ins = warp_sum(ins);
    if ((threadIdx.x & 31) == 0) {
        if (explored) atomicAdd(&c->explored, explored);
        if (pruned) atomicAdd(&c->pruned, pruned);
        if (ins) atomicAdd(&c->inserted, ins);
    }

    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) last = atomicAdd(&c->done, 1ull) == gridDim.x - 1;
    __syncthreads();
    if (!last || threadIdx.x != 0) return;
    __threadfence();
    volatile Ctr *vc = c;
    const unsigned long long live0 = vc->live, nf = vc->front[par];
    unsigned long long status = vc->status;
    if (np > live0 && !status) status = 3;
    if (np == 0 && live0 > 0 && !status) status = 1;
    const unsigned long long live = np > live0 ? nf : live0 - np + nf;
    vc->live = live;
    vc->status = status;
    vc->deleted = vc->deleted + np;
    if (np && !finished) vc->iters = vc->iters + 1;
    vc->front[par ^ 1u] = 0;
    vc->done = 0;
    volatile unsigned long long *r = ring;
    r[2 * slot] = vc->finished ? 0ull : live;      // a finished search reports an empty heap
    r[2 * slot + 1] = status;
    __threadfence_system();
}

// Garbage collection: keeps the deleted keys whose bound still beats the
// incumbent (into `kept`) and updates the live count.
__global__ void __launch_bounds__(RT) ks_filter(const unsigned long long *all, Ctr *c,
                                                unsigned long long *kept)
{
    __shared__ bool last;
    const unsigned long long np = c->gc_popped, umax = c->umax;
    const unsigned long long best = c->best;
    for (unsigned long long b = (unsigned long long)blockIdx.x * RT; b < np;
         b += (unsigned long long)gridDim.x * RT) {
        const unsigned long long idx = b + threadIdx.x;
        bool keep = false;
        unsigned long long key = 0;
        if (idx < np) {
            key = all[idx];
            keep = umax - (key >> 32) > best;
        }
        const unsigned mask = __ballot_sync(FULL, keep);
        if (mask == 0) continue;
        const int lane = threadIdx.x & 31, leader = __ffs(mask) - 1;
        unsigned long long pos = 0;
        if (lane == leader) pos = atomicAdd(&c->gc_kept, (unsigned long long)__popc(mask));
        pos = __shfl_sync(FULL, pos, leader);
        if (keep) kept[pos + __popc(mask & ((1u << lane) - 1u))] = key;
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) last = atomicAdd(&c->done, 1ull) == gridDim.x - 1;
    __syncthreads();
    if (!last || threadIdx.x != 0) return;
    __threadfence();
    volatile Ctr *vc = c;
    vc->live = vc->gc_kept;
    vc->gc_runs = vc->gc_runs + 1;
    vc->gc_dropped = vc->gc_dropped + (np - vc->gc_kept);
    vc->done = 0;
}

__global__ void ks_gc_reset(Ctr *c)
{
    c->gc_popped = 0;
    c->gc_kept = 0;
}

int cuda_err(cudaError_t e) { return e == cudaSuccess ? GHEAP_OK : GHEAP_ERR_CUDA; }

}  // namespace

struct knapsack_s {
    int device;
    int sm_count;
    uint32_t max_items;
    uint64_t max_nodes;
    uint32_t batch;
    uint64_t gc_threshold;
    gheap_t heap;
    uint32_t *d_w, *d_v;                // sorted items
    unsigned long long *d_pw, *d_pv;    // prefix sums
    uint4 *d_pool;                      // node records (i, P, W, -)
    unsigned long long *d_batch;        // keys of one deleteMin
    unsigned long long *d_front;        // keys of one insert (2 per popped key)
    unsigned long long *d_gc_all;       // garbage collection: every key, then
    unsigned long long *d_gc_kept;      //   the kept ones
    Ctr *d_ctr;
    app::Loop loop;
};

namespace {

int enqueue_iteration(knapsack_t s, uint32_t par, uint32_t slot, cudaStream_t st)
{
    Ctr *c = s->d_ctr;
    Items it = {s->d_w, s->d_v, s->d_pw, s->d_pv};
    const uint64_t blocks = (s->batch + RT - 1) / RT;
    const unsigned grid = (unsigned)(blocks < (uint64_t)s->sm_count * 8 ? blocks : (uint64_t)s->sm_count * 8);
    int rc = heap_delete_min(s->heap, s->d_batch, s->batch, reinterpret_cast<uint64_t *>(&c->popped), st);
    if (rc != GHEAP_OK) return rc;
    ks_expand<<<grid, RT, 0, st>>>(it, s->d_batch, c, par, s->d_front, s->d_pool, s->max_nodes,
                                   s->loop.d_ring, slot);
    if (cudaGetLastError() != cudaSuccess) return GHEAP_ERR_CUDA;
    return heap_insert_dev(s->heap, s->d_front, reinterpret_cast<const uint64_t *>(&c->front[par]),
                           2ull * s->batch, st);
}

// One garbage-collection pass on `st` (synchronizes at its end).
int collect(knapsack_t s, cudaStream_t st, unsigned long long *kept)
{
    Ctr *c = s->d_ctr;
    ks_gc_reset<<<1, 1, 0, st>>>(c);
    if (cudaGetLastError() != cudaSuccess) return GHEAP_ERR_CUDA;
    int rc = heap_delete_min(s->heap, s->d_gc_all, s->max_nodes,
                             reinterpret_cast<uint64_t *>(&c->gc_popped), st);
    if (rc != GHEAP_OK) return rc;
    ks_filter<<<(unsigned)s->sm_count * 4, RT, 0, st>>>(s->d_gc_all, c, s->d_gc_kept);
    if (cudaGetLastError() != cudaSuccess) return GHEAP_ERR_CUDA;
    rc = heap_insert_dev(s->heap, s->d_gc_kept, reinterpret_cast<const uint64_t *>(&c->gc_kept),
                         s->max_nodes, st);
    if (rc != GHEAP_OK) return rc;
    if (cudaStreamSynchronize(st) != cudaSuccess) return GHEAP_ERR_CUDA;
    if (cudaMemcpy(kept, &c->gc_kept, sizeof(*kept), cudaMemcpyDeviceToHost) != cudaSuccess)
        return GHEAP_ERR_CUDA;
    return heap_sync(s->heap);
}

}  // namespace

extern "C" {

gheap_t knapsack_heap(knapsack_t s)
{
    return s ? s->heap : nullptr;
}

int knapsack_destroy(knapsack_t s)
{
    if (!s) return GHEAP_ERR_ARG;
    cudaSetDevice(s->device);
    app::loop_free(s->loop);
    if (s->heap) heap_destroy(s->heap);
    cudaFree(s->d_w);
    cudaFree(s->d_v);
    cudaFree(s->d_pw);
    cudaFree(s->d_pv);
    cudaFree(s->d_pool);
    cudaFree(s->d_batch);
    cudaFree(s->d_front);
    cudaFree(s->d_gc_all);
    cudaFree(s->d_gc_kept);
    cudaFree(s->d_ctr);
    delete s;
    return GHEAP_OK;
}

int knapsack_create(knapsack_t *out, uint32_t max_items, uint64_t max_nodes, uint32_t k,
                    uint32_t batch, uint64_t gc_threshold)
{
    if (!out) return GHEAP_ERR_ARG;
    *out = nullptr;
    if (max_items == 0 || max_items > MAX_ITEMS || batch == 0) return GHEAP_ERR_ARG;
    if (max_nodes == 0) max_nodes = 1ull << 26;
    if (max_nodes > 0xFFFFFFFFull) return GHEAP_ERR_ARG;
    knapsack_t s = new (std::nothrow) knapsack_s();
    if (!s) return GHEAP_ERR_OOM;
    if (cudaGetDevice(&s->device) != cudaSuccess) { delete s; return GHEAP_ERR_CUDA; }
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, s->device) != cudaSuccess) { delete s; return GHEAP_ERR_CUDA; }
    s->sm_count = prop.multiProcessorCount;
    s->max_items = max_items;
    s->max_nodes = max_nodes;
    s->batch = batch;
    s->gc_threshold = gc_threshold;
    // every heap key names a distinct node record
    // the iterations' insert launches carry no deletes: bottom-up inserts
    // (targets reserved without the root lock)
    int rc = heap_create(&s->heap, max_nodes, k, 8, GHEAP_FLAG_BOTTOM_UP, 0);
    if (rc != GHEAP_OK) { s->heap = nullptr; knapsack_destroy(s); return rc; }
    bool ok = cudaMalloc(&s->d_w, (size_t)max_items * 4) == cudaSuccess &&
              cudaMalloc(&s->d_v, (size_t)max_items * 4) == cudaSuccess &&
              cudaMalloc(&s->d_pw, ((size_t)max_items + 1) * 8) == cudaSuccess &&
              cudaMalloc(&s->d_pv, ((size_t)max_items + 1) * 8) == cudaSuccess &&
              cudaMalloc(&s->d_pool, (size_t)max_nodes * sizeof(uint4)) == cudaSuccess &&
              cudaMalloc(&s->d_batch, (size_t)batch * 8) == cudaSuccess &&
              cudaMalloc(&s->d_front, (size_t)batch * 16) == cudaSuccess &&
              cudaMalloc(&s->d_ctr, sizeof(Ctr)) == cudaSuccess;
    if (ok && gc_threshold)
        ok = cudaMalloc(&s->d_gc_all, (size_t)max_nodes * 8) == cudaSuccess &&
             cudaMalloc(&s->d_gc_kept, (size_t)max_nodes * 8) == cudaSuccess;
    if (!ok) { knapsack_destroy(s); return GHEAP_ERR_OOM; }
    rc = app::loop_init(s->loop);
    if (rc != GHEAP_OK) { knapsack_destroy(s); return rc; }
    *out = s;
    return GHEAP_OK;
}

int knapsack_set_launch(knapsack_t s, uint32_t ctas, uint32_t items_per_thread)
{
    if (!s) return GHEAP_ERR_ARG;
    app::loop_drop(s->loop);
    return heap_set_launch(s->heap, ctas, items_per_thread);
}

int knapsack_run(knapsack_t s, const uint32_t *d_w, const uint32_t *d_v, uint32_t n, uint32_t capacity,
                 knapsack_stats *stats, void *stream)
{
    if (!s || !d_w || !d_v || n == 0 || n > s->max_items) return GHEAP_ERR_ARG;
    if (cudaSetDevice(s->device) != cudaSuccess) return GHEAP_ERR_CUDA;
    cudaStream_t st = (cudaStream_t)stream;
    Ctr *c = s->d_ctr;
    // the captured iterations use only buffers of the context
    if (!app::loop_ready(s->loop)) {
        const int rc = app::loop_capture(s->loop, [&](uint32_t par, uint32_t slot, cudaStream_t cs) {
            return enqueue_iteration(s, par, slot, cs);
        });
        if (rc != GHEAP_OK) return rc;
    }
    int rc = heap_reset(s->heap, stream);
    if (rc != GHEAP_OK) return rc;
    if (cudaMemsetAsync(c, 0, sizeof(Ctr), st) != cudaSuccess) return GHEAP_ERR_CUDA;
    ks_prepare<<<1, PREP_T, 0, st>>>(d_w, d_v, n, capacity, s->d_w, s->d_v, s->d_pw, s->d_pv,
                                     s->d_pool, s->d_front, c);
    if (cudaGetLastError() != cudaSuccess) return GHEAP_ERR_CUDA;
    // the bound is stored in 32 bits of the key: the values must sum below 2^32
    unsigned long long umax = 0;
    if (cudaMemcpyAsync(&umax, &c->umax, sizeof(umax), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return GHEAP_ERR_CUDA;
    if (umax >= 0xFFFFFFFFull) return GHEAP_ERR_ARG;
    rc = heap_insert(s->heap, s->d_front, 1, stream);
    if (rc != GHEAP_OK) return rc;

    unsigned long long status = 0, floor = 0;
    rc = app::loop_run(
        s->loop, st, &status,
        [&](unsigned long long live) {
            return s->gc_threshold && live > s->gc_threshold && live > 2 * floor;
        },
        [&](cudaStream_t cs) { return collect(s, cs, &floor); });
    if (rc != GHEAP_OK) return rc;
    if (cudaStreamSynchronize(st) != cudaSuccess) return GHEAP_ERR_CUDA;
    rc = heap_sync(s->heap);
    if (rc != GHEAP_OK) return rc;
    if (status == 2) return GHEAP_ERR_FULL;
    if (status) return GHEAP_ERR_STATE;
    Ctr hc;
    if (cudaMemcpy(&hc, c, sizeof(Ctr), cudaMemcpyDeviceToHost) != cudaSuccess) return GHEAP_ERR_CUDA;
    if (stats) {
        stats->best = hc.best;
        stats->iterations = hc.iters;
        stats->keys_deleted = hc.deleted;
        stats->explored = hc.explored;
        stats->pruned = hc.pruned;
        stats->keys_inserted = hc.inserted;
        stats->nodes = hc.nodes < s->max_nodes ? hc.nodes : s->max_nodes;
        stats->gc_runs = hc.gc_runs;
        stats->gc_dropped = hc.gc_dropped;
    }
    return cuda_err(cudaGetLastError());
}

}  // extern "C"

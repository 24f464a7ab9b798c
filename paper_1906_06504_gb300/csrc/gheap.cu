// gheap.cu -- C ABI of the GB300 generalized concurrent heap (include/gheap.h).
//
// Host side: device memory layout, launch shapes, capacity accounting and
// error reporting.  All heap arithmetic runs in the persistent kernel of
// gheap_kernel.cuh (TD-INS/TD-DEL and BU-INS/TD-DEL heaps of arXiv 1906.06504,
// Sections 3-4).
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include <atomic>
#include <chrono>
#include <deque>
#include <mutex>
#include <thread>
#include <vector>

#include "gheap.h"
#include "gheap_kernel.cuh"

struct gheap_s {
    int device;
    uint32_t k;
    uint32_t key_bytes;
    uint32_t flags;
    uint64_t capacity;       // keys
    uint32_t max_nodes;      // storage slots 1..max_nodes
    void *d_keys;
    uint32_t *d_state;
    void *d_buf;
    gh::Hdr *d_hdr;
    gh::Ctl *d_ctl;
    gheap_log_entry *d_log;
    uint64_t log_cap;
    unsigned long long *d_stats;
    uint32_t ctas;           // 0 = one block per SM
    uint32_t ipt;            // merge outputs per thread: 2, 4 or 8
    uint64_t timeout_ns;
    uint32_t del_yields;     // root hand-backs before a DEL marks an in-flight target
    int sm_count;
    int sticky;              // host copy of a sticky device error
    uint64_t size_upper;     // upper bound on the keys held
    uint32_t call_id;
};

namespace {

int cuda_err(cudaError_t e) { return e == cudaSuccess ? GHEAP_OK : GHEAP_ERR_CUDA; }

// heap_debug_hold_root: holds the root's ticket lock forever.
__global__ void take_root_ticket(gh::Hdr *hdr) { atomicAdd(&hdr->next, 1ull); }

int map_dev_err(uint32_t e)
{
    switch (e) {
    case gh::E_NONE: return GHEAP_OK;
    case gh::E_TIMEOUT: return GHEAP_ERR_TIMEOUT;
    case gh::E_FULL: return GHEAP_ERR_FULL;
    default: return GHEAP_ERR_STATE;
    }
}

// Threads per block: the merge threads (2k/ipt merge outputs each, at least
// one warp, at most 512) plus the control warp and the release warp.
uint32_t merge_threads_for(uint32_t k, uint32_t ipt)
{
    uint32_t t = 2 * k / ipt;
    if (t < 32) t = 32;
    return t;
}

uint32_t threads_for(uint32_t k, uint32_t ipt) { return merge_threads_for(k, ipt) + 64; }

// Merge threads allowed by the kernel's launch bound for this merge width.
uint32_t max_merge_threads(uint32_t ipt) { return ipt >= 8 ? 256 : 512; }

// What a launch needs besides the kernel parameters.  `per_sm_default`:
// blocks per SM when ctas is 0.
struct Shape {
    uint32_t k, ipt, ctas;
    uint32_t per_sm_default = 1;
    int sm_count;
    gh::Ctl *d_ctl;
};

template <typename K, int IPT>
int launch_t(const Shape &sp, gh::Params<K> &p, uint64_t n_ops, cudaStream_t s)
{
    // a heap-set list with no input keys holds only DELs (an INS there is its
    // heap's sticky error): the delete-only walk, ops naming their heaps
    auto kern = p.mode == gh::MODE_DELETE ? gh::heap_kernel<K, IPT, true>
                : (p.mode == gh::MODE_SET && p.in == nullptr && p.out != nullptr)
                    ? gh::heap_kernel<K, IPT, true, true>
                    : gh::heap_kernel<K, IPT, false>;
    const uint32_t threads = threads_for(sp.k, IPT);
    const size_t smem = 6u * (size_t)sp.k * sizeof(K);
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return GHEAP_ERR_CUDA;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, (int)threads, smem);
    if (e != cudaSuccess || per_sm < 1) return GHEAP_ERR_CUDA;
    // default: one block per SM on a single heap, whose operations all pass
    // its root lock (more blocks only add waiters: measured flat to slightly
    // slower from 16 to 512 blocks at k = 1024), two on a heap set; an
    // explicit count is clamped only by residency
    const uint64_t resident = (uint64_t)per_sm * sp.sm_count;
    const uint32_t dflt = per_sm < (int)sp.per_sm_default ? (uint32_t)per_sm : sp.per_sm_default;
    uint64_t grid = sp.ctas ? sp.ctas : (uint64_t)dflt * sp.sm_count;
    if (grid > resident) grid = resident;
    if (grid > n_ops) grid = n_ops;
    if (grid == 0) return GHEAP_OK;
    // the control block is zero here: zeroed at creation and reset, and put
    // back to zero by the last block of every launch
    kern<<<(unsigned)grid, threads, smem, s>>>(p);
    return cuda_err(cudaGetLastError());
}

template <typename K>
int launch_k(const Shape &sp, gh::Params<K> &p, uint64_t n_ops, cudaStream_t s)
{
    switch (sp.ipt) {
    case 4: return launch_t<K, 4>(sp, p, n_ops, s);
    case 8: return launch_t<K, 8>(sp, p, n_ops, s);
    case 16: return launch_t<K, 16>(sp, p, n_ops, s);
    default: return GHEAP_ERR_ARG;
    }
}

Shape shape_of(gheap_t h)
{
    Shape sp;
    sp.k = h->k;
    sp.ipt = h->ipt;
    sp.ctas = h->ctas;
    sp.sm_count = h->sm_count;
    sp.d_ctl = h->d_ctl;
    return sp;
}

template <typename K>
gh::Params<K> base_params(gheap_t h, uint32_t mode)
{
    gh::Params<K> p;
    memset(&p, 0, sizeof(p));
    p.h.keys = static_cast<K *>(h->d_keys);
    p.h.state = h->d_state;
    p.h.buf = static_cast<K *>(h->d_buf);
    p.h.hdr = h->d_hdr;
    p.h.log = h->d_log;
    p.h.log_cap = h->log_cap;
    p.h.max_nodes = h->max_nodes;
    p.ctl = h->d_ctl;
    p.stats = (h->flags & GHEAP_FLAG_STATS) ? h->d_stats : nullptr;
    p.k = h->k;
    p.timeout_ns = h->timeout_ns;
    p.del_yields = h->del_yields;
    p.mode = mode;
    p.bu = (h->flags & GHEAP_FLAG_BOTTOM_UP) ? 1u : 0u;
    p.call_id = ++h->call_id;
    return p;
}

int launch(gheap_t h, uint32_t mode, const void *in, void *out, uint64_t n,
           const gheap_op *ops, uint64_t n_ops, uint32_t *out_counts, uint64_t *out_total,
           cudaStream_t s)
{
    uint64_t launch_ops = mode == gh::MODE_OPS ? n_ops : (n + h->k - 1) / h->k;
    if (h->key_bytes == 4) {
        gh::Params<uint32_t> p = base_params<uint32_t>(h, mode);
        p.in = static_cast<const uint32_t *>(in);
        p.out = static_cast<uint32_t *>(out);
        p.n = n;
        p.ops = ops;
        p.n_ops = n_ops;
        p.out_counts = out_counts;
        p.out_total = reinterpret_cast<unsigned long long *>(out_total);
        return launch_k<uint32_t>(shape_of(h), p, launch_ops, s);
    } else {
        gh::Params<uint64_t> p = base_params<uint64_t>(h, mode);
        p.in = static_cast<const uint64_t *>(in);
        p.out = static_cast<uint64_t *>(out);
        p.n = n;
        p.ops = ops;
        p.n_ops = n_ops;
        p.out_counts = out_counts;
        p.out_total = reinterpret_cast<unsigned long long *>(out_total);
        return launch_k<uint64_t>(shape_of(h), p, launch_ops, s);
    }
}

// Reads the exact size and the sticky device error (synchronizes).
int read_state(gheap_t h, uint64_t *size_out)
{
    if (cudaSetDevice(h->device) != cudaSuccess) return GHEAP_ERR_CUDA;
    if (cudaDeviceSynchronize() != cudaSuccess) return GHEAP_ERR_CUDA;
    gh::Hdr hd;
    if (cudaMemcpy(&hd, h->d_hdr, sizeof(hd), cudaMemcpyDeviceToHost) != cudaSuccess)
        return GHEAP_ERR_CUDA;
    int rc = map_dev_err(hd.err);
    if (rc != GHEAP_OK) h->sticky = rc;
    uint64_t size = (uint64_t)gh::rw_m(hd.root) * h->k + gh::rw_s(hd.root);
    h->size_upper = size;
    if (size_out) *size_out = size;
    return rc;
}

}  // namespace

extern "C" {

const char *heap_strerror(int code)
{
    switch (code) {
    case GHEAP_OK: return "ok";
    case GHEAP_ERR_ARG: return "invalid argument";
    case GHEAP_ERR_OOM: return "device allocation failed";
    case GHEAP_ERR_FULL: return "heap capacity exceeded";
    case GHEAP_ERR_TIMEOUT: return "a bounded lock wait gave up";
    case GHEAP_ERR_CUDA: return "CUDA runtime error";
    case GHEAP_ERR_STATE: return "impossible node state observed on the device";
    case GHEAP_ERR_TOO_LARGE: return "more keys than the fixed scratch of heap_sort_noalloc holds";
    default: return "unknown error";
    }
}

uint64_t heap_slot_to_node(uint64_t j)
{
    if (j == 0) return 0;
    uint32_t d = 63u - (uint32_t)__builtin_clzll(j);
    if (d == 0) return j;
    uint64_t o = j - (1ull << d), r = 0;
    for (uint32_t i = 0; i < d; i++) {
        r = (r << 1) | (o & 1ull);
        o >>= 1;
    }
    return (1ull << d) + r;
}

int heap_create(gheap_t *out, uint64_t capacity_keys, uint32_t k, uint32_t key_bytes,
                uint32_t flags, uint64_t log_capacity)
{
    if (!out) return GHEAP_ERR_ARG;
    *out = nullptr;
    if (k < 1 || k > 2048 || (k & (k - 1)) != 0) return GHEAP_ERR_ARG;
    if (key_bytes != 4 && key_bytes != 8) return GHEAP_ERR_ARG;
    if (capacity_keys == 0) return GHEAP_ERR_ARG;
    uint64_t nodes = capacity_keys / k + 1;
    if (nodes >= (1ull << 30)) return GHEAP_ERR_ARG;

    gheap_t h = (gheap_t)calloc(1, sizeof(gheap_s));
    if (!h) return GHEAP_ERR_OOM;
    if (cudaGetDevice(&h->device) != cudaSuccess) { free(h); return GHEAP_ERR_CUDA; }
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, h->device) != cudaSuccess) { free(h); return GHEAP_ERR_CUDA; }
    h->sm_count = prop.multiProcessorCount;
    h->k = k;
    h->key_bytes = key_bytes;
    h->flags = flags;
    h->capacity = capacity_keys;
    h->max_nodes = (uint32_t)nodes;
    h->ctas = 0;
    h->ipt = k >= 2048 ? 16 : 8;
    h->timeout_ns = 2000000000ull;
    h->del_yields = gh::DEL_YIELDS;
    h->log_cap = log_capacity;

    size_t key_bytes_total = ((size_t)h->max_nodes + 1) * k * key_bytes;
    bool ok = cudaMalloc(&h->d_keys, key_bytes_total) == cudaSuccess &&
              cudaMalloc((void **)&h->d_state, ((size_t)h->max_nodes + 1) * sizeof(uint32_t)) == cudaSuccess &&
              cudaMalloc(&h->d_buf, (size_t)k * key_bytes) == cudaSuccess &&
              cudaMalloc((void **)&h->d_hdr, sizeof(gh::Hdr)) == cudaSuccess &&
              cudaMalloc((void **)&h->d_ctl, sizeof(gh::Ctl)) == cudaSuccess &&
              cudaMalloc((void **)&h->d_stats, gh::N_STATS * sizeof(unsigned long long)) == cudaSuccess;
    if (ok && log_capacity)
        ok = cudaMalloc((void **)&h->d_log, log_capacity * sizeof(gheap_log_entry)) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        heap_destroy(h);
        return GHEAP_ERR_OOM;
    }
    int rc = heap_reset(h, nullptr);
    if (rc == GHEAP_OK && cudaDeviceSynchronize() != cudaSuccess) rc = GHEAP_ERR_CUDA;
    if (rc != GHEAP_OK) {
        heap_destroy(h);
        return rc;
    }
    *out = h;
    return GHEAP_OK;
}

int heap_destroy(gheap_t h)
{
    if (!h) return GHEAP_ERR_ARG;
    cudaSetDevice(h->device);
    cudaDeviceSynchronize();
    cudaFree(h->d_keys);
    cudaFree(h->d_state);
    cudaFree(h->d_buf);
    cudaFree(h->d_hdr);
    cudaFree(h->d_ctl);
    cudaFree(h->d_log);
    cudaFree(h->d_stats);
    free(h);
    return GHEAP_OK;
}

int heap_reset(gheap_t h, void *stream)
{
    if (!h) return GHEAP_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    if (cudaSetDevice(h->device) != cudaSuccess) return GHEAP_ERR_CUDA;
    cudaError_t e = cudaMemsetAsync(h->d_state, 0, ((size_t)h->max_nodes + 1) * sizeof(uint32_t), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->d_hdr, 0, sizeof(gh::Hdr), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->d_ctl, 0, sizeof(gh::Ctl), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->d_stats, 0, gh::N_STATS * sizeof(unsigned long long), s);
    if (e != cudaSuccess) return GHEAP_ERR_CUDA;
    h->sticky = GHEAP_OK;
    h->size_upper = 0;
    return GHEAP_OK;
}

int heap_set_launch(gheap_t h, uint32_t ctas, uint32_t items_per_thread)
{
    if (!h) return GHEAP_ERR_ARG;
    if (items_per_thread != 4 && items_per_thread != 8 && items_per_thread != 16)
        return GHEAP_ERR_ARG;
    if (merge_threads_for(h->k, items_per_thread) > max_merge_threads(items_per_thread))
        return GHEAP_ERR_ARG;
    h->ctas = ctas;
    h->ipt = items_per_thread;
    return GHEAP_OK;
}

int heap_set_timeout(gheap_t h, uint64_t ns)
{
    if (!h || ns == 0) return GHEAP_ERR_ARG;
    h->timeout_ns = ns;
    return GHEAP_OK;
}

int heap_set_stats(gheap_t h, uint32_t on)
{
    if (!h) return GHEAP_ERR_ARG;
    h->flags = on ? (h->flags | GHEAP_FLAG_STATS) : (h->flags & ~GHEAP_FLAG_STATS);
    return GHEAP_OK;
}

int heap_set_yields(gheap_t h, uint32_t n)
{
    if (!h) return GHEAP_ERR_ARG;
    h->del_yields = n;
    return GHEAP_OK;
}

int heap_insert(gheap_t h, const void *d_keys, uint64_t n, void *stream)
{
    if (!h) return GHEAP_ERR_ARG;
    if (h->sticky) return h->sticky;
    if (n == 0) return GHEAP_OK;
    if (!d_keys) return GHEAP_ERR_ARG;
    if (cudaSetDevice(h->device) != cudaSuccess) return GHEAP_ERR_CUDA;
    if (h->size_upper + n > h->capacity) {
        uint64_t size = 0;
        int rc = read_state(h, &size);
        if (rc != GHEAP_OK) return rc;
        if (size + n > h->capacity) return GHEAP_ERR_FULL;
    }
    h->size_upper += n;
    return launch(h, gh::MODE_INSERT, d_keys, nullptr, n, nullptr, 0, nullptr, nullptr,
                  (cudaStream_t)stream);
}

int heap_insert_dev(gheap_t h, const void *d_keys, const uint64_t *d_n, uint64_t max_n,
                    void *stream)
{
    if (!h) return GHEAP_ERR_ARG;
    if (h->sticky) return h->sticky;
    if (max_n == 0) return GHEAP_OK;
    if (!d_keys || !d_n) return GHEAP_ERR_ARG;
    if (cudaSetDevice(h->device) != cudaSuccess) return GHEAP_ERR_CUDA;
    // the count is not known here: the device checks the node storage (E_FULL),
    // and the host bound saturates so that a later heap_insert re-reads the size
    h->size_upper = max_n > h->capacity - h->size_upper ? h->capacity : h->size_upper + max_n;
    cudaStream_t s = (cudaStream_t)stream;
    const uint64_t launch_ops = (max_n + h->k - 1) / h->k;
    if (h->key_bytes == 4) {
        gh::Params<uint32_t> p = base_params<uint32_t>(h, gh::MODE_INSERT);
        p.in = static_cast<const uint32_t *>(d_keys);
        p.n = max_n;
        p.n_dev = reinterpret_cast<const unsigned long long *>(d_n);
        return launch_k<uint32_t>(shape_of(h), p, launch_ops, s);
    }
    gh::Params<uint64_t> p = base_params<uint64_t>(h, gh::MODE_INSERT);
    p.in = static_cast<const uint64_t *>(d_keys);
    p.n = max_n;
    p.n_dev = reinterpret_cast<const unsigned long long *>(d_n);
    return launch_k<uint64_t>(shape_of(h), p, launch_ops, s);
}

int heap_delete_min(gheap_t h, void *d_out, uint64_t n, uint64_t *d_count, void *stream)
{
    if (!h) return GHEAP_ERR_ARG;
    if (h->sticky) return h->sticky;
    if (cudaSetDevice(h->device) != cudaSuccess) return GHEAP_ERR_CUDA;
    if (n == 0) {
        if (d_count)
            return cuda_err(cudaMemsetAsync(d_count, 0, sizeof(uint64_t), (cudaStream_t)stream));
        return GHEAP_OK;
    }
    if (!d_out) return GHEAP_ERR_ARG;
    // *d_count is written by the launch's last block
    return launch(h, gh::MODE_DELETE, nullptr, d_out, n, nullptr, 0, nullptr, d_count,
                  (cudaStream_t)stream);
}

int heap_ops(gheap_t h, const gheap_op *d_ops, uint64_t n_ops, const void *d_in_keys,
             void *d_out_keys, uint32_t *d_out_counts, uint64_t max_insert_keys, void *stream)
{
    if (!h) return GHEAP_ERR_ARG;
    if (h->sticky) return h->sticky;
    if (n_ops == 0) return GHEAP_OK;
    if (!d_ops) return GHEAP_ERR_ARG;
    if (cudaSetDevice(h->device) != cudaSuccess) return GHEAP_ERR_CUDA;
    if (h->size_upper + max_insert_keys > h->capacity) {
        uint64_t size = 0;
        int rc = read_state(h, &size);
        if (rc != GHEAP_OK) return rc;
        if (size + max_insert_keys > h->capacity) return GHEAP_ERR_FULL;
    }
    h->size_upper += max_insert_keys;
    return launch(h, gh::MODE_OPS, d_in_keys, d_out_keys, 0, d_ops, n_ops, d_out_counts, nullptr,
                  (cudaStream_t)stream);
}

int heap_sync(gheap_t h)
{
    if (!h) return GHEAP_ERR_ARG;
    return read_state(h, nullptr);
}

int heap_size(gheap_t h, uint64_t *out)
{
    if (!h || !out) return GHEAP_ERR_ARG;
    return read_state(h, out);
}

int heap_get_log(gheap_t h, gheap_log_entry *host_buf, uint64_t cap, uint64_t *n_copied,
                 uint64_t *n_total)
{
    if (!h) return GHEAP_ERR_ARG;
    int rc = read_state(h, nullptr);
    gh::Hdr hd;
    if (cudaMemcpy(&hd, h->d_hdr, sizeof(hd), cudaMemcpyDeviceToHost) != cudaSuccess)
        return GHEAP_ERR_CUDA;
    uint64_t total = hd.seq;
    uint64_t avail = total < h->log_cap ? total : h->log_cap;
    uint64_t n = avail < cap ? avail : cap;
    if (n && host_buf) {
        if (cudaMemcpy(host_buf, h->d_log, n * sizeof(gheap_log_entry), cudaMemcpyDeviceToHost) !=
            cudaSuccess)
            return GHEAP_ERR_CUDA;
    }
    if (n_copied) *n_copied = host_buf ? n : 0;
    if (n_total) *n_total = total;
    return rc;
}

int heap_snapshot(gheap_t h, void *host_keys, uint32_t *host_state, void *host_buf,
                  uint64_t *hdr)
{
    if (!h) return GHEAP_ERR_ARG;
    int rc = read_state(h, nullptr);
    gh::Hdr hd;
    if (cudaMemcpy(&hd, h->d_hdr, sizeof(hd), cudaMemcpyDeviceToHost) != cudaSuccess)
        return GHEAP_ERR_CUDA;
    size_t slots = (size_t)h->max_nodes + 1;
    if (host_keys &&
        cudaMemcpy(host_keys, h->d_keys, slots * h->k * h->key_bytes, cudaMemcpyDeviceToHost) !=
            cudaSuccess)
        return GHEAP_ERR_CUDA;
    if (host_state) {
        if (cudaMemcpy(host_state, h->d_state, slots * sizeof(uint32_t), cudaMemcpyDeviceToHost) !=
            cudaSuccess)
            return GHEAP_ERR_CUDA;
        // the root is guarded by the header's root lock, not by a state word
        host_state[1] = gh::rw_m(hd.root) >= 1 ? gh::ST_AVAIL : gh::ST_EMPTY;
    }
    if (host_buf &&
        cudaMemcpy(host_buf, h->d_buf, (size_t)h->k * h->key_bytes, cudaMemcpyDeviceToHost) !=
            cudaSuccess)
        return GHEAP_ERR_CUDA;
    if (hdr) {
        hdr[0] = gh::rw_m(hd.root);
        hdr[1] = gh::rw_s(hd.root);
        hdr[2] = hd.seq;
    }
    return rc;
}

int heap_geometry(gheap_t h, uint64_t *max_nodes, uint32_t *k, uint32_t *key_bytes)
{
    if (!h) return GHEAP_ERR_ARG;
    if (max_nodes) *max_nodes = h->max_nodes;
    if (k) *k = h->k;
    if (key_bytes) *key_bytes = h->key_bytes;
    return GHEAP_OK;
}

// ---------------------------------------------------------------------------
// heap sets
// ---------------------------------------------------------------------------

}  // extern "C"

struct gheapset_s {
    int device;
    uint32_t n;
    uint32_t k;
    uint32_t key_bytes;
    uint32_t flags;
    uint32_t ipt;
    uint32_t ctas;
    int sm_count;
    uint32_t call_id;
    uint64_t timeout_ns;
    gheap_t *heaps;            // NULL for an empty slot
    uint8_t *owned;            // heaps[i] was created by the set
    void *d_table;             // gh::HeapView<K>[n]
    gh::Ctl *d_ctl;
    unsigned long long *d_stats;
    uint32_t *d_no_del;        // GHEAP_FLAG_BOTTOM_UP: the launch's list holds no DEL
};

namespace {

// Clears *no_del when the op list holds an op other than INS (the flag was
// set beforehand): a launch with only inserts may insert bottom-up.
__global__ void set_scan_no_del(const gheapset_op *ops, unsigned long long n, uint32_t *no_del)
{
    for (unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; i < n;
         i += (unsigned long long)gridDim.x * blockDim.x)
        if ((ops[i].kind_n >> 24) != GHEAP_OP_INS) *no_del = 0;
}

}  // namespace

struct gheapset_graph_s {
    cudaGraph_t graph;
    cudaGraphExec_t exec;
};

namespace {

template <typename K>
int set_launch(gheapset_t S, const gheapset_op *ops, uint64_t n_ops, const void *in, void *out,
               uint32_t *counts, const uint64_t *req_base, uint64_t *req_cursor, cudaStream_t st)
{
    gh::Params<K> p;
    memset(&p, 0, sizeof(p));
    p.ctl = S->d_ctl;
    p.stats = (S->flags & GHEAP_FLAG_STATS) ? S->d_stats : nullptr;
    p.k = S->k;
    p.mode = gh::MODE_SET;
    p.call_id = ++S->call_id;
    p.timeout_ns = S->timeout_ns;
    p.del_yields = gh::DEL_YIELDS;
    p.in = static_cast<const K *>(in);
    p.out = static_cast<K *>(out);
    p.n_ops = n_ops;
    p.out_counts = counts;
    p.table = static_cast<const gh::HeapView<K> *>(S->d_table);
    p.sops = ops;
    p.n_heaps = S->n;
    p.req_base = reinterpret_cast<const unsigned long long *>(req_base);
    p.req_cursor = reinterpret_cast<unsigned long long *>(req_cursor);
    if ((S->flags & GHEAP_FLAG_BOTTOM_UP) && n_ops) {
        // the kernel inserts bottom-up only when no DEL shares the launch
        if (cudaMemsetAsync(S->d_no_del, 0xFF, sizeof(uint32_t), st) != cudaSuccess)
            return GHEAP_ERR_CUDA;
        const uint64_t blocks = (n_ops + 255) / 256;
        const unsigned grid = (unsigned)(blocks < (uint64_t)S->sm_count * 2 ? blocks
                                                                         : (uint64_t)S->sm_count * 2);
        set_scan_no_del<<<grid, 256, 0, st>>>(ops, n_ops, S->d_no_del);
        if (cudaGetLastError() != cudaSuccess) return GHEAP_ERR_CUDA;
        p.set_bu = S->d_no_del;
    }
    Shape sp;
    sp.k = S->k;
    sp.ipt = S->ipt;
    sp.ctas = S->ctas;
    sp.per_sm_default = 2;
    sp.sm_count = S->sm_count;
    sp.d_ctl = S->d_ctl;
    return launch_k<K>(sp, p, n_ops, st);
}

template <typename K>
void fill_view(gh::HeapView<K> &v, gheap_t h)
{
    memset(&v, 0, sizeof(v));
    v.keys = static_cast<K *>(h->d_keys);
    v.state = h->d_state;
    v.buf = static_cast<K *>(h->d_buf);
    v.hdr = h->d_hdr;
    v.log = h->d_log;
    v.log_cap = h->log_cap;
    v.max_nodes = h->max_nodes;
}

}  // namespace

extern "C" {

int heapset_create(gheapset_t *out, uint32_t n_heaps, const uint64_t *capacities, uint32_t k,
                   uint32_t key_bytes, uint32_t flags, uint64_t log_capacity)
{
    if (!out || !capacities || n_heaps == 0) return GHEAP_ERR_ARG;
    *out = nullptr;
    gheapset_t S = (gheapset_t)calloc(1, sizeof(gheapset_s));
    if (!S) return GHEAP_ERR_OOM;
    S->heaps = (gheap_t *)calloc(n_heaps, sizeof(gheap_t));
    S->owned = (uint8_t *)calloc(n_heaps, 1);
    if (!S->heaps || !S->owned) { free(S->heaps); free(S->owned); free(S); return GHEAP_ERR_OOM; }
    S->n = n_heaps;
    S->k = k;
    S->key_bytes = key_bytes;
    S->flags = flags;
    S->timeout_ns = 2000000000ull;
    if (k < 1 || k > 2048 || (k & (k - 1)) != 0 || (key_bytes != 4 && key_bytes != 8)) {
        heapset_destroy(S);
        return GHEAP_ERR_ARG;
    }
    int rc = GHEAP_OK;
    for (uint32_t i = 0; i < n_heaps && rc == GHEAP_OK; i++) {
        if (capacities[i] == 0) continue;
        rc = heap_create(&S->heaps[i], capacities[i], k, key_bytes, 0, log_capacity);
        S->owned[i] = rc == GHEAP_OK;
    }
    if (rc != GHEAP_OK) {
        heapset_destroy(S);
        return rc;
    }
    cudaDeviceProp prop;
    if (cudaGetDevice(&S->device) != cudaSuccess ||
        cudaGetDeviceProperties(&prop, S->device) != cudaSuccess) {
        heapset_destroy(S);
        return GHEAP_ERR_CUDA;
    }
    S->sm_count = prop.multiProcessorCount;
    S->ipt = k >= 2048 ? 16 : 8;
    S->ctas = 0;
    size_t vb = key_bytes == 4 ? sizeof(gh::HeapView<uint32_t>) : sizeof(gh::HeapView<uint64_t>);
    void *host = calloc(n_heaps, vb);
    bool ok = host != nullptr &&
              cudaMalloc(&S->d_table, (size_t)n_heaps * vb) == cudaSuccess &&
              cudaMalloc((void **)&S->d_ctl, sizeof(gh::Ctl)) == cudaSuccess &&
              cudaMalloc((void **)&S->d_stats, gh::N_STATS * sizeof(unsigned long long)) == cudaSuccess &&
              cudaMalloc((void **)&S->d_no_del, sizeof(uint32_t)) == cudaSuccess;
    if (ok) {
        for (uint32_t i = 0; i < n_heaps; i++) {
            if (!S->heaps[i]) continue;   // calloc left the view zero: empty slot
            if (key_bytes == 4) fill_view(static_cast<gh::HeapView<uint32_t> *>(host)[i], S->heaps[i]);
            else fill_view(static_cast<gh::HeapView<uint64_t> *>(host)[i], S->heaps[i]);
        }
        ok = cudaMemcpy(S->d_table, host, (size_t)n_heaps * vb, cudaMemcpyHostToDevice) == cudaSuccess &&
             cudaMemset(S->d_stats, 0, gh::N_STATS * sizeof(unsigned long long)) == cudaSuccess &&
             cudaMemset(S->d_ctl, 0, sizeof(gh::Ctl)) == cudaSuccess;
    }
    free(host);
    if (!ok) {
        cudaGetLastError();
        heapset_destroy(S);
        return GHEAP_ERR_OOM;
    }
    *out = S;
    return GHEAP_OK;
}

int heapset_destroy(gheapset_t S)
{
    if (!S) return GHEAP_ERR_ARG;
    if (S->heaps) {
        for (uint32_t i = 0; i < S->n; i++)
            if (S->heaps[i] && S->owned && S->owned[i]) heap_destroy(S->heaps[i]);
        free(S->heaps);
    }
    free(S->owned);
    cudaFree(S->d_table);
    cudaFree(S->d_ctl);
    cudaFree(S->d_stats);
    cudaFree(S->d_no_del);
    free(S);
    return GHEAP_OK;
}

gheap_t heapset_heap(gheapset_t S, uint32_t i)
{
    if (!S || i >= S->n) return nullptr;
    return S->heaps[i];
}

int heapset_set_launch(gheapset_t S, uint32_t ctas, uint32_t items_per_thread)
{
    if (!S) return GHEAP_ERR_ARG;
    if (items_per_thread != 4 && items_per_thread != 8 && items_per_thread != 16)
        return GHEAP_ERR_ARG;
    if (merge_threads_for(S->k, items_per_thread) > max_merge_threads(items_per_thread))
        return GHEAP_ERR_ARG;
    S->ctas = ctas;
    S->ipt = items_per_thread;
    return GHEAP_OK;
}

int heapset_set_timeout(gheapset_t S, uint64_t ns)
{
    if (!S || ns == 0) return GHEAP_ERR_ARG;
    S->timeout_ns = ns;
    for (uint32_t i = 0; i < S->n; i++)
        if (S->heaps[i]) heap_set_timeout(S->heaps[i], ns);
    return GHEAP_OK;
}

int heapset_bind(gheapset_t S, uint32_t i, gheap_t h, void *stream)
{
    if (!S || !h || i >= S->n || S->heaps[i]) return GHEAP_ERR_ARG;
    if (h->k != S->k || h->key_bytes != S->key_bytes) return GHEAP_ERR_ARG;
    if (cudaSetDevice(S->device) != cudaSuccess) return GHEAP_ERR_CUDA;
    cudaError_t e;
    if (S->key_bytes == 4) {
        gh::HeapView<uint32_t> v;
        fill_view(v, h);
        e = cudaMemcpyAsync(static_cast<gh::HeapView<uint32_t> *>(S->d_table) + i, &v, sizeof(v),
                            cudaMemcpyHostToDevice, (cudaStream_t)stream);
    } else {
        gh::HeapView<uint64_t> v;
        fill_view(v, h);
        e = cudaMemcpyAsync(static_cast<gh::HeapView<uint64_t> *>(S->d_table) + i, &v, sizeof(v),
                            cudaMemcpyHostToDevice, (cudaStream_t)stream);
    }
    // the view lives on this stack frame: wait for the copy before returning
    if (e == cudaSuccess) e = cudaStreamSynchronize((cudaStream_t)stream);
    if (e != cudaSuccess) return GHEAP_ERR_CUDA;
    h->timeout_ns = S->timeout_ns;
    S->heaps[i] = h;
    S->owned[i] = 0;
    return GHEAP_OK;
}

int heapset_unbind(gheapset_t S, uint32_t i, void *stream)
{
    if (!S || i >= S->n || !S->heaps[i]) return GHEAP_ERR_ARG;
    if (cudaSetDevice(S->device) != cudaSuccess) return GHEAP_ERR_CUDA;
    size_t vb = S->key_bytes == 4 ? sizeof(gh::HeapView<uint32_t>) : sizeof(gh::HeapView<uint64_t>);
    cudaError_t e = cudaMemsetAsync(static_cast<char *>(S->d_table) + (size_t)i * vb, 0, vb,
                                    (cudaStream_t)stream);
    if (e != cudaSuccess) return GHEAP_ERR_CUDA;
    if (S->owned[i]) heap_destroy(S->heaps[i]);   // synchronizes the device first
    S->heaps[i] = nullptr;
    S->owned[i] = 0;
    return GHEAP_OK;
}

int heapset_ops(gheapset_t S, const gheapset_op *d_ops, uint64_t n_ops, const void *d_in_keys,
                void *d_out_keys, uint32_t *d_out_counts, void *stream)
{
    if (!S) return GHEAP_ERR_ARG;
    if (n_ops == 0) return GHEAP_OK;
    if (!d_ops) return GHEAP_ERR_ARG;
    if (cudaSetDevice(S->device) != cudaSuccess) return GHEAP_ERR_CUDA;
    if (S->key_bytes == 4)
        return set_launch<uint32_t>(S, d_ops, n_ops, d_in_keys, d_out_keys, d_out_counts,
                                    nullptr, nullptr, (cudaStream_t)stream);
    return set_launch<uint64_t>(S, d_ops, n_ops, d_in_keys, d_out_keys, d_out_counts, nullptr,
                                nullptr, (cudaStream_t)stream);
}

int heapset_ops_req(gheapset_t S, const gheapset_op *d_ops, uint64_t n_ops,
                    const void *d_in_keys, void *d_out_keys, uint32_t *d_out_counts,
                    const uint64_t *d_req_base, uint64_t *d_req_cursor, void *stream)
{
    if (!S) return GHEAP_ERR_ARG;
    if (n_ops == 0) return GHEAP_OK;
    if (!d_ops) return GHEAP_ERR_ARG;
    if (cudaSetDevice(S->device) != cudaSuccess) return GHEAP_ERR_CUDA;
    if (S->key_bytes == 4)
        return set_launch<uint32_t>(S, d_ops, n_ops, d_in_keys, d_out_keys, d_out_counts,
                                    d_req_base, d_req_cursor, (cudaStream_t)stream);
    return set_launch<uint64_t>(S, d_ops, n_ops, d_in_keys, d_out_keys, d_out_counts,
                                d_req_base, d_req_cursor, (cudaStream_t)stream);
}

int heapset_get_stats(gheapset_t S, uint64_t *out, uint32_t n)
{
    if (!S || !out || n > gh::N_STATS) return GHEAP_ERR_ARG;
    if (cudaSetDevice(S->device) != cudaSuccess) return GHEAP_ERR_CUDA;
    if (cudaDeviceSynchronize() != cudaSuccess) return GHEAP_ERR_CUDA;
    unsigned long long tmp[gh::N_STATS];
    if (cudaMemcpy(tmp, S->d_stats, sizeof(tmp), cudaMemcpyDeviceToHost) != cudaSuccess)
        return GHEAP_ERR_CUDA;
    for (uint32_t i = 0; i < n; i++) out[i] = tmp[i];
    return GHEAP_OK;
}

int heapset_sync(gheapset_t S)
{
    if (!S) return GHEAP_ERR_ARG;
    int first = GHEAP_OK;
    if (cudaSetDevice(S->device) != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess)
        return GHEAP_ERR_CUDA;
    for (uint32_t i = 0; i < S->n; i++) {
        if (!S->heaps[i]) continue;
        int rc = heap_sync(S->heaps[i]);
        if (rc != GHEAP_OK && first == GHEAP_OK) first = rc;
    }
    return first;
}

int heapset_reset(gheapset_t S, void *stream)
{
    if (!S) return GHEAP_ERR_ARG;
    for (uint32_t i = 0; i < S->n; i++) {
        if (!S->heaps[i]) continue;
        int rc = heap_reset(S->heaps[i], stream);
        if (rc != GHEAP_OK) return rc;
    }
    if (cudaMemsetAsync(S->d_ctl, 0, sizeof(gh::Ctl), (cudaStream_t)stream) != cudaSuccess)
        return GHEAP_ERR_CUDA;
    return cuda_err(cudaMemsetAsync(S->d_stats, 0, gh::N_STATS * sizeof(unsigned long long),
                                    (cudaStream_t)stream));
}

int heapset_graph_create(gheapset_t S, const gheapset_op *d_ops, uint64_t n_ops,
                         const void *d_in_keys, void *d_out_keys, uint32_t *d_out_counts,
                         gheapset_graph_t *out)
{
    if (!S || !out) return GHEAP_ERR_ARG;
    *out = nullptr;
    if (cudaSetDevice(S->device) != cudaSuccess) return GHEAP_ERR_CUDA;
    cudaStream_t cs;
    if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) return GHEAP_ERR_CUDA;
    gheapset_graph_t G = (gheapset_graph_t)calloc(1, sizeof(gheapset_graph_s));
    if (!G) { cudaStreamDestroy(cs); return GHEAP_ERR_OOM; }
    int rc = GHEAP_OK;
    if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) != cudaSuccess) rc = GHEAP_ERR_CUDA;
    if (rc == GHEAP_OK) {
        rc = heapset_ops(S, d_ops, n_ops, d_in_keys, d_out_keys, d_out_counts, cs);
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamEndCapture(cs, &g);
        if (rc == GHEAP_OK && e != cudaSuccess) rc = GHEAP_ERR_CUDA;
        G->graph = g;
        if (rc == GHEAP_OK && cudaGraphInstantiate(&G->exec, g, 0) != cudaSuccess) rc = GHEAP_ERR_CUDA;
    }
    cudaStreamDestroy(cs);
    if (rc != GHEAP_OK) {
        cudaGetLastError();
        heapset_graph_destroy(G);
        return rc;
    }
    *out = G;
    return GHEAP_OK;
}

int heapset_graph_launch(gheapset_graph_t G, void *stream)
{
    if (!G || !G->exec) return GHEAP_ERR_ARG;
    return cuda_err(cudaGraphLaunch(G->exec, (cudaStream_t)stream));
}

int heapset_graph_destroy(gheapset_graph_t G)
{
    if (!G) return GHEAP_ERR_ARG;
    if (G->exec) cudaGraphExecDestroy(G->exec);
    if (G->graph) cudaGraphDestroy(G->graph);
    free(G);
    return GHEAP_OK;
}

// ---------------------------------------------------------------------------
// allocation-free sort (heap_sort_noalloc): the heap in a fixed scratch array
// ---------------------------------------------------------------------------

}  // extern "C"

namespace {

constexpr uint32_t NA_K = 1024;
constexpr uint32_t NA_MAX_NODES = (uint32_t)(GHEAP_NOALLOC_MAX_KEYS / NA_K) + 1;
constexpr size_t NA_SLOTS = (size_t)NA_MAX_NODES + 1;
constexpr size_t na_round(size_t b) { return (b + 255) / 256 * 256; }
// The status word of the last call comes first, outside the region each call
// clears, so that the next call can still read it.
constexpr size_t NA_OFF_STATUS = 0;
constexpr size_t NA_OFF_HDR = 256;
constexpr size_t NA_OFF_CTL = NA_OFF_HDR + na_round(sizeof(gh::Hdr));
constexpr size_t NA_OFF_CNT = NA_OFF_CTL + na_round(sizeof(gh::Ctl));
constexpr size_t NA_OFF_STATE = NA_OFF_CNT + 256;
constexpr size_t NA_OFF_BUF = NA_OFF_STATE + na_round(NA_SLOTS * sizeof(uint32_t));
constexpr size_t NA_OFF_KEYS = NA_OFF_BUF + na_round(NA_K * sizeof(uint32_t));
constexpr size_t NA_BYTES = NA_OFF_KEYS + NA_SLOTS * NA_K * sizeof(uint32_t);

constexpr int NA_MAX_DEVICES = 64;
// per-device address of the array, filled once under its std::call_once
std::atomic<unsigned char *> na_base[NA_MAX_DEVICES];
std::once_flag na_once[NA_MAX_DEVICES];

// After the delete launch: when it wrote fewer than n keys (a bounded wait
// gave up, or the device saw an impossible state), the rest of d_out gets the
// key maximum and the status word the device error; otherwise the status
// word is cleared.
__global__ void na_finish(unsigned char *base, uint32_t *d_out, unsigned long long n)
{
    const unsigned long long got = *reinterpret_cast<const unsigned long long *>(base + NA_OFF_CNT);
    const uint32_t err = reinterpret_cast<const gh::Hdr *>(base + NA_OFF_HDR)->err;
    const unsigned long long from = got < n ? got : n;
    for (unsigned long long i = from + blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x;
         i < n; i += (unsigned long long)gridDim.x * blockDim.x)
        d_out[i] = 0xFFFFFFFFu;
    if (blockIdx.x == 0 && threadIdx.x == 0)
        *reinterpret_cast<uint32_t *>(base + NA_OFF_STATUS) =
            err != gh::E_NONE ? err : (got < n ? (uint32_t)gh::E_STATE : (uint32_t)gh::E_NONE);
}

}  // namespace

// The last call's status word, then the header, launch counters, a count
// word, node states, the partial buffer and (max_nodes + 1) node batches of
// one k = 1024 heap, each section 256-aligned.
static __device__ __align__(256) unsigned char g_noalloc_scratch[NA_BYTES];

extern "C" {

int heap_sort_noalloc(const uint32_t *d_in, uint32_t *d_out, uint64_t n, void *stream)
{
    if (n > GHEAP_NOALLOC_MAX_KEYS) return GHEAP_ERR_TOO_LARGE;
    if (n == 0) return GHEAP_OK;
    if (!d_in || !d_out) return GHEAP_ERR_ARG;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return GHEAP_ERR_CUDA;
    if (dev < 0 || dev >= NA_MAX_DEVICES) return GHEAP_ERR_ARG;
    // once per device, with that device current: the host-side name of the
    // array is not its device address
    std::call_once(na_once[dev], [dev] {
        unsigned char *b = nullptr;
        if (cudaGetSymbolAddress((void **)&b, g_noalloc_scratch) == cudaSuccess && b)
            na_base[dev].store(b);
    });
    unsigned char *base = na_base[dev].load();
    if (!base) return GHEAP_ERR_CUDA;
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return GHEAP_ERR_CUDA;
    cudaStream_t s = (cudaStream_t)stream;
    // the previous call's status (it is complete once the stream is: calls on
    // one stream are ordered); a failure is reported now, once
    uint32_t last = gh::E_NONE;
    if (cudaMemcpyAsync(&last, base + NA_OFF_STATUS, sizeof(last), cudaMemcpyDeviceToHost, s) !=
            cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return GHEAP_ERR_CUDA;
    if (last != gh::E_NONE) {
        if (cudaMemsetAsync(base + NA_OFF_STATUS, 0, sizeof(uint32_t), s) != cudaSuccess)
            return GHEAP_ERR_CUDA;
        return map_dev_err(last);
    }
    // the root word, ticket counter, error word, launch counters and node
    // states must start at zero; keys and the partial buffer need not
    if (cudaMemsetAsync(base + NA_OFF_HDR, 0, NA_OFF_BUF - NA_OFF_HDR, s) != cudaSuccess)
        return GHEAP_ERR_CUDA;
    gh::Params<uint32_t> p;
    memset(&p, 0, sizeof(p));
    p.h.keys = reinterpret_cast<uint32_t *>(base + NA_OFF_KEYS);
    p.h.state = reinterpret_cast<uint32_t *>(base + NA_OFF_STATE);
    p.h.buf = reinterpret_cast<uint32_t *>(base + NA_OFF_BUF);
    p.h.hdr = reinterpret_cast<gh::Hdr *>(base + NA_OFF_HDR);
    p.h.max_nodes = NA_MAX_NODES;
    p.ctl = reinterpret_cast<gh::Ctl *>(base + NA_OFF_CTL);
    p.k = NA_K;
    p.timeout_ns = 2000000000ull;
    Shape sp;
    sp.k = NA_K;
    sp.ipt = 8;
    sp.ctas = 0;
    sp.sm_count = sms;
    sp.d_ctl = p.ctl;
    const uint64_t n_ops = (n + NA_K - 1) / NA_K;
    p.mode = gh::MODE_INSERT;
    p.call_id = 1;
    p.in = d_in;
    p.n = n;
    int rc = launch_k<uint32_t>(sp, p, n_ops, s);
    if (rc != GHEAP_OK) return rc;
    p.mode = gh::MODE_DELETE;
    p.call_id = 2;
    p.in = nullptr;
    p.out = d_out;
    p.out_total = reinterpret_cast<unsigned long long *>(base + NA_OFF_CNT);
    rc = launch_k<uint32_t>(sp, p, n_ops, s);
    if (rc != GHEAP_OK) return rc;
    na_finish<<<(unsigned)sms, 256, 0, s>>>(base, d_out, n);
    return cuda_err(cudaGetLastError());
}

int heap_debug_hold_root(gheap_t h, void *stream)
{
    if (!h) return GHEAP_ERR_ARG;
    if (cudaSetDevice(h->device) != cudaSuccess) return GHEAP_ERR_CUDA;
    // draw the root's next ticket and never release it
    take_root_ticket<<<1, 1, 0, (cudaStream_t)stream>>>(h->d_hdr);
    return cuda_err(cudaGetLastError());
}

int heap_get_stats(gheap_t h, uint64_t *out, uint32_t n)
{
    if (!h || !out || n > gh::N_STATS) return GHEAP_ERR_ARG;
    int rc = read_state(h, nullptr);
    unsigned long long tmp[gh::N_STATS];
    if (cudaMemcpy(tmp, h->d_stats, sizeof(tmp), cudaMemcpyDeviceToHost) != cudaSuccess)
        return GHEAP_ERR_CUDA;
    for (uint32_t i = 0; i < n; i++) out[i] = tmp[i];
    return rc;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// serving ring: one persistent launch over a heap set, fed from host memory
// ---------------------------------------------------------------------------

namespace {

enum : uint8_t { RQ_FREE = 0, RQ_INFLIGHT = 1, RQ_DONE = 2, RQ_TAKEN = 3 };

// The native serving loop's completion scan ends after this many requests in
// a row still running (ring_poll).
constexpr uint64_t POLL_RUN = 512;

struct RingReq {
    uint64_t seq;
    uint64_t op_end;                 // ring position after its last op
    uint64_t in_start, in_end;       // input-arena positions (INS)
    uint64_t out_start, out_end;     // output-arena positions (DEL)
    uint64_t n;
    uint32_t heap;
    uint32_t kind;
    uint8_t state;
};

// Contiguous space of n units in a circular arena of `cap` units whose
// allocations are freed in order: returns the start position (monotonic),
// skipping the arena's end when the chunk would wrap, or UINT64_MAX.
uint64_t arena_take(uint64_t &tail, uint64_t freed, uint64_t cap, uint64_t n)
{
    uint64_t pos = tail;
    if (pos % cap + n > cap) pos = (pos / cap + 1) * cap;
    if (pos + n - freed > cap) return UINT64_MAX;
    tail = pos + n;
    return pos;
}

template <typename T>
bool host_map(T **h, T **d, size_t count)
{
    if (cudaHostAlloc((void **)h, count * sizeof(T), cudaHostAllocMapped) != cudaSuccess) {
        *h = nullptr;
        return false;
    }
    memset(*h, 0, count * sizeof(T));
    return cudaHostGetDevicePointer((void **)d, *h, 0) == cudaSuccess;
}

}  // namespace

struct gheap_ring_s {
    gheapset_t set;
    int device;
    uint32_t n_slots;
    uint64_t op_cap, in_cap, out_cap;         // ring entries, arena keys
    cudaStream_t stream;
    // pinned host memory, with the device's view of each block
    gh::RingOp *ops, *d_ops;
    unsigned long long *tail, *d_tail;
    uint32_t *stop, *d_stop;
    gh::RingDone *done, *d_done;
    uint32_t *req_ops, *d_req_ops;
    unsigned long long *req_seq, *d_req_seq;
    unsigned long long *req_base, *d_req_base;
    unsigned char *in_keys, *d_in_keys;
    unsigned char *out_keys, *d_out_keys;
    // device memory
    uint32_t *d_ops_done, *d_status, *d_err;
    unsigned long long *d_cursor;
    gh::Ctl *d_ctl;
    // host bookkeeping
    RingReq *reqs;
    uint64_t next_seq, oldest;
    uint64_t op_tail, op_free, in_tail, in_free, out_tail, out_free;
    uint64_t consumed;                        // ring positions run by earlier launches
    uint64_t *heap_ticket;                    // next root ticket per heap
    bool running;
    uint64_t idle_ns;
};

namespace {

int ring_read_ticket(gheap_ring_t r, uint32_t i)
{
    gheap_t h = r->set->heaps[i];
    if (!h) {
        r->heap_ticket[i] = 0;
        return GHEAP_OK;
    }
    cudaStream_t s;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) return GHEAP_ERR_CUDA;
    unsigned long long next = 0;
    cudaError_t e = cudaMemcpyAsync(&next, &h->d_hdr->next, sizeof(next), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaStreamDestroy(s);
    if (e != cudaSuccess) return GHEAP_ERR_CUDA;
    r->heap_ticket[i] = next;
    return GHEAP_OK;
}

template <typename K>
int ring_launch(gheap_ring_t r)
{
    gheapset_t S = r->set;
    gh::Params<K> p;
    memset(&p, 0, sizeof(p));
    p.ctl = r->d_ctl;
    p.stats = (S->flags & GHEAP_FLAG_STATS) ? S->d_stats : nullptr;
    p.k = S->k;
    p.mode = gh::MODE_RING;
    p.call_id = ++S->call_id;
    p.timeout_ns = S->timeout_ns;
    p.del_yields = 0;              // tickets are fixed: a DEL waits for its INS
    p.in = reinterpret_cast<const K *>(r->d_in_keys);
    p.out = reinterpret_cast<K *>(r->d_out_keys);
    p.table = static_cast<const gh::HeapView<K> *>(S->d_table);
    p.n_heaps = S->n;
    p.req_base = r->d_req_base;
    p.req_cursor = r->d_cursor;
    p.ring_ops = r->d_ops;
    p.ring_cap = r->op_cap;
    p.ring_base = r->consumed;
    p.ring_tail = r->d_tail;
    p.ring_stop = r->d_stop;
    p.ring_req_ops = r->d_req_ops;
    p.ring_req_seq = r->d_req_seq;
    p.ring_done = r->d_done;
    p.ring_ops_done = r->d_ops_done;
    p.ring_status = r->d_status;
    p.ring_err = r->d_err;
    p.ring_idle_ns = r->idle_ns;
    Shape sp;
    sp.k = S->k;
    sp.ipt = S->ipt;
    sp.ctas = S->ctas;
    sp.per_sm_default = 2;
    sp.sm_count = S->sm_count;
    sp.d_ctl = r->d_ctl;
    return launch_k<K>(sp, p, ~0ull, r->stream);
}

int status_code(uint32_t bits)
{
    if (bits & (1u << gh::E_TIMEOUT)) return GHEAP_ERR_TIMEOUT;
    if (bits & (1u << gh::E_FULL)) return GHEAP_ERR_FULL;
    if (bits) return GHEAP_ERR_STATE;
    return GHEAP_OK;
}

}  // namespace

extern "C" {

int heapring_destroy(gheap_ring_t r);

int heapring_create(gheap_ring_t *out, gheapset_t set, uint32_t max_requests,
                    uint64_t max_ops, uint64_t in_keys, uint64_t out_keys)
{
    if (!out || !set || max_requests == 0 || max_ops == 0 || in_keys == 0 || out_keys == 0)
        return GHEAP_ERR_ARG;
    *out = nullptr;
    uint64_t cap = 1;
    while (cap < max_ops) cap <<= 1;
    gheap_ring_t r = (gheap_ring_t)calloc(1, sizeof(gheap_ring_s));
    if (!r) return GHEAP_ERR_OOM;
    r->set = set;
    r->device = set->device;
    r->n_slots = max_requests;
    r->op_cap = cap;
    r->in_cap = in_keys;
    r->out_cap = out_keys;
    r->idle_ns = 10000000000ull;
    const size_t kb = set->key_bytes;
    r->reqs = (RingReq *)calloc(max_requests, sizeof(RingReq));
    r->heap_ticket = (uint64_t *)calloc(set->n, sizeof(uint64_t));
    bool ok = r->reqs && r->heap_ticket && cudaSetDevice(r->device) == cudaSuccess &&
              cudaStreamCreateWithFlags(&r->stream, cudaStreamNonBlocking) == cudaSuccess &&
              host_map(&r->ops, &r->d_ops, cap) && host_map(&r->tail, &r->d_tail, 1) &&
              host_map(&r->stop, &r->d_stop, 1) &&
              host_map(&r->done, &r->d_done, max_requests) &&
              host_map(&r->req_ops, &r->d_req_ops, max_requests) &&
              host_map(&r->req_seq, &r->d_req_seq, max_requests) &&
              host_map(&r->req_base, &r->d_req_base, max_requests) &&
              host_map(&r->in_keys, &r->d_in_keys, in_keys * kb) &&
              host_map(&r->out_keys, &r->d_out_keys, out_keys * kb) &&
              cudaMalloc((void **)&r->d_ops_done, max_requests * sizeof(uint32_t)) == cudaSuccess &&
              cudaMalloc((void **)&r->d_status, max_requests * sizeof(uint32_t)) == cudaSuccess &&
              cudaMalloc((void **)&r->d_err, sizeof(uint32_t)) == cudaSuccess &&
              cudaMalloc((void **)&r->d_cursor, max_requests * sizeof(unsigned long long)) == cudaSuccess &&
              cudaMalloc((void **)&r->d_ctl, sizeof(gh::Ctl)) == cudaSuccess;
    if (ok) {
        ok = cudaMemsetAsync(r->d_ops_done, 0, max_requests * sizeof(uint32_t), r->stream) == cudaSuccess &&
             cudaMemsetAsync(r->d_status, 0, max_requests * sizeof(uint32_t), r->stream) == cudaSuccess &&
             cudaMemsetAsync(r->d_err, 0, sizeof(uint32_t), r->stream) == cudaSuccess &&
             cudaMemsetAsync(r->d_cursor, 0, max_requests * sizeof(unsigned long long), r->stream) == cudaSuccess &&
             cudaMemsetAsync(r->d_ctl, 0, sizeof(gh::Ctl), r->stream) == cudaSuccess &&
             cudaStreamSynchronize(r->stream) == cudaSuccess;
    }
    for (uint32_t i = 0; ok && i < set->n; i++) ok = ring_read_ticket(r, i) == GHEAP_OK;
    if (!ok) {
        cudaGetLastError();
        heapring_destroy(r);
        return GHEAP_ERR_OOM;
    }
    *out = r;
    return GHEAP_OK;
}

int heapring_attach(gheap_ring_t r, uint32_t i)
{
    if (!r || i >= r->set->n) return GHEAP_ERR_ARG;
    if (cudaSetDevice(r->device) != cudaSuccess) return GHEAP_ERR_CUDA;
    return ring_read_ticket(r, i);
}

int heapring_start(gheap_ring_t r)
{
    if (!r) return GHEAP_ERR_ARG;
    if (r->running) return GHEAP_OK;
    if (cudaSetDevice(r->device) != cudaSuccess) return GHEAP_ERR_CUDA;
    __atomic_store_n(r->stop, 0u, __ATOMIC_RELEASE);
    const int rc = r->set->key_bytes == 4 ? ring_launch<uint32_t>(r) : ring_launch<uint64_t>(r);
    if (rc == GHEAP_OK) r->running = true;
    return rc;
}

int heapring_stop(gheap_ring_t r)
{
    if (!r) return GHEAP_ERR_ARG;
    if (!r->running) return GHEAP_OK;
    if (cudaSetDevice(r->device) != cudaSuccess) return GHEAP_ERR_CUDA;
    __atomic_store_n(r->stop, 1u, __ATOMIC_RELEASE);
    cudaError_t e = cudaStreamSynchronize(r->stream);
    r->running = false;
    // every published operation ran before the launch ended
    r->consumed = r->op_tail;
    if (e != cudaSuccess) return GHEAP_ERR_CUDA;
    uint32_t err = 0;
    e = cudaMemcpyAsync(&err, r->d_err, sizeof(err), cudaMemcpyDeviceToHost, r->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(r->stream);
    if (e != cudaSuccess) return GHEAP_ERR_CUDA;
    return err ? GHEAP_ERR_TIMEOUT : GHEAP_OK;
}

}  // extern "C"

namespace {

// Appends one request (not yet published).  Returns 1 when appended (id in
// *id), 0 when the ring, an arena or the request slots are full, or
// GHEAP_ERR_ARG for a malformed request.
int ring_append(gheap_ring_t r, uint32_t h, uint32_t kind, uint64_t n, const unsigned char *src,
                uint64_t *id)
{
    gheapset_t S = r->set;
    const uint32_t k = S->k;
    const size_t kb = S->key_bytes;
    if (h >= S->n || !S->heaps[h] || n == 0 || (kind != GHEAP_OP_INS && kind != GHEAP_OP_DEL) ||
        (kind == GHEAP_OP_INS && !src))
        return GHEAP_ERR_ARG;
    if (r->next_seq - r->oldest >= r->n_slots) return 0;
    const uint64_t n_ops = (n + k - 1) / k;
    if (r->op_tail + n_ops - r->op_free > r->op_cap) return 0;
    uint64_t in_pos = 0, out_pos = 0;
    uint64_t in_tail = r->in_tail, out_tail = r->out_tail;
    if (kind == GHEAP_OP_INS) {
        in_pos = arena_take(in_tail, r->in_free, r->in_cap, n);
        if (in_pos == UINT64_MAX) return 0;
    } else {
        out_pos = arena_take(out_tail, r->out_free, r->out_cap, n);
        if (out_pos == UINT64_MAX) return 0;
    }
    const uint64_t seq = r->next_seq;
    const uint32_t slot = (uint32_t)(seq % r->n_slots);
    RingReq &q = r->reqs[slot];
    q.seq = seq;
    q.heap = h;
    q.kind = kind;
    q.n = n;
    q.in_start = kind == GHEAP_OP_INS ? in_pos : r->in_tail;
    q.in_end = in_tail;
    q.out_start = kind == GHEAP_OP_DEL ? out_pos : r->out_tail;
    q.out_end = out_tail;
    r->in_tail = in_tail;
    r->out_tail = out_tail;
    r->req_ops[slot] = (uint32_t)n_ops;
    r->req_seq[slot] = seq;
    r->req_base[slot] = kind == GHEAP_OP_DEL ? out_pos % r->out_cap : 0;
    if (kind == GHEAP_OP_INS) memcpy(r->in_keys + (in_pos % r->in_cap) * kb, src, n * kb);
    for (uint64_t j = 0; j < n_ops; j++) {
        gh::RingOp &o = r->ops[r->op_tail % r->op_cap];
        const uint32_t m = (uint32_t)(n - j * k < k ? n - j * k : k);
        o.heap = h;
        o.kind_n = (kind << 24) | (kind == GHEAP_OP_DEL ? GHEAPSET_CURSOR : 0u) | m;
        o.offset = kind == GHEAP_OP_INS ? in_pos % r->in_cap + j * k : slot;
        o.ticket = r->heap_ticket[h]++;
        o.req = slot;
        o._pad = 0;
        r->op_tail++;
    }
    q.op_end = r->op_tail;
    q.state = RQ_INFLIGHT;
    r->next_seq++;
    *id = seq;
    return 1;
}

// Publishes every appended entry: one release store of the tail after them.
void ring_publish(gheap_ring_t r)
{
    __atomic_store_n(r->tail, (unsigned long long)r->op_tail, __ATOMIC_RELEASE);
}

// Marks completed and reports up to `max` requests in submission order,
// scanning from the oldest one in flight; the scan ends after `run` requests
// in a row that are still running (the ring runs operations in order, so
// the finished ones are mostly the oldest; a later one is found by a later
// call).  Returns the count.
uint32_t ring_poll(gheap_ring_t r, uint64_t *ids, uint64_t *counts, int32_t *status, uint32_t max,
                   uint64_t run)
{
    uint32_t c = 0;
    uint64_t busy = 0;
    for (uint64_t s = r->oldest; s < r->next_seq && c < max && busy < run; s++) {
        const uint32_t slot = (uint32_t)(s % r->n_slots);
        RingReq &q = r->reqs[slot];
        if (q.state != RQ_INFLIGHT) continue;
        if (__atomic_load_n(&r->done[slot].seq, __ATOMIC_ACQUIRE) != s + 1) {
            busy++;
            continue;
        }
        busy = 0;
        q.state = RQ_DONE;
        ids[c] = s;
        if (counts) counts[c] = q.kind == GHEAP_OP_DEL ? r->done[slot].count : q.n;
        if (status) status[c] = status_code(r->done[slot].status);
        c++;
    }
    return c;
}

}  // namespace

extern "C" {

int heapring_submit(gheap_ring_t r, uint32_t n_req, const uint32_t *heaps, const uint32_t *kinds,
                    const uint64_t *sizes, const void *keys, uint64_t *ids)
{
    if (!r || (n_req && (!heaps || !kinds || !sizes))) return GHEAP_ERR_ARG;
    const size_t kb = r->set->key_bytes;
    const unsigned char *src = static_cast<const unsigned char *>(keys);
    uint32_t i = 0;
    for (; i < n_req; i++) {
        uint64_t id = 0;
        const int rc = ring_append(r, heaps[i], kinds[i], sizes[i],
                                   kinds[i] == GHEAP_OP_INS ? src : nullptr, &id);
        if (rc < 0) {
            if (i == 0) return rc;
            break;
        }
        if (rc == 0) break;
        if (kinds[i] == GHEAP_OP_INS) src += sizes[i] * kb;
        if (ids) ids[i] = id;
    }
    ring_publish(r);
    return (int)i;
}

int heapring_poll(gheap_ring_t r, uint64_t *ids, uint64_t *counts, int32_t *status, uint32_t max,
                  uint32_t *n_done)
{
    if (!r || !n_done || (max && !ids)) return GHEAP_ERR_ARG;
    *n_done = ring_poll(r, ids, counts, status, max, UINT64_MAX);
    return GHEAP_OK;
}

int heapring_take(gheap_ring_t r, uint32_t n, const uint64_t *ids, void *host_out, uint64_t cap,
                  uint64_t *counts)
{
    if (!r || (n && !ids)) return GHEAP_ERR_ARG;
    const size_t kb = r->set->key_bytes;
    unsigned char *dst = static_cast<unsigned char *>(host_out);
    uint64_t used = 0;
    for (uint32_t i = 0; i < n; i++) {
        const uint64_t id = ids[i];
        if (id >= r->next_seq || id < r->oldest) return GHEAP_ERR_ARG;
        const uint32_t slot = (uint32_t)(id % r->n_slots);
        RingReq &q = r->reqs[slot];
        if (q.seq != id || q.state != RQ_DONE) return GHEAP_ERR_ARG;
        uint64_t cnt = 0;
        if (q.kind == GHEAP_OP_DEL) {
            cnt = r->done[slot].count;
            if (used + cnt > cap || (cnt && !dst)) return GHEAP_ERR_ARG;
            memcpy(dst + used * kb, r->out_keys + (q.out_start % r->out_cap) * kb, cnt * kb);
            used += cnt;
        }
        if (counts) counts[i] = cnt;
        q.state = RQ_TAKEN;
    }
    // free the arenas, the op entries and the slots of the oldest requests taken
    while (r->oldest < r->next_seq) {
        RingReq &o = r->reqs[r->oldest % r->n_slots];
        if (o.state != RQ_TAKEN) break;
        r->op_free = o.op_end;
        if (o.in_end > r->in_free) r->in_free = o.in_end;
        if (o.out_end > r->out_free) r->out_free = o.out_end;
        o.state = RQ_FREE;
        r->oldest++;
    }
    return GHEAP_OK;
}

int heapring_pending(gheap_ring_t r, uint64_t *in_flight)
{
    if (!r || !in_flight) return GHEAP_ERR_ARG;
    *in_flight = r->next_seq - r->oldest;
    return GHEAP_OK;
}

int heapring_serve(gheap_ring_t r, uint64_t n_req, const double *arrival, const uint32_t *heaps,
                   const uint32_t *kinds, const uint64_t *sizes, const void *keys,
                   const uint64_t *capacities, uint64_t *held, int realtime, void *out,
                   uint64_t *out_counts, double *t_submit, double *t_done, int32_t *status)
{
    if (!r || (n_req && (!arrival || !heaps || !kinds || !sizes || !capacities || !held ||
                         !out_counts || !t_submit || !t_done || !status)))
        return GHEAP_ERR_ARG;
    if (!r->running) return GHEAP_ERR_ARG;
    gheapset_t S = r->set;
    const uint32_t nh = S->n;
    const size_t kb = S->key_bytes;
    const unsigned char *in = static_cast<const unsigned char *>(keys);
    unsigned char *dst = static_cast<unsigned char *>(out);
    // each insert's keys and each deleteMin's output place, in request order
    std::vector<uint64_t> key_off(n_req), out_off(n_req);
    uint64_t ko = 0, oo = 0;
    for (uint64_t i = 0; i < n_req; i++) {
        key_off[i] = ko;
        out_off[i] = oo;
        if (kinds[i] == GHEAP_OP_INS) ko += sizes[i];
        else oo += sizes[i];
        out_counts[i] = 0;
        t_submit[i] = t_done[i] = -1.0;
        status[i] = GHEAP_OK;
    }
    std::vector<std::deque<uint64_t>> queue(nh);
    std::vector<uint64_t> busy(nh, 0);
    std::vector<uint8_t> blocked(nh, 0), listed(nh, 0);
    std::deque<uint32_t> ready;             // heaps with queued requests, not blocked
    const uint64_t base = r->next_seq;      // ids from here on are this call's submissions
    std::vector<uint64_t> req_of;           // request index of id base + j
    req_of.reserve(n_req);
    std::vector<uint64_t> ids(r->n_slots), counts(r->n_slots);
    std::vector<int32_t> sts(r->n_slots);
    const uint64_t arena = r->in_cap < r->out_cap ? r->in_cap : r->out_cap;
    const auto t0 = std::chrono::steady_clock::now();
    auto now_s = [&]() {
        return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    };
    uint64_t next = 0, done = 0, inflight = 0;
    double last_progress = 0.0;
    auto finish = [&](uint64_t i, int32_t st, double t) {
        status[i] = st;
        t_done[i] = t;
        done++;
    };
    while (done < n_req) {
        double now = now_s();
        bool progress = false;
        // arrivals, in order
        while (next < n_req && (!realtime || arrival[next] <= now)) {
            const uint32_t h = heaps[next];
            if (h >= nh || !S->heaps[h] || sizes[next] == 0 ||
                (kinds[next] != GHEAP_OP_INS && kinds[next] != GHEAP_OP_DEL)) {
                finish(next, GHEAP_ERR_ARG, now);
            } else {
                queue[h].push_back(next);
                if (!listed[h] && !blocked[h]) {
                    listed[h] = 1;
                    ready.push_back(h);
                }
            }
            next++;
            progress = true;
        }
        // completions: take each deleteMin's keys into its place
        uint32_t nd = 0;
        // with many requests in flight a full scan of them on every pass
        // would cost more than the completions it finds
        nd = ring_poll(r, ids.data(), counts.data(), sts.data(), r->n_slots, POLL_RUN);
        now = now_s();
        for (uint32_t j = 0; j < nd; j++) {
            const uint64_t i = req_of[ids[j] - base];
            const uint32_t h = heaps[i];
            uint64_t got = 0;
            heapring_take(r, 1, &ids[j], kinds[i] == GHEAP_OP_DEL ? dst + out_off[i] * kb : nullptr,
                          kinds[i] == GHEAP_OP_DEL ? sizes[i] : 0, &got);
            out_counts[i] = kinds[i] == GHEAP_OP_DEL ? got : sizes[i];
            if (kinds[i] == GHEAP_OP_DEL) held[h] -= got;
            busy[h]--;
            inflight--;
            if (blocked[h]) {
                blocked[h] = 0;
                if (!queue[h].empty() && !listed[h]) {
                    listed[h] = 1;
                    ready.push_back(h);
                }
            }
            finish(i, sts[j], now);
            progress = true;
        }
        // submissions: every ready heap's queue in order, until one must wait
        bool appended = false, full = false;
        for (size_t round = ready.size(); round > 0 && !full; --round) {
            const uint32_t h = ready.front();
            ready.pop_front();
            listed[h] = 0;
            auto &qh = queue[h];
            while (!qh.empty()) {
                const uint64_t i = qh.front();
                const uint64_t n = sizes[i];
                const bool ins = kinds[i] == GHEAP_OP_INS;
                if (n > arena || (ins && n > capacities[h])) {
                    qh.pop_front();
                    finish(i, ins && n > capacities[h] ? GHEAP_ERR_FULL : GHEAP_ERR_ARG, now);
                    continue;
                }
                if (ins && held[h] + n > capacities[h]) {
                    if (busy[h] == 0) {
                        // nothing ahead of it can make room: refuse it
                        qh.pop_front();
                        finish(i, GHEAP_ERR_FULL, now);
                        continue;
                    }
                    blocked[h] = 1;        // waits for this heap's completions
                    break;
                }
                uint64_t id = 0;
                const int rc = ring_append(r, h, kinds[i], n, ins ? in + key_off[i] * kb : nullptr,
                                           &id);
                if (rc < 0) {
                    qh.pop_front();
                    finish(i, rc, now);
                    continue;
                }
                if (rc == 0) {
                    full = true;           // the ring is full: retry after completions
                    break;
                }
                qh.pop_front();
                req_of.push_back(i);
                t_submit[i] = now;
                if (ins) held[h] += n;
                busy[h]++;
                inflight++;
                appended = true;
            }
            if (!qh.empty() && !blocked[h] && !listed[h]) {
                listed[h] = 1;
                ready.push_back(h);
            }
        }
        if (appended) {
            ring_publish(r);
            progress = true;
        }
        if (progress) {
            last_progress = now;
            continue;
        }
        if (inflight == 0 && ready.empty() && next < n_req && realtime) {
            // idle until the next arrival
            const double wait = arrival[next] - now_s();
            if (wait > 2e-4) std::this_thread::sleep_for(std::chrono::duration<double>(wait - 1e-4));
            last_progress = now_s();
            continue;
        }
        if (now - last_progress > 60.0) return GHEAP_ERR_TIMEOUT;
    }
    return GHEAP_OK;
}

int heapring_destroy(gheap_ring_t r)
{
    if (!r) return GHEAP_ERR_ARG;
    heapring_stop(r);
    cudaSetDevice(r->device);
    cudaFreeHost(r->ops);
    cudaFreeHost(r->tail);
    cudaFreeHost(r->stop);
    cudaFreeHost(r->done);
    cudaFreeHost(r->req_ops);
    cudaFreeHost(r->req_seq);
    cudaFreeHost(r->req_base);
    cudaFreeHost(r->in_keys);
    cudaFreeHost(r->out_keys);
    cudaFree(r->d_ops_done);
    cudaFree(r->d_status);
    cudaFree(r->d_err);
    cudaFree(r->d_cursor);
    cudaFree(r->d_ctl);
    if (r->stream) cudaStreamDestroy(r->stream);
    free(r->reqs);
    free(r->heap_ticket);
    free(r);
    return GHEAP_OK;
}

}  // extern "C"

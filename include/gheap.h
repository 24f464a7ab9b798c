/*
 * gheap.h -- C ABI of the GB300 generalized concurrent heap.
 *
 * Implements the TD-INS/TD-DEL concurrent heap of "Accelerating Concurrent
 * Heap on GPUs" (Chen, Hua, Huang, Bierema, Zhang, Zhang; arXiv 1906.06504),
 * and its BU-INS/TD-DEL variant (GHEAP_FLAG_BOTTOM_UP, Section 3.3.4):
 * a min-heap whose nodes each hold k sorted keys (Section 3.1), insert and
 * deleteMin as top-down walks that MergeAndSort one k-batch per level
 * (Section 3.2; bottom-up inserts rise from their target instead),
 * per-node multi-state locks taken parent before child
 * (Section 3.3.1), a partial buffer at the root for batches smaller than k
 * (Section 3.3.2) and bit-reversal target placement (Section 4.3).  Every
 * operation runs on one thread block of a persistent CUDA kernel; the whole
 * heap lives in device memory.
 *
 * Conventions for every entry point:
 *   - Return value: GHEAP_OK (0) or a negative GHEAP_ERR_* code.
 *   - Key buffers passed in are DEVICE pointers owned by the caller, holding
 *     `key_bytes`-wide unsigned integers (uint32_t or uint64_t) in native
 *     byte order; they must stay valid until the work enqueued on `stream`
 *     has finished.  Heap memory is owned by the library.
 *   - `stream` is a cudaStream_t passed as void* (NULL = the legacy default
 *     stream).  Work is enqueued asynchronously and ordered on that stream.
 *   - Device-side failures (a lock wait that gave up, GHEAP_ERR_TIMEOUT; an
 *     insert past the node storage, GHEAP_ERR_FULL) are sticky: they are
 *     reported by heap_sync() and by every later call on the same heap, and
 *     the heap must then be reset or destroyed.
 *   - A heap may be used from one host thread at a time.
 */
#ifndef GHEAP_H
#define GHEAP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct gheap_s *gheap_t;

#define GHEAP_OK 0
#define GHEAP_ERR_ARG (-1)     /* bad argument: null pointer, k, key_bytes */
#define GHEAP_ERR_OOM (-2)     /* device allocation failed                 */
#define GHEAP_ERR_FULL (-3)    /* insert would exceed capacity_keys        */
#define GHEAP_ERR_TIMEOUT (-4) /* a bounded lock wait gave up (sticky)     */
#define GHEAP_ERR_CUDA (-5)    /* a CUDA runtime call failed               */
#define GHEAP_ERR_STATE (-6)   /* device found an impossible node state    */
#define GHEAP_ERR_TOO_LARGE (-7) /* beyond the fixed scratch of heap_sort_noalloc */

/* heap_create flags */
#define GHEAP_FLAG_STATS 1u    /* count node loads/stores and merges       */
#define GHEAP_FLAG_BOTTOM_UP 2u /* heap_insert / heap_insert_dev insert
    bottom-up (BU-INS, Sections 3.2.2 and 3.3.4): a full batch is placed at
    the target node and rises, merging with each parent (which keeps the k
    smallest), until the parent's maximum is at most the batch's minimum or
    the root is reached; it holds the root only to reserve the target.  An
    insert is linearized under its last lock.  Launches that mix inserts and
    deletes (heap_ops, heap sets) still insert top-down.                    */

/* One entry of the linearization record (Section 3.3.3): the operation that
 * held the root lock in that position.  kind_n = (kind << 24) | n with kind
 * GHEAP_OP_INS or GHEAP_OP_DEL and n the keys inserted or returned.  `ref` is
 * the input key offset of an insert chunk (heap_insert), the output key
 * offset of a delete (heap_delete_min), or the op index (heap_ops). */
typedef struct {
    uint32_t call_id;
    uint32_t kind_n;
    uint64_t ref;
} gheap_log_entry;

#define GHEAP_OP_INS 1u
#define GHEAP_OP_DEL 2u

/* One operation of heap_ops.  INS: insert n (1..k) keys read from
 * in_keys[offset .. offset+n).  DEL: delete up to n (1..k) smallest keys and
 * write them ascending to out_keys[offset ..); the count goes to
 * out_counts[i]. */
typedef struct {
    uint32_t kind;
    uint32_t n;
    uint64_t offset;
} gheap_op;

/* Creates an empty heap able to hold `capacity_keys` keys in nodes of `k`
 * keys (Section 3.1: node i occupies keys [i*k, (i+1)*k) of one array).
 * k: a power of two in [1, 2048].  key_bytes: 4 or 8.  flags: GHEAP_FLAG_*.
 * log_capacity: number of linearization-record entries kept (0 = none).
 * Allocates all device memory on the current CUDA device; errors: ARG, OOM,
 * CUDA. */
int heap_create(gheap_t *out, uint64_t capacity_keys, uint32_t k,
                uint32_t key_bytes, uint32_t flags, uint64_t log_capacity);

/* Frees the heap and its device memory (synchronizes the device first). */
int heap_destroy(gheap_t h);

/* Launch shape of the persistent kernels: `ctas` thread blocks (0 = one per
 * SM; a larger count is clamped to the blocks that fit on the device at
 * once), each of 2k/items_per_thread merge threads
 * (at least 32; at most 512 for items_per_thread 4, 256 for 8 and 16) plus
 * one control warp that takes the node locks and one release warp that
 * releases them for deleteMin; items_per_thread in {4, 8, 16}.
 * The paper's best setting is k = 1024 with 512 threads (Section 5.4), i.e.
 * items_per_thread = 4; the default is 8 (256 merge threads and more
 * registers per thread, measured faster on GB300), 16 for k = 2048. */
int heap_set_launch(gheap_t h, uint32_t ctas, uint32_t items_per_thread);

/* Bound on every lock wait, in nanoseconds (default 2e9).  A wait that runs
 * out sets the sticky GHEAP_ERR_TIMEOUT and the kernel returns. */
int heap_set_timeout(gheap_t h, uint64_t ns);

/* Turns the device counters of heap_get_stats on or off for later launches
 * (GHEAP_FLAG_STATS at creation turns them on from the start).  Counting
 * costs time: a run that counts is not a timed run. */
int heap_set_stats(gheap_t h, uint32_t on);

/* INS/DEL cooperation (Section 3.3.2): a DEL whose last node is the target of
 * an INS still on its way down marks that target and waits, holding the
 * root, until the INS delivers its keys -- the paper's protocol, n = 0 (the
 * default).  The INS checks its target at every level and, once marked,
 * hands over the keys it carries after the level it is on, so the wait is
 * one level step.  With n > 0 the DEL first hands the root back and queues
 * again up to n times, so that the operations behind it proceed meanwhile;
 * only the root order changes, never what a DEL returns for its place in
 * that order. */
int heap_set_yields(gheap_t h, uint32_t n);

/* Inserts n keys (Section 3.2.2 top-down INS, Section 3.3.2 partial
 * buffer).  The keys are split into ceil(n/k) INS operations of consecutive
 * chunks of k (the last may be partial), run concurrently by the persistent
 * thread blocks.  Returns GHEAP_ERR_FULL, and enqueues nothing, when the
 * heap could exceed capacity_keys. */
int heap_insert(gheap_t h, const void *d_keys, uint64_t n, void *stream);

/* heap_insert with the key count in device memory: inserts the first
 * min(*d_n, max_n) keys of d_keys (device), *d_n being read when the work
 * runs on `stream`, so a kernel enqueued before it may produce the count.
 * Nothing synchronizes.  The capacity is checked on the device only: an
 * insert that finds no free node sets the sticky GHEAP_ERR_FULL (reported by
 * heap_sync and later calls), and the keys of that insert are lost. */
int heap_insert_dev(gheap_t h, const void *d_keys, const uint64_t *d_n, uint64_t max_n,
                    void *stream);

/* Deletes the min(n, size) smallest keys (Section 3.2.1 DEL) as ceil(n/k)
 * DEL operations and writes them to d_out in the order the operations held
 * the root, which is ascending when no insert runs concurrently.  When
 * d_count is not NULL it receives (device uint64_t) the number written. */
int heap_delete_min(gheap_t h, void *d_out, uint64_t n, uint64_t *d_count,
                    void *stream);

/* Runs an arbitrary list of INS/DEL operations concurrently (the mixed
 * insert/delete workload of Section 5.5).  d_ops: device array of n_ops
 * gheap_op.  max_insert_keys: the caller's bound on the keys the list
 * inserts, used for the capacity check.  d_out_counts: device uint32_t per
 * op (DEL: keys returned; INS: n), may be NULL.  d_in_keys must be a valid
 * device array when the list holds an INS, and d_out_keys when it holds a
 * DEL: the operations are on the device, so the host cannot check this, and
 * the kernel dereferences the pointer. */
int heap_ops(gheap_t h, const gheap_op *d_ops, uint64_t n_ops,
             const void *d_in_keys, void *d_out_keys, uint32_t *d_out_counts,
             uint64_t max_insert_keys, void *stream);

/* Waits for all work on the heap's last stream and returns its sticky device
 * error, if any. */
int heap_sync(gheap_t h);

/* Number of keys in the heap (synchronizes). */
int heap_size(gheap_t h, uint64_t *out);

/* Empties the heap, clears its linearization record and any sticky error
 * (enqueued on `stream`). */
int heap_reset(gheap_t h, void *stream);

/* Copies up to `cap` linearization-record entries to host memory, in root
 * order, and the total number of operations recorded so far to *n_total
 * (synchronizes).  Entries beyond log_capacity are not kept; a heap created
 * with log_capacity 0 keeps no record and counts nothing (*n_total = 0). */
int heap_get_log(gheap_t h, gheap_log_entry *host_buf, uint64_t cap,
                 uint64_t *n_copied, uint64_t *n_total);

/* Copies a quiescent heap to host memory (synchronizes): host_keys receives
 * (max_nodes+1)*k keys indexed by storage slot, host_state (max_nodes+1)
 * uint32_t node states (1 = occupied), host_buf k keys (the partial buffer),
 * hdr[0] = full nodes, hdr[1] = partial-buffer keys, hdr[2] = operations
 * recorded.  Storage slot j holds the j-th allocated node, whose tree
 * position is given by heap_slot_to_node().  Any pointer may be NULL. */
int heap_snapshot(gheap_t h, void *host_keys, uint32_t *host_state,
                  void *host_buf, uint64_t *hdr);

/* Shape queries: node capacity in nodes (max_nodes) and k. */
int heap_geometry(gheap_t h, uint64_t *max_nodes, uint32_t *k,
                  uint32_t *key_bytes);

/* Tree position (1-based, children of p are 2p and 2p+1) of storage slot
 * j >= 1: the bit-reversal permutation within the slot's level
 * (Section 4.3).  The map is its own inverse. */
uint64_t heap_slot_to_node(uint64_t j);

/* Device counters when created with GHEAP_FLAG_STATS (synchronizes), n <= 24:
 * out[0] node loads, out[1] node stores, out[2] merges, out[3] merges skipped
 * as disjoint (Section 4.3), out[4] INS ops, out[5] DEL ops, out[6] lock
 * waits that spun, out[7] sum of root-hold time in ns; then SM cycles seen
 * by the operating block per phase: DEL root-lock wait [8], DEL root step
 * before the children [9], DEL child-lock waits [10], child loads [11],
 * merges [12], stores + releases [13], DEL sift levels [14], INS root-lock
 * wait [15], INS batch sort [16], INS node-lock waits [17], INS level steps
 * [18], INS levels [19]; DELs that received the keys of an INS whose target
 * they had marked (Section 3.3.2) [20], root hand-backs of DELs waiting for
 * such an INS (heap_set_yields) [21], children a DEL found reserved as the
 * target of an INS still on its way down and treated as absent [22], INSs
 * that handed their keys to a DEL that had marked their target, at the
 * level they were on, instead of carrying them to it [23]. */
int heap_get_stats(gheap_t h, uint64_t *out, uint32_t n);

/* Test hook for the bounded waits: marks the root lock as held, with no
 * holder that will ever release it, so that every later operation's wait
 * runs out (GHEAP_ERR_TIMEOUT after the heap_set_timeout bound) instead of
 * completing.  The paper has no counterpart; heap_reset() undoes it. */
int heap_debug_hold_root(gheap_t h, void *stream);

/* ------------------------------------------------------------------------
 * Heap sets: many independent heaps driven by one persistent launch.
 *
 * Each heap of a set is an ordinary generalized heap with its own root lock,
 * so operations on different heaps never wait for each other; operations on
 * the same heap are linearized by that heap's root as for a single heap
 * (Section 3.3.3).  One launch runs a list of operations that name their
 * heap; the persistent thread blocks take them in list order.
 * ------------------------------------------------------------------------ */

typedef struct gheapset_s *gheapset_t;

/* One operation of heapset_ops: heap index, kind_n = (GHEAP_OP_INS or
 * GHEAP_OP_DEL) << 24 | flags | n (1..k), and the key offset into the
 * launch's input (INS) or output (DEL) array.  With GHEAPSET_CURSOR (DEL
 * only), `offset` is instead a request index r: the op writes its keys at
 * d_req_base[r] + d_req_cursor[r] and advances d_req_cursor[r] by its count
 * while it holds the heap's root, so that the DELs of one request fill one
 * contiguous ascending result whatever order they run in. */
typedef struct {
    uint32_t heap;
    uint32_t kind_n;
    uint64_t offset;
} gheapset_op;

#define GHEAPSET_CURSOR (1u << 23)

/* Creates a set of n_heaps slots; capacities[i] (host array) is heap i's
 * capacity in keys, 0 for an empty slot (see heapset_bind).  k, key_bytes,
 * flags and log_capacity (per heap) as for heap_create.  With
 * GHEAP_FLAG_BOTTOM_UP, a set launch whose op list holds no DEL inserts
 * bottom-up (a small kernel checks the list on the device before the
 * launch); lists with DELs insert top-down.  All heaps live on the current
 * device. */
int heapset_create(gheapset_t *out, uint32_t n_heaps, const uint64_t *capacities, uint32_t k,
                   uint32_t key_bytes, uint32_t flags, uint64_t log_capacity);

/* Frees every heap of the set (synchronizes the device first). */
int heapset_destroy(gheapset_t s);

/* Heap i of the set (NULL for an empty slot), for the single-heap calls
 * (heap_size, heap_get_log, heap_snapshot, heap_reset, ...). */
gheap_t heapset_heap(gheapset_t s, uint32_t i);

/* Puts heap h (created by heap_create with the set's k and key_bytes, owned
 * by the caller) into empty slot i, enqueued on `stream`; later launches on
 * that stream see it.  Errors: ARG (slot taken, shape mismatch). */
int heapset_bind(gheapset_t s, uint32_t i, gheap_t h, void *stream);

/* Empties slot i (enqueued on `stream`); ops naming it are skipped.  A heap
 * the set created is destroyed after the device is synchronized; a bound
 * heap goes back to its owner. */
int heapset_unbind(gheapset_t s, uint32_t i, void *stream);

/* The set's operation counters (created with GHEAP_FLAG_STATS), summed over
 * every launch on the set, in the order and meaning of heap_get_stats; n <=
 * 24 (synchronizes). */
int heapset_get_stats(gheapset_t s, uint64_t *out, uint32_t n);

/* Launch shape and wait bound, as heap_set_launch / heap_set_timeout, except
 * that ctas = 0 means two blocks per SM (operations on different heaps run
 * in parallel). */
int heapset_set_launch(gheapset_t s, uint32_t ctas, uint32_t items_per_thread);
int heapset_set_timeout(gheapset_t s, uint64_t ns);

/* Runs d_ops[0..n_ops) (device gheapset_op array) in one persistent launch.
 * INS reads keys from d_in_keys[offset..], DEL writes the keys it removes,
 * ascending, to d_out_keys[offset..] and its count to d_out_counts[i]
 * (INS: n, or 0 when skipped).  An op whose heap already holds a sticky
 * error is skipped; an insert beyond a heap's node storage sets that heap's
 * GHEAP_ERR_FULL.  Capacities are not checked on the host.  d_out_keys must
 * be a valid device array when the list holds a DEL (the host cannot see
 * the operations; the kernel dereferences it).  With d_in_keys
 * NULL (and d_out_keys given) the list must hold only DELs: it runs the
 * delete-only specialisation of the kernel (one block per SM, the root
 * step's node fetches by TMA), and an INS in it sets its heap's
 * GHEAP_ERR_STATE while the other heaps go on. */
int heapset_ops(gheapset_t s, const gheapset_op *d_ops, uint64_t n_ops, const void *d_in_keys,
                void *d_out_keys, uint32_t *d_out_counts, void *stream);

/* heapset_ops with per-request cursors for GHEAPSET_CURSOR DELs: device
 * uint64_t arrays indexed by request (d_req_cursor is read and advanced; the
 * caller zeroes it). */
int heapset_ops_req(gheapset_t s, const gheapset_op *d_ops, uint64_t n_ops,
                    const void *d_in_keys, void *d_out_keys, uint32_t *d_out_counts,
                    const uint64_t *d_req_base, uint64_t *d_req_cursor, void *stream);

/* Waits for the device and returns the first sticky error of any heap. */
int heapset_sync(gheapset_t s);

/* Empties every heap and clears their records and errors (on `stream`). */
int heapset_reset(gheapset_t s, void *stream);

/* CUDA-graph form of heapset_ops: records the launch for the given arrays
 * once (stream capture) and replays it with heapset_graph_launch; the arrays
 * must stay valid while the graph exists. */
typedef struct gheapset_graph_s *gheapset_graph_t;
int heapset_graph_create(gheapset_t s, const gheapset_op *d_ops, uint64_t n_ops,
                         const void *d_in_keys, void *d_out_keys, uint32_t *d_out_counts,
                         gheapset_graph_t *out);
int heapset_graph_launch(gheapset_graph_t g, void *stream);
int heapset_graph_destroy(gheapset_graph_t g);

/* ------------------------------------------------------------------------
 * Serving ring: continuous batching over a heap set.
 *
 * One persistent launch serves insert and deleteMin requests on the heaps of
 * a set while the host keeps adding requests.  The requests, their input keys
 * and their results live in pinned host memory that the GPU reads and writes
 * directly (coherently over NVLink-C2C on a Grace host, over PCIe elsewhere):
 * the host appends a request's operations to a ring and publishes the ring's
 * tail with one release store; the launch's thread blocks take operations in
 * ring order as soon as they are published, so a request that arrives while
 * others run starts at once and runs beside them; the block that finishes a
 * request's last operation writes its completion record to host memory.
 * Every heap takes its requests in submission order: the host numbers each
 * heap's operations with that heap's root tickets (Section 3.3.3's root lock
 * order), so whichever blocks pick them up, they hold the root in that order
 * and each result is the one the same requests give one call at a time.  A
 * DEL whose last node is an INS target still in flight marks it and waits
 * for the keys (Section 3.3.2; heap_set_yields does not apply here).
 *
 * Requests: an insert of n >= 1 keys (ceil(n/k) INS operations) or a
 * deleteMin of up to n >= 1 keys (ceil(n/k) DEL operations whose results
 * fill one contiguous, ascending output).  Any number of requests may be in
 * flight per heap, up to the ring's limits.  Heaps of the set must be driven
 * only through the ring while it runs, and no other launch on the set may
 * overlap it.  Heap memory must not be freed (heapset_unbind, heap_destroy)
 * while the ring runs: stop it first, and destroy the ring before its set.
 * A ring is driven by one host thread at a time (its host-side bookkeeping
 * takes no lock).
 * ------------------------------------------------------------------------ */
typedef struct gheap_ring_s *gheap_ring_t;

/* A ring over `set` with room for max_requests requests in flight,
 * max_ops operation entries (rounded up to a power of two), in_keys input
 * keys and out_keys output keys (all in pinned host memory; the set's key
 * width).  Reads each bound heap's next root ticket (synchronizes).  The
 * ring is not running until heapring_start. */
int heapring_create(gheap_ring_t *out, gheapset_t set, uint32_t max_requests,
                    uint64_t max_ops, uint64_t in_keys, uint64_t out_keys);

/* Stops the launch if it runs (heapring_stop) and frees the ring. */
int heapring_destroy(gheap_ring_t r);

/* After heapset_bind of heap i while the ring is stopped or running: reads
 * that heap's next root ticket (synchronizes a private stream only). */
int heapring_attach(gheap_ring_t r, uint32_t i);

/* Launches the persistent serving kernel on the ring's own stream (a no-op
 * when it runs).  It runs until heapring_stop; a launch that receives no
 * operation for 10 s ends with an error that heapring_stop reports. */
int heapring_start(gheap_ring_t r);

/* Asks the launch to end once every published operation has run, and waits
 * for it.  Returns GHEAP_ERR_TIMEOUT when the launch ended on its idle bound. */
int heapring_stop(gheap_ring_t r);

/* Appends up to n_req requests: heap index, kind (GHEAP_OP_INS or
 * GHEAP_OP_DEL) and size per request; `keys` (host memory) holds the insert
 * requests' keys back to back, in request order.  The keys are copied, so
 * the caller may reuse `keys` on return.  Each accepted request's id goes to
 * ids[i].  Returns how many requests were accepted (in order; fewer when the
 * ring, an arena or the request slots are full: poll, take and retry), or
 * GHEAP_ERR_ARG for a malformed first request (an empty heap slot, n = 0).
 * The requests are published before the call returns. */
int heapring_submit(gheap_ring_t r, uint32_t n_req, const uint32_t *heaps, const uint32_t *kinds,
                    const uint64_t *sizes, const void *keys, uint64_t *ids);

/* Reports up to `max` requests that completed since they were submitted and
 * were not reported before: ids, counts (insert: n; deleteMin: keys
 * returned) and status (GHEAP_OK, or the sticky device error of the heap
 * that failed an operation of the request).  Does not wait. */
int heapring_poll(gheap_ring_t r, uint64_t *ids, uint64_t *counts, int32_t *status, uint32_t max,
                  uint32_t *n_done);

/* Takes n completed requests: their deleteMin keys (each request's keys
 * ascending) are copied to host_out back to back in the order of ids (at
 * most cap keys in all), counts[i] = the keys request ids[i] returned (0 for
 * an insert), and the requests' slots and arena space are freed.  Every
 * completed request must be taken once.  GHEAP_ERR_ARG (nothing further
 * taken) for an id that is not completed or already taken, or when cap is
 * too small. */
int heapring_take(gheap_ring_t r, uint32_t n, const uint64_t *ids, void *host_out, uint64_t cap,
                  uint64_t *counts);

/* Requests submitted and not yet taken. */
int heapring_pending(gheap_ring_t r, uint64_t *in_flight);

/* A whole serving session on a running ring, the host loop in native code:
 * request i arrives at arrival[i] seconds after the call starts (ascending;
 * with realtime = 0 all have arrived at the start), names heap heaps[i] (a
 * bound heap of the set), kind kinds[i] and size sizes[i]; `keys` holds the
 * inserts' keys back to back in request order.  Each heap takes its requests
 * in arrival order, several in flight at once.  An insert that could take its
 * heap past capacities[h] keys (held[h] = keys the heap holds at the start,
 * updated as the session runs) waits while earlier requests of that heap are
 * in flight and is refused with GHEAP_ERR_FULL when none are; one larger than
 * the heap, or a request larger than a key arena, is refused at once.  Out:
 * each deleteMin's keys (ascending) at out[sum of the sizes of the deleteMins
 * before it], out_counts[i] (keys returned, or n for an insert), t_submit[i]
 * and t_done[i] (seconds from the start when it entered the ring and when its
 * completion was seen; -1 if it never entered) and status[i].  Returns when
 * every request is done, or GHEAP_ERR_TIMEOUT when nothing completed for 60
 * s while requests were in flight. */
int heapring_serve(gheap_ring_t r, uint64_t n_req, const double *arrival, const uint32_t *heaps,
                   const uint32_t *kinds, const uint64_t *sizes, const void *keys,
                   const uint64_t *capacities, uint64_t *held, int realtime, void *out,
                   uint64_t *out_counts, double *t_submit, double *t_done, int32_t *status);

/* ------------------------------------------------------------------------
 * Allocation-free entry point.  The paper has no counterpart: this is an
 * interface for callers that must not allocate device memory -- code whose
 * device memory is all reserved up front by a pool or budget it does not own,
 * and paths that cannot accept the latency or the implicit synchronization of
 * a cudaMalloc.
 *
 * heap_sort_noalloc inserts the n uint32_t keys of d_in (device) into a
 * temporary generalized heap with k = 1024 and deletes them all into d_out
 * (device, n keys, ascending) -- the same kernels and the same result as
 * heap_create + heap_insert + heap_delete_min.  Instead of allocating, the
 * heap lives in one fixed scratch array compiled into this library (about
 * 4.2 MB of device memory, held by every GPU that loads the library until the
 * process exits).  The caller passes only the input and output buffers.
 *
 *   - n may be at most GHEAP_NOALLOC_MAX_KEYS; larger n returns
 *     GHEAP_ERR_TOO_LARGE and enqueues nothing.  n = 0 does nothing.
 *   - The first call on each device looks up that device's address of the
 *     scratch array (a synchronous CUDA runtime query, once, even when host
 *     threads race to make that call) with that device current; make that
 *     first call before any stream capture.  No call allocates.
 *   - Every call shares the one scratch array: calls whose work overlaps on
 *     the GPU (different streams, or other host threads) race and corrupt
 *     each other.  Each call clears the heap state it needs, so a call never
 *     depends on what the previous call left in the array.
 *   - Device-side lock waits are bounded as for heap_insert.  When one runs
 *     out (or the device sees an impossible node state) the call's output is
 *     incomplete: the keys it did not write are set to 0xFFFFFFFF, and the
 *     failure is kept in the scratch array.  The next call on the same stream
 *     first waits for the stream, reads that record, and, if the previous call
 *     failed, returns its error (GHEAP_ERR_TIMEOUT or GHEAP_ERR_STATE),
 *     clears the record and enqueues nothing; a call after it runs normally.
 *     Every call therefore synchronizes `stream` once before it enqueues.
 *   - The scratch address is looked up once per device for the life of the
 *     process; after a cudaDeviceReset the library must not be called again
 *     on that device.
 * ------------------------------------------------------------------------ */
#define GHEAP_NOALLOC_MAX_KEYS (1ull << 20)
int heap_sort_noalloc(const uint32_t *d_in, uint32_t *d_out, uint64_t n, void *stream);

/* Human-readable text of an error code. */
const char *heap_strerror(int code);

#ifdef __cplusplus
}
#endif

#endif /* GHEAP_H */

/*
 * gheap_apps.h -- applications of the generalized concurrent heap
 * (arXiv 1906.06504, Section 5.7), built on the C ABI of gheap.h.
 *
 * Conventions are those of gheap.h: GHEAP_OK or a negative GHEAP_ERR_* code;
 * graph and output arrays are DEVICE pointers owned by the caller; `stream`
 * is a cudaStream_t passed as void*.  A context may be used from one host
 * thread at a time and owns all the device memory it allocates.
 */
#ifndef GHEAP_APPS_H
#define GHEAP_APPS_H

#include <stdint.h>

#include "gheap.h"

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------------------
 * Single-source shortest paths with the heap as the priority queue of the
 * active vertices (Section 5.7.1).  Heap keys are 64-bit:
 * (tentative distance << 32) | vertex, so the heap orders active vertices
 * by distance, ties by vertex id.  Each iteration
 *   1. deletes the `batch` smallest keys (heap_delete_min),
 *   2. drops stale keys (distance above the vertex's current distance),
 *   3. relaxes the out-edges of the rest: nd = d + w(e) lowers dist[u] by
 *      atomicMin when nd < dist[u],
 *   4. inserts (nd << 32 | u) for every lowering (heap_insert_dev),
 * until the heap is empty.  Every lowering is inserted and every current key
 * is expanded, so the result is the exact shortest-path distance whatever
 * order the batches take (a label-correcting method): bit-identical to
 * textbook Dijkstra.
 *
 * Graph: CSR with rowptr[n_vertices + 1] (uint64_t), col[n_edges] and
 * w[n_edges] (uint32_t), edges of v in [rowptr[v], rowptr[v+1]).  Output:
 * dist[n_vertices] (uint32_t), UINT32_MAX for unreachable vertices; path
 * lengths of 2^32 - 1 or more are not representable and count as
 * unreachable.
 * ------------------------------------------------------------------------ */
typedef struct sssp_s *sssp_t;

typedef struct {
    uint64_t iterations;     /* deleteMin batches issued                     */
    uint64_t keys_deleted;   /* keys those batches returned                  */
    uint64_t visited;        /* current (not stale) keys: vertices expanded  */
    uint64_t edges;          /* out-edges scanned from the visited vertices  */
    uint64_t keys_inserted;  /* distance lowerings inserted into the heap    */
} sssp_stats;

/* Creates a context for graphs of up to n_vertices vertices and n_edges
 * edges.  k: heap node capacity (power of two in [1, 2048]); batch: keys
 * deleted per iteration (>= 1); heap_capacity: keys the heap can hold
 * (0 = n_edges + n_vertices + 1).  Allocates the heap (8-byte keys), a
 * delete buffer of `batch` keys and an insert buffer of n_edges keys.
 * Errors: ARG (a zero size, n_vertices >= 2^32 - 1), OOM, CUDA. */
int sssp_create(sssp_t *out, uint32_t n_vertices, uint64_t n_edges, uint32_t k,
                uint32_t batch, uint64_t heap_capacity);
int sssp_destroy(sssp_t s);

/* The context's heap (owned by the context), e.g. for heap_get_stats after
 * heap_set_stats; NULL for a NULL context. */
gheap_t sssp_heap(sssp_t s);

/* Launch shape of the heap operations (see heap_set_launch). */
int sssp_set_launch(sssp_t s, uint32_t ctas, uint32_t items_per_thread);

/* Computes dist[] from `source` on the context's stream and returns when it
 * is done (it synchronizes, also once at the start to read a check of the
 * graph's out-degrees: a graph with no vertex above 2048 out-edges runs each
 * iteration without the kernel that spreads such vertices over the grid).
 * The graph must fit the sizes given at creation; n_vertices here may be
 * smaller.  `stats` (host, may be NULL)
 * receives the counters above.  Errors: ARG (source >= n_vertices, a null
 * pointer, sizes above the context's), FULL (more live keys than
 * heap_capacity), TIMEOUT, STATE, CUDA. */
int sssp_run(sssp_t s, const uint64_t *d_rowptr, const uint32_t *d_col, const uint32_t *d_w,
             uint32_t n_vertices, uint64_t n_edges, uint32_t source, uint32_t *d_dist,
             sssp_stats *stats, void *stream);

/* ------------------------------------------------------------------------
 * 0/1 knapsack by best-first branch and bound with the heap as the queue of
 * open search nodes (Section 5.7.2).  Items are sorted by value/weight
 * descending (exact 64-bit cross products; weightless items first; equal
 * ratios keep the input order).  A node fixes the first i sorted items and
 * holds (i, profit, weight) in a node pool; its bound is the floor of the
 * linear relaxation (Dantzig): the profit, every following item up to the
 * first that does not fit, and the fitting fraction of that one.  Heap keys
 * are ((sum of values - bound) << 32) | node id: the largest bound first.
 * Each iteration deletes `batch` keys, drops those whose bound no longer
 * beats the incumbent, branches the rest on their next item (take if it
 * fits, skip), raises the incumbent with leaves and with each child's greedy
 * completion, and inserts the children whose bound beats the incumbent.  The
 * search ends when the heap is empty or the best bound left does not beat
 * the incumbent; the incumbent is then the optimum, the same value a dynamic
 * program gives.  With gc_threshold > 0, whenever the heap holds more keys
 * than that (and more than twice what the last pass kept), a filter pass
 * deletes every key and re-inserts those whose bound still beats the
 * incumbent (the paper's garbage collection).
 *
 * Inputs: w[n], v[n] (uint32_t, device), 1 <= n <= max_items, capacity.
 * The values must sum below 2^32 - 1 (GHEAP_ERR_ARG otherwise).
 * ------------------------------------------------------------------------ */
typedef struct knapsack_s *knapsack_t;

typedef struct {
    uint64_t best;           /* the optimum total value                     */
    uint64_t iterations;     /* deleteMin batches that expanded nodes       */
    uint64_t keys_deleted;   /* keys those batches returned                 */
    uint64_t explored;       /* nodes branched (bound beat the incumbent)   */
    uint64_t pruned;         /* popped nodes whose bound no longer did      */
    uint64_t keys_inserted;  /* children inserted                           */
    uint64_t nodes;          /* node records allocated                      */
    uint64_t gc_runs;        /* filter passes                               */
    uint64_t gc_dropped;     /* keys they removed                           */
} knapsack_stats;

/* max_items <= 4096.  max_nodes: node records (and heap keys) the search may
 * allocate, < 2^32 (0 = 2^26).  k, batch: heap node capacity and keys
 * deleted per iteration.  Allocates 24 bytes per node record (pool and
 * heap), plus 16 more when gc_threshold > 0.  Errors: ARG, OOM, CUDA. */
int knapsack_create(knapsack_t *out, uint32_t max_items, uint64_t max_nodes, uint32_t k,
                    uint32_t batch, uint64_t gc_threshold);
int knapsack_destroy(knapsack_t s);

/* The context's heap (owned by the context); NULL for a NULL context. */
gheap_t knapsack_heap(knapsack_t s);
int knapsack_set_launch(knapsack_t s, uint32_t ctas, uint32_t items_per_thread);

/* Solves one instance on `stream` and returns when done (synchronizes).
 * `stats` (host, may be NULL) receives the optimum and the counters.
 * Errors: ARG, FULL (more node records than max_nodes), TIMEOUT, STATE, CUDA. */
int knapsack_run(knapsack_t s, const uint32_t *d_w, const uint32_t *d_v, uint32_t n,
                 uint32_t capacity, knapsack_stats *stats, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* GHEAP_APPS_H */

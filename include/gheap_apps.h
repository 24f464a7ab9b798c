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

/* Launch shape of the heap operations (see heap_set_launch). */
int sssp_set_launch(sssp_t s, uint32_t ctas, uint32_t items_per_thread);

/* Computes dist[] from `source` on the context's stream and returns when it
 * is done (it synchronizes).  The graph must fit the sizes given at
 * creation; n_vertices here may be smaller.  `stats` (host, may be NULL)
 * receives the counters above.  Errors: ARG (source >= n_vertices, a null
 * pointer, sizes above the context's), FULL (more live keys than
 * heap_capacity), TIMEOUT, STATE, CUDA. */
int sssp_run(sssp_t s, const uint64_t *d_rowptr, const uint32_t *d_col, const uint32_t *d_w,
             uint32_t n_vertices, uint64_t n_edges, uint32_t source, uint32_t *d_dist,
             sssp_stats *stats, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* GHEAP_APPS_H */

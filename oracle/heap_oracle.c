/*
 * heap_oracle.c -- CPU oracle for the generalized concurrent heap of
 * "Accelerating Concurrent Heap on GPUs" (Chen et al., arXiv 1906.06504).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or
 * call this file: only the tests, __graft_entry__.smoke() and the CPU-baseline
 * leg of bench.py use it.  It shares no code, header, table or helper with the
 * CUDA implementation in paper_1906_06504_gb300/csrc.
 *
 * What it computes, and why that is the oracle:
 *   The heap is linearizable (Section 3.3.3, Theorem 1): every operation takes
 *   effect at a point inside its hold of the root lock, and a DEL returns the
 *   root batch, i.e. the k smallest keys of the multiset at that point
 *   (Section 3.2, the MergeAndSort postconditions and Property 3).  So, given
 *   the order in which operations held the root, every DEL output is fixed by
 *   a plain sequential priority queue.  This file is that priority queue: the
 *   textbook array binary heap of Section 2.1 (bottom-up insert by sift-up,
 *   delete-min by moving the last leaf to the root and sifting down), over
 *   64-bit unsigned keys (32-bit keys are widened by the caller).
 *
 * Also here, each a plain definition written out:
 *   - orc_merge_and_sort: the MergeAndSort operation of Section 3.2.1 by its
 *     definition (sort the concatenation, split at k).
 *   - orc_check_properties: Properties 1-3 of Section 3.1 checked on a heap
 *     snapshot.
 *   - orc_dijkstra: textbook Dijkstra over the binary heap (Section 5.7.1
 *     application; distances are unique, so any correct SSSP must match).
 *   - orc_knapsack_dp: textbook O(n*C) dynamic program for 0/1 knapsack
 *     (Section 5.7.2 application; the optimum value is unique).
 *
 * Everything is single-threaded and unoptimised on purpose.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------ */
/* Binary-heap priority queue (Section 2.1).                                 */
/* ------------------------------------------------------------------------ */

typedef struct {
    uint64_t *a;   /* a[0] is the root; children of i are 2i+1 and 2i+2 */
    size_t n;
    size_t cap;
} orc_pq;

orc_pq *orc_pq_new(size_t cap_hint)
{
    orc_pq *q = (orc_pq *)calloc(1, sizeof(orc_pq));
    if (!q) return NULL;
    q->cap = cap_hint ? cap_hint : 16;
    q->a = (uint64_t *)malloc(q->cap * sizeof(uint64_t));
    if (!q->a) { free(q); return NULL; }
    return q;
}

void orc_pq_free(orc_pq *q)
{
    if (!q) return;
    free(q->a);
    free(q);
}

size_t orc_pq_size(const orc_pq *q) { return q->n; }

/* Insert one key: place it in the first empty leaf, then swap it with its
 * parent while it is smaller (the bottom-up insertion of Section 2.1). */
static int pq_push1(orc_pq *q, uint64_t key)
{
    if (q->n == q->cap) {
        size_t nc = q->cap * 2;
        uint64_t *na = (uint64_t *)realloc(q->a, nc * sizeof(uint64_t));
        if (!na) return -1;
        q->a = na;
        q->cap = nc;
    }
    size_t i = q->n++;
    q->a[i] = key;
    while (i > 0) {
        size_t p = (i - 1) / 2;
        if (q->a[i] < q->a[p]) {
            uint64_t t = q->a[i]; q->a[i] = q->a[p]; q->a[p] = t;
            i = p;
        } else {
            break;
        }
    }
    return 0;
}

/* Delete the minimum: take the root, move the last leaf to the root, then
 * repeatedly swap it with its smaller child while that child is smaller
 * (delete-min of Section 2.1). */
static uint64_t pq_pop1(orc_pq *q)
{
    uint64_t top = q->a[0];
    q->n--;
    if (q->n > 0) {
        q->a[0] = q->a[q->n];
        size_t i = 0;
        for (;;) {
            size_t l = 2 * i + 1, r = l + 1, c;
            if (l >= q->n) break;
            c = l;
            if (r < q->n && q->a[r] < q->a[l]) c = r;
            if (q->a[c] < q->a[i]) {
                uint64_t t = q->a[i]; q->a[i] = q->a[c]; q->a[c] = t;
                i = c;
            } else {
                break;
            }
        }
    }
    return top;
}

int orc_pq_push(orc_pq *q, const uint64_t *keys, size_t n)
{
    for (size_t i = 0; i < n; i++)
        if (pq_push1(q, keys[i]) != 0) return -1;
    return 0;
}

/* Pops min(n, size) keys in ascending order into out; returns the count. */
size_t orc_pq_pop(orc_pq *q, uint64_t *out, size_t n)
{
    size_t c = 0;
    while (c < n && q->n > 0) out[c++] = pq_pop1(q);
    return c;
}

/* 32-bit convenience wrappers (the keys of the raw-heap workloads). */
int orc_pq_push_u32(orc_pq *q, const uint32_t *keys, size_t n)
{
    for (size_t i = 0; i < n; i++)
        if (pq_push1(q, (uint64_t)keys[i]) != 0) return -1;
    return 0;
}

size_t orc_pq_pop_u32(orc_pq *q, uint32_t *out, size_t n)
{
    size_t c = 0;
    while (c < n && q->n > 0) out[c++] = (uint32_t)pq_pop1(q);
    return c;
}

/* ------------------------------------------------------------------------ */
/* MergeAndSort by definition (Section 3.2.1).                               */
/* ------------------------------------------------------------------------ */

static int cmp_u64(const void *x, const void *y)
{
    uint64_t a = *(const uint64_t *)x, b = *(const uint64_t *)y;
    return (a > b) - (a < b);
}

/* (small, large) = MergeAndSort(a[0..na), b[0..nb)): `small` receives the
 * k_small smallest keys of the concatenation, ascending, and `large` the
 * remaining na+nb-k_small keys, ascending.  With na = nb = k_small = k this
 * is the paper's operation (its "hi" batch is `small`, its "lo" batch is
 * `large`).  Returns 0, or -1 on allocation failure. */
int orc_merge_and_sort(const uint64_t *a, size_t na, const uint64_t *b,
                       size_t nb, size_t k_small, uint64_t *small,
                       uint64_t *large)
{
    size_t n = na + nb;
    if (k_small > n) return -1;
    uint64_t *t = (uint64_t *)malloc((n ? n : 1) * sizeof(uint64_t));
    if (!t) return -1;
    memcpy(t, a, na * sizeof(uint64_t));
    memcpy(t + na, b, nb * sizeof(uint64_t));
    qsort(t, n, sizeof(uint64_t), cmp_u64);
    memcpy(small, t, k_small * sizeof(uint64_t));
    memcpy(large, t + k_small, (n - k_small) * sizeof(uint64_t));
    free(t);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Properties 1-3 of the generalized heap (Section 3.1).                     */
/* ------------------------------------------------------------------------ */

/* Snapshot layout: nodes are numbered from 1 (root) in the implicit binary
 * tree (children of i are 2i and 2i+1); node i's k keys are at
 * nodes[i*k .. i*k+k); present[i] != 0 marks an occupied node; slots 0 of
 * both arrays are unused.  buf[0..s) is the partial buffer.
 *
 * Returns 0 when every property holds.  Otherwise returns the first violated
 * check and stores the offending node in *where:
 *   1  Property 1 (child min >= parent max)
 *   2  Property 2 (each node ascending)
 *   3  Property 3 (buffer ascending, buffer min >= root max)
 *   4  structure: an occupied node whose parent is not occupied, or a buffer
 *      of k or more keys (the buffer holds at most k-1)
 */
int orc_check_properties(const uint64_t *nodes, const uint8_t *present,
                         size_t n_slots, size_t k, const uint64_t *buf,
                         size_t s, size_t *where)
{
    *where = 0;
    if (k > 0 && s >= k) return 4;
    for (size_t i = 1; i < n_slots; i++) {
        if (!present[i]) continue;
        const uint64_t *c = nodes + i * k;
        for (size_t j = 0; j + 1 < k; j++)
            if (c[j] > c[j + 1]) { *where = i; return 2; }
        if (i > 1) {
            size_t p = i / 2;
            if (!present[p]) { *where = i; return 4; }
            const uint64_t *pn = nodes + p * k;
            uint64_t pmax = pn[0], cmin = c[0];
            for (size_t j = 0; j < k; j++) {
                if (pn[j] > pmax) pmax = pn[j];
                if (c[j] < cmin) cmin = c[j];
            }
            if (cmin < pmax) { *where = i; return 1; }
        }
    }
    for (size_t j = 0; j + 1 < s; j++)
        if (buf[j] > buf[j + 1]) { *where = 0; return 3; }
    if (s > 0 && n_slots > 1 && present[1]) {
        const uint64_t *root = nodes + k;
        uint64_t rmax = root[0];
        for (size_t j = 0; j < k; j++)
            if (root[j] > rmax) rmax = root[j];
        uint64_t bmin = buf[0];
        for (size_t j = 0; j < s; j++)
            if (buf[j] < bmin) bmin = buf[j];
        if (bmin < rmax) { *where = 1; return 3; }
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Textbook Dijkstra (application of Section 5.7.1).                         */
/* ------------------------------------------------------------------------ */

/* Graph in CSR form: the out-edges of v are col[rowptr[v] .. rowptr[v+1])
 * with weights w[...].  dist[v] receives the shortest distance from src, or
 * UINT32_MAX when v is unreachable.  Queue keys pack (distance << 32 | v) so
 * that equal distances are ordered by vertex.  Returns 0, or -1 on
 * allocation failure. */
int orc_dijkstra(uint32_t n, const uint64_t *rowptr, const uint32_t *col,
                 const uint32_t *w, uint32_t src, uint32_t *dist)
{
    for (uint32_t v = 0; v < n; v++) dist[v] = UINT32_MAX;
    if (src >= n) return 0;
    orc_pq *q = orc_pq_new(1024);
    if (!q) return -1;
    dist[src] = 0;
    if (pq_push1(q, (uint64_t)src) != 0) { orc_pq_free(q); return -1; }
    while (q->n > 0) {
        uint64_t top = pq_pop1(q);
        uint32_t d = (uint32_t)(top >> 32), u = (uint32_t)top;
        if (d != dist[u]) continue;            /* stale entry */
        for (uint64_t e = rowptr[u]; e < rowptr[u + 1]; e++) {
            uint32_t v = col[e];
            uint64_t nd = (uint64_t)d + w[e];
            if (nd < dist[v]) {
                dist[v] = (uint32_t)nd;
                if (pq_push1(q, (nd << 32) | v) != 0) { orc_pq_free(q); return -1; }
            }
        }
    }
    orc_pq_free(q);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Textbook 0/1 knapsack dynamic program (application of Section 5.7.2).     */
/* ------------------------------------------------------------------------ */

/* best[c] = the largest total value of a subset of the items seen so far with
 * total weight <= c; items are taken one at a time, capacities descending.
 * Returns the optimum, or UINT64_MAX on allocation failure. */
uint64_t orc_knapsack_dp(uint32_t n, const uint32_t *w, const uint32_t *v,
                         uint64_t cap)
{
    uint64_t *best = (uint64_t *)calloc(cap + 1, sizeof(uint64_t));
    if (!best) return UINT64_MAX;
    for (uint32_t i = 0; i < n; i++) {
        if (w[i] > cap) continue;
        for (uint64_t c = cap; c >= w[i]; c--) {
            uint64_t cand = best[c - w[i]] + v[i];
            if (cand > best[c]) best[c] = cand;
            if (c == 0) break;
        }
    }
    uint64_t r = best[cap];
    free(best);
    return r;
}

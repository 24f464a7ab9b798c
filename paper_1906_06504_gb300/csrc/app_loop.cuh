// app_loop.cuh -- the iteration driver shared by the heap applications
// (SSSP and knapsack branch-and-bound, Section 5.7).
//
// An application iteration is a fixed sequence of stream operations (a
// deleteMin batch, the application's kernels, an insert whose count is on the
// device).  The driver captures UNROLL iterations into each of two CUDA
// graphs; the application's last kernel of every iteration writes
// (live keys, status) of its graph's slot into mapped host memory.  The host
// launches the two graphs alternately and reads one graph's slot while the
// other runs, so the device never idles waiting for the host until the heap
// has run empty (live == 0) or the application reported a status (an error,
// or an early finish it encodes as live == 0).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "gheap.h"

namespace app {

constexpr int UNROLL = 4;   // iterations per graph; even, so parities alternate

struct Loop {
    cudaStream_t cap_stream = nullptr;          // capture stream
    cudaEvent_t ev[2] = {nullptr, nullptr};
    cudaGraphExec_t exec[2] = {nullptr, nullptr};
    unsigned long long *h_ring = nullptr;       // mapped host memory: 2 words per slot
    unsigned long long *d_ring = nullptr;
};

inline int loop_init(Loop &L)
{
    if (cudaHostAlloc(&L.h_ring, 4 * sizeof(unsigned long long), cudaHostAllocMapped) != cudaSuccess)
        return GHEAP_ERR_CUDA;
    if (cudaHostGetDevicePointer(&L.d_ring, L.h_ring, 0) != cudaSuccess) return GHEAP_ERR_CUDA;
    if (cudaStreamCreateWithFlags(&L.cap_stream, cudaStreamNonBlocking) != cudaSuccess)
        return GHEAP_ERR_CUDA;
    for (int i = 0; i < 2; i++)
        if (cudaEventCreateWithFlags(&L.ev[i], cudaEventDisableTiming) != cudaSuccess)
            return GHEAP_ERR_CUDA;
    return GHEAP_OK;
}

inline void loop_drop(Loop &L)
{
    for (int i = 0; i < 2; i++) {
        if (L.exec[i]) cudaGraphExecDestroy(L.exec[i]);
        L.exec[i] = nullptr;
    }
}

inline void loop_free(Loop &L)
{
    loop_drop(L);
    if (L.h_ring) cudaFreeHost(L.h_ring);
    for (int i = 0; i < 2; i++)
        if (L.ev[i]) cudaEventDestroy(L.ev[i]);
    if (L.cap_stream) cudaStreamDestroy(L.cap_stream);
    L = Loop();
}

inline bool loop_ready(const Loop &L) { return L.exec[0] && L.exec[1]; }

// Captures both graphs; enqueue(parity, slot, stream) enqueues one iteration
// that reports to ring slot `slot` and returns a GHEAP code.
template <class F>
int loop_capture(Loop &L, F &&enqueue)
{
    loop_drop(L);
    for (int i = 0; i < 2; i++) {
        if (cudaStreamBeginCapture(L.cap_stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
            return GHEAP_ERR_CUDA;
        int rc = GHEAP_OK;
        for (int u = 0; u < UNROLL && rc == GHEAP_OK; u++)
            rc = enqueue((uint32_t)(u & 1), (uint32_t)i, L.cap_stream);
        cudaGraph_t graph = nullptr;
        const cudaError_t e = cudaStreamEndCapture(L.cap_stream, &graph);
        if (rc == GHEAP_OK && e != cudaSuccess) rc = GHEAP_ERR_CUDA;
        if (rc == GHEAP_OK && cudaGraphInstantiate(&L.exec[i], graph, 0) != cudaSuccess) {
            L.exec[i] = nullptr;
            rc = GHEAP_ERR_CUDA;
        }
        if (graph) cudaGraphDestroy(graph);
        if (rc != GHEAP_OK) {
            cudaGetLastError();
            loop_drop(L);
            return rc;
        }
    }
    return GHEAP_OK;
}

// Launches the graphs alternately on `st` until a report shows live == 0 or
// a non-zero status (returned in *status).  After each report with live > 0,
// want(live) may ask for an intervention: the driver then lets the stream
// drain, re-reads the latest report, calls act(st) (which enqueues work on
// st and returns a GHEAP code) and starts both graphs again.
template <class W, class A>
int loop_run(Loop &L, cudaStream_t st, unsigned long long *status, W &&want, A &&act)
{
    *status = 0;
    for (;;) {
        for (int i = 0; i < 2; i++) {
            if (cudaGraphLaunch(L.exec[i], st) != cudaSuccess) return GHEAP_ERR_CUDA;
            if (cudaEventRecord(L.ev[i], st) != cudaSuccess) return GHEAP_ERR_CUDA;
        }
        bool restart = false;
        for (int j = 0; !restart; j ^= 1) {
            if (cudaEventSynchronize(L.ev[j]) != cudaSuccess) return GHEAP_ERR_CUDA;
            const volatile unsigned long long *r = L.h_ring;
            unsigned long long live = r[2 * j];
            *status = r[2 * j + 1];
            if (live == 0 || *status) return GHEAP_OK;
            if (want(live)) {
                if (cudaStreamSynchronize(st) != cudaSuccess) return GHEAP_ERR_CUDA;
                live = r[2 * (j ^ 1)];
                *status = r[2 * (j ^ 1) + 1];
                if (live == 0 || *status) return GHEAP_OK;
                const int rc = act(st);
                if (rc != GHEAP_OK) return rc;
                restart = true;
            } else {
                if (cudaGraphLaunch(L.exec[j], st) != cudaSuccess) return GHEAP_ERR_CUDA;
                if (cudaEventRecord(L.ev[j], st) != cudaSuccess) return GHEAP_ERR_CUDA;
            }
        }
    }
}

}  // namespace app

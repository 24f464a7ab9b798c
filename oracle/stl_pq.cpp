/*
 * stl_pq.cpp -- the sequential CPU baseline of the paper's Table 1 (Section
 * 5.2): the C++ standard library's priority queue (a binary heap over a
 * vector), used as a min-queue of 32-bit keys.
 *
 * Test and CPU-baseline infrastructure only, like the rest of this directory:
 * only the tests and the CPU-baseline legs of bench.py load it.  It shares
 * nothing with the CUDA implementation.
 *
 * stl_insert_delete_u32 runs the phased raw-heap workload: push all n keys,
 * then pop them all into out (ascending).  Returns the seconds spent in the
 * pushes and pops (a steady clock around them), or a negative value when the
 * queue's storage could not be allocated.
 */
#include <chrono>
#include <cstddef>
#include <cstdint>
#include <functional>
#include <new>
#include <queue>
#include <vector>

extern "C" double stl_insert_delete_u32(const uint32_t *keys, size_t n, uint32_t *out)
{
    try {
        std::vector<uint32_t> store;
        store.reserve(n);
        std::priority_queue<uint32_t, std::vector<uint32_t>, std::greater<uint32_t>> q(
            std::greater<uint32_t>(), std::move(store));
        const auto t0 = std::chrono::steady_clock::now();
        for (size_t i = 0; i < n; ++i) q.push(keys[i]);
        for (size_t i = 0; i < n; ++i) {
            out[i] = q.top();
            q.pop();
        }
        const auto t1 = std::chrono::steady_clock::now();
        return std::chrono::duration<double>(t1 - t0).count();
    } catch (const std::bad_alloc &) {
        return -1.0;
    }
}

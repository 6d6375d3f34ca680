// Device and page-locked host allocations of the library, in one place.
//
// Every allocation the library makes goes through dmalloc / hmalloc and every
// release through dfree / hfree, so that
//   * a host-side test can make the k-th allocation fail as if the device were out
//     of memory (sdf_debug_fail_alloc) and check that each entry point then returns
//     SDF_ERR_OOM and leaks nothing (sdf_debug_alloc_live), without touching the GPU;
//   * the live allocations and their bytes can be counted.
// Allocation is never on the hot path of a check (scratch is grown, not churned),
// so the bookkeeping under a mutex costs nothing that matters.
#include <cuda_runtime.h>

#include <atomic>
#include <mutex>
#include <unordered_map>

#include "internal.h"

namespace {

std::mutex g_mu;
std::unordered_map<void*, size_t> g_live;   // pointer -> bytes, device and host alike
std::atomic<long long> g_countdown{0};      // > 0: the allocation that takes it to 0 fails

// True if this allocation is the one chosen to fail.
bool injected_failure() {
    long long c = g_countdown.load();
    while (c > 0) {
        if (g_countdown.compare_exchange_weak(c, c - 1)) return c == 1;
    }
    return false;
}

cudaError_t track(cudaError_t e, void* p, size_t bytes) {
    if (e == cudaSuccess && p) {
        std::lock_guard<std::mutex> lk(g_mu);
        g_live[p] = bytes;
    }
    return e;
}

void untrack(void* p) {
    if (!p) return;
    std::lock_guard<std::mutex> lk(g_mu);
    g_live.erase(p);
}

}  // namespace

namespace sdf {

cudaError_t dmalloc_raw(void** p, size_t bytes) {
    *p = nullptr;
    if (injected_failure()) return cudaErrorMemoryAllocation;
    return track(cudaMalloc(p, bytes), *p, bytes);
}

cudaError_t hmalloc_raw(void** p, size_t bytes) {
    *p = nullptr;
    if (injected_failure()) return cudaErrorMemoryAllocation;
    return track(cudaHostAlloc(p, bytes, cudaHostAllocDefault), *p, bytes);
}

cudaError_t amalloc3d(cudaArray_t* a, int n) {
    *a = nullptr;
    if (injected_failure()) return cudaErrorMemoryAllocation;
    const cudaChannelFormatDesc fd = cudaCreateChannelDesc<float>();
    return track(cudaMalloc3DArray(a, &fd, make_cudaExtent((size_t)n, (size_t)n, (size_t)n)), (void*)*a,
                 (size_t)n * n * n * sizeof(float));
}

void afree(cudaArray_t a) {
    if (!a) return;
    untrack((void*)a);
    cudaFreeArray(a);
}

void dfree(void* p) {
    if (!p) return;
    untrack(p);
    cudaFree(p);
}

void hfree(void* p) {
    if (!p) return;
    untrack(p);
    cudaFreeHost(p);
}

}  // namespace sdf

extern "C" {

int sdf_debug_fail_alloc(int64_t countdown) {
    if (countdown < 0) return SDF_ERR_INVALID_ARG;
    g_countdown.store((long long)countdown);
    return SDF_OK;
}

int sdf_debug_alloc_live(int64_t* count, int64_t* bytes, int64_t* countdown) {
    std::lock_guard<std::mutex> lk(g_mu);
    long long b = 0;
    for (const auto& kv : g_live) b += (long long)kv.second;
    if (count) *count = (int64_t)g_live.size();
    if (bytes) *bytes = (int64_t)b;
    if (countdown) *countdown = (int64_t)g_countdown.load();
    return SDF_OK;
}

}  // extern "C"

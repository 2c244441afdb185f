// alloc.cu -- counted allocation wrappers with injectable failure (see alloc.h).
#include "alloc.h"
#include "poisson.h"

#include <atomic>

namespace pcg {
namespace {
std::atomic<int> g_fail_in{0};     // > 0: allocations until the one that fails
std::atomic<long long> g_live{0};

bool injected_failure() {
    int c = g_fail_in.load(std::memory_order_relaxed);
    while (c > 0) {
        if (g_fail_in.compare_exchange_weak(c, c - 1, std::memory_order_relaxed))
            return c == 1;
    }
    return false;
}
}  // namespace

cudaError_t lib_malloc(void** p, size_t bytes) {
    *p = nullptr;
    if (injected_failure()) return cudaErrorMemoryAllocation;
    const cudaError_t e = cudaMalloc(p, bytes);
    if (e == cudaSuccess) g_live.fetch_add(1, std::memory_order_relaxed);
    else *p = nullptr;
    return e;
}

cudaError_t lib_malloc_host(void** p, size_t bytes) {
    *p = nullptr;
    if (injected_failure()) return cudaErrorMemoryAllocation;
    const cudaError_t e = cudaMallocHost(p, bytes);
    if (e == cudaSuccess) g_live.fetch_add(1, std::memory_order_relaxed);
    else *p = nullptr;
    return e;
}

void lib_free(void* p) {
    if (!p) return;
    cudaFree(p);
    g_live.fetch_sub(1, std::memory_order_relaxed);
}

void lib_free_host(void* p) {
    if (!p) return;
    cudaFreeHost(p);
    g_live.fetch_sub(1, std::memory_order_relaxed);
}

void lib_fail_alloc(int n) { g_fail_in.store(n, std::memory_order_relaxed); }

long long lib_live_allocs() { return g_live.load(std::memory_order_relaxed); }

}  // namespace pcg

extern "C" int poisson_test_fail_alloc(int n) {
    if (n < 0) return POISSON_EINVAL;
    pcg::lib_fail_alloc(n);
    return POISSON_OK;
}

extern "C" int poisson_test_live_allocations(long long* out) {
    if (!out) return POISSON_EINVAL;
    *out = pcg::lib_live_allocs();
    return POISSON_OK;
}

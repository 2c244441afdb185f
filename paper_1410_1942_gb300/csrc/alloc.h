// alloc.h -- the library's device and pinned-host allocations.
//
// Every cudaMalloc / cudaMallocHost / cudaFree / cudaFreeHost of the library goes through these
// wrappers, which count the live allocations and can be told to fail the n-th following
// allocation as if the device (or the host's pinned pool) were out of memory
// (poisson_test_fail_alloc): the error paths of creation, planning, staging and batching are
// then exercised on the host, without exhausting a GPU.
#pragma once

#include <cuda_runtime.h>

#include <cstddef>

namespace pcg {

cudaError_t lib_malloc(void** p, size_t bytes);
cudaError_t lib_malloc_host(void** p, size_t bytes);
void lib_free(void* p);        // null: nothing
void lib_free_host(void* p);   // null: nothing
void lib_fail_alloc(int n);    // the n-th following allocation fails (0: none)
long long lib_live_allocs();   // allocations made and not yet freed

}  // namespace pcg

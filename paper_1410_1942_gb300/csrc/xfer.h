// xfer.h -- moving user arrays between host and device memory.
#pragma once

#include <cuda_runtime.h>

#include <cstddef>

namespace pcg {

// Copies `bytes` from src to dst on stream st, asynchronously like cudaMemcpyAsync (the host
// array must stay valid and unchanged until the stream has passed the copy); kind is
// cudaMemcpyHostToDevice, cudaMemcpyDeviceToHost or cudaMemcpyDeviceToDevice.  A transfer of at
// least XFER_MIN_BYTES whose host side is pinned memory mapped into the current device's address
// space runs as a kernel that reads or writes the host array through that mapping; pageable host
// memory, smaller transfers and device-to-device copies go through cudaMemcpyAsync.
constexpr size_t XFER_MIN_BYTES = size_t(1) << 20;
cudaError_t copy_user(void* dst, const void* src, size_t bytes, cudaMemcpyKind kind,
                      cudaStream_t st);

}  // namespace pcg

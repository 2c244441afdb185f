// xfer.cu -- host<->device transfers of user arrays (the right side, the start and the
// solution, the density field, operator and projection arrays given in host memory).
//
// Pinned host memory is mapped into the device's address space, so the SMs can move an array in
// it with their own loads and stores over the CPU-GPU link.  The copy engine walks a large
// transfer in address order, and when the translations of its host pages are no longer cached
// (after a long solve has streamed gigabytes of device memory) it pays for them one page after
// another: on GB300 with 64 KiB host pages a 1 GiB transfer then took 31-140 ms against 5 ms
// when repeated at once.  Here every block streams its own contiguous chunk, so several hundred
// host pages are translated at the same time: 12-18 ms cold, 6-7 ms warm.
#include <cstdint>

#include "kernels.h"
#include "xfer.h"

namespace pcg {

constexpr int XFER_T = 256;
constexpr int XFER_BLOCKS_PER_SM = 8;

// dst[i] = src[i] for i in this block's chunk [per b, per (b + 1)) of [0, n).
template <typename T>
__global__ void __launch_bounds__(XFER_T) k_xfer(T* __restrict__ dst, const T* __restrict__ src,
                                                 size_t n, size_t per) {
    const size_t b0 = per * blockIdx.x;
    const size_t b1 = (b0 + per < n) ? b0 + per : n;
    for (size_t i = b0 + threadIdx.x; i < b1; i += XFER_T) dst[i] = src[i];
}

// The device address of pinned host memory, or null (pageable, managed or device memory).
static void* mapped_host(const void* p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return a.type == cudaMemoryTypeHost ? a.devicePointer : nullptr;
}

template <typename T>
static cudaError_t launch_xfer(void* dst, const void* src, size_t n, cudaStream_t st) {
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    size_t blocks = (n + XFER_T - 1) / XFER_T;
    const size_t cap = (size_t)XFER_BLOCKS_PER_SM * (size_t)(sms > 0 ? sms : 1);
    if (blocks > cap) blocks = cap;
    const size_t per = (n + blocks - 1) / blocks;
    k_xfer<T><<<(unsigned)blocks, XFER_T, 0, st>>>(static_cast<T*>(dst), static_cast<const T*>(src),
                                                   n, per);
    g_kernel_launches.fetch_add(1, std::memory_order_relaxed);
    return cudaGetLastError();
}

cudaError_t copy_user(void* dst, const void* src, size_t bytes, cudaMemcpyKind kind,
                      cudaStream_t st) {
    if (bytes == 0) return cudaSuccess;
    void* d = nullptr;
    const void* s = nullptr;
    if (bytes >= XFER_MIN_BYTES && kind == cudaMemcpyHostToDevice) {
        d = dst;
        s = mapped_host(src);
    } else if (bytes >= XFER_MIN_BYTES && kind == cudaMemcpyDeviceToHost) {
        d = mapped_host(dst);
        s = src;
    }
    if (!d || !s) return cudaMemcpyAsync(dst, src, bytes, kind, st);
    const uintptr_t align = reinterpret_cast<uintptr_t>(d) | reinterpret_cast<uintptr_t>(s);
    size_t unit = 0;
    cudaError_t e;
    if ((align & 15) == 0) {
        unit = 16;
        e = launch_xfer<double2>(d, s, bytes / 16, st);
    } else if ((align & 7) == 0) {
        unit = 8;
        e = launch_xfer<double>(d, s, bytes / 8, st);
    } else {
        return cudaMemcpyAsync(dst, src, bytes, kind, st);
    }
    if (e != cudaSuccess) return e;
    const size_t head = bytes - bytes % unit;
    if (head == bytes) return cudaSuccess;
    // the last bytes % unit bytes (the original pointers: cudaMemcpyAsync takes host addresses)
    return cudaMemcpyAsync(static_cast<char*>(dst) + head, static_cast<const char*>(src) + head,
                           bytes - head, kind, st);
}

}  // namespace pcg

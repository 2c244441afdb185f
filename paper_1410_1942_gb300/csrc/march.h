// march.h -- host interface of the TMA plane-marching CG kernels (march.cu).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include "internal.cuh"

namespace pcg {

// Tensor maps of one FP32 inner solve: halo boxes (32+8) x (ty+2) x 1 for z, both p buffers and
// eta (BF16: (32+16) x (ty+2)), centre boxes 32 x ty x 1 for x and r.
struct MarchMaps {
    CUtensorMap z, pa, pb, eta, x, r;
    int ty = 8;
    bool bf16 = false;
};

bool march_supported(const Dims& d);
bool march_maps(MarchMaps* mm, const Dims& d, int ty, const float* z, const float* pa,
                const float* pb, const void* eta, bool bf16, const float* x, const float* r);
int march_smem_a(int ty, bool bf16);
int march_smem_b(int ty, bool bf16);
int march_occupancy(int ty, bool bf16, bool a_side);
size_t march_blocks(const Dims& d, int ty, int kchunk);

// phase A: reads z and p_in (pa if pin_is_a else pb) with eta, writes p_out.
void launch_march_a(const Dims& d, int kchunk, const MarchMaps& mm, bool pin_is_a, float* p_out,
                    Scalars* sc, double* part, cudaStream_t st);
// phase B: reads p (pa if p_is_a else pb), eta, x, r; writes x, r, z.
void launch_march_b(const Dims& d, int kchunk, const MarchMaps& mm, bool p_is_a, float* x,
                    float* r, float* z, Scalars* sc, double* part, cudaStream_t st);

}  // namespace pcg

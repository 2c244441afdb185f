// march.h -- host interface of the TMA plane-marching CG kernels (march.cu).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include "internal.cuh"

namespace pcg {

// One kernel variant: 32 x tyt threads, each owning cx x cy cells; tile width x height cells.
struct MarchVariant {
    int id, cx, cy, tyt, width, height;
};

// Tensor maps of one FP32 inner solve for one variant: halo boxes (width+8) x (height+2) x 1
// for z and both p buffers, (width+8 or +16 for BF16) x (height+2) for eta, centre boxes
// width x height x 1 for x and r.
struct MarchMaps {
    CUtensorMap z, pa, pb, eta, x, r;
    int variant = 0;
    bool bf16 = false;
};

bool march_supported(const Dims& d);
int march_variant_count();
MarchVariant march_variant(int id);
int march_find_variant(int cx, int cy, int tyt);  // -1 if there is none
bool march_maps(MarchMaps* mm, const Dims& d, int variant, const float* z, const float* pa,
                const float* pb, const void* eta, bool bf16, const float* x, const float* r);
int march_occupancy(int variant, bool bf16);       // resident CTAs per SM (min of both phases)
size_t march_blocks(const Dims& d, int variant, int kchunk);
size_t march_max_blocks(const Dims& d, int kchunk);

// phase A: reads z and p_in (pa if pin_is_a else pb) with eta, writes p_out.
void launch_march_a(const Dims& d, int kchunk, const MarchMaps& mm, bool pin_is_a, float* p_out,
                    Scalars* sc, double* part, cudaStream_t st);
// phase B: reads p (pa if p_is_a else pb), eta, x, r; writes x, r, z.
void launch_march_b(const Dims& d, int kchunk, const MarchMaps& mm, bool p_is_a, float* x,
                    float* r, float* z, Scalars* sc, double* part, cudaStream_t st);

}  // namespace pcg

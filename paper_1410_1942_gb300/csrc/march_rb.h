// march_rb.h -- host interface of the red-black SSOR plane-marching kernels (march_rb.cu).
#pragma once

#include "march_dev.cuh"

namespace pcg {

// Kernels of the red-black family (variant family 3): (CX, CY, TYT, NS) of each instantiation;
// tile 64 x CY TYT cells (full resolution; CX = 2: one lane per compressed column), TYT consumer
// warps and a producer warp, an NS-stage ring (at least 7).
#define RB_CONFIGS(X) X(2, 2, 4, 8) X(2, 2, 4, 7) X(2, 1, 8, 8) X(2, 2, 8, 7)
Cg1Kernel rb_kernel(int cx, int cy, int tyt, int ns);  // null kernels if not instantiated

// Start of an inner solve on the black Schur complement: from the full-size right side r, the
// red relaxation d_R = r_R / D_R and the reduced right side r_B + C d_R; u = D_B^-1 of it, s^,
// w^, p and x zeroed (all compressed black vectors of n/2 floats); the scalars set with
// |r|^2 of the full r (stop when the residual falls to tol2 times it).
template <typename E>
void launch_rb_init(const Dims& d, const E* eta, const float* r, float* u, float* s, float* w,
                    float* p, float* x, Scalars* sc, double* part, double tol2, int max_iter,
                    cudaStream_t st);
// End of the inner solve: out_B = x_B, out_R = D_R^-1 (r_R + C x_B) (full size).
template <typename E>
void launch_rb_finish(const Dims& d, const E* eta, const float* r, const float* xb, float* out,
                      cudaStream_t st);

}  // namespace pcg

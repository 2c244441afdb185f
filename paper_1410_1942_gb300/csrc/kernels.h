// kernels.h -- host-side launchers of the libpoisson kernels (see kernels.cu).
#pragma once

#include "internal.cuh"

#include <atomic>

namespace pcg {

// Launches kernel k with programmatic stream serialization: it may start launching while the
// previous kernel of the stream drains (the kernel must begin with pdl_entry()).
template <typename... KArgs, typename... Args>
inline void launch_pdl(void (*k)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                       Args... args) {
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    cudaLaunchKernelEx(&cfg, k, static_cast<KArgs>(args)...);
}

constexpr int TX = 32;  // threads (cells) per tile along x
constexpr int TY = 8;   // ... along y

void launch_setup(const Dims& d, const double* F, double ra, double rw, double* bx, double* by,
                  double* bz, double* diag, double* dinv, double* top, double* rinv2,
                  float* eta32, __nv_bfloat16* eta16, const Apertures& ap, unsigned* bad,
                  cudaStream_t st);
void launch_scale(long long n, const double* s, double a, double* b, cudaStream_t st,
                  const double* vol = nullptr);
void launch_update64(long long n, double* x, const float* dlt, cudaStream_t st);
void launch_narrow_f32(long long n, const double* a, float* b, cudaStream_t st);
void launch_widen_f32(long long n, const float* a, double* b, cudaStream_t st);
// rows padded with `pad` ghost columns each side holding the other end of the row (periodic x)
void launch_pad_rows_f32(const Dims& d, int pad, const float* src, float* dst, cudaStream_t st);
void launch_pad_rows_bf16(const Dims& d, int pad, const __nv_bfloat16* src, __nv_bfloat16* dst,
                          cudaStream_t st);
void launch_fill_f32(long long n, float* p, float v, cudaStream_t st);
void launch_fill_bf16(long long n, __nv_bfloat16* p, float v, cudaStream_t st);
void launch_residual64(const Dims& d, int kc, const CoefFaces64& c, const double* b,
                       const double* x, double* r, Scalars* sc, double* part, cudaStream_t st);
void launch_residual64_f32(const Dims& d, int kc, const CoefFaces64& c, const double* b,
                           const double* x, float* r, Scalars* sc, double* part, cudaStream_t st);

template <typename V, typename Coef>
void launch_apply(const Dims& d, int kc, const Coef& c, const double* x, double* y,
                  cudaStream_t st);
template <typename V, typename Coef>
void launch_jacobi(const Dims& d, int kc, const Coef& c, const double* r, double* z,
                   cudaStream_t st);
template <typename V, typename Coef>
void launch_cg_init(const Dims& d, int kc, const Coef& c, const V* r, V* z, Scalars* sc,
                    double* part, double tol2, int rel_to_b, int max_iter, cudaStream_t st);
template <typename V, typename Coef>
void launch_cg_a(const Dims& d, int kc, const Coef& c, const V* z, const V* p_in, V* p_out,
                 Scalars* sc, double* part, cudaStream_t st);
template <typename V, typename Coef>
void launch_cg_b(const Dims& d, int kc, const Coef& c, const V* p, V* x, V* r, V* z,
                 Scalars* sc, double* part, cudaStream_t st);

// red-black SSOR (see kernels.cu): start (z = M^-1 r without the w(2-w) factor, scalars set),
// phase B with the two sweeps and the beta/stopping update, and the checking apply
// (out = M^-1 r including the factor; zbuf: n values of type V).
template <typename V, typename Coef>
void launch_ssor_init(const Dims& d, int kc, const Coef& c, const V* r, V* z, double omega,
                      Scalars* sc, double* part, double tol2, int rel_to_b, int max_iter,
                      cudaStream_t st);
template <typename V, typename Coef>
void launch_cg_b_ssor(const Dims& d, int kc, const Coef& c, const V* p, V* x, V* r, V* z,
                      double omega, Scalars* sc, double* part, cudaStream_t st);
template <typename V, typename Coef>
void launch_ssor_apply(const Dims& d, int kc, const Coef& c, const double* r, V* zbuf,
                       double omega, double* out, cudaStream_t st);

// Batched column kernels over a job table (jobs.cuh); blocks = total blocks of all jobs.
struct JobDev;
void launch_batch_update(const JobDev* jobs, int njobs, int blocks, cudaStream_t st);
void launch_batch_residual(const JobDev* jobs, int njobs, int blocks, cudaStream_t st);
void launch_batch_init(const JobDev* jobs, int njobs, int blocks, cudaStream_t st);

extern std::atomic<unsigned long long> g_kernel_launches;

}  // namespace pcg

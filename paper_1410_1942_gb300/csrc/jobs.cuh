// jobs.cuh -- device-side job table of a batch of independent solves.
//
// The batched FP64 residual, CG start and refinement update run every job of a batch in one
// launch: blocks [blk_off, blk_off + blocks) of the grid belong to a job, which uses the
// column-kernel geometry (32 x 8 threads, kc planes per thread) of its own grid and its own
// scalars and partial sums.
#pragma once

#include "internal.cuh"

namespace pcg {

struct JobDev {
    Dims d;
    int kc;        // planes per thread
    int gx, gy;    // blocks in x and y (gz = blocks / (gx gy))
    int blk_off;   // first block of the job in the launch
    int blocks;    // blocks of the job
    int bf16;      // inner coefficients in BF16
    // FP64 operator and vectors
    const double *bx, *by, *bz, *diag;
    const double* b64;
    double* x64;
    // FP32 inner vectors
    float *d32, *r32, *z32, *pa32;
    float *sa32, *wa32;  // zeroed by the init (read, times zero, by the one-sweep kernels)
    const float* eta32;
    const __nv_bfloat16* eta16;
    Scalars* sc;       // this job's scalars (contiguous array of the batch)
    double* partials;  // 2 * blocks doubles
    // host-set controls of the next inner solve
    double tol2;   // stop when r.r <= tol2 r0.r0
    int max_iter;  // iteration cap of the inner solve
    int active;    // 0: the job takes no part (finished); its scalars say CONVERGED
};

// Block -> job lookup by bisection over blk_off (jobs sorted by blk_off).
__device__ __forceinline__ int job_of_block(const JobDev* jobs, int njobs, int bid) {
    int lo = 0, hi = njobs - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (jobs[mid].blk_off <= bid) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// grid_sum over the blocks of one job: partials[local * NV + q]; the job's last block adds them
// in block order and returns true with the totals.
template <int NV>
__device__ __forceinline__ bool job_sum(double (&v)[NV], double* partials, unsigned int* ticket,
                                        unsigned nblocks, unsigned local, double (&tot)[NV],
                                        double* smem) {
    const int tid = threadIdx.x + blockDim.x * threadIdx.y;
    const int nthreads = blockDim.x * blockDim.y;
    __shared__ unsigned int s_last;
    block_sum<NV>(v, smem);
    if (tid == 0) {
#pragma unroll
        for (int q = 0; q < NV; ++q) partials[(size_t)local * NV + q] = v[q];
        __threadfence();
        const unsigned t = atomicAdd(ticket, 1u);
        s_last = (t == nblocks - 1) ? 1u : 0u;
    }
    __syncthreads();
    if (!s_last) return false;
    __threadfence();
    double acc[NV];
#pragma unroll
    for (int q = 0; q < NV; ++q) acc[q] = 0.0;
    for (unsigned b = tid; b < nblocks; b += nthreads)
#pragma unroll
        for (int q = 0; q < NV; ++q) acc[q] += __ldcg(&partials[(size_t)b * NV + q]);
    block_sum<NV>(acc, smem);
    if (tid == 0) {
#pragma unroll
        for (int q = 0; q < NV; ++q) smem[q] = acc[q];
        *ticket = 0u;
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < NV; ++q) tot[q] = smem[q];
    __syncthreads();
    return true;
}

}  // namespace pcg

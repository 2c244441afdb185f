// internal.cuh -- device-side building blocks shared by the libpoisson kernels.
//
// Operator (Formulation, eqs. (density) and (pois)): for cell c with neighbours n,
//   (A v)_c = D_c v_c - sum_n w_cn v_n,   D_c = sum_n w_cn + w_top,
// w_cn = 2 / (rho_c + rho_n) on interior faces, 0 on the Neumann walls, and w_top = 2 / rho_c on
// the top face (Dirichlet p = 0, ghost -v_c).  A = -h^2 div_h((1/rho) grad_h).
//
// Two coefficient sources implement it:
//   * FP64 face arrays (bx, by, bz = coefficient of the low face of each cell, diag) built once
//     per density -- the exact operator of the FP64 residual and of the plain FP64 PCG;
//   * eta = rho / 2 per cell in FP32 or BF16, from which the inner solver forms each face on the
//     fly as 1 / (eta_c + eta_n) (and the top term as 1 / eta_c).  The sum is commutative, so
//     both cells of a face see the same coefficient: the reduced-precision operator stays a
//     symmetric weighted graph Laplacian whose diagonal is the sum of its own faces.
#pragma once

#include <type_traits>

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

namespace pcg {

struct Dims {
    int nx, ny, nz;
    int sxy;        // nx * ny
    int n;          // nx * ny * nz (< 2^31, checked at create)
    int walls = 0;  // side/bottom walls with p = 0 (POISSON_WALL_* bits); the top always has p = 0;
                    // bit PERIODIC_X: x periodic (cell 0 and cell nx-1 of a row are neighbours)
};

constexpr int PERIODIC_X = 32;
constexpr int CUT_CELLS = 64;  // face open fractions and cell fluid fractions are in use

// Open fractions of the MAC faces and fluid fractions of the cells (free-slip cut cells); all
// null when the handle has none.
struct Apertures {
    const double *ax, *ay, *az, *vol;
};

// A Dirichlet side/bottom wall (Dims::walls bit) puts p = 0 on its face: the wall face gets the
// coefficient 2/rho_c = 1/eta_c, which counts in the diagonal, while the value beyond the wall
// contributes nothing (the kernels read it as 0: zero-filled halo, or no neighbour term).
// Per-solve CG scalars, updated on the device by the last block of each reduction.
struct Scalars {
    double rz;      // (r, z) of the current iterate
    double pq;      // (p, A p)
    double alpha;
    double beta;
    double rr;      // (r, r)
    double rr0;     // (r, r) at the start of the (inner) solve
    double stop2;   // stop when rr <= stop2
    double bb;      // (b, b) -- written by the residual reduction
    int iter;       // CG iterations done in this solve
    int max_iter;   // cap
    int done;       // 0 running, 1 converged, 2 breakdown, 3 iteration cap, 4 wait timed out
    unsigned int ticket;  // arrivals of the current reduction
};

enum Done { RUNNING = 0, CONVERGED = 1, BREAKDOWN = 2, CAPPED = 3, TIMEDOUT = 4 };

// Hardware reciprocal (MUFU), flush-to-zero: deterministic for a given input.
__device__ __forceinline__ float rcp_approx(float x) {
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Programmatic dependent launch: a kernel launched with programmatic stream serialization
// (launch_pdl) may start while the kernel before it in the stream is still running.  It waits
// here, before touching global memory, until that kernel has completed and its writes are
// visible, and lets the next kernel of the stream begin launching.  Without the launch attribute
// both instructions do nothing.
__device__ __forceinline__ void pdl_entry() {
    asm volatile("griddepcontrol.wait;\n" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory");
}

// ------------------------------------------------------------------ block reductions (FP64)
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Sums NV doubles over the block; the result is valid in thread 0.  smem: 32 * NV doubles.
template <int NV>
__device__ __forceinline__ void block_sum(double (&v)[NV], double* smem) {
    const int tid = threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
    const int nthreads = blockDim.x * blockDim.y * blockDim.z;
    const int lane = tid & 31, warp = tid >> 5, nwarps = (nthreads + 31) >> 5;
#pragma unroll
    for (int q = 0; q < NV; ++q) v[q] = warp_sum(v[q]);
    if (lane == 0) {
#pragma unroll
        for (int q = 0; q < NV; ++q) smem[warp * NV + q] = v[q];
    }
    __syncthreads();
    if (warp == 0) {
#pragma unroll
        for (int q = 0; q < NV; ++q) {
            double t = (lane < nwarps) ? smem[lane * NV + q] : 0.0;
            v[q] = warp_sum(t);
        }
    }
    __syncthreads();
}

// Grid-wide deterministic reduction: every block stores its NV partial sums to
// partials[block * NV + q]; the last block to arrive adds them in block order and returns true
// in all of its threads with the totals in `tot` (valid in every thread of that block).
template <int NV>
__device__ __forceinline__ bool grid_sum(double (&v)[NV], double* partials, unsigned int* ticket,
                                         double (&tot)[NV], double* smem) {
    const int tid = threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
    const int nthreads = blockDim.x * blockDim.y * blockDim.z;
    const unsigned int nblocks = gridDim.x * gridDim.y * gridDim.z;
    const unsigned int bid = blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z);
    __shared__ unsigned int s_last;
    block_sum<NV>(v, smem);
    if (tid == 0) {
#pragma unroll
        for (int q = 0; q < NV; ++q) partials[(size_t)bid * NV + q] = v[q];
        __threadfence();
        unsigned int t = atomicAdd(ticket, 1u);
        s_last = (t == nblocks - 1) ? 1u : 0u;
    }
    __syncthreads();
    if (!s_last) return false;
    __threadfence();
    double acc[NV];
#pragma unroll
    for (int q = 0; q < NV; ++q) acc[q] = 0.0;
    for (unsigned int b = tid; b < nblocks; b += nthreads) {
#pragma unroll
        for (int q = 0; q < NV; ++q) acc[q] += __ldcg(&partials[(size_t)b * NV + q]);
    }
    block_sum<NV>(acc, smem);
    if (tid == 0) {
#pragma unroll
        for (int q = 0; q < NV; ++q) smem[q] = acc[q];
        *ticket = 0u;  // ready for the next reduction (stream-ordered)
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < NV; ++q) tot[q] = smem[q];
    __syncthreads();
    return true;
}

// ------------------------------------------------------------------ coefficient policies
// weights(): the six face coefficients and the diagonal of cell (i, j, k).
template <typename T>
struct Stencil {
    T xm, xp, ym, yp, zm, zp, D;
};

struct CoefFaces64 {
    const double* bx;
    const double* by;
    const double* bz;
    const double* diag;
    const double* dinv;  // 1/diag (FP64 Jacobi); may be null
    __device__ __forceinline__ void weights(const Dims& d, int c, int i, int j, int k,
                                            Stencil<double>& w) const {
        w.xm = bx[c];  // periodic x: the wrap face of cell 0, else 0 at i = 0
        w.xp = (i + 1 < d.nx) ? bx[c + 1] : ((d.walls & PERIODIC_X) ? bx[c + 1 - d.nx] : 0.0);
        w.ym = by[c];
        w.yp = (j + 1 < d.ny) ? by[c + d.nx] : 0.0;
        w.zm = bz[c];
        w.zp = (k + 1 < d.nz) ? bz[c + d.sxy] : 0.0;
        w.D = diag[c];
    }
};

// The FP32 copies of the FP64 faces and diagonal: the inner operator of cut-cell handles (their
// face coefficients carry the open fractions, which the on-the-fly faces from rho/2 cannot).
struct CoefFaces32 {
    const float* bx;
    const float* by;
    const float* bz;
    const float* diag;
    __device__ __forceinline__ void weights(const Dims& d, int c, int i, int j, int k,
                                            Stencil<float>& w) const {
        w.xm = bx[c];
        w.xp = (i + 1 < d.nx) ? bx[c + 1] : ((d.walls & PERIODIC_X) ? bx[c + 1 - d.nx] : 0.f);
        w.ym = by[c];
        w.yp = (j + 1 < d.ny) ? by[c + d.nx] : 0.f;
        w.zm = bz[c];
        w.zp = (k + 1 < d.nz) ? bz[c + d.sxy] : 0.f;
        w.D = diag[c];
    }
};

// sum_n w_cn v_n with v = load(e)
template <typename V, typename L>
__device__ __forceinline__ V nb_sum(const Dims& d, const Stencil<V>& w, int c, int i, int j,
                                    int k, L load) {
    V s = 0;
    const bool per = d.walls & PERIODIC_X;
    if (i > 0) s += w.xm * load(c - 1);
    else if (per) s += w.xm * load(c + d.nx - 1);
    if (i + 1 < d.nx) s += w.xp * load(c + 1);
    else if (per) s += w.xp * load(c + 1 - d.nx);
    if (j > 0) s += w.ym * load(c - d.nx);
    if (j + 1 < d.ny) s += w.yp * load(c + d.nx);
    if (k > 0) s += w.zm * load(c - d.sxy);
    if (k + 1 < d.nz) s += w.zp * load(c + d.sxy);
    return s;
}

template <typename E>
__device__ __forceinline__ float eta_load(const E* p, int c);
template <>
__device__ __forceinline__ float eta_load<float>(const float* p, int c) { return __ldg(p + c); }
template <>
__device__ __forceinline__ float eta_load<__nv_bfloat16>(const __nv_bfloat16* p, int c) {
    return __bfloat162float(p[c]);
}

// The face coefficients and diagonal of cell (i, j, k) from rho/2 of the cell (ec) and of its six
// neighbours (a value across a wall or the top face is not used).  At a Dirichlet wall the face
// coefficient is 1/eta_c, and nb_sum never reads past the wall.
__device__ __forceinline__ void eta_stencil(const Dims& d, int i, int j, int k, float ec,
                                            float exm, float exp_, float eym, float eyp,
                                            float ezm, float ezp, Stencil<float>& w) {
    const float ew = rcp_approx(ec);
    const bool per = d.walls & PERIODIC_X;
    w.xm = (i > 0 || per) ? rcp_approx(ec + exm) : ((d.walls & 1) ? ew : 0.f);
    w.xp = (i + 1 < d.nx || per) ? rcp_approx(ec + exp_) : ((d.walls & 2) ? ew : 0.f);
    w.ym = (j > 0) ? rcp_approx(ec + eym) : ((d.walls & 4) ? ew : 0.f);
    w.yp = (j + 1 < d.ny) ? rcp_approx(ec + eyp) : ((d.walls & 8) ? ew : 0.f);
    w.zm = (k > 0) ? rcp_approx(ec + ezm) : ((d.walls & 16) ? ew : 0.f);
    const bool top = (k + 1 == d.nz);
    const float wzp = top ? ew : rcp_approx(ec + ezp);
    w.zp = top ? 0.f : wzp;
    w.D = w.xm + w.xp + w.ym + w.yp + w.zm + wzp;
}

template <typename E>
struct CoefEta {
    const E* eta;
    __device__ __forceinline__ void weights(const Dims& d, int c, int i, int j, int k,
                                            Stencil<float>& w) const {
        const bool per = d.walls & PERIODIC_X;
        const float ec = eta_load(eta, c);
        const float exm = (i > 0 || per) ? eta_load(eta, i > 0 ? c - 1 : c + d.nx - 1) : 0.f;
        const float exp_ = (i + 1 < d.nx || per) ? eta_load(eta, i + 1 < d.nx ? c + 1 : c + 1 - d.nx)
                                                 : 0.f;
        const float eym = (j > 0) ? eta_load(eta, c - d.nx) : 0.f;
        const float eyp = (j + 1 < d.ny) ? eta_load(eta, c + d.nx) : 0.f;
        const float ezm = (k > 0) ? eta_load(eta, c - d.sxy) : 0.f;
        const float ezp = (k + 1 < d.nz) ? eta_load(eta, c + d.sxy) : 0.f;
        eta_stencil(d, i, j, k, ec, exm, exp_, eym, eyp, ezm, ezp, w);
    }
};

// rho/2's element type of a CoefEta policy
template <typename C>
using EtaOf = std::remove_const_t<std::remove_pointer_t<decltype(C::eta)>>;

template <typename C>
struct is_coef_eta { static constexpr bool value = false; };
template <typename E>
struct is_coef_eta<CoefEta<E>> { static constexpr bool value = true; };

}  // namespace pcg

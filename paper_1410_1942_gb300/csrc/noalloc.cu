// noalloc.cu -- poisson_residual_noalloc: the FP64 relative residual of a pressure field, with
// no device allocation at call time.
//
// Some callers cannot allocate device memory at the moment they want to check a pressure
// field: a simulation step loop that must not pay cudaMalloc's latency or cudaFree's implicit
// device synchronisation, a process whose device memory is owned by another allocator under a
// fixed budget (a framework's caching pool, a preallocated arena) where a direct cudaMalloc
// fails or fragments it, or code that forbids dynamic allocation after initialisation.  For
// them this file computes ||b - A p||_2 / ||b||_2 (b = -h^2 s, A the FP64 operator built from
// F on the fly) in one kernel whose only scratch -- the per-block partial sums, the block
// ticket and the result -- lives in the static device array below.  The caller passes every
// input and the output; the array is sized for NOALLOC_MAX_BLOCKS blocks (64 KiB) and every GPU
// that loads this library holds it until the process exits.
#include <algorithm>
#include <cmath>
#include <mutex>

#include "poisson.h"
#include "capi_internal.h"
#include "internal.cuh"
#include "kernels.h"

namespace {

constexpr int NA_TX = 32, NA_TY = 8;        // threads per block (x, y); one cell column each
constexpr int NOALLOC_MAX_BLOCKS = 4096;    // partial-sum slots in the static array
constexpr int NA_RESULT = 2 * NOALLOC_MAX_BLOCKS;  // the result, then the ticket counter
constexpr int NA_TICKET = NA_RESULT + 1;
constexpr int NA_DOUBLES = NA_TICKET + 1;

// The scratch: [0, 2 MAXB) partials (r.r, b.b per block), [NA_RESULT] relative residual,
// [NA_TICKET] the arrival counter of the last-block reduction (as an unsigned int).
static __device__ __align__(256) double g_noalloc_scratch[NA_DOUBLES];

__device__ __forceinline__ double rho_at(const double* F, int c, double ra, double rw) {
    return __dadd_rn(ra, __dmul_rn(F[c], __dadd_rn(rw, -ra)));
}

// One thread per (i, j) column segment of kc planes: r = b - A p with the faces
// 2/(rho_c + rho_n), the top Dirichlet term 2/rho_c, and the diagonal summed in the set-up
// kernels' order; then a block sum, a partial per block, and the last block's ordered total.
__global__ void __launch_bounds__(NA_TX * NA_TY)
    k_residual_noalloc(pcg::Dims d, int kc, double h2, const double* __restrict__ F, double ra,
                       double rw, const double* __restrict__ s, const double* __restrict__ p,
                       double* scratch) {
    __shared__ double smem[64];
    const int i = blockIdx.x * NA_TX + threadIdx.x;
    const int j = blockIdx.y * NA_TY + threadIdx.y;
    const int k0 = blockIdx.z * kc, k1 = min(d.nz, k0 + kc);
    double rr = 0.0, bb = 0.0;
    if (i < d.nx && j < d.ny) {
        for (int k = k0; k < k1; ++k) {
            const int c = i + d.nx * (j + d.ny * k);
            const double rc = rho_at(F, c, ra, rw);
            const double wxm = (i > 0) ? 2.0 / __dadd_rn(rc, rho_at(F, c - 1, ra, rw)) : 0.0;
            const double wym = (j > 0) ? 2.0 / __dadd_rn(rc, rho_at(F, c - d.nx, ra, rw)) : 0.0;
            const double wzm = (k > 0) ? 2.0 / __dadd_rn(rc, rho_at(F, c - d.sxy, ra, rw)) : 0.0;
            const double wxp = (i + 1 < d.nx) ? 2.0 / __dadd_rn(rc, rho_at(F, c + 1, ra, rw)) : 0.0;
            const double wyp = (j + 1 < d.ny) ? 2.0 / __dadd_rn(rc, rho_at(F, c + d.nx, ra, rw)) : 0.0;
            const bool top = (k + 1 == d.nz);
            const double wzp = top ? 0.0 : 2.0 / __dadd_rn(rc, rho_at(F, c + d.sxy, ra, rw));
            double D = __dadd_rn(__dadd_rn(wxm, wym), wzm);
            D = __dadd_rn(D, wxp);
            D = __dadd_rn(D, wyp);
            D = __dadd_rn(D, top ? 2.0 / rc : wzp);
            double nb = 0.0;
            if (i > 0) nb += wxm * p[c - 1];
            if (i + 1 < d.nx) nb += wxp * p[c + 1];
            if (j > 0) nb += wym * p[c - d.nx];
            if (j + 1 < d.ny) nb += wyp * p[c + d.nx];
            if (k > 0) nb += wzm * p[c - d.sxy];
            if (!top) nb += wzp * p[c + d.sxy];
            const double b = __dmul_rn(-h2, s[c]);
            const double r = b - (D * p[c] - nb);
            rr += r * r;
            bb += b * b;
        }
    }
    double v[2] = {rr, bb}, tot[2];
    unsigned int* ticket = reinterpret_cast<unsigned int*>(scratch + NA_TICKET);
    if (pcg::grid_sum<2>(v, scratch, ticket, tot, smem)) {
        if (threadIdx.x == 0 && threadIdx.y == 0)
            scratch[NA_RESULT] = (tot[1] > 0.0) ? sqrt(tot[0] / tot[1]) : 0.0;
    }
}

// The array's device address, looked up once per device with that device current.
std::mutex g_mu;
constexpr int NA_MAX_DEVICES = 64;
double* g_scratch_ptr[NA_MAX_DEVICES] = {};

int scratch_for_current_device(double** out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= NA_MAX_DEVICES) {
        cudaGetLastError();
        return POISSON_ECUDA;
    }
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_scratch_ptr[dev]) {
        void* ptr = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
        if (e != cudaSuccess || !ptr) {
            cudaGetLastError();
            return POISSON_ECUDA;
        }
        g_scratch_ptr[dev] = static_cast<double*>(ptr);
    }
    *out = g_scratch_ptr[dev];
    return POISSON_OK;
}

}  // namespace

extern "C" int poisson_residual_noalloc(int nx, int ny, int nz, double h, const double* F,
                                        double rho_air, double rho_water, const double* rhs,
                                        const double* p, double* rel_residual, void* stream) {
    if (nx <= 0 || ny <= 0 || nz <= 0 || !(h > 0.0) || !std::isfinite(h) || !(rho_air > 0.0) ||
        !(rho_water > 0.0) || !std::isfinite(rho_air) || !std::isfinite(rho_water) || !F ||
        !rhs || !p || !rel_residual)
        return POISSON_EINVAL;
    const long long n = (long long)nx * ny * nz;
    if (n >= (1LL << 31)) return POISSON_EINVAL;
    const long long tiles = (long long)((nx + NA_TX - 1) / NA_TX) * ((ny + NA_TY - 1) / NA_TY);
    if (tiles > NOALLOC_MAX_BLOCKS) return POISSON_ETOOLARGE;
    if (!is_device_ptr(F) || !is_device_ptr(rhs) || !is_device_ptr(p)) return POISSON_EINVAL;
    double* scratch = nullptr;
    int rc = scratch_for_current_device(&scratch);
    if (rc != POISSON_OK) return rc;
    // z-planes per thread: about 2048 blocks, never more than the array holds
    long long kc = std::max(1LL, (nz * tiles + 2047) / 2048);
    while (tiles * ((nz + kc - 1) / kc) > NOALLOC_MAX_BLOCKS) ++kc;
    const pcg::Dims d{nx, ny, nz, nx * ny, (int)n};
    const dim3 grid((nx + NA_TX - 1) / NA_TX, (ny + NA_TY - 1) / NA_TY,
                    (unsigned)((nz + kc - 1) / kc));
    cudaStream_t st = (cudaStream_t)stream;
    // the ticket must start at zero (the last block also resets it)
    if (cudaMemsetAsync(scratch + NA_TICKET, 0, sizeof(double), st) != cudaSuccess) {
        cudaGetLastError();
        return POISSON_ECUDA;
    }
    k_residual_noalloc<<<grid, dim3(NA_TX, NA_TY), 0, st>>>(d, (int)kc, h * h, F, rho_air,
                                                            rho_water, rhs, p, scratch);
    pcg::g_kernel_launches.fetch_add(1, std::memory_order_relaxed);
    if (cudaGetLastError() != cudaSuccess) return POISSON_ECUDA;
    const bool dev_out = is_device_ptr(rel_residual);
    if (cudaMemcpyAsync(rel_residual, scratch + NA_RESULT, sizeof(double),
                        dev_out ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                        st) != cudaSuccess) {
        cudaGetLastError();
        return POISSON_ECUDA;
    }
    if (!dev_out && cudaStreamSynchronize(st) != cudaSuccess) {
        cudaGetLastError();
        return POISSON_ECUDA;
    }
    return POISSON_OK;
}

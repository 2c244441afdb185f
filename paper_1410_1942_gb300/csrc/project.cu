// project.cu -- the projection around the pressure solve: the divergence of a face velocity
// (the solve's source) and the velocity correction by the pressure gradient.
//
// Numerical Time Integration: each stage forms a provisional velocity u* on the faces of the
// cells (MAC grid), solves div((1/rho) grad p) = div(u*)/dt, and corrects
// u = u* - dt (1/rho) grad p.  The correction uses the operator's own face coefficients
// (2/(rho_c + rho_n) on interior faces; 1/rho_c with p = 0 on the top face, at half a cell from
// the centre), so div_h(u) / dt = div_h(u*) / dt - L p exactly: the divergence left behind is the
// solve's residual, (A p - b) / h^2.
//
// Both passes are elementwise over cells (one thread per cell, its three low faces plus the top
// face on the last layer): HBM-bound, a few tens of bytes per cell, once per solve.  They are FP64
// throughout and evaluate every expression in one fixed order with rounded intrinsics, so the
// results do not depend on FMA contraction.
#include <cmath>

#include "alloc.h"
#include "poisson.h"
#include "capi_internal.h"
#include "internal.cuh"
#include "kernels.h"
#include "xfer.h"

namespace {

using pcg::copy_user;
using pcg::Dims;
using pcg::lib_free;
using pcg::lib_malloc;

constexpr int PT = 256;

inline unsigned blocks_of(long long n) { return (unsigned)((n + PT - 1) / PT); }

// s_c = ((u_{i+1} - u_i) + (v_{j+1} - v_j) + (w_{k+1} - w_k)) / (h dt)
__global__ void __launch_bounds__(PT) k_divergence(Dims d, double hd, const double* __restrict__ u,
                                                   const double* __restrict__ v,
                                                   const double* __restrict__ w,
                                                   double* __restrict__ s, pcg::Apertures ap) {
    const long long t = blockIdx.x * (long long)PT + threadIdx.x;
    if (t >= d.n) return;
    const int c = (int)t;
    const int i = c % d.nx, j = (c / d.nx) % d.ny, k = c / d.sxy;
    const long long fu = i + (long long)(d.nx + 1) * (j + (long long)d.ny * k);
    const long long fv = i + (long long)d.nx * (j + (long long)(d.ny + 1) * k);
    if (ap.vol) {
        // cut cells: fluxes a u, divided by the cell's fluid fraction; 0 in inactive cells
        if (!(ap.vol[c] > 0.0)) {
            s[c] = 0.0;
            return;
        }
        const long long up = c + (long long)d.sxy;
        const double du = __dsub_rn(__dmul_rn(ap.ax[fu + 1], u[fu + 1]), __dmul_rn(ap.ax[fu], u[fu]));
        const double dv = __dsub_rn(__dmul_rn(ap.ay[fv + d.nx], v[fv + d.nx]),
                                    __dmul_rn(ap.ay[fv], v[fv]));
        const double dw = __dsub_rn(__dmul_rn(ap.az[up], w[up]), __dmul_rn(ap.az[c], w[c]));
        s[c] = __ddiv_rn(__ddiv_rn(__dadd_rn(__dadd_rn(du, dv), dw), hd), ap.vol[c]);
        return;
    }
    const double du = __dsub_rn(u[fu + 1], u[fu]);
    const double dv = __dsub_rn(v[fv + d.nx], v[fv]);
    const double dw = __dsub_rn(w[c + (long long)d.sxy], w[c]);
    s[c] = __ddiv_rn(__dadd_rn(__dadd_rn(du, dv), dw), hd);
}

// q - dt (beta ((p_hi - p_lo) / h)), in that order
__device__ __forceinline__ double corrected(double q, double dt, double beta, double p_hi,
                                            double p_lo, double h) {
    return __dsub_rn(q, __dmul_rn(dt, __dmul_rn(beta, __ddiv_rn(__dsub_rn(p_hi, p_lo), h))));
}

__global__ void __launch_bounds__(PT) k_project(Dims d, double h, double dt,
                                                const double* __restrict__ bx,
                                                const double* __restrict__ by,
                                                const double* __restrict__ bz,
                                                const double* __restrict__ top,
                                                const double* __restrict__ rinv2,
                                                const double* __restrict__ p, double* __restrict__ u,
                                                double* __restrict__ v, double* __restrict__ w,
                                                pcg::Apertures ap) {
    const long long t = blockIdx.x * (long long)PT + threadIdx.x;
    if (t >= d.n) return;
    const int c = (int)t;
    const int i = c % d.nx, j = (c / d.nx) % d.ny, k = c / d.sxy;
    const double pc = p[c];
    const long long fu = i + (long long)(d.nx + 1) * (j + (long long)d.ny * k);
    const long long fv = i + (long long)d.nx * (j + (long long)(d.ny + 1) * k);
    // cut cells: an open face's own coefficient is the cut coefficient over its open fraction
    auto beta = [&](const double* a, long long f, double b) {
        return a ? (b != 0.0 ? __ddiv_rn(b, a[f]) : 0.0) : b;
    };
    if (i > 0) {
        u[fu] = corrected(u[fu], dt, beta(ap.ax, fu, bx[c]), pc, p[c - 1], h);
    } else if (d.walls & pcg::PERIODIC_X) {
        // periodic x: faces 0 and nx are one face, corrected from face 0 and written to both
        const double q = corrected(u[fu], dt, beta(ap.ax, fu, bx[c]), pc, p[c + d.nx - 1], h);
        u[fu] = q;
        u[fu + d.nx] = q;
    }
    if (j > 0) v[fv] = corrected(v[fv], dt, beta(ap.ay, fv, by[c]), pc, p[c - d.nx], h);
    if (k > 0) w[c] = corrected(w[c], dt, beta(ap.az, c, bz[c]), pc, p[c - d.sxy], h);
    if (ap.vol && !(ap.vol[c] > 0.0)) return;  // inactive: no boundary faces
    auto open = [&](const double* a, long long f) { return !a || a[f] > 0.0; };
    if (k + 1 == d.nz && open(ap.az, c + (long long)d.sxy)) {
        // top face: p = 0 there; (1/rho_c) (0 - p_c) / (h/2) = (2/rho_c) ((0 - p_c) / h)
        const long long f = c + (long long)d.sxy;
        w[f] = corrected(w[f], dt, top[c - k * d.sxy], 0.0, pc, h);
    }
    if (d.walls & POISSON_WALLS_ALL) {
        // Dirichlet walls: p = 0 on the wall face, (2/rho_c) times the difference to 0 over h
        const double t = rinv2[c];
        if ((d.walls & 1) && i == 0 && open(ap.ax, fu)) u[fu] = corrected(u[fu], dt, t, pc, 0.0, h);
        if ((d.walls & 2) && i == d.nx - 1 && open(ap.ax, fu + 1))
            u[fu + 1] = corrected(u[fu + 1], dt, t, 0.0, pc, h);
        if ((d.walls & 4) && j == 0 && open(ap.ay, fv)) v[fv] = corrected(v[fv], dt, t, pc, 0.0, h);
        if ((d.walls & 8) && j == d.ny - 1 && open(ap.ay, fv + d.nx))
            v[fv + d.nx] = corrected(v[fv + d.nx], dt, t, 0.0, pc, h);
        if ((d.walls & 16) && k == 0 && open(ap.az, c)) w[c] = corrected(w[c], dt, t, pc, 0.0, h);
    }
}

// The reduced-pressure force (Entrance and Exit Boundary Conditions, hydrostatic-pressure
// method): the solve is for P_r = P - rho g (z - z_o), and the momentum equations carry
// -(z - z_o) (1/rho) d(rho g)/dx_i.  On the face between the low cell (density rl) and the high
// cell (rh) at height zf: f = -(zf - z_o) g (2/(rl + rh)) (rh - rl) / h, with the operator's face
// coefficient 2/(rl + rh), evaluated in this order.  Boundary faces get none (H continued beyond
// the boundary without change along its normal).
__device__ __forceinline__ double reduced_force(double rl, double rh, double zf, double zo,
                                                double g, double h) {
    const double a = __dmul_rn(__dsub_rn(zf, zo), g);
    const double b = __dmul_rn(__ddiv_rn(2.0, __dadd_rn(rl, rh)), __dsub_rn(rh, rl));
    return __ddiv_rn(-__dmul_rn(a, b), h);
}

__device__ __forceinline__ double rho_of(const double* F, long long c, double ra, double rw) {
    return __dadd_rn(ra, __dmul_rn(F[c], __dsub_rn(rw, ra)));
}

// u_f <- u_f + dt f on the low faces of every cell (one thread per cell); the periodic wrap face
// is written to faces 0 and nx.
__global__ void __launch_bounds__(PT) k_hydrostatic_force(Dims d, double h, const double* __restrict__ F,
                                                          double ra, double rw, double g, double zo,
                                                          double dt, double* __restrict__ u,
                                                          double* __restrict__ v,
                                                          double* __restrict__ w) {
    const long long t = blockIdx.x * (long long)PT + threadIdx.x;
    if (t >= d.n) return;
    const int c = (int)t;
    const int i = c % d.nx, j = (c / d.nx) % d.ny, k = c / d.sxy;
    const long long fu = i + (long long)(d.nx + 1) * (j + (long long)d.ny * k);
    const long long fv = i + (long long)d.nx * (j + (long long)(d.ny + 1) * k);
    const double rc = rho_of(F, c, ra, rw);
    const double zc = __dmul_rn(__dadd_rn((double)k, 0.5), h);  // height of the x and y faces
    if (i > 0) {
        u[fu] = __dadd_rn(u[fu], __dmul_rn(dt, reduced_force(rho_of(F, c - 1, ra, rw), rc, zc, zo, g, h)));
    } else if (d.walls & pcg::PERIODIC_X) {
        const double q = __dadd_rn(
            u[fu], __dmul_rn(dt, reduced_force(rho_of(F, c + d.nx - 1, ra, rw), rc, zc, zo, g, h)));
        u[fu] = q;
        u[fu + d.nx] = q;
    }
    if (j > 0)
        v[fv] = __dadd_rn(v[fv], __dmul_rn(dt, reduced_force(rho_of(F, c - d.nx, ra, rw), rc, zc, zo, g, h)));
    if (k > 0)
        w[c] = __dadd_rn(w[c], __dmul_rn(dt, reduced_force(rho_of(F, c - d.sxy, ra, rw), rc,
                                                           __dmul_rn((double)k, h), zo, g, h)));
}

// Device copies of caller arrays: the caller's pointer if it is device memory, else a temporary
// filled from the host (and, for outputs, copied back by flush()).
struct Staged {
    double* dev = nullptr;
    double* host = nullptr;
    size_t bytes = 0;
    bool owned = false;
    int stage(const double* p, size_t n, bool load, cudaStream_t st) {
        bytes = n * sizeof(double);
        if (is_device_ptr(p)) {
            dev = const_cast<double*>(p);
            return POISSON_OK;
        }
        host = const_cast<double*>(p);
        if (lib_malloc((void**)&dev, bytes) != cudaSuccess) {
            cudaGetLastError();
            dev = nullptr;
            return POISSON_ENOMEM;
        }
        owned = true;
        if (load && copy_user(dev, p, bytes, cudaMemcpyHostToDevice, st) != cudaSuccess) {
            cudaGetLastError();
            return POISSON_ECUDA;
        }
        return POISSON_OK;
    }
    int flush(cudaStream_t st) {
        if (!owned) return POISSON_OK;
        if (copy_user(host, dev, bytes, cudaMemcpyDeviceToHost, st) != cudaSuccess) {
            cudaGetLastError();
            return POISSON_ECUDA;
        }
        return POISSON_OK;
    }
    ~Staged() {
        if (owned && dev) lib_free(dev);
    }
};

int finish(cudaStream_t st) {
    const cudaError_t e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return POISSON_ECUDA;
    }
    return POISSON_OK;
}

}  // namespace

extern "C" int poisson_divergence(poisson_t* H, const double* u, const double* v, const double* w,
                                  double dt, double* s) {
    if (!H || !u || !v || !w || !s || !(dt > 0.0) || !std::isfinite(dt)) return POISSON_EINVAL;
    const Dims d = H->d;
    const size_t nu = (size_t)(d.nx + 1) * d.ny * d.nz, nv = (size_t)d.nx * (d.ny + 1) * d.nz,
                 nw = (size_t)d.sxy * (d.nz + 1);
    Staged U, V, W, S;
    int rc = U.stage(u, nu, true, H->st);
    if (rc == POISSON_OK) rc = V.stage(v, nv, true, H->st);
    if (rc == POISSON_OK) rc = W.stage(w, nw, true, H->st);
    if (rc == POISSON_OK) rc = S.stage(s, (size_t)d.n, false, H->st);
    if (rc != POISSON_OK) {
        finish(H->st);
        return rc;
    }
    k_divergence<<<blocks_of(d.n), PT, 0, H->st>>>(d, H->h * dt, U.dev, V.dev, W.dev, S.dev,
                                                  H->apertures());
    pcg::g_kernel_launches.fetch_add(1, std::memory_order_relaxed);
    if (cudaGetLastError() != cudaSuccess) rc = POISSON_ECUDA;
    if (rc == POISSON_OK) rc = S.flush(H->st);
    const int rs = finish(H->st);
    return rc != POISSON_OK ? rc : rs;
}

extern "C" int poisson_project(poisson_t* H, double* u, double* v, double* w, const double* p,
                               double dt) {
    if (!H || !u || !v || !w || !p || !(dt > 0.0) || !std::isfinite(dt)) return POISSON_EINVAL;
    if (!H->ready) return POISSON_ENOTREADY;
    const Dims d = H->d;
    const size_t nu = (size_t)(d.nx + 1) * d.ny * d.nz, nv = (size_t)d.nx * (d.ny + 1) * d.nz,
                 nw = (size_t)d.sxy * (d.nz + 1);
    Staged U, V, W, P;
    int rc = U.stage(u, nu, true, H->st);
    if (rc == POISSON_OK) rc = V.stage(v, nv, true, H->st);
    if (rc == POISSON_OK) rc = W.stage(w, nw, true, H->st);
    if (rc == POISSON_OK) rc = P.stage(p, (size_t)d.n, true, H->st);
    if (rc != POISSON_OK) {
        finish(H->st);
        return rc;
    }
    k_project<<<blocks_of(d.n), PT, 0, H->st>>>(d, H->h, dt, H->bx, H->by, H->bz, H->top64,
                                                H->rinv2, P.dev, U.dev, V.dev, W.dev,
                                                H->apertures());
    pcg::g_kernel_launches.fetch_add(1, std::memory_order_relaxed);
    if (cudaGetLastError() != cudaSuccess) rc = POISSON_ECUDA;
    if (rc == POISSON_OK) rc = U.flush(H->st);
    if (rc == POISSON_OK) rc = V.flush(H->st);
    if (rc == POISSON_OK) rc = W.flush(H->st);
    const int rs = finish(H->st);
    return rc != POISSON_OK ? rc : rs;
}

extern "C" int poisson_hydrostatic_force(poisson_t* H, const double* F, double rho_air,
                                         double rho_water, double g, double z_o, double dt,
                                         double* u, double* v, double* w) {
    if (!H || !F || !u || !v || !w || !(rho_air > 0.0) || !(rho_water > 0.0) ||
        !std::isfinite(rho_air) || !std::isfinite(rho_water) || !std::isfinite(g) ||
        !std::isfinite(z_o) || !std::isfinite(dt))
        return POISSON_EINVAL;
    const Dims d = H->d;
    const size_t nu = (size_t)(d.nx + 1) * d.ny * d.nz, nv = (size_t)d.nx * (d.ny + 1) * d.nz,
                 nw = (size_t)d.sxy * (d.nz + 1);
    Staged Fs, U, V, W;
    int rc = Fs.stage(F, (size_t)d.n, true, H->st);
    if (rc == POISSON_OK) rc = U.stage(u, nu, true, H->st);
    if (rc == POISSON_OK) rc = V.stage(v, nv, true, H->st);
    if (rc == POISSON_OK) rc = W.stage(w, nw, true, H->st);
    if (rc != POISSON_OK) {
        finish(H->st);
        return rc;
    }
    k_hydrostatic_force<<<blocks_of(d.n), PT, 0, H->st>>>(d, H->h, Fs.dev, rho_air, rho_water, g,
                                                          z_o, dt, U.dev, V.dev, W.dev);
    pcg::g_kernel_launches.fetch_add(1, std::memory_order_relaxed);
    if (cudaGetLastError() != cudaSuccess) rc = POISSON_ECUDA;
    if (rc == POISSON_OK) rc = U.flush(H->st);
    if (rc == POISSON_OK) rc = V.flush(H->st);
    if (rc == POISSON_OK) rc = W.flush(H->st);
    const int rs = finish(H->st);
    return rc != POISSON_OK ? rc : rs;
}

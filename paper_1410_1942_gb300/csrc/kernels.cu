// kernels.cu -- operator setup, FP64 residual/refinement and the PCG phase kernels.
//
// PCG (Introduction: preconditioned conjugate gradients on the second-order variable-coefficient
// Poisson equation) is split at its two global reductions into two fused passes per iteration:
//
//   phase A:  p = z + beta p_old;  q = A p (not stored);  sum p.q          -> alpha = rz / pq
//   phase B:  q = A p (recomputed); x += alpha p;  r -= alpha q;  z = M^{-1} r;
//             sum r.z and r.r                                            -> beta, convergence
//
// Recomputing q in phase B costs one more stencil evaluation but saves writing and re-reading q.
// p is double-buffered (phase A reads neighbours of p_old while writing p).  All CG scalars live
// in device memory (struct Scalars); the last block of each reduction updates them, and every
// kernel returns at once when the solve is finished, so chunks of iterations can be queued
// without host round trips.
#include "internal.cuh"
#include "kernels.h"
#include "jobs.cuh"
#include "plane_tile.cuh"

#include <algorithm>
#include <atomic>

namespace pcg {

// ------------------------------------------------------------------ operator setup (FP64)
// rho = rho_air + F (rho_water - rho_air) with explicit rounding (no contraction) so the FP64
// face arrays are reproducible bit for bit.
__device__ __forceinline__ double rho_of(double F, double ra, double rw) {
    return __dadd_rn(ra, __dmul_rn(F, __dadd_rn(rw, -ra)));
}

// bad: set to 1 when some cell's density is not a positive finite number (F non-finite, or so
// far outside [0, 1] that rho <= 0): the operator is then not SPD
__global__ void k_setup_faces(Dims d, const double* __restrict__ F, double ra, double rw,
                              double* __restrict__ bx, double* __restrict__ by,
                              double* __restrict__ bz, float* __restrict__ eta32,
                              __nv_bfloat16* __restrict__ eta16, Apertures ap,
                              unsigned* __restrict__ bad) {
    const long long tid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (tid >= d.n) return;
    const int c = (int)tid;
    const int i = c % d.nx, j = (c / d.nx) % d.ny, k = c / d.sxy;
    const double rc = rho_of(F[c], ra, rw);
    if (!(rc > 0.0) || !isfinite(rc)) *bad = 1u;
    // periodic x: the low face of cell 0 couples it to cell nx-1 of its row
    bx[c] = (i > 0 || (d.walls & PERIODIC_X))
                ? 2.0 / __dadd_rn(rc, rho_of(F[i > 0 ? c - 1 : c + d.nx - 1], ra, rw))
                : 0.0;
    by[c] = (j > 0) ? 2.0 / __dadd_rn(rc, rho_of(F[c - d.nx], ra, rw)) : 0.0;
    bz[c] = (k > 0) ? 2.0 / __dadd_rn(rc, rho_of(F[c - d.sxy], ra, rw)) : 0.0;
    if (ap.ax) {
        // cut cells: each face scaled by its open fraction; closed next to a cell with no fluid
        const long long fu = i + (long long)(d.nx + 1) * (j + (long long)d.ny * k);
        const long long fv = i + (long long)d.nx * (j + (long long)(d.ny + 1) * k);
        const bool act = ap.vol[c] > 0.0;
        const int cxm = i > 0 ? c - 1 : c + d.nx - 1;
        bx[c] = (act && ap.vol[cxm] > 0.0) ? __dmul_rn(ap.ax[fu], bx[c]) : 0.0;
        by[c] = (act && j > 0 && ap.vol[c - d.nx] > 0.0) ? __dmul_rn(ap.ay[fv], by[c]) : 0.0;
        bz[c] = (act && k > 0 && ap.vol[c - d.sxy] > 0.0) ? __dmul_rn(ap.az[c], bz[c]) : 0.0;
    }
    const double e = 0.5 * rc;
    if (eta32) eta32[c] = (float)e;
    if (eta16) eta16[c] = __float2bfloat16_rn((float)e);
}

// diag = bx[c] + by[c] + bz[c] + high faces (+ 2/rho_c on the top layer) (+ 2/rho_c for each
// Dirichlet side/bottom wall the cell touches, x-, x+, y-, y+, z-), summed in that order;
// top[i + nx j] = 2/rho_c of the top layer; rinv2[c] = 2/rho_c (only with Dirichlet walls).
__global__ void k_setup_diag(Dims d, const double* __restrict__ F, double ra, double rw,
                             const double* __restrict__ bx, const double* __restrict__ by,
                             const double* __restrict__ bz, double* __restrict__ diag,
                             double* __restrict__ dinv, double* __restrict__ top,
                             double* __restrict__ rinv2, Apertures ap) {
    const long long tid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (tid >= d.n) return;
    const int c = (int)tid;
    const int i = c % d.nx, j = (c / d.nx) % d.ny, k = c / d.sxy;
    const double t = 2.0 / rho_of(F[c], ra, rw);  // a boundary face's coefficient (unscaled)
    if (k + 1 == d.nz && top) top[c - k * d.sxy] = t;
    if (rinv2) rinv2[c] = t;
    if (ap.vol && !(ap.vol[c] > 0.0)) {
        // cut cells: a cell with no fluid is inactive
        diag[c] = 1.0;
        if (dinv) dinv[c] = 1.0;
        return;
    }
    const long long fu = i + (long long)(d.nx + 1) * (j + (long long)d.ny * k);
    const long long fv = i + (long long)d.nx * (j + (long long)(d.ny + 1) * k);
    // a boundary term, scaled by its face's open fraction with cut cells
    auto bnd = [&](const double* a, long long f) { return a ? __dmul_rn(a[f], t) : t; };
    double s = __dadd_rn(__dadd_rn(bx[c], by[c]), bz[c]);
    if (i + 1 < d.nx) s = __dadd_rn(s, bx[c + 1]);
    else if (d.walls & PERIODIC_X) s = __dadd_rn(s, bx[c + 1 - d.nx]);
    if (j + 1 < d.ny) s = __dadd_rn(s, by[c + d.nx]);
    if (k + 1 < d.nz) s = __dadd_rn(s, bz[c + d.sxy]);
    else s = __dadd_rn(s, bnd(ap.az, c + (long long)d.sxy));
    if ((d.walls & 1) && i == 0) s = __dadd_rn(s, bnd(ap.ax, fu));
    if ((d.walls & 2) && i == d.nx - 1) s = __dadd_rn(s, bnd(ap.ax, fu + 1));
    if ((d.walls & 4) && j == 0) s = __dadd_rn(s, bnd(ap.ay, fv));
    if ((d.walls & 8) && j == d.ny - 1) s = __dadd_rn(s, bnd(ap.ay, fv + d.nx));
    if ((d.walls & 16) && k == 0) s = __dadd_rn(s, bnd(ap.az, c));
    diag[c] = s;
    if (dinv) dinv[c] = 1.0 / s;
}

// b = a s, or a (vol s) with cut cells (vol: fluid fractions, may be null)
__global__ void k_scale(long long n, const double* __restrict__ s, double a,
                        const double* __restrict__ vol, double* __restrict__ b) {
    const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t < n) b[t] = __dmul_rn(a, vol ? __dmul_rn(vol[t], s[t]) : s[t]);
}

__global__ void k_update64(long long n, double* __restrict__ x, const float* __restrict__ dlt) {
    const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t < n) x[t] += (double)dlt[t];
}

template <typename T>
__global__ void k_narrow(long long n, const double* __restrict__ a, T* __restrict__ b) {
    const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t < n) b[t] = (T)a[t];
}

template <typename T>
__global__ void k_widen(long long n, const T* __restrict__ a, double* __restrict__ b) {
    const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t < n) b[t] = (double)a[t];
}

template <typename T>
__global__ void k_fill(long long n, T* __restrict__ p, float v) {
    const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t < n) p[t] = (T)v;
}

// ------------------------------------------------------------------ stencil helpers
#define COL_LOOP_BEGIN                                                         \
    const int i = blockIdx.x * TX + threadIdx.x;                               \
    const int j = blockIdx.y * TY + threadIdx.y;                               \
    const int k0 = blockIdx.z * kc;                                            \
    const int k1 = min(d.nz, k0 + kc);                                         \
    if (i < d.nx && j < d.ny)                                                  \
        for (int k = k0; k < k1; ++k) {                                        \
            const int c = i + d.nx * (j + d.ny * k);

#define COL_LOOP_END }

template <typename V, typename Coef>
__device__ __forceinline__ V inv_diag(const Coef& coef, int c, const Stencil<V>& w);

template <>
__device__ __forceinline__ double inv_diag<double, CoefFaces64>(const CoefFaces64& coef, int c,
                                                                const Stencil<double>& w) {
    return coef.dinv ? coef.dinv[c] : 1.0 / w.D;
}
template <>
__device__ __forceinline__ float inv_diag<float, CoefEta<float>>(const CoefEta<float>&, int,
                                                                 const Stencil<float>& w) {
    return rcp_approx(w.D);
}
template <>
__device__ __forceinline__ float inv_diag<float, CoefEta<__nv_bfloat16>>(
    const CoefEta<__nv_bfloat16>&, int, const Stencil<float>& w) {
    return rcp_approx(w.D);
}
template <>
__device__ __forceinline__ float inv_diag<float, CoefFaces32>(const CoefFaces32&, int,
                                                              const Stencil<float>& w) {
    return rcp_approx(w.D);
}

// ------------------------------------------------------------------ FP64 residual
// r = b - A x with the FP64 operator; writes r (as R) and reduces (r.r, b.b) into sc->rr, sc->bb.
template <typename R>
__global__ void __launch_bounds__(TX * TY) k_residual64(Dims d, CoefFaces64 coef, int kc,
                                                       const double* __restrict__ b,
                                                       const double* __restrict__ x,
                                                       R* __restrict__ r, Scalars* sc,
                                                       double* partials) {
    __shared__ double smem[64];
    double rr = 0.0, bb = 0.0;
    auto ld = [&](int e) { return x[e]; };
    COL_LOOP_BEGIN
        Stencil<double> w;
        coef.weights(d, c, i, j, k, w);
        const double ax = w.D * x[c] - nb_sum(d, w, c, i, j, k, ld);
        const double bc = b[c];
        const double rc = bc - ax;
        r[c] = (R)rc;
        rr += rc * rc;
        bb += bc * bc;
    COL_LOOP_END
    double v[2] = {rr, bb}, tot[2];
    if (grid_sum<2>(v, partials, &sc->ticket, tot, smem)) {
        if (threadIdx.x == 0 && threadIdx.y == 0) {
            sc->rr = tot[0];
            sc->bb = tot[1];
        }
    }
}

// ------------------------------------------------------------------ y = A x, z = D^{-1} r
template <typename V, typename Coef>
__global__ void __launch_bounds__(TX * TY) k_apply(Dims d, Coef coef, int kc,
                                                  const double* __restrict__ x,
                                                  double* __restrict__ y) {
    auto ld = [&](int e) { return (V)x[e]; };
    COL_LOOP_BEGIN
        Stencil<V> w;
        coef.weights(d, c, i, j, k, w);
        y[c] = (double)(w.D * ld(c) - nb_sum(d, w, c, i, j, k, ld));
    COL_LOOP_END
}

template <typename V, typename Coef>
__global__ void __launch_bounds__(TX * TY) k_jacobi(Dims d, Coef coef, int kc,
                                                   const double* __restrict__ r,
                                                   double* __restrict__ z) {
    COL_LOOP_BEGIN
        Stencil<V> w;
        coef.weights(d, c, i, j, k, w);
        z[c] = (double)((V)r[c] * inv_diag<V, Coef>(coef, c, w));
    COL_LOOP_END
}

// ------------------------------------------------------------------ PCG passes
// init: z = D^{-1} r, rz = r.z, rr0 = r.r; stop2 = tol2 * (rel_to_b ? bb : rr0).
template <typename V, typename Coef>
__global__ void __launch_bounds__(TX * TY) k_cg_init(Dims d, Coef coef, int kc,
                                                    const V* __restrict__ r, V* __restrict__ z,
                                                    Scalars* sc, double* partials, double tol2,
                                                    int rel_to_b, int max_iter) {
    __shared__ double smem[64];
    V rz = 0, rr = 0;
    COL_LOOP_BEGIN
        Stencil<V> w;
        coef.weights(d, c, i, j, k, w);
        const V rc = r[c];
        const V zc = rc * inv_diag<V, Coef>(coef, c, w);
        z[c] = zc;
        rz += rc * zc;
        rr += rc * rc;
    COL_LOOP_END
    double v[2] = {(double)rz, (double)rr}, tot[2];
    if (grid_sum<2>(v, partials, &sc->ticket, tot, smem)) {
        if (threadIdx.x == 0 && threadIdx.y == 0) {
            sc->rz = tot[0];
            sc->rr = tot[1];
            sc->rr0 = tot[1];
            sc->beta = 0.0;
            sc->alpha = 0.0;
            sc->iter = 0;
            sc->max_iter = max_iter;
            sc->stop2 = tol2 * (rel_to_b ? sc->bb : tot[1]);
            sc->done = (tot[1] <= sc->stop2) ? CONVERGED : RUNNING;
            if (!isfinite(tot[0]) || !isfinite(tot[1])) sc->done = BREAKDOWN;
        }
    }
}

template <typename V, typename Coef>
__global__ void __launch_bounds__(TX * TY) k_cg_a(Dims d, Coef coef, int kc,
                                                 const V* __restrict__ z,
                                                 const V* __restrict__ p_in,
                                                 V* __restrict__ p_out, Scalars* sc,
                                                 double* partials) {
    pdl_entry();
    __shared__ double smem[64];
    if (sc->done) return;
    const V beta = (V)sc->beta;
    auto pn = [&](int e) { return z[e] + beta * p_in[e]; };
    V acc = 0;
    COL_LOOP_BEGIN
        Stencil<V> w;
        coef.weights(d, c, i, j, k, w);
        const V pc = pn(c);
        const V q = w.D * pc - nb_sum(d, w, c, i, j, k, pn);
        acc += pc * q;
        p_out[c] = pc;
    COL_LOOP_END
    double v[1] = {(double)acc}, tot[1];
    if (grid_sum<1>(v, partials, &sc->ticket, tot, smem)) {
        if (threadIdx.x == 0 && threadIdx.y == 0) {
            const double pq = tot[0];
            if (!(pq > 0.0) || !isfinite(pq)) {
                sc->done = BREAKDOWN;
            } else {
                sc->pq = pq;
                sc->alpha = sc->rz / pq;
            }
        }
    }
}

// Phase A on the rho/2 operator, marching the thread's column in z with the values of the planes
// k-1, k, k+1 in registers and the loads of plane k+2 issued before plane k is computed (the
// plain k_cg_a leaves one plane's loads in flight per thread, which bounds it by latency).  Same
// arithmetic, in the same order, as k_cg_a with CoefEta.
template <typename E>
__global__ void __launch_bounds__(TX * TY) k_cg_a_eta(Dims d, CoefEta<E> coef, int kc,
                                                     const float* __restrict__ z,
                                                     const float* __restrict__ p_in,
                                                     float* __restrict__ p_out, Scalars* sc,
                                                     double* partials) {
    pdl_entry();
    __shared__ double smem[64];
    if (sc->done) return;
    const float beta = (float)sc->beta;
    const int i = blockIdx.x * TX + threadIdx.x;
    const int j = blockIdx.y * TY + threadIdx.y;
    const int k0 = blockIdx.z * kc;
    const int k1 = min(d.nz, k0 + kc);
    float acc = 0.f;
    if (i < d.nx && j < d.ny) {
        const bool per = d.walls & PERIODIC_X;
        const bool hxm = i > 0 || per, hxp = i + 1 < d.nx || per, hym = j > 0, hyp = j + 1 < d.ny;
        const int oxm = i > 0 ? -1 : d.nx - 1, oxp = i + 1 < d.nx ? 1 : 1 - d.nx;
        auto pn = [&](int e) { return z[e] + beta * p_in[e]; };
        auto et = [&](int e) { return eta_load(coef.eta, e); };
        int c = i + d.nx * (j + d.ny * k0);
        float pm = 0.f, em = 0.f, pp = 0.f, ep = 0.f, pq = 0.f, eq = 0.f;
        if (k0 > 0) { pm = pn(c - d.sxy); em = et(c - d.sxy); }
        float p0 = pn(c), e0 = et(c);
        if (k0 + 1 < d.nz) { pp = pn(c + d.sxy); ep = et(c + d.sxy); }
        for (int k = k0; k < k1; ++k, c += d.sxy) {
            if (k + 1 < k1 && k + 2 < d.nz) { pq = pn(c + 2 * d.sxy); eq = et(c + 2 * d.sxy); }
            Stencil<float> w;
            eta_stencil(d, i, j, k, e0, hxm ? et(c + oxm) : 0.f, hxp ? et(c + oxp) : 0.f,
                        hym ? et(c - d.nx) : 0.f, hyp ? et(c + d.nx) : 0.f, em, ep, w);
            float s = 0.f;
            if (hxm) s += w.xm * pn(c + oxm);
            if (hxp) s += w.xp * pn(c + oxp);
            if (hym) s += w.ym * pn(c - d.nx);
            if (hyp) s += w.yp * pn(c + d.nx);
            if (k > 0) s += w.zm * pm;
            if (k + 1 < d.nz) s += w.zp * pp;
            const float q = w.D * p0 - s;
            acc += p0 * q;
            p_out[c] = p0;
            pm = p0; em = e0;
            p0 = pp; e0 = ep;
            pp = pq; ep = eq;
        }
    }
    double v[1] = {(double)acc}, tot[1];
    if (grid_sum<1>(v, partials, &sc->ticket, tot, smem)) {
        if (threadIdx.x == 0 && threadIdx.y == 0) {
            const double pq2 = tot[0];
            if (!(pq2 > 0.0) || !isfinite(pq2)) {
                sc->done = BREAKDOWN;
            } else {
                sc->pq = pq2;
                sc->alpha = sc->rz / pq2;
            }
        }
    }
}

// k_cg_a_eta with the x and y neighbours of plane k from a shared plane (plane_tile.cuh): the
// same arithmetic in the same order, two global loads of p per cell and plane (z, p_in) plus the
// halo's share.  Grids with plane_tiles_fit only.
template <typename E>
__global__ void __launch_bounds__(TX * TY) k_cg_a_sm(Dims d, CoefEta<E> coef, int kc,
                                                    const float* __restrict__ z,
                                                    const float* __restrict__ p_in,
                                                    float* __restrict__ p_out, Scalars* sc,
                                                    double* partials) {
    pdl_entry();
    __shared__ double smem[64];
    __shared__ float Ps[2][PT_N], Es[2][PT_N];
    if (sc->done) return;
    const float beta = (float)sc->beta;
    const int i = blockIdx.x * TX + threadIdx.x;
    const int j = blockIdx.y * TY + threadIdx.y;
    const int k0 = blockIdx.z * kc;
    const int k1 = min(d.nz, k0 + kc);
    const bool act = j < d.ny;  // i < nx: whole tiles along x
    const int ci = pt_index(threadIdx.x, threadIdx.y);
    int hx, hy;
    const bool hs = pt_halo_slot(threadIdx.x + TX * threadIdx.y, hx, hy);
    const int gx = blockIdx.x * TX + hx, gy = blockIdx.y * TY + hy;
    const bool hv = hs && gx >= 0 && gx < d.nx && gy >= 0 && gy < d.ny;
    const int hi = hs ? pt_index(hx, hy) : 0;
    const bool hxm = i > 0, hxp = i + 1 < d.nx, hym = j > 0, hyp = j + 1 < d.ny;
    auto pn = [&](int e) { return z[e] + beta * p_in[e]; };
    auto et = [&](int e) { return eta_load(coef.eta, e); };
    int c = i + d.nx * (j + d.ny * k0);
    int h = gx + d.nx * (gy + d.ny * k0);
    float pm = 0.f, em = 0.f, p0 = 0.f, e0 = 0.f, pp = 0.f, ep = 0.f, pq = 0.f, eq = 0.f;
    if (act) {
        if (k0 > 0) { pm = pn(c - d.sxy); em = et(c - d.sxy); }
        p0 = pn(c);
        e0 = et(c);
        if (k0 + 1 < d.nz) { pp = pn(c + d.sxy); ep = et(c + d.sxy); }
    }
    float hp = 0.f, he = 0.f, hpn = 0.f, hen = 0.f;
    if (hv) { hp = pn(h); he = et(h); }
    float acc = 0.f;
    for (int k = k0; k < k1; ++k, c += d.sxy, h += d.sxy) {
        const int b = (k - k0) & 1;
        Ps[b][ci] = p0;
        Es[b][ci] = e0;
        if (hs) { Ps[b][hi] = hp; Es[b][hi] = he; }
        if (act && k + 1 < k1 && k + 2 < d.nz) { pq = pn(c + 2 * d.sxy); eq = et(c + 2 * d.sxy); }
        if (hv && k + 1 < k1) { hpn = pn(h + d.sxy); hen = et(h + d.sxy); }
        __syncthreads();
        if (act) {
            const float* P = Ps[b];
            const float* Ee = Es[b];
            Stencil<float> w;
            eta_stencil(d, i, j, k, e0, hxm ? Ee[ci - 1] : 0.f, hxp ? Ee[ci + 1] : 0.f,
                        hym ? Ee[ci - PT_W] : 0.f, hyp ? Ee[ci + PT_W] : 0.f, em, ep, w);
            float s = 0.f;
            if (hxm) s += w.xm * P[ci - 1];
            if (hxp) s += w.xp * P[ci + 1];
            if (hym) s += w.ym * P[ci - PT_W];
            if (hyp) s += w.yp * P[ci + PT_W];
            if (k > 0) s += w.zm * pm;
            if (k + 1 < d.nz) s += w.zp * pp;
            const float q = w.D * p0 - s;
            acc += p0 * q;
            p_out[c] = p0;
        }
        pm = p0; em = e0;
        p0 = pp; e0 = ep;
        pp = pq; ep = eq;
        hp = hpn; he = hen;
    }
    double v[1] = {(double)acc}, tot[1];
    if (grid_sum<1>(v, partials, &sc->ticket, tot, smem)) {
        if (threadIdx.x == 0 && threadIdx.y == 0) {
            const double pq2 = tot[0];
            if (!(pq2 > 0.0) || !isfinite(pq2)) {
                sc->done = BREAKDOWN;
            } else {
                sc->pq = pq2;
                sc->alpha = sc->rz / pq2;
            }
        }
    }
}

// k_cg_a_sm with 2 x 2 cells per thread (quad_march, plane_tile.cuh): p = z + beta p_in and
// (p, A p) on QX x QY tiles of kc planes.  Grids with quad_tiles_fit only.
struct BodyCgA {
    static constexpr int NX = 0;
    const float* in[1];
    float* p_out;
    int nx;
    float acc = 0.f;
    __device__ __forceinline__ void cell(int c, int, int, int, const Quad& u, const Quad& q,
                                         const Quad&, const Quad*) {
#pragma unroll
        for (int a = 0; a < 2; ++a)
#pragma unroll
            for (int b = 0; b < 2; ++b) acc += u.v[a][b] * q.v[a][b];
        st2(p_out, c, u.v[0][0], u.v[0][1]);
        st2(p_out, c + nx, u.v[1][0], u.v[1][1]);
    }
};

template <typename E>
__global__ void __launch_bounds__(TX * TY, QB_CG_A) k_cg_a_q(Dims d, CoefEta<E> coef, int kc,
                                                                const float* __restrict__ z,
                                                                const float* __restrict__ p_in,
                                                                float* __restrict__ p_out,
                                                                Scalars* sc, double* partials) {
    pdl_entry();
    __shared__ double smem[64];
    if (sc->done) return;
    FieldSum F{z, p_in, (float)sc->beta};
    BodyCgA B{{nullptr}, p_out, d.nx};
    quad_march(d, coef.eta, kc, F, B);
    double v[1] = {(double)B.acc}, tot[1];
    if (grid_sum<1>(v, partials, &sc->ticket, tot, smem)) {
        if (threadIdx.x == 0 && threadIdx.y == 0) {
            const double pq2 = tot[0];
            if (!(pq2 > 0.0) || !isfinite(pq2)) {
                sc->done = BREAKDOWN;
            } else {
                sc->pq = pq2;
                sc->alpha = sc->rz / pq2;
            }
        }
    }
}

// Phase A on FP32 faces (cut-cell handles), 2 x 2 cells per thread: as k_cg_a_q.
__global__ void __launch_bounds__(TX * TY, QB_FACES) k_cg_a_fq(Dims d, CoefFaces32 coef, int kc,
                                                              const float* __restrict__ z,
                                                              const float* __restrict__ p_in,
                                                              float* __restrict__ p_out,
                                                              Scalars* sc, double* partials) {
    pdl_entry();
    __shared__ double smem[64];
    if (sc->done) return;
    FieldSum F{z, p_in, (float)sc->beta};
    BodyCgA B{{nullptr}, p_out, d.nx};
    quad_march_faces(d, coef, kc, F, B);
    double v[1] = {(double)B.acc}, tot[1];
    if (grid_sum<1>(v, partials, &sc->ticket, tot, smem)) {
        if (threadIdx.x == 0 && threadIdx.y == 0) {
            const double pq2 = tot[0];
            if (!(pq2 > 0.0) || !isfinite(pq2)) {
                sc->done = BREAKDOWN;
            } else {
                sc->pq = pq2;
                sc->alpha = sc->rz / pq2;
            }
        }
    }
}

// Jacobi phase B on FP32 faces, 2 x 2 cells per thread: x += alpha p; r -= alpha A p;
// z = r rcp(D); sums (r, z), (r, r) and the decision, as k_cg_b.
struct BodyCgBJ {
    static constexpr int NX = 2;
    const float* in[NX];
    float* x;
    float* r;
    float* z;
    float alpha;
    int nx;
    float rz = 0.f, rr = 0.f;
    __device__ __forceinline__ void cell(int c, int, int, int, const Quad& u, const Quad& q,
                                         const Quad& D, const Quad* X) {
        Quad xn, rn, zn;
#pragma unroll
        for (int a = 0; a < 2; ++a)
#pragma unroll
            for (int b = 0; b < 2; ++b) {
                xn.v[a][b] = X[0].v[a][b] + alpha * u.v[a][b];
                rn.v[a][b] = X[1].v[a][b] - alpha * q.v[a][b];
                zn.v[a][b] = rn.v[a][b] * rcp_approx(D.v[a][b]);
                rz += rn.v[a][b] * zn.v[a][b];
                rr += rn.v[a][b] * rn.v[a][b];
            }
        st2(x, c, xn.v[0][0], xn.v[0][1]);
        st2(x, c + nx, xn.v[1][0], xn.v[1][1]);
        st2(r, c, rn.v[0][0], rn.v[0][1]);
        st2(r, c + nx, rn.v[1][0], rn.v[1][1]);
        st2(z, c, zn.v[0][0], zn.v[0][1]);
        st2(z, c + nx, zn.v[1][0], zn.v[1][1]);
    }
};

__global__ void __launch_bounds__(TX * TY, QB_FACES) k_cg_b_fq(Dims d, CoefFaces32 coef, int kc,
                                                              const float* __restrict__ p,
                                                              float* __restrict__ x,
                                                              float* __restrict__ r,
                                                              float* __restrict__ z, Scalars* sc,
                                                              double* partials) {
    pdl_entry();
    __shared__ double smem[64];
    if (sc->done) return;
    FieldPlain F{p};
    BodyCgBJ B{{x, r}, x, r, z, (float)sc->alpha, d.nx};
    quad_march_faces(d, coef, kc, F, B);
    double v[2] = {(double)B.rz, (double)B.rr}, tot[2];
    if (grid_sum<2>(v, partials, &sc->ticket, tot, smem)) {
        if (threadIdx.x == 0 && threadIdx.y == 0) {
            const double rz_new = tot[0], rr_new = tot[1];
            sc->iter += 1;
            sc->rr = rr_new;
            if (!isfinite(rz_new) || !isfinite(rr_new) || rz_new < 0.0) {
                sc->done = BREAKDOWN;
            } else if (rr_new <= sc->stop2) {
                sc->done = CONVERGED;
            } else if (sc->iter >= sc->max_iter) {
                sc->done = CAPPED;
            } else {
                sc->beta = rz_new / sc->rz;
                sc->rz = rz_new;
            }
        }
    }
}

template <typename V, typename Coef>
__global__ void __launch_bounds__(TX * TY) k_cg_b(Dims d, Coef coef, int kc,
                                                 const V* __restrict__ p, V* __restrict__ x,
                                                 V* __restrict__ r, V* __restrict__ z,
                                                 Scalars* sc, double* partials) {
    __shared__ double smem[64];
    if (sc->done) return;
    const V alpha = (V)sc->alpha;
    auto ld = [&](int e) { return p[e]; };
    V rz = 0, rr = 0;
    COL_LOOP_BEGIN
        Stencil<V> w;
        coef.weights(d, c, i, j, k, w);
        const V pc = p[c];
        const V q = w.D * pc - nb_sum(d, w, c, i, j, k, ld);
        x[c] += alpha * pc;
        const V rn = r[c] - alpha * q;
        const V zn = rn * inv_diag<V, Coef>(coef, c, w);
        r[c] = rn;
        z[c] = zn;
        rz += rn * zn;
        rr += rn * rn;
    COL_LOOP_END
    double v[2] = {(double)rz, (double)rr}, tot[2];
    if (grid_sum<2>(v, partials, &sc->ticket, tot, smem)) {
        if (threadIdx.x == 0 && threadIdx.y == 0) {
            const double rz_new = tot[0], rr_new = tot[1];
            sc->iter += 1;
            sc->rr = rr_new;
            if (!isfinite(rz_new) || !isfinite(rr_new) || rz_new < 0.0) {
                sc->done = BREAKDOWN;
            } else if (rr_new <= sc->stop2) {
                sc->done = CONVERGED;
            } else if (sc->iter >= sc->max_iter) {
                sc->done = CAPPED;
            } else {
                sc->beta = rz_new / sc->rz;
                sc->rz = rz_new;
            }
        }
    }
}

// ------------------------------------------------------------------ red-black SSOR
// M = (D - wE) D^-1 (D - wE^T) / (w (2 - w)) in red-black order (red = (i+j+k) even first),
// applied as: y_R = r_R / D_R; y_B = (r_B + w sum_{red nbrs} w_f y_R) / D_B;
// t_R = y_R + w (sum_{black nbrs} w_f y_B) / D_R, t_B = y_B; z = w (2 - w) t.  Inside PCG the
// constant factor w (2 - w) is left out (it rescales the search directions, not the iterates);
// poisson_precond_apply applies it.  Each sweep updates one colour and reads only the other.
__device__ __forceinline__ bool is_red(int i, int j, int k) { return ((i + j + k) & 1) == 0; }

// phase B of SSOR-PCG: q = A p (recomputed), x += alpha p, r -= alpha q, z_R = r_R / D_R; sums r.r
template <typename V, typename Coef>
__global__ void __launch_bounds__(TX * TY) k_cg_b_ssor(Dims d, Coef coef, int kc,
                                                      const V* __restrict__ p, V* __restrict__ x,
                                                      V* __restrict__ r, V* __restrict__ z,
                                                      Scalars* sc, double* partials) {
    __shared__ double smem[64];
    if (sc->done) return;
    const V alpha = (V)sc->alpha;
    auto ld = [&](int e) { return p[e]; };
    V rr = 0;
    COL_LOOP_BEGIN
        Stencil<V> w;
        coef.weights(d, c, i, j, k, w);
        const V pc = p[c];
        const V q = w.D * pc - nb_sum(d, w, c, i, j, k, ld);
        x[c] += alpha * pc;
        const V rn = r[c] - alpha * q;
        r[c] = rn;
        if (is_red(i, j, k)) z[c] = rn * inv_diag<V, Coef>(coef, c, w);
        rr += rn * rn;
    COL_LOOP_END
    double v[1] = {(double)rr}, tot[1];
    if (grid_sum<1>(v, partials, &sc->ticket, tot, smem)) {
        if (threadIdx.x == 0 && threadIdx.y == 0) sc->rr = tot[0];
    }
}

// SSOR start from r: z_R = r_R / D_R (the black sweep and k_ssor_red follow); sums r.r and sets
// the solve's scalars like k_cg_init.  R is the type r is read as (V, or double for the
// checking entry point).
template <typename V, typename Coef, typename R>
__global__ void __launch_bounds__(TX * TY) k_ssor_first(Dims d, Coef coef, int kc,
                                                       const R* __restrict__ r, V* __restrict__ z,
                                                       Scalars* sc, double* partials, double tol2,
                                                       int rel_to_b, int max_iter) {
    __shared__ double smem[64];
    V rr = 0;
    COL_LOOP_BEGIN
        const V rc = (V)r[c];
        if (is_red(i, j, k)) {
            Stencil<V> w;
            coef.weights(d, c, i, j, k, w);
            z[c] = rc * inv_diag<V, Coef>(coef, c, w);
        }
        rr += rc * rc;
    COL_LOOP_END
    if (!sc) return;
    double v[1] = {(double)rr}, tot[1];
    if (grid_sum<1>(v, partials, &sc->ticket, tot, smem)) {
        if (threadIdx.x == 0 && threadIdx.y == 0) {
            sc->rr = tot[0];
            sc->rr0 = tot[0];
            sc->beta = 0.0;
            sc->alpha = 0.0;
            sc->iter = 0;
            sc->max_iter = max_iter;
            sc->stop2 = tol2 * (rel_to_b ? sc->bb : tot[0]);
            sc->done = (tot[0] <= sc->stop2) ? CONVERGED : RUNNING;
            if (!isfinite(tot[0])) sc->done = BREAKDOWN;
            sc->rz = 0.0;
        }
    }
}

// black sweep: z_B = (r_B + w sum_{red nbrs} w_f z) / D_B
template <typename V, typename Coef, typename R>
__global__ void __launch_bounds__(TX * TY) k_ssor_black(Dims d, Coef coef, int kc,
                                                       const R* __restrict__ r,
                                                       V* __restrict__ z, double omega,
                                                       const Scalars* sc) {
    if (sc && sc->done) return;
    const V om = (V)omega;
    auto ld = [&](int e) { return z[e]; };
    COL_LOOP_BEGIN
        if (!is_red(i, j, k)) {
            Stencil<V> w;
            coef.weights(d, c, i, j, k, w);
            z[c] = ((V)r[c] + om * nb_sum(d, w, c, i, j, k, ld)) * inv_diag<V, Coef>(coef, c, w);
        }
    COL_LOOP_END
}

// red sweep: z_R += w (sum_{black nbrs} w_f z) / D_R; then, inside PCG, sums r.z and updates
// beta and the stopping state (mode 1), or only stores rz after the start (mode 0).
template <typename V, typename Coef>
__global__ void __launch_bounds__(TX * TY) k_ssor_red(Dims d, Coef coef, int kc,
                                                     const V* __restrict__ r, V* __restrict__ z,
                                                     double omega, Scalars* sc, double* partials,
                                                     int mode) {
    __shared__ double smem[64];
    if (sc->done) return;
    const V om = (V)omega;
    auto ld = [&](int e) { return z[e]; };
    V rz = 0;
    COL_LOOP_BEGIN
        V zc = z[c];
        if (is_red(i, j, k)) {
            Stencil<V> w;
            coef.weights(d, c, i, j, k, w);
            zc += om * nb_sum(d, w, c, i, j, k, ld) * inv_diag<V, Coef>(coef, c, w);
            z[c] = zc;
        }
        rz += r[c] * zc;
    COL_LOOP_END
    double v[1] = {(double)rz}, tot[1];
    if (grid_sum<1>(v, partials, &sc->ticket, tot, smem)) {
        if (threadIdx.x == 0 && threadIdx.y == 0) {
            const double rz_new = tot[0];
            if (mode == 0) {
                sc->rz = rz_new;
                if (!isfinite(rz_new) || !(rz_new > 0.0)) sc->done = BREAKDOWN;
            } else {
                sc->iter += 1;
                if (!isfinite(rz_new) || rz_new < 0.0 || !isfinite(sc->rr)) {
                    sc->done = BREAKDOWN;
                } else if (sc->rr <= sc->stop2) {
                    sc->done = CONVERGED;
                } else if (sc->iter >= sc->max_iter) {
                    sc->done = CAPPED;
                } else {
                    sc->beta = rz_new / sc->rz;
                    sc->rz = rz_new;
                }
            }
        }
    }
}

// red sweep of the checking entry point: z_R += w (sum w_f z_B) / D_R (no reduction)
template <typename V, typename Coef>
__global__ void __launch_bounds__(TX * TY) k_ssor_red_plain(Dims d, Coef coef, int kc,
                                                           V* __restrict__ z, double omega) {
    const V om = (V)omega;
    auto ld = [&](int e) { return z[e]; };
    COL_LOOP_BEGIN
        if (is_red(i, j, k)) {
            Stencil<V> w;
            coef.weights(d, c, i, j, k, w);
            z[c] += om * nb_sum(d, w, c, i, j, k, ld) * inv_diag<V, Coef>(coef, c, w);
        }
    COL_LOOP_END
}

template <typename V>
__global__ void k_scale_out(long long n, const V* __restrict__ z, double a, double* __restrict__ o) {
    const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t < n) o[t] = a * (double)z[t];
}

// ------------------------------------------------------------------ batched jobs
// One launch over every job of a batch; block -> job by bisection over the job table.
#define JOB_LOOP_BEGIN(J)                                                          \
    const int jb_ = job_of_block(jobs, njobs, blockIdx.x);                        \
    const JobDev& J = jobs[jb_];                                                   \
    const unsigned local_ = blockIdx.x - J.blk_off;                                \
    const Dims d = J.d;                                                            \
    const int kc = J.kc;                                                           \
    const int bx_ = local_ % J.gx, by_ = (local_ / J.gx) % J.gy, bz_ = local_ / (J.gx * J.gy); \
    const int i = bx_ * TX + threadIdx.x;                                          \
    const int j = by_ * TY + threadIdx.y;                                          \
    const int k0 = bz_ * kc;                                                       \
    const int k1 = min(d.nz, k0 + kc);

// x64 += d; d = 0; p_a = 0 (the inner solve of the next refinement step starts from zero).
__global__ void __launch_bounds__(TX * TY) k_batch_update(const JobDev* jobs, int njobs) {
    JOB_LOOP_BEGIN(J)
    if (!J.active || i >= d.nx || j >= d.ny) return;
    for (int k = k0; k < k1; ++k) {
        const int c = i + d.nx * (j + d.ny * k);
        J.x64[c] += (double)J.d32[c];
        J.d32[c] = 0.f;
        J.pa32[c] = 0.f;
    }
}

// r32 = (float)(b - A64 x64); (r.r, b.b) -> the job's scalars rr, bb.
__global__ void __launch_bounds__(TX * TY) k_batch_residual(const JobDev* jobs, int njobs) {
    __shared__ double smem[64];
    JOB_LOOP_BEGIN(J)
    if (!J.active) return;  // whole job skipped: its blocks never reach the reduction
    const CoefFaces64 coef{J.bx, J.by, J.bz, J.diag, nullptr};
    const double* x = J.x64;
    auto ld = [&](int e) { return x[e]; };
    double rr = 0.0, bb = 0.0;
    if (i < d.nx && j < d.ny)
        for (int k = k0; k < k1; ++k) {
            const int c = i + d.nx * (j + d.ny * k);
            Stencil<double> w;
            coef.weights(d, c, i, j, k, w);
            const double ax = w.D * x[c] - nb_sum(d, w, c, i, j, k, ld);
            const double bc = J.b64[c];
            const double rc = bc - ax;
            J.r32[c] = (float)rc;
            rr += rc * rc;
            bb += bc * bc;
        }
    double v[2] = {rr, bb}, tot[2];
    if (job_sum<2>(v, J.partials, &J.sc->ticket, (unsigned)J.blocks, local_, tot, smem)) {
        if (threadIdx.x == 0 && threadIdx.y == 0) {
            J.sc->rr = tot[0];
            J.sc->bb = tot[1];
        }
    }
}

// z = D^-1 r (Jacobi start of the inner FP32 PCG), rz, rr0, stop2 = tol2 rr0; an inactive job
// is marked CONVERGED so the persistent PCG skips it.
template <typename E>
__device__ __forceinline__ void batch_init_body(const JobDev& J, const Dims& d, int i, int j,
                                                int k0, int k1, const E* eta, float& rz,
                                                float& rr) {
    const CoefEta<E> coef{eta};
    if (i < d.nx && j < d.ny)
        for (int k = k0; k < k1; ++k) {
            const int c = i + d.nx * (j + d.ny * k);
            Stencil<float> w;
            coef.weights(d, c, i, j, k, w);
            const float rc = J.r32[c];
            const float zc = rc * rcp_approx(w.D);
            J.z32[c] = zc;
            J.sa32[c] = 0.f;
            J.wa32[c] = 0.f;
            rz += rc * zc;
            rr += rc * rc;
        }
}

__global__ void __launch_bounds__(TX * TY) k_batch_init(const JobDev* jobs, int njobs) {
    __shared__ double smem[64];
    JOB_LOOP_BEGIN(J)
    if (!J.active) {
        if (local_ == 0 && threadIdx.x == 0 && threadIdx.y == 0) {
            J.sc->done = CONVERGED;
            J.sc->iter = 0;
        }
        return;
    }
    float rz = 0.f, rr = 0.f;
    if (J.bf16) batch_init_body(J, d, i, j, k0, k1, J.eta16, rz, rr);
    else batch_init_body(J, d, i, j, k0, k1, J.eta32, rz, rr);
    double v[2] = {(double)rz, (double)rr}, tot[2];
    if (job_sum<2>(v, J.partials, &J.sc->ticket, (unsigned)J.blocks, local_, tot, smem)) {
        if (threadIdx.x == 0 && threadIdx.y == 0) {
            Scalars* sc = J.sc;
            sc->rz = tot[0];
            sc->rr = tot[1];
            sc->rr0 = tot[1];
            sc->beta = 0.0;
            sc->alpha = 0.0;
            sc->iter = 0;
            sc->max_iter = J.max_iter;
            sc->stop2 = J.tol2 * tot[1];
            sc->done = (tot[1] <= sc->stop2) ? CONVERGED : RUNNING;
            if (!isfinite(tot[0]) || !isfinite(tot[1])) sc->done = BREAKDOWN;
        }
    }
}

// Rows padded with `pad` ghost columns on each side (periodic x): the data at column i + pad,
// the ghosts holding the other end of the row.
template <typename T>
__global__ void k_pad_rows(Dims d, int pad, const T* __restrict__ src, T* __restrict__ dst) {
    const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t >= d.n) return;
    const int c = (int)t;
    const int i = c % d.nx, row = c / d.nx;
    const long long base = (long long)(d.nx + 2 * pad) * row + pad;
    const T v = src[c];
    dst[base + i] = v;
    if (i < pad) dst[base + i + d.nx] = v;
    if (i >= d.nx - pad) dst[base + i - d.nx] = v;
}

// ------------------------------------------------------------------ host launchers
int quad_kc(const Dims& d, int blocks_per_sm) {
    static const int sms = [] {  // (initialised once, thread-safe)
        int dev = 0, n = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) {
            cudaGetLastError();
            n = 152;
        }
        return n;
    }();
    // blocks take time ~ kc + 2 (their planes plus the two look-ahead planes of the prologue);
    // the grid takes ceil(blocks / resident blocks) of those
    const long long tiles = (long long)(d.nx / QX) * ((d.ny + QY - 1) / QY);
    const long long slots = (long long)sms * blocks_per_sm;
    long long kc = 64, best = -1;
    for (long long k = 2; k <= 64; k += 2) {
        const long long blocks = tiles * ((d.nz + k - 1) / k);
        const long long t = ((blocks + slots - 1) / slots) * (k + 2);
        // (a handle's reduction partials hold at least 4096 blocks)
        if (blocks <= 4096 && (best < 0 || t < best)) { best = t; kc = k; }
        if (k >= d.nz) break;
    }
    return (int)kc;
}

std::atomic<unsigned long long> g_kernel_launches{0};
static inline void counted(int k) { g_kernel_launches.fetch_add((unsigned long long)k, std::memory_order_relaxed); }

static inline dim3 grid_of(const Dims& d, int kc) {
    return dim3((d.nx + TX - 1) / TX, (d.ny + TY - 1) / TY, (d.nz + kc - 1) / kc);
}
static inline unsigned blocks1d(long long n) { return (unsigned)((n + 255) / 256); }

void launch_setup(const Dims& d, const double* F, double ra, double rw, double* bx, double* by,
                  double* bz, double* diag, double* dinv, double* top, double* rinv2,
                  float* eta32, __nv_bfloat16* eta16, const Apertures& ap, unsigned* bad,
                  cudaStream_t st) {
    k_setup_faces<<<blocks1d(d.n), 256, 0, st>>>(d, F, ra, rw, bx, by, bz, eta32, eta16, ap, bad);
    k_setup_diag<<<blocks1d(d.n), 256, 0, st>>>(d, F, ra, rw, bx, by, bz, diag, dinv, top, rinv2,
                                                ap);
    counted(2);
}

void launch_scale(long long n, const double* s, double a, double* b, cudaStream_t st,
                  const double* vol) {
    k_scale<<<blocks1d(n), 256, 0, st>>>(n, s, a, vol, b);
    counted(1);
}

void launch_update64(long long n, double* x, const float* dlt, cudaStream_t st) {
    k_update64<<<blocks1d(n), 256, 0, st>>>(n, x, dlt);
    counted(1);
}

void launch_fill_f32(long long n, float* p, float v, cudaStream_t st) {
    k_fill<float><<<blocks1d(n), 256, 0, st>>>(n, p, v);
    counted(1);
}

void launch_fill_bf16(long long n, __nv_bfloat16* p, float v, cudaStream_t st) {
    k_fill<__nv_bfloat16><<<blocks1d(n), 256, 0, st>>>(n, p, v);
    counted(1);
}

void launch_pad_rows_f32(const Dims& d, int pad, const float* src, float* dst, cudaStream_t st) {
    k_pad_rows<float><<<blocks1d(d.n), 256, 0, st>>>(d, pad, src, dst);
    counted(1);
}

void launch_pad_rows_bf16(const Dims& d, int pad, const __nv_bfloat16* src, __nv_bfloat16* dst,
                          cudaStream_t st) {
    k_pad_rows<__nv_bfloat16><<<blocks1d(d.n), 256, 0, st>>>(d, pad, src, dst);
    counted(1);
}

void launch_narrow_f32(long long n, const double* a, float* b, cudaStream_t st) {
    k_narrow<float><<<blocks1d(n), 256, 0, st>>>(n, a, b);
    counted(1);
}

void launch_widen_f32(long long n, const float* a, double* b, cudaStream_t st) {
    k_widen<float><<<blocks1d(n), 256, 0, st>>>(n, a, b);
    counted(1);
}

void launch_residual64(const Dims& d, int kc, const CoefFaces64& c, const double* b,
                       const double* x, double* r, Scalars* sc, double* part, cudaStream_t st) {
    k_residual64<double><<<grid_of(d, kc), dim3(TX, TY), 0, st>>>(d, c, kc, b, x, r, sc, part);
    counted(1);
}

void launch_residual64_f32(const Dims& d, int kc, const CoefFaces64& c, const double* b,
                           const double* x, float* r, Scalars* sc, double* part, cudaStream_t st) {
    k_residual64<float><<<grid_of(d, kc), dim3(TX, TY), 0, st>>>(d, c, kc, b, x, r, sc, part);
    counted(1);
}

template <typename V, typename Coef>
void launch_apply(const Dims& d, int kc, const Coef& c, const double* x, double* y,
                  cudaStream_t st) {
    k_apply<V, Coef><<<grid_of(d, kc), dim3(TX, TY), 0, st>>>(d, c, kc, x, y);
    counted(1);
}

template <typename V, typename Coef>
void launch_jacobi(const Dims& d, int kc, const Coef& c, const double* r, double* z,
                   cudaStream_t st) {
    k_jacobi<V, Coef><<<grid_of(d, kc), dim3(TX, TY), 0, st>>>(d, c, kc, r, z);
    counted(1);
}

template <typename V, typename Coef>
void launch_cg_init(const Dims& d, int kc, const Coef& c, const V* r, V* z, Scalars* sc,
                    double* part, double tol2, int rel_to_b, int max_iter, cudaStream_t st) {
    k_cg_init<V, Coef><<<grid_of(d, kc), dim3(TX, TY), 0, st>>>(d, c, kc, r, z, sc, part, tol2,
                                                                rel_to_b, max_iter);
    counted(1);
}

template <typename V, typename Coef>
void launch_cg_a(const Dims& d, int kc, const Coef& c, const V* z, const V* p_in, V* p_out,
                 Scalars* sc, double* part, cudaStream_t st) {
    if constexpr (is_coef_eta<Coef>::value) {
        if (quad_tiles_fit(d))
            launch_pdl(k_cg_a_q<EtaOf<Coef>>, quad_grid(d, quad_kc(d, QB_CG_A)), dim3(TX, TY), 0, st, d, c,
                       quad_kc(d, QB_CG_A), z, p_in,
                                                                       p_out, sc, part);
        else if (plane_tiles_fit(d))
            launch_pdl(k_cg_a_sm<EtaOf<Coef>>, grid_of(d, kc), dim3(TX, TY), 0, st, d, c, kc, z, p_in, p_out, sc, part);
        else
            launch_pdl(k_cg_a_eta<EtaOf<Coef>>, grid_of(d, kc), dim3(TX, TY), 0, st, d, c, kc, z, p_in, p_out, sc,
                                                                part);
    } else if constexpr (std::is_same<Coef, CoefFaces32>::value) {
        if (quad_tiles_fit(d))
            launch_pdl(k_cg_a_fq, quad_grid(d, quad_kc(d, QB_FACES)), dim3(TX, TY), 0, st, d, c,
                       quad_kc(d, QB_FACES), z, p_in, p_out, sc, part);
        else
            launch_pdl(k_cg_a<V, Coef>, grid_of(d, kc), dim3(TX, TY), 0, st, d, c, kc, z, p_in,
                       p_out, sc, part);
    } else
        launch_pdl(k_cg_a<V, Coef>, grid_of(d, kc), dim3(TX, TY), 0, st, d, c, kc, z, p_in, p_out, sc, part);
    counted(1);
}

template <typename V, typename Coef>
void launch_cg_b(const Dims& d, int kc, const Coef& c, const V* p, V* x, V* r, V* z,
                 Scalars* sc, double* part, cudaStream_t st) {
    if constexpr (std::is_same<Coef, CoefFaces32>::value) {
        if (quad_tiles_fit(d)) {
            launch_pdl(k_cg_b_fq, quad_grid(d, quad_kc(d, QB_FACES)), dim3(TX, TY), 0, st, d, c,
                       quad_kc(d, QB_FACES), p, x, r, z, sc, part);
            counted(1);
            return;
        }
    }
    k_cg_b<V, Coef><<<grid_of(d, kc), dim3(TX, TY), 0, st>>>(d, c, kc, p, x, r, z, sc, part);
    counted(1);
}

template <typename V, typename Coef>
void launch_ssor_init(const Dims& d, int kc, const Coef& c, const V* r, V* z, double omega,
                      Scalars* sc, double* part, double tol2, int rel_to_b, int max_iter,
                      cudaStream_t st) {
    k_ssor_first<V, Coef, V><<<grid_of(d, kc), dim3(TX, TY), 0, st>>>(d, c, kc, r, z, sc, part,
                                                                      tol2, rel_to_b, max_iter);
    k_ssor_black<V, Coef, V><<<grid_of(d, kc), dim3(TX, TY), 0, st>>>(d, c, kc, r, z, omega, sc);
    k_ssor_red<V, Coef><<<grid_of(d, kc), dim3(TX, TY), 0, st>>>(d, c, kc, r, z, omega, sc, part, 0);
    counted(3);
}

template <typename V, typename Coef>
void launch_cg_b_ssor(const Dims& d, int kc, const Coef& c, const V* p, V* x, V* r, V* z,
                      double omega, Scalars* sc, double* part, cudaStream_t st) {
    k_cg_b_ssor<V, Coef><<<grid_of(d, kc), dim3(TX, TY), 0, st>>>(d, c, kc, p, x, r, z, sc, part);
    k_ssor_black<V, Coef, V><<<grid_of(d, kc), dim3(TX, TY), 0, st>>>(d, c, kc, r, z, omega, sc);
    k_ssor_red<V, Coef><<<grid_of(d, kc), dim3(TX, TY), 0, st>>>(d, c, kc, r, z, omega, sc, part, 1);
    counted(3);
}

template <typename V, typename Coef>
void launch_ssor_apply(const Dims& d, int kc, const Coef& c, const double* r, V* zbuf,
                       double omega, double* out, cudaStream_t st) {
    k_ssor_first<V, Coef, double><<<grid_of(d, kc), dim3(TX, TY), 0, st>>>(
        d, c, kc, r, zbuf, nullptr, nullptr, 0.0, 0, 0);
    k_ssor_black<V, Coef, double><<<grid_of(d, kc), dim3(TX, TY), 0, st>>>(d, c, kc, r, zbuf,
                                                                           omega, nullptr);
    k_ssor_red_plain<V, Coef><<<grid_of(d, kc), dim3(TX, TY), 0, st>>>(d, c, kc, zbuf, omega);
    k_scale_out<V><<<blocks1d(d.n), 256, 0, st>>>(d.n, zbuf, omega * (2.0 - omega), out);
    counted(4);
}

void launch_batch_update(const JobDev* jobs, int njobs, int blocks, cudaStream_t st) {
    k_batch_update<<<blocks, dim3(TX, TY), 0, st>>>(jobs, njobs);
    counted(1);
}

void launch_batch_residual(const JobDev* jobs, int njobs, int blocks, cudaStream_t st) {
    k_batch_residual<<<blocks, dim3(TX, TY), 0, st>>>(jobs, njobs);
    counted(1);
}

void launch_batch_init(const JobDev* jobs, int njobs, int blocks, cudaStream_t st) {
    k_batch_init<<<blocks, dim3(TX, TY), 0, st>>>(jobs, njobs);
    counted(1);
}

#define INSTANTIATE(V, C)                                                                   \
    template void launch_apply<V, C>(const Dims&, int, const C&, const double*, double*,     \
                                     cudaStream_t);                                         \
    template void launch_jacobi<V, C>(const Dims&, int, const C&, const double*, double*,    \
                                      cudaStream_t);                                        \
    template void launch_cg_init<V, C>(const Dims&, int, const C&, const V*, V*, Scalars*,   \
                                       double*, double, int, int, cudaStream_t);            \
    template void launch_cg_a<V, C>(const Dims&, int, const C&, const V*, const V*, V*,     \
                                    Scalars*, double*, cudaStream_t);                       \
    template void launch_cg_b<V, C>(const Dims&, int, const C&, const V*, V*, V*, V*,       \
                                    Scalars*, double*, cudaStream_t);                       \
    template void launch_ssor_init<V, C>(const Dims&, int, const C&, const V*, V*, double,  \
                                         Scalars*, double*, double, int, int, cudaStream_t); \
    template void launch_cg_b_ssor<V, C>(const Dims&, int, const C&, const V*, V*, V*, V*,  \
                                         double, Scalars*, double*, cudaStream_t);          \
    template void launch_ssor_apply<V, C>(const Dims&, int, const C&, const double*, V*,    \
                                          double, double*, cudaStream_t);

INSTANTIATE(double, CoefFaces64)
INSTANTIATE(float, CoefEta<float>)
INSTANTIATE(float, CoefEta<__nv_bfloat16>)
INSTANTIATE(float, CoefFaces32)

}  // namespace pcg

// mg.cu -- the multigrid V-cycle preconditioner of the column-kernel PCG (see mg.h).
//
// All kernels are elementwise over the cells of one level.  The Galerkin setup runs one thread per
// coarse cell over its (up to 8) fine cells, the restriction one thread per coarse cell on the
// finest level and one per fine cell below; the prolongation + post-smoothing runs in the column
// layout of the PCG kernels (the fine one carries the (r, z) reduction, so its blocks must match
// the handle's reduction partials); the bottom levels and the coarsest run in one block.  Every
// kernel of a PCG iteration returns at once when the solve has finished.
#include <atomic>

#include "alloc.h"
#include "poisson.h"
#include "mg.h"
#include "kernels.h"
#include "plane_tile.cuh"

namespace pcg {
namespace {

constexpr int MT = 256;         // threads of the one-thread-per-coarse-cell kernels
constexpr int COARSE_T = 1024;  // threads of the coarsest-level block

inline unsigned blocks_of(long long n) { return (unsigned)((n + MT - 1) / MT); }
inline dim3 cols(const Dims& d, int kc) {
    return dim3((d.nx + TX - 1) / TX, (d.ny + TY - 1) / TY, (d.nz + kc - 1) / kc);
}
inline void counted(int k) {
    g_kernel_launches.fetch_add((unsigned long long)k, std::memory_order_relaxed);
}

// The stored operator of a coarse level, in the handle's inner precision.
template <typename V>
struct LevelCoef;
template <>
struct LevelCoef<double> {
    using type = CoefFaces64;
    __host__ __device__ static type make(const double* bx, const double* by, const double* bz, const double* dg) {
        return CoefFaces64{bx, by, bz, dg, nullptr};
    }
    static type of(const MgHier& m, int l) {
        return CoefFaces64{(const double*)m.bx[l], (const double*)m.by[l], (const double*)m.bz[l],
                           (const double*)m.diag[l], nullptr};
    }
};
template <>
struct LevelCoef<float> {
    using type = CoefFaces32;
    __host__ __device__ static type make(const float* bx, const float* by, const float* bz, const float* dg) {
        return CoefFaces32{bx, by, bz, dg};
    }
    static type of(const MgHier& m, int l) {
        return CoefFaces32{(const float*)m.bx[l], (const float*)m.by[l], (const float*)m.bz[l],
                           (const float*)m.diag[l]};
    }
};

// The policy as CoefFaces32 where it is one (the quad face kernels' launches are compiled for
// every policy but taken only for FP32 faces).
template <typename Coef>
inline CoefFaces32 faces32_of(const Coef& c) {
    if constexpr (std::is_same<Coef, CoefFaces32>::value) {
        return c;
    } else {
        (void)c;
        return CoefFaces32{};
    }
}

__device__ __forceinline__ void coarse_index(const Dims& dc, int I, int& ic, int& jc, int& kc) {
    ic = I % dc.nx;
    jc = (I / dc.nx) % dc.ny;
    kc = I / dc.sxy;
}

// A_c = P^T A P: the coarse low face is the sum of the fine low faces of the block's first layer;
// the diagonal is the sum of the block's diagonals minus twice the faces inside the block.
// Accumulated in FP64.
template <typename T, typename V>
__global__ void __launch_bounds__(MT) k_mg_galerkin(Dims df, const T* __restrict__ bx,
                                                    const T* __restrict__ by,
                                                    const T* __restrict__ bz,
                                                    const T* __restrict__ diag, Dims dc, int fx,
                                                    int fy, int fz, V* __restrict__ cbx,
                                                    V* __restrict__ cby, V* __restrict__ cbz,
                                                    V* __restrict__ cdiag) {
    const long long t = blockIdx.x * (long long)MT + threadIdx.x;
    if (t >= dc.n) return;
    const int I = (int)t;
    int ic, jc, kc;
    coarse_index(dc, I, ic, jc, kc);
    const int i0 = ic * fx, j0 = jc * fy, k0 = kc * fz;
    const int i1 = min(i0 + fx, df.nx), j1 = min(j0 + fy, df.ny), k1 = min(k0 + fz, df.nz);
    double BX = 0.0, BY = 0.0, BZ = 0.0, D = 0.0;
    for (int k = k0; k < k1; ++k)
        for (int j = j0; j < j1; ++j)
            for (int i = i0; i < i1; ++i) {
                const int c = i + df.nx * (j + df.ny * k);
                D += (double)diag[c];
                if (i == i0) BX += (double)bx[c]; else D -= 2.0 * (double)bx[c];
                if (j == j0) BY += (double)by[c]; else D -= 2.0 * (double)by[c];
                if (k == k0) BZ += (double)bz[c]; else D -= 2.0 * (double)bz[c];
            }
    cbx[I] = (V)BX;
    cby[I] = (V)BY;
    cbz[I] = (V)BZ;
    cdiag[I] = (V)D;
}

// P^T (r - A x) at coarse cell I: the residuals of its (up to 8) fine cells, added x fastest.
template <typename V, typename Coef>
__device__ __forceinline__ V restrict_at(const Dims& df, const Coef& coef, const V* r, const V* x,
                                         const Dims& dc, int fx, int fy, int fz, int I) {
    int ic, jc, kc;
    coarse_index(dc, I, ic, jc, kc);
    const int i0 = ic * fx, j0 = jc * fy, k0 = kc * fz;
    const int i1 = min(i0 + fx, df.nx), j1 = min(j0 + fy, df.ny), k1 = min(k0 + fz, df.nz);
    auto ld = [&](int e) { return x[e]; };
    V s = 0;
    for (int k = k0; k < k1; ++k)
        for (int j = j0; j < j1; ++j)
            for (int i = i0; i < i1; ++i) {
                const int c = i + df.nx * (j + df.ny * k);
                Stencil<V> w;
                coef.weights(df, c, i, j, k, w);
                s += r[c] - (w.D * x[c] - nb_sum(df, w, c, i, j, k, ld));
            }
    return s;
}

// r_c = P^T (r - A x) over the block of each coarse cell; x_c = w r_c / D_c (the coarse level's
// pre-smoothing from zero).  One thread per coarse cell: the finest level.
template <typename V, typename Coef>
__global__ void __launch_bounds__(MT) k_mg_restrict(Dims df, Coef coef, const V* __restrict__ r,
                                                    const V* __restrict__ x, Dims dc, int fx,
                                                    int fy, int fz, const V* __restrict__ cdiag,
                                                    V* __restrict__ rc, V* __restrict__ xc,
                                                    V omega, const Scalars* sc) {
    pdl_entry();
    if (sc && sc->done) return;
    const long long t = blockIdx.x * (long long)MT + threadIdx.x;
    if (t >= dc.n) return;
    const int I = (int)t;
    const V s = restrict_at(df, coef, r, x, dc, fx, fy, fz, I);
    rc[I] = s;
    xc[I] = omega * s / cdiag[I];
}

// The same with eight consecutive threads per coarse cell, one per child (bit 0 of the lane: +x,
// bit 1: +y, bit 2: +z), the children's residuals added by a fixed shuffle tree: the coarse
// levels, whose few cells would leave one thread per coarse cell walking eight stencils alone.
// (On the finest level the eight-lane pattern halves the coalescing and is slower.)
template <typename V, typename Coef>
__global__ void __launch_bounds__(MT) k_mg_restrict8(Dims df, Coef coef, const V* __restrict__ r,
                                                    const V* __restrict__ x, Dims dc, int fx,
                                                    int fy, int fz, const V* __restrict__ cdiag,
                                                    V* __restrict__ rc, V* __restrict__ xc,
                                                    V omega, const Scalars* sc) {
    pdl_entry();
    if (sc && sc->done) return;
    const long long t = blockIdx.x * (long long)MT + threadIdx.x;
    const long long I = t >> 3;
    const int q = threadIdx.x & 7;
    const int qx = q & 1, qy = (q >> 1) & 1, qz = q >> 2;
    V s = 0;
    if (I < dc.n) {
        int ic, jc, kc;
        coarse_index(dc, (int)I, ic, jc, kc);
        const int i = ic * fx + qx, j = jc * fy + qy, k = kc * fz + qz;
        if (qx < fx && qy < fy && qz < fz && i < df.nx && j < df.ny && k < df.nz) {
            const int c = i + df.nx * (j + df.ny * k);
            auto ld = [&](int e) { return x[e]; };
            Stencil<V> w;
            coef.weights(df, c, i, j, k, w);
            s = r[c] - (w.D * x[c] - nb_sum(df, w, c, i, j, k, ld));
        }
    }
    s += __shfl_xor_sync(0xffffffffu, s, 1);
    s += __shfl_xor_sync(0xffffffffu, s, 2);
    s += __shfl_xor_sync(0xffffffffu, s, 4);
    if (q == 0 && I < dc.n) {
        rc[I] = s;
        xc[I] = omega * s / cdiag[I];
    }
}

// Coarsest level, inside one block: x holds the first damped Jacobi sweep from zero; sweeps - 1
// more follow (__syncthreads between sweeps), the iterates alternating between the two
// shared-memory buffers when the level fits (at most MG_COARSE_MAX cells), else between x and y;
// the result ends in y.
template <typename V, typename Coef>
__device__ __forceinline__ void coarsest_sweeps(const Dims& d, const Coef& coef, const V* r, V* x,
                                                V* y, V omega, int sweeps,
                                                V (*buf)[MG_COARSE_MAX]) {
    const bool in_smem = d.n <= MG_COARSE_MAX;
    V* src = x;
    V* dst = y;
    if (in_smem) {
        for (int c = threadIdx.x; c < d.n; c += blockDim.x) buf[0][c] = x[c];
        __syncthreads();
        src = buf[0];
        dst = buf[1];
    }
    for (int m = 1; m < sweeps; ++m) {
        auto ld = [&](int e) { return src[e]; };
        for (int c = threadIdx.x; c < d.n; c += blockDim.x) {
            const int i = c % d.nx, j = (c / d.nx) % d.ny, k = c / d.sxy;
            Stencil<V> w;
            coef.weights(d, c, i, j, k, w);
            const V xc = src[c];
            dst[c] = xc + omega * (r[c] - (w.D * xc - nb_sum(d, w, c, i, j, k, ld))) / w.D;
        }
        __syncthreads();
        V* t = src;
        src = dst;
        dst = t;
    }
    if (src != y)
        for (int c = threadIdx.x; c < d.n; c += blockDim.x) y[c] = src[c];
}

// y = xt + w D^-1 (r - A xt) at cell c = (i, j, k), with xt = x + a e(parent) at the cell and its
// neighbours: one cell of the prolongation + post-smoothing, terms in nb_sum's order.
template <typename V, typename Coef>
__device__ __forceinline__ V smooth_at(const Dims& d, const Coef& coef, const V* r, const V* x,
                                       const V* e, const Dims& dc, int sx, int sy, int sz,
                                       V alpha, V omega, int c, int i, int j, int k) {
    const bool per = d.walls & PERIODIC_X;
    auto xt = [&](int ii, int jj, int kk) -> V {
        return x[ii + d.nx * (jj + d.ny * kk)] +
               alpha * e[(ii >> sx) + dc.nx * ((jj >> sy) + dc.ny * (kk >> sz))];
    };
    Stencil<V> w;
    coef.weights(d, c, i, j, k, w);
    V s = 0;
    if (i > 0) s += w.xm * xt(i - 1, j, k);
    else if (per) s += w.xm * xt(d.nx - 1, j, k);
    if (i + 1 < d.nx) s += w.xp * xt(i + 1, j, k);
    else if (per) s += w.xp * xt(0, j, k);
    if (j > 0) s += w.ym * xt(i, j - 1, k);
    if (j + 1 < d.ny) s += w.yp * xt(i, j + 1, k);
    if (k > 0) s += w.zm * xt(i, j, k - 1);
    if (k + 1 < d.nz) s += w.zp * xt(i, j, k + 1);
    const V xc = xt(i, j, k);
    return xc + omega * (r[c] - (w.D * xc - s)) / w.D;
}

// The bottom of the V-cycle in one block: the levels from b (whose r and pre-smoothed x the
// previous restriction wrote) to the coarsest -- restrictions down, the coarsest sweeps,
// prolongation + post-smoothing up to level b, whose y it leaves for the next finer level.  The
// level arrays are written and read by the same block between __syncthreads, so they are read
// with plain loads.
constexpr int MG_BOTTOM_LEVELS = 8;
constexpr int MG_BOTTOM_CELLS = 2048;  // largest level handled in the block

template <typename V>
struct Bottom {
    int nb;  // levels b .. b + nb - 1 (the coarsest)
    Dims d[MG_BOTTOM_LEVELS];
    int f[MG_BOTTOM_LEVELS][3];
    const V *bx[MG_BOTTOM_LEVELS], *by[MG_BOTTOM_LEVELS], *bz[MG_BOTTOM_LEVELS],
        *diag[MG_BOTTOM_LEVELS];
    V *r[MG_BOTTOM_LEVELS], *x[MG_BOTTOM_LEVELS], *y[MG_BOTTOM_LEVELS];
};

template <typename V>
__global__ void __launch_bounds__(COARSE_T) k_mg_bottom(Bottom<V> B, V omega, V alpha, int sweeps,
                                                        const Scalars* sc) {
    pdl_entry();
    __shared__ V buf[2][MG_COARSE_MAX];
    if (sc && sc->done) return;
    using LC = LevelCoef<V>;
    for (int q = 0; q + 1 < B.nb; ++q) {
        const auto cf = LC::make(B.bx[q], B.by[q], B.bz[q], B.diag[q]);
        const Dims& dc = B.d[q + 1];
        for (int I = threadIdx.x; I < dc.n; I += blockDim.x) {
            const V v = restrict_at(B.d[q], cf, (const V*)B.r[q], (const V*)B.x[q], dc, B.f[q][0],
                                    B.f[q][1], B.f[q][2], I);
            B.r[q + 1][I] = v;
            B.x[q + 1][I] = omega * v / B.diag[q + 1][I];
        }
        __syncthreads();
    }
    const int cq = B.nb - 1;
    coarsest_sweeps(B.d[cq], LC::make(B.bx[cq], B.by[cq], B.bz[cq], B.diag[cq]),
                    (const V*)B.r[cq], B.x[cq], B.y[cq], omega, sweeps, buf);
    __syncthreads();
    for (int q = B.nb - 2; q >= 0; --q) {
        const auto cf = LC::make(B.bx[q], B.by[q], B.bz[q], B.diag[q]);
        const Dims& d = B.d[q];
        for (int c = threadIdx.x; c < d.n; c += blockDim.x) {
            const int i = c % d.nx, j = (c / d.nx) % d.ny, k = c / d.sxy;
            B.y[q][c] = smooth_at(d, cf, (const V*)B.r[q], (const V*)B.x[q], (const V*)B.y[q + 1],
                                  B.d[q + 1], B.f[q][0] - 1, B.f[q][1] - 1, B.f[q][2] - 1, alpha,
                                  omega, c, i, j, k);
        }
        __syncthreads();
    }
}

// Sums (r, z) over the grid; the last block stores rz after the start (mode 0) or, inside PCG
// (mode 1), counts the iteration and sets beta or the stopping state, like the SSOR red sweep.
template <typename V>
__device__ __forceinline__ void reduce_rz(V rz, Scalars* sc, double* partials, double* smem,
                                          int mode) {
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

// Prolongation + post-smoothing: xt = x + a P e;  y = xt + w D^-1 (r - A xt).  On the fine
// level (mode >= 0) also sums (r, y) and, like the SSOR red sweep, either stores rz after the
// start (mode 0) or sets beta and the stopping state (mode 1).
template <typename V, typename Coef>
__global__ void __launch_bounds__(TX * TY) k_mg_smooth(Dims d, Coef coef, int kc,
                                                      const V* __restrict__ r,
                                                      const V* __restrict__ x,
                                                      const V* __restrict__ e, Dims dc, int sx,
                                                      int sy, int sz, V alpha, V omega,
                                                      V* __restrict__ y, Scalars* sc,
                                                      double* partials, int mode) {
    pdl_entry();
    __shared__ double smem[64];
    if (sc && sc->done) return;
    V rz = 0;
    const int i = blockIdx.x * TX + threadIdx.x;
    const int j = blockIdx.y * TY + threadIdx.y;
    const int k0 = blockIdx.z * kc;
    const int k1 = min(d.nz, k0 + kc);
    if (i < d.nx && j < d.ny)
        for (int k = k0; k < k1; ++k) {
            const int c = i + d.nx * (j + d.ny * k);
            const V yc = smooth_at(d, coef, r, x, e, dc, sx, sy, sz, alpha, omega, c, i, j, k);
            y[c] = yc;
            rz += r[c] * yc;
        }
    if (mode < 0 || !sc) return;
    reduce_rz(rz, sc, partials, smem, mode);
}

// The fine-level kernels on the rho/2 operator, marching the thread's column in z with planes
// k-1, k, k+1 in registers and the loads of the next planes issued before plane k is computed
// (the plain versions leave one plane's loads in flight per thread).  Same arithmetic, in the
// same order, as k_mg_cg_b and k_mg_smooth with CoefEta.
template <typename E>
__global__ void __launch_bounds__(TX * TY) k_mg_cg_b_eta(Dims d, CoefEta<E> coef, int kc,
                                                        const float* __restrict__ p,
                                                        float* __restrict__ x,
                                                        float* __restrict__ r,
                                                        float* __restrict__ x0, float omega,
                                                        Scalars* sc, double* partials) {
    pdl_entry();
    __shared__ double smem[64];
    if (sc->done) return;
    const float alpha = (float)sc->alpha;
    const int i = blockIdx.x * TX + threadIdx.x;
    const int j = blockIdx.y * TY + threadIdx.y;
    const int k0 = blockIdx.z * kc;
    const int k1 = min(d.nz, k0 + kc);
    float rr = 0.f;
    if (i < d.nx && j < d.ny) {
        const bool per = d.walls & PERIODIC_X;
        const bool hxm = i > 0 || per, hxp = i + 1 < d.nx || per, hym = j > 0, hyp = j + 1 < d.ny;
        const int oxm = i > 0 ? -1 : d.nx - 1, oxp = i + 1 < d.nx ? 1 : 1 - d.nx;
        auto et = [&](int e) { return eta_load(coef.eta, e); };
        int c = i + d.nx * (j + d.ny * k0);
        float pm = 0.f, em = 0.f, pp = 0.f, ep = 0.f, pq = 0.f, eq = 0.f, xn = 0.f, rn = 0.f;
        if (k0 > 0) { pm = p[c - d.sxy]; em = et(c - d.sxy); }
        float p0 = p[c], e0 = et(c), xc = x[c], rc = r[c];
        if (k0 + 1 < d.nz) { pp = p[c + d.sxy]; ep = et(c + d.sxy); }
        for (int k = k0; k < k1; ++k, c += d.sxy) {
            if (k + 1 < k1) {
                xn = x[c + d.sxy];
                rn = r[c + d.sxy];
                if (k + 2 < d.nz) { pq = p[c + 2 * d.sxy]; eq = et(c + 2 * d.sxy); }
            }
            Stencil<float> w;
            eta_stencil(d, i, j, k, e0, hxm ? et(c + oxm) : 0.f, hxp ? et(c + oxp) : 0.f,
                        hym ? et(c - d.nx) : 0.f, hyp ? et(c + d.nx) : 0.f, em, ep, w);
            float s = 0.f;
            if (hxm) s += w.xm * p[c + oxm];
            if (hxp) s += w.xp * p[c + oxp];
            if (hym) s += w.ym * p[c - d.nx];
            if (hyp) s += w.yp * p[c + d.nx];
            if (k > 0) s += w.zm * pm;
            if (k + 1 < d.nz) s += w.zp * pp;
            const float q = w.D * p0 - s;
            x[c] = xc + alpha * p0;
            const float rnew = rc - alpha * q;
            r[c] = rnew;
            x0[c] = omega * rnew / w.D;
            rr += rnew * rnew;
            pm = p0; em = e0;
            p0 = pp; e0 = ep;
            pp = pq; ep = eq;
            xc = xn; rc = rn;
        }
    }
    double v[1] = {(double)rr}, tot[1];
    if (grid_sum<1>(v, partials, &sc->ticket, tot, smem)) {
        if (threadIdx.x == 0 && threadIdx.y == 0) sc->rr = tot[0];
    }
}

template <typename E>
__global__ void __launch_bounds__(TX * TY, 5) k_mg_smooth_eta(Dims d, CoefEta<E> coef, int kc,
                                                             const float* __restrict__ r,
                                                             const float* __restrict__ x,
                                                             const float* __restrict__ e,
                                                             Dims dc, int sx, int sy, int sz,
                                                             float alpha, float omega,
                                                             float* __restrict__ y, Scalars* sc,
                                                             double* partials, int mode) {
    pdl_entry();
    __shared__ double smem[64];
    if (sc && sc->done) return;
    const int i = blockIdx.x * TX + threadIdx.x;
    const int j = blockIdx.y * TY + threadIdx.y;
    const int k0 = blockIdx.z * kc;
    const int k1 = min(d.nz, k0 + kc);
    float rz = 0.f;
    if (i < d.nx && j < d.ny) {
        const bool per = d.walls & PERIODIC_X;
        const bool hxm = i > 0 || per, hxp = i + 1 < d.nx || per, hym = j > 0, hyp = j + 1 < d.ny;
        const int oxm = i > 0 ? -1 : d.nx - 1, oxp = i + 1 < d.nx ? 1 : 1 - d.nx;
        // parents: x and y offsets of the cell's and its x/y neighbours' aggregates
        const int pc = (i >> sx) + dc.nx * (j >> sy);
        const int pxm = ((i + oxm) >> sx) + dc.nx * (j >> sy);
        const int pxp = ((i + oxp) >> sx) + dc.nx * (j >> sy);
        const int pym = (i >> sx) + dc.nx * ((hym ? j - 1 : j) >> sy);
        const int pyp = (i >> sx) + dc.nx * ((hyp ? j + 1 : j) >> sy);
        auto et = [&](int q) { return eta_load(coef.eta, q); };
        auto xt = [&](int c, int pk) { return x[c] + alpha * e[pc + pk]; };
        int c = i + d.nx * (j + d.ny * k0);
        float tm = 0.f, em = 0.f, tp = 0.f, ep = 0.f, tq = 0.f, eq = 0.f, rn = 0.f;
        if (k0 > 0) { tm = xt(c - d.sxy, dc.sxy * ((k0 - 1) >> sz)); em = et(c - d.sxy); }
        float t0 = xt(c, dc.sxy * (k0 >> sz)), e0 = et(c), rc = r[c];
        if (k0 + 1 < d.nz) { tp = xt(c + d.sxy, dc.sxy * ((k0 + 1) >> sz)); ep = et(c + d.sxy); }
        for (int k = k0; k < k1; ++k, c += d.sxy) {
            if (k + 1 < k1) {
                rn = r[c + d.sxy];
                if (k + 2 < d.nz) {
                    tq = xt(c + 2 * d.sxy, dc.sxy * ((k + 2) >> sz));
                    eq = et(c + 2 * d.sxy);
                }
            }
            const int pk = dc.sxy * (k >> sz);
            Stencil<float> w;
            eta_stencil(d, i, j, k, e0, hxm ? et(c + oxm) : 0.f, hxp ? et(c + oxp) : 0.f,
                        hym ? et(c - d.nx) : 0.f, hyp ? et(c + d.nx) : 0.f, em, ep, w);
            float s = 0.f;
            if (hxm) s += w.xm * (x[c + oxm] + alpha * e[pxm + pk]);
            if (hxp) s += w.xp * (x[c + oxp] + alpha * e[pxp + pk]);
            if (hym) s += w.ym * (x[c - d.nx] + alpha * e[pym + pk]);
            if (hyp) s += w.yp * (x[c + d.nx] + alpha * e[pyp + pk]);
            if (k > 0) s += w.zm * tm;
            if (k + 1 < d.nz) s += w.zp * tp;
            const float yc = t0 + omega * (rc - (w.D * t0 - s)) / w.D;
            y[c] = yc;
            rz += rc * yc;
            tm = t0; em = e0;
            t0 = tp; e0 = ep;
            tp = tq; ep = eq;
            rc = rn;
        }
    }
    if (mode < 0 || !sc) return;
    reduce_rz(rz, sc, partials, smem, mode);
}

// k_mg_cg_b_eta and k_mg_smooth_eta with the x and y neighbours of plane k from a shared plane
// (plane_tile.cuh): the same arithmetic in the same order.  Grids with plane_tiles_fit only.
template <typename E>
__global__ void __launch_bounds__(TX * TY) k_mg_cg_b_sm(Dims d, CoefEta<E> coef, int kc,
                                                       const float* __restrict__ p,
                                                       float* __restrict__ x,
                                                       float* __restrict__ r,
                                                       float* __restrict__ x0, float omega,
                                                       Scalars* sc, double* partials) {
    pdl_entry();
    __shared__ double smem[64];
    __shared__ float Ps[2][PT_N], Es[2][PT_N];
    if (sc->done) return;
    const float alpha = (float)sc->alpha;
    const int i = blockIdx.x * TX + threadIdx.x;
    const int j = blockIdx.y * TY + threadIdx.y;
    const int k0 = blockIdx.z * kc;
    const int k1 = min(d.nz, k0 + kc);
    const bool act = j < d.ny;
    const int ci = pt_index(threadIdx.x, threadIdx.y);
    int hx, hy;
    const bool hs = pt_halo_slot(threadIdx.x + TX * threadIdx.y, hx, hy);
    const int gx = blockIdx.x * TX + hx, gy = blockIdx.y * TY + hy;
    const bool hv = hs && gx >= 0 && gx < d.nx && gy >= 0 && gy < d.ny;
    const int hi = hs ? pt_index(hx, hy) : 0;
    const bool hxm = i > 0, hxp = i + 1 < d.nx, hym = j > 0, hyp = j + 1 < d.ny;
    auto et = [&](int e) { return eta_load(coef.eta, e); };
    int c = i + d.nx * (j + d.ny * k0);
    int h = gx + d.nx * (gy + d.ny * k0);
    float pm = 0.f, em = 0.f, p0 = 0.f, e0 = 0.f, pp = 0.f, ep = 0.f, pq = 0.f, eq = 0.f;
    float xc = 0.f, rc = 0.f, xn = 0.f, rn = 0.f;
    if (act) {
        if (k0 > 0) { pm = p[c - d.sxy]; em = et(c - d.sxy); }
        p0 = p[c];
        e0 = et(c);
        xc = x[c];
        rc = r[c];
        if (k0 + 1 < d.nz) { pp = p[c + d.sxy]; ep = et(c + d.sxy); }
    }
    float hp = 0.f, he = 0.f, hpn = 0.f, hen = 0.f;
    if (hv) { hp = p[h]; he = et(h); }
    float rr = 0.f;
    for (int k = k0; k < k1; ++k, c += d.sxy, h += d.sxy) {
        const int b = (k - k0) & 1;
        Ps[b][ci] = p0;
        Es[b][ci] = e0;
        if (hs) { Ps[b][hi] = hp; Es[b][hi] = he; }
        if (act && k + 1 < k1) {
            xn = x[c + d.sxy];
            rn = r[c + d.sxy];
            if (k + 2 < d.nz) { pq = p[c + 2 * d.sxy]; eq = et(c + 2 * d.sxy); }
        }
        if (hv && k + 1 < k1) { hpn = p[h + d.sxy]; hen = et(h + d.sxy); }
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
            x[c] = xc + alpha * p0;
            const float rnew = rc - alpha * q;
            r[c] = rnew;
            x0[c] = omega * rnew / w.D;
            rr += rnew * rnew;
        }
        pm = p0; em = e0;
        p0 = pp; e0 = ep;
        pp = pq; ep = eq;
        xc = xn; rc = rn;
        hp = hpn; he = hen;
    }
    double v[1] = {(double)rr}, tot[1];
    if (grid_sum<1>(v, partials, &sc->ticket, tot, smem)) {
        if (threadIdx.x == 0 && threadIdx.y == 0) sc->rr = tot[0];
    }
}

template <typename E>
__global__ void __launch_bounds__(TX * TY) k_mg_smooth_sm(Dims d, CoefEta<E> coef, int kc,
                                                         const float* __restrict__ r,
                                                         const float* __restrict__ x,
                                                         const float* __restrict__ e, Dims dc,
                                                         int sx, int sy, int sz, float alpha,
                                                         float omega, float* __restrict__ y,
                                                         Scalars* sc, double* partials,
                                                         int mode) {
    pdl_entry();
    __shared__ double smem[64];
    __shared__ float Ts[2][PT_N], Es[2][PT_N];
    if (sc && sc->done) return;
    const int i = blockIdx.x * TX + threadIdx.x;
    const int j = blockIdx.y * TY + threadIdx.y;
    const int k0 = blockIdx.z * kc;
    const int k1 = min(d.nz, k0 + kc);
    const bool act = j < d.ny;
    const int ci = pt_index(threadIdx.x, threadIdx.y);
    int hx, hy;
    const bool hs = pt_halo_slot(threadIdx.x + TX * threadIdx.y, hx, hy);
    const int gx = blockIdx.x * TX + hx, gy = blockIdx.y * TY + hy;
    const bool hv = hs && gx >= 0 && gx < d.nx && gy >= 0 && gy < d.ny;
    const int hi = hs ? pt_index(hx, hy) : 0;
    const bool hxm = i > 0, hxp = i + 1 < d.nx, hym = j > 0, hyp = j + 1 < d.ny;
    // parents (x and y offsets of the aggregates) of the cell and of the halo cell
    const int pc = (i >> sx) + dc.nx * (j >> sy);
    const int ph = hv ? (gx >> sx) + dc.nx * (gy >> sy) : 0;
    auto et = [&](int q) { return eta_load(coef.eta, q); };
    int c = i + d.nx * (j + d.ny * k0);
    int h = gx + d.nx * (gy + d.ny * k0);
    float tm = 0.f, em = 0.f, t0 = 0.f, e0 = 0.f, tp = 0.f, ep = 0.f, tq = 0.f, eq = 0.f;
    float rc = 0.f, rn = 0.f;
    if (act) {
        if (k0 > 0) { tm = x[c - d.sxy] + alpha * e[pc + dc.sxy * ((k0 - 1) >> sz)]; em = et(c - d.sxy); }
        t0 = x[c] + alpha * e[pc + dc.sxy * (k0 >> sz)];
        e0 = et(c);
        rc = r[c];
        if (k0 + 1 < d.nz) {
            tp = x[c + d.sxy] + alpha * e[pc + dc.sxy * ((k0 + 1) >> sz)];
            ep = et(c + d.sxy);
        }
    }
    float ht = 0.f, he = 0.f, htn = 0.f, hen = 0.f;
    if (hv) { ht = x[h] + alpha * e[ph + dc.sxy * (k0 >> sz)]; he = et(h); }
    float rz = 0.f;
    for (int k = k0; k < k1; ++k, c += d.sxy, h += d.sxy) {
        const int b = (k - k0) & 1;
        Ts[b][ci] = t0;
        Es[b][ci] = e0;
        if (hs) { Ts[b][hi] = ht; Es[b][hi] = he; }
        if (act && k + 1 < k1) {
            rn = r[c + d.sxy];
            if (k + 2 < d.nz) {
                tq = x[c + 2 * d.sxy] + alpha * e[pc + dc.sxy * ((k + 2) >> sz)];
                eq = et(c + 2 * d.sxy);
            }
        }
        if (hv && k + 1 < k1) {
            htn = x[h + d.sxy] + alpha * e[ph + dc.sxy * ((k + 1) >> sz)];
            hen = et(h + d.sxy);
        }
        __syncthreads();
        if (act) {
            const float* T = Ts[b];
            const float* Ee = Es[b];
            Stencil<float> w;
            eta_stencil(d, i, j, k, e0, hxm ? Ee[ci - 1] : 0.f, hxp ? Ee[ci + 1] : 0.f,
                        hym ? Ee[ci - PT_W] : 0.f, hyp ? Ee[ci + PT_W] : 0.f, em, ep, w);
            float s = 0.f;
            if (hxm) s += w.xm * T[ci - 1];
            if (hxp) s += w.xp * T[ci + 1];
            if (hym) s += w.ym * T[ci - PT_W];
            if (hyp) s += w.yp * T[ci + PT_W];
            if (k > 0) s += w.zm * tm;
            if (k + 1 < d.nz) s += w.zp * tp;
            const float yc = t0 + omega * (rc - (w.D * t0 - s)) / w.D;
            y[c] = yc;
            rz += rc * yc;
        }
        tm = t0; em = e0;
        t0 = tp; e0 = ep;
        tp = tq; ep = eq;
        rc = rn;
        ht = htn; he = hen;
    }
    if (mode < 0 || !sc) return;
    reduce_rz(rz, sc, partials, smem, mode);
}

// ------------------------------------------------------------------ fine passes, 2 x 2 per thread
// The fine-level passes of the V-cycle PCG on QX x QY tiles with 2 x 2 cells per thread
// (quad_march in plane_tile.cuh): the same arithmetic per cell as k_mg_cg_b_sm, the finest
// k_mg_restrict and k_mg_smooth_sm.  Grids with quad_tiles_fit only (their aggregates are 2 x 2
// in x-y).
// Stencil field of the post-smoothing: u = x + alpha e(parent) (the prolongation).
struct FieldProlong {
    const float* x;
    const float* e;
    Dims dc;
    int sz;
    float alpha;
    __device__ __forceinline__ float par(int i, int j, int k) const {
        return e[(i >> 1) + dc.nx * ((j >> 1) + dc.ny * (k >> sz))];
    }
    // raw parts: a = x, b = e(parent) (one parent for a pair, i even)
    __device__ __forceinline__ void raw(int c, int i, int j, int k, float2& a, float2& b) const {
        a = ld2(x, c);
        const float pe = par(i, j, k);
        b = make_float2(pe, pe);
    }
    __device__ __forceinline__ void raw1(int c, int i, int j, int k, float& a, float& b) const {
        a = x[c];
        b = par(i, j, k);
    }
    __device__ __forceinline__ float comb(float a, float b) const { return a + alpha * b; }
};

// Phase B of MG-PCG: x += alpha p; r -= alpha A p; x0 = w D^-1 r; (r, r).  Inputs x, r.
struct BodyCgB {
    static constexpr int NX = 2;
    const float* in[NX];
    float* x;
    float* r;
    float* x0;
    float alpha, omega;
    int nx;
    float rr = 0.f;
    __device__ __forceinline__ void cell(int c, int, int, int, const Quad& u, const Quad& q,
                                         const Quad& D, const Quad* X) {
        Quad xn, rn, zn;
#pragma unroll
        for (int a = 0; a < 2; ++a)
#pragma unroll
            for (int b = 0; b < 2; ++b) {
                xn.v[a][b] = X[0].v[a][b] + alpha * u.v[a][b];
                rn.v[a][b] = X[1].v[a][b] - alpha * q.v[a][b];
                zn.v[a][b] = omega * rn.v[a][b] / D.v[a][b];
                rr += rn.v[a][b] * rn.v[a][b];
            }
        st2(x, c, xn.v[0][0], xn.v[0][1]);
        st2(x, c + nx, xn.v[1][0], xn.v[1][1]);
        st2(r, c, rn.v[0][0], rn.v[0][1]);
        st2(r, c + nx, rn.v[1][0], rn.v[1][1]);
        st2(x0, c, zn.v[0][0], zn.v[0][1]);
        st2(x0, c + nx, zn.v[1][0], zn.v[1][1]);
    }
};

// The finest restriction: r_c = P^T (r - A x0) over each 2 x 2 x fz block (children added x
// fastest, then y, then z, as restrict_at), x_c = w r_c / D_c.  Input r.
struct BodyRestrict {
    static constexpr int NX = 1;
    const float* in[NX];
    float* rc;
    float* xc;
    const float* cdiag;
    Dims dc;
    int nz, fz;
    float omega;
    float s = 0.f;
    __device__ __forceinline__ void cell(int, int x0, int y0, int k, const Quad&, const Quad& q,
                                         const Quad&, const Quad* X) {
#pragma unroll
        for (int a = 0; a < 2; ++a)
#pragma unroll
            for (int b = 0; b < 2; ++b) s += X[0].v[a][b] - q.v[a][b];
        if (fz == 1 || (k & 1) || k + 1 == nz) {
            const int I = (x0 >> 1) + dc.nx * ((y0 >> 1) + dc.ny * (fz == 1 ? k : k >> 1));
            rc[I] = s;
            xc[I] = omega * s / cdiag[I];
            s = 0.f;
        }
    }
};

// The fine post-smoothing: y = t + w D^-1 (r - A t), t = x0 + alpha e(parent); (r, y).  Input r.
struct BodySmooth {
    static constexpr int NX = 1;
    const float* in[NX];
    float* y;
    float omega;
    int nx;
    float rz = 0.f;
    __device__ __forceinline__ void cell(int c, int, int, int, const Quad& u, const Quad& q,
                                         const Quad& D, const Quad* X) {
        Quad yn;
#pragma unroll
        for (int a = 0; a < 2; ++a)
#pragma unroll
            for (int b = 0; b < 2; ++b) {
                yn.v[a][b] = u.v[a][b] + omega * (X[0].v[a][b] - q.v[a][b]) / D.v[a][b];
                rz += X[0].v[a][b] * yn.v[a][b];
            }
        st2(y, c, yn.v[0][0], yn.v[0][1]);
        st2(y, c + nx, yn.v[1][0], yn.v[1][1]);
    }
};

template <typename E>
__global__ void __launch_bounds__(TX * TY, QB_CG_B) k_mg_cg_b_q(Dims d, CoefEta<E> coef, int kc,
                                                         const float* __restrict__ p,
                                                         float* __restrict__ x,
                                                         float* __restrict__ r,
                                                         float* __restrict__ x0, float omega,
                                                         Scalars* sc, double* partials) {
    pdl_entry();
    __shared__ double smem[64];
    if (sc->done) return;
    FieldPlain F{p};
    BodyCgB B{{x, r}, x, r, x0, (float)sc->alpha, omega, d.nx};
    quad_march(d, coef.eta, kc, F, B);
    double v[1] = {(double)B.rr}, tot[1];
    if (grid_sum<1>(v, partials, &sc->ticket, tot, smem)) {
        if (threadIdx.x == 0 && threadIdx.y == 0) sc->rr = tot[0];
    }
}

template <typename E>
__global__ void __launch_bounds__(TX * TY, QB_RESTRICT) k_mg_restrict_q(Dims d, CoefEta<E> coef, int kc,
                                                             const float* __restrict__ r,
                                                             const float* __restrict__ x, Dims dc,
                                                             int fz, const float* __restrict__ cdiag,
                                                             float* __restrict__ rc,
                                                             float* __restrict__ xc, float omega,
                                                             const Scalars* sc) {
    pdl_entry();
    if (sc && sc->done) return;
    FieldPlain F{x};
    BodyRestrict B{{r}, rc, xc, cdiag, dc, d.nz, fz, omega};
    quad_march(d, coef.eta, kc, F, B);
}

template <typename E>
__global__ void __launch_bounds__(TX * TY, QB_SMOOTH) k_mg_smooth_q(Dims d, CoefEta<E> coef, int kc,
                                                           const float* __restrict__ r,
                                                           const float* __restrict__ x,
                                                           const float* __restrict__ e, Dims dc,
                                                           int sz, float alpha, float omega,
                                                           float* __restrict__ y, Scalars* sc,
                                                           double* partials, int mode) {
    pdl_entry();
    __shared__ double smem[64];
    if (sc && sc->done) return;
    FieldProlong F{x, e, dc, sz, alpha};
    BodySmooth B{{r}, y, omega, d.nx};
    quad_march(d, coef.eta, kc, F, B);
    if (mode < 0 || !sc) return;
    reduce_rz(B.rz, sc, partials, smem, mode);
}

// The same three passes on FP32 faces (quad_march_faces): the fine level of cut-cell handles
// and the coarse levels of every FP32/BF16 hierarchy whose grid takes quad tiles.
__global__ void __launch_bounds__(TX * TY, QB_FACES) k_mg_cg_b_fq(Dims d, CoefFaces32 coef, int kc,
                                                                 const float* __restrict__ p,
                                                                 float* __restrict__ x,
                                                                 float* __restrict__ r,
                                                                 float* __restrict__ x0,
                                                                 float omega, Scalars* sc,
                                                                 double* partials) {
    pdl_entry();
    __shared__ double smem[64];
    if (sc->done) return;
    FieldPlain F{p};
    BodyCgB B{{x, r}, x, r, x0, (float)sc->alpha, omega, d.nx};
    quad_march_faces(d, coef, kc, F, B);
    double v[1] = {(double)B.rr}, tot[1];
    if (grid_sum<1>(v, partials, &sc->ticket, tot, smem)) {
        if (threadIdx.x == 0 && threadIdx.y == 0) sc->rr = tot[0];
    }
}

__global__ void __launch_bounds__(TX * TY, QB_FACES) k_mg_restrict_fq(Dims d, CoefFaces32 coef,
                                                                     int kc,
                                                                     const float* __restrict__ r,
                                                                     const float* __restrict__ x,
                                                                     Dims dc, int fz,
                                                                     const float* __restrict__ cdiag,
                                                                     float* __restrict__ rc,
                                                                     float* __restrict__ xc,
                                                                     float omega,
                                                                     const Scalars* sc) {
    pdl_entry();
    if (sc && sc->done) return;
    FieldPlain F{x};
    BodyRestrict B{{r}, rc, xc, cdiag, dc, d.nz, fz, omega};
    quad_march_faces(d, coef, kc, F, B);
}

__global__ void __launch_bounds__(TX * TY, QB_FACES) k_mg_smooth_fq(Dims d, CoefFaces32 coef,
                                                                   int kc,
                                                                   const float* __restrict__ r,
                                                                   const float* __restrict__ x,
                                                                   const float* __restrict__ e,
                                                                   Dims dc, int sz, float alpha,
                                                                   float omega,
                                                                   float* __restrict__ y,
                                                                   Scalars* sc, double* partials,
                                                                   int mode) {
    pdl_entry();
    __shared__ double smem[64];
    if (sc && sc->done) return;
    FieldProlong F{x, e, dc, sz, alpha};
    BodySmooth B{{r}, y, omega, d.nx};
    quad_march_faces(d, coef, kc, F, B);
    if (mode < 0 || !sc) return;
    reduce_rz(B.rz, sc, partials, smem, mode);
}

// Start of the preconditioned solve: x0 = w D^-1 r on the fine level; with scalars, sums r.r
// and sets them like k_cg_init (rz follows from the V-cycle's last kernel).
template <typename V, typename Coef>
__global__ void __launch_bounds__(TX * TY) k_mg_first(Dims d, Coef coef, int kc,
                                                     const V* __restrict__ r,
                                                     V* __restrict__ x0, V omega, Scalars* sc,
                                                     double* partials, double tol2, int rel_to_b,
                                                     int max_iter) {
    pdl_entry();
    __shared__ double smem[64];
    V rr = 0;
    const int i = blockIdx.x * TX + threadIdx.x;
    const int j = blockIdx.y * TY + threadIdx.y;
    const int k0 = blockIdx.z * kc;
    const int k1 = min(d.nz, k0 + kc);
    if (i < d.nx && j < d.ny)
        for (int k = k0; k < k1; ++k) {
            const int c = i + d.nx * (j + d.ny * k);
            Stencil<V> w;
            coef.weights(d, c, i, j, k, w);
            const V rc = r[c];
            x0[c] = omega * rc / w.D;
            rr += rc * rc;
        }
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

// Phase B of MG-PCG: q = A p (recomputed); x += alpha p; r -= alpha q; x0 = w D^-1 r; sums r.r.
template <typename V, typename Coef>
__global__ void __launch_bounds__(TX * TY) k_mg_cg_b(Dims d, Coef coef, int kc,
                                                    const V* __restrict__ p, V* __restrict__ x,
                                                    V* __restrict__ r, V* __restrict__ x0,
                                                    V omega, Scalars* sc, double* partials) {
    pdl_entry();
    __shared__ double smem[64];
    if (sc->done) return;
    const V alpha = (V)sc->alpha;
    auto ld = [&](int e) { return p[e]; };
    V rr = 0;
    const int i = blockIdx.x * TX + threadIdx.x;
    const int j = blockIdx.y * TY + threadIdx.y;
    const int k0 = blockIdx.z * kc;
    const int k1 = min(d.nz, k0 + kc);
    if (i < d.nx && j < d.ny)
        for (int k = k0; k < k1; ++k) {
            const int c = i + d.nx * (j + d.ny * k);
            Stencil<V> w;
            coef.weights(d, c, i, j, k, w);
            const V pc = p[c];
            const V q = w.D * pc - nb_sum(d, w, c, i, j, k, ld);
            x[c] += alpha * pc;
            const V rn = r[c] - alpha * q;
            r[c] = rn;
            x0[c] = omega * rn / w.D;
            rr += rn * rn;
        }
    double v[1] = {(double)rr}, tot[1];
    if (grid_sum<1>(v, partials, &sc->ticket, tot, smem)) {
        if (threadIdx.x == 0 && threadIdx.y == 0) sc->rr = tot[0];
    }
}

// z = V_0(r) given x[0] = w D^-1 r: restrictions down, the coarsest sweeps, prolongation +
// post-smoothing up; the fine smoothing writes z (and reduces r.z when mode >= 0).
template <typename V, typename Coef>
void vcycle(MgHier* m, const Dims& d, int kc, const Coef& coef, const V* r, V* z, Scalars* sc,
            double* part, int mode, cudaStream_t st) {
    using LC = LevelCoef<V>;
    const int L = m->nlev;
    const V om = (V)MG_OMEGA, al = (V)MG_ALPHA;
    // levels b .. L-1 run in one block (at most MG_BOTTOM_CELLS cells each, b >= 1)
    int b = L - 1;
    while (b - 1 >= 1 && m->d[b - 1].n <= MG_BOTTOM_CELLS && L - (b - 1) <= MG_BOTTOM_LEVELS) --b;
    for (int l = 0; l < b; ++l) {
        const Dims& df = m->d[l];
        const Dims& dc = m->d[l + 1];
        const int* f = m->f[l];
        bool done = false;
        if constexpr (std::is_same<V, float>::value) {
            // FP32 faces: the fine level of a cut-cell handle, or a coarse level
            if (quad_tiles_fit(df) && (l > 0 || std::is_same<Coef, CoefFaces32>::value)) {
                const CoefFaces32 cf = l > 0 ? LevelCoef<float>::of(*m, l) : faces32_of(coef);
                launch_pdl(k_mg_restrict_fq, quad_grid(df, quad_kc(df, QB_FACES)), dim3(TX, TY), 0,
                           st, df, cf, quad_kc(df, QB_FACES), l > 0 ? (const V*)m->r[l] : r,
                           (const V*)m->x[l], dc, f[2], (const V*)m->diag[l + 1],
                           (V*)m->r[l + 1], (V*)m->x[l + 1], om, sc);
                done = true;
            }
        }
        if constexpr (is_coef_eta<Coef>::value) {
            if (!done && l == 0 && quad_tiles_fit(df)) {
                launch_pdl(k_mg_restrict_q<EtaOf<Coef>>, quad_grid(df, quad_kc(df, QB_RESTRICT)),
                           dim3(TX, TY), 0, st, df, coef, quad_kc(df, QB_RESTRICT), r, (const V*)m->x[0], dc, f[2], (const V*)m->diag[1],
                    (V*)m->r[1], (V*)m->x[1], om, sc);
                done = true;
            }
        }
        if (done) {
        } else if (l == 0)
            launch_pdl(k_mg_restrict<V, Coef>, blocks_of(dc.n), MT, 0, st,
                df, coef, r, (const V*)m->x[0], dc, f[0], f[1], f[2], (const V*)m->diag[1],
                (V*)m->r[1], (V*)m->x[1], om, sc);
        else
            launch_pdl(k_mg_restrict8<V, typename LC::type>, blocks_of(8LL * dc.n), MT, 0, st,
                df, LC::of(*m, l), (const V*)m->r[l], (const V*)m->x[l], dc, f[0], f[1], f[2],
                (const V*)m->diag[l + 1], (V*)m->r[l + 1], (V*)m->x[l + 1], om, sc);
    }
    Bottom<V> B{};
    B.nb = L - b;
    for (int q = 0; q < B.nb; ++q) {
        const int l = b + q;
        B.d[q] = m->d[l];
        for (int a = 0; a < 3; ++a) B.f[q][a] = m->f[l][a];
        B.bx[q] = (const V*)m->bx[l];
        B.by[q] = (const V*)m->by[l];
        B.bz[q] = (const V*)m->bz[l];
        B.diag[q] = (const V*)m->diag[l];
        B.r[q] = (V*)m->r[l];
        B.x[q] = (V*)m->x[l];
        B.y[q] = (V*)m->y[l];
    }
    launch_pdl(k_mg_bottom<V>, 1, COARSE_T, 0, st, B, om, al, MG_COARSE_SWEEPS, sc);
    for (int l = b - 1; l >= 1; --l) {
        const int* f = m->f[l];
        if constexpr (std::is_same<V, float>::value) {
            if (quad_tiles_fit(m->d[l])) {
                launch_pdl(k_mg_smooth_fq, quad_grid(m->d[l], quad_kc(m->d[l], QB_FACES)),
                           dim3(TX, TY), 0, st, m->d[l], LevelCoef<float>::of(*m, l),
                           quad_kc(m->d[l], QB_FACES), (const V*)m->r[l], (const V*)m->x[l],
                           (const V*)m->y[l + 1], m->d[l + 1], f[2] - 1, al, om, (V*)m->y[l], sc,
                           nullptr, -1);
                continue;
            }
        }
        launch_pdl(k_mg_smooth<V, typename LC::type>, cols(m->d[l], 1), dim3(TX, TY), 0, st,
            m->d[l], LC::of(*m, l), 1, (const V*)m->r[l], (const V*)m->x[l],
            (const V*)m->y[l + 1], m->d[l + 1], f[0] - 1, f[1] - 1, f[2] - 1, al, om,
            (V*)m->y[l], sc, nullptr, -1);
    }
    const int* f = m->f[0];
    if constexpr (is_coef_eta<Coef>::value) {
        if (quad_tiles_fit(d))
            launch_pdl(k_mg_smooth_q<EtaOf<Coef>>, quad_grid(d, quad_kc(d, QB_SMOOTH)), dim3(TX, TY),
                       0, st, d, coef, quad_kc(d, QB_SMOOTH), r, (const V*)m->x[0], (const V*)m->y[1], m->d[1], f[2] - 1,
                al, om, z, sc, part, mode);
        else if (plane_tiles_fit(d))
            launch_pdl(k_mg_smooth_sm<EtaOf<Coef>>, cols(d, kc), dim3(TX, TY), 0, st,
                d, coef, kc, r, (const V*)m->x[0], (const V*)m->y[1], m->d[1], f[0] - 1,
                f[1] - 1, f[2] - 1, al, om, z, sc, part, mode);
        else
            launch_pdl(k_mg_smooth_eta<EtaOf<Coef>>, cols(d, kc), dim3(TX, TY), 0, st,
                d, coef, kc, r, (const V*)m->x[0], (const V*)m->y[1], m->d[1], f[0] - 1,
                f[1] - 1, f[2] - 1, al, om, z, sc, part, mode);
    } else if (std::is_same<Coef, CoefFaces32>::value && quad_tiles_fit(d)) {
        launch_pdl(k_mg_smooth_fq, quad_grid(d, quad_kc(d, QB_FACES)), dim3(TX, TY), 0, st, d,
                   faces32_of(coef), quad_kc(d, QB_FACES), (const float*)r,
                   (const float*)m->x[0], (const float*)m->y[1], m->d[1], f[2] - 1, (float)al,
                   (float)om, (float*)z, sc, part, mode);
    } else
        launch_pdl(k_mg_smooth<V, Coef>, cols(d, kc), dim3(TX, TY), 0, st,
            d, coef, kc, r, (const V*)m->x[0], (const V*)m->y[1], m->d[1], f[0] - 1, f[1] - 1,
            f[2] - 1, al, om, z, sc, part, mode);
    counted(2 * b + 1);
}

}  // namespace

int mg_plan(const Dims& fine, MgHier* m) {
    *m = MgHier{};
    m->d[0] = fine;
    int L = 1;
    while (L < MG_MAX_LEVELS) {
        const Dims& c = m->d[L - 1];
        const bool per = c.walls & PERIODIC_X;
        const int fx = per ? ((c.nx % 2 == 0 && c.nx >= 4) ? 2 : 1) : (c.nx > 1 ? 2 : 1);
        const int fy = c.ny > 1 ? 2 : 1, fz = c.nz > 1 ? 2 : 1;
        if (fx * fy * fz == 1) break;
        if (L > 1 && c.n <= MG_COARSE_MAX) break;
        m->f[L - 1][0] = fx;
        m->f[L - 1][1] = fy;
        m->f[L - 1][2] = fz;
        Dims nd{};
        nd.nx = (c.nx + fx - 1) / fx;
        nd.ny = (c.ny + fy - 1) / fy;
        nd.nz = (c.nz + fz - 1) / fz;
        nd.sxy = nd.nx * nd.ny;
        nd.n = nd.sxy * nd.nz;
        nd.walls = c.walls & PERIODIC_X;  // wall terms live in the Galerkin diagonal
        m->d[L++] = nd;
    }
    m->nlev = L;
    return L;
}

int mg_alloc(MgHier* m, bool dbl) {
    m->dbl = dbl;
    const size_t es = dbl ? sizeof(double) : sizeof(float);
    auto al = [&](void** p, size_t n) {
        if (lib_malloc(p, es * n) != cudaSuccess) {
            cudaGetLastError();
            *p = nullptr;
            return false;
        }
        return true;
    };
    bool ok = al(&m->x[0], (size_t)m->d[0].n);
    for (int l = 1; ok && l < m->nlev; ++l) {
        const size_t n = (size_t)m->d[l].n;
        ok = al(&m->bx[l], n) && al(&m->by[l], n) && al(&m->bz[l], n) && al(&m->diag[l], n) &&
             al(&m->r[l], n) && al(&m->x[l], n) && al(&m->y[l], n);
    }
    if (!ok) {
        mg_free(m);
        return POISSON_ENOMEM;
    }
    return POISSON_OK;
}

void mg_free(MgHier* m) {
    for (int l = 0; l < MG_MAX_LEVELS; ++l)
        for (void** p : {&m->bx[l], &m->by[l], &m->bz[l], &m->diag[l], &m->r[l], &m->x[l], &m->y[l]})
            if (*p) {
                lib_free(*p);
                *p = nullptr;
            }
}

template <typename V>
static void setup_typed(MgHier* m, const double* bx, const double* by, const double* bz,
                        const double* diag, cudaStream_t st) {
    for (int l = 0; l + 1 < m->nlev; ++l) {
        const Dims& df = m->d[l];
        const Dims& dc = m->d[l + 1];
        const int* f = m->f[l];
        V *cbx = (V*)m->bx[l + 1], *cby = (V*)m->by[l + 1], *cbz = (V*)m->bz[l + 1],
          *cd = (V*)m->diag[l + 1];
        if (l == 0)
            k_mg_galerkin<double, V><<<blocks_of(dc.n), MT, 0, st>>>(
                df, bx, by, bz, diag, dc, f[0], f[1], f[2], cbx, cby, cbz, cd);
        else
            k_mg_galerkin<V, V><<<blocks_of(dc.n), MT, 0, st>>>(
                df, (const V*)m->bx[l], (const V*)m->by[l], (const V*)m->bz[l],
                (const V*)m->diag[l], dc, f[0], f[1], f[2], cbx, cby, cbz, cd);
    }
    counted(m->nlev - 1);
}

void mg_setup(MgHier* m, const double* bx, const double* by, const double* bz,
              const double* diag, cudaStream_t st) {
    if (m->dbl)
        setup_typed<double>(m, bx, by, bz, diag, st);
    else
        setup_typed<float>(m, bx, by, bz, diag, st);
}

template <typename V, typename Coef>
void mg_init(MgHier* m, const Dims& d, int kc, const Coef& coef, const V* r, V* z, Scalars* sc,
             double* part, double tol2, int rel_to_b, int max_iter, cudaStream_t st) {
    launch_pdl(k_mg_first<V, Coef>, cols(d, kc), dim3(TX, TY), 0, st,
        d, coef, kc, r, (V*)m->x[0], (V)MG_OMEGA, sc, part, tol2, rel_to_b, max_iter);
    counted(1);
    vcycle<V, Coef>(m, d, kc, coef, r, z, sc, part, 0, st);
}

template <typename V, typename Coef>
void mg_cg_b(MgHier* m, const Dims& d, int kc, const Coef& coef, const V* p, V* x, V* r, V* z,
             Scalars* sc, double* part, cudaStream_t st) {
    if constexpr (is_coef_eta<Coef>::value) {
        if (quad_tiles_fit(d))
            launch_pdl(k_mg_cg_b_q<EtaOf<Coef>>, quad_grid(d, quad_kc(d, QB_CG_B)), dim3(TX, TY), 0,
                       st, d, coef, quad_kc(d, QB_CG_B), p, x, r, (V*)m->x[0], (V)MG_OMEGA, sc, part);
        else if (plane_tiles_fit(d))
            launch_pdl(k_mg_cg_b_sm<EtaOf<Coef>>, cols(d, kc), dim3(TX, TY), 0, st, d, coef, kc, p, x, r,
                                                               (V*)m->x[0], (V)MG_OMEGA, sc,
                                                               part);
        else
            launch_pdl(k_mg_cg_b_eta<EtaOf<Coef>>, cols(d, kc), dim3(TX, TY), 0, st, d, coef, kc, p, x, r,
                                                                (V*)m->x[0], (V)MG_OMEGA, sc,
                                                                part);
    } else if (std::is_same<Coef, CoefFaces32>::value && quad_tiles_fit(d)) {
        launch_pdl(k_mg_cg_b_fq, quad_grid(d, quad_kc(d, QB_FACES)), dim3(TX, TY), 0, st, d,
                   faces32_of(coef), quad_kc(d, QB_FACES), (const float*)p, (float*)x, (float*)r,
                   (float*)m->x[0], (float)MG_OMEGA, sc, part);
    } else
        launch_pdl(k_mg_cg_b<V, Coef>, cols(d, kc), dim3(TX, TY), 0, st, d, coef, kc, p, x, r,
                                                                (V*)m->x[0], (V)MG_OMEGA, sc,
                                                                part);
    counted(1);
    vcycle<V, Coef>(m, d, kc, coef, r, z, sc, part, 1, st);
}

template <typename V, typename Coef>
void mg_apply(MgHier* m, const Dims& d, int kc, const Coef& coef, const V* r, V* z,
              cudaStream_t st) {
    launch_pdl(k_mg_first<V, Coef>, cols(d, kc), dim3(TX, TY), 0, st,
        d, coef, kc, r, (V*)m->x[0], (V)MG_OMEGA, nullptr, nullptr, 0.0, 0, 0);
    counted(1);
    vcycle<V, Coef>(m, d, kc, coef, r, z, nullptr, nullptr, -1, st);
}

#define MG_INSTANTIATE(V, C)                                                                   \
    template void mg_init<V, C>(MgHier*, const Dims&, int, const C&, const V*, V*, Scalars*,   \
                                double*, double, int, int, cudaStream_t);                      \
    template void mg_cg_b<V, C>(MgHier*, const Dims&, int, const C&, const V*, V*, V*, V*,     \
                                Scalars*, double*, cudaStream_t);                              \
    template void mg_apply<V, C>(MgHier*, const Dims&, int, const C&, const V*, V*,            \
                                 cudaStream_t);

MG_INSTANTIATE(double, CoefFaces64)
MG_INSTANTIATE(float, CoefEta<float>)
MG_INSTANTIATE(float, CoefEta<__nv_bfloat16>)
MG_INSTANTIATE(float, CoefFaces32)

}  // namespace pcg

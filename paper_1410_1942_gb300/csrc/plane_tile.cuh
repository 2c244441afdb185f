// plane_tile.cuh -- shared-memory x-y planes of the column kernels' TX x TY tiles with a one-cell
// halo, for the fine-level z-marching kernels of the rho/2 operator (k_cg_a_sm in kernels.cu,
// k_mg_cg_b_sm and k_mg_smooth_sm in mg.cu).
//
// Those kernels march a thread's cell column in z with planes k-1, k, k+1 in registers.  Their x
// and y neighbours come from a shared plane instead of from global memory: every thread stores
// its own value of plane k, the threads with a halo slot store the ring's values (loaded a plane
// ahead), and one barrier per plane (two buffers) publishes them.  A cell then issues two or
// three global loads per plane instead of a dozen.
#pragma once

#include "internal.cuh"
#include "kernels.h"

namespace pcg {

constexpr int PT_W = TX + 2, PT_H = TY + 2, PT_N = PT_W * PT_H;

// Halo slot of the block's thread t = threadIdx.x + TX threadIdx.y: the row below the tile
// (t < TX), the row above (TX <= t < 2 TX), the column to the left (next TY) and to the right
// (next TY); (hx, hy) relative to the tile's first cell.  false: the thread has no slot.
__device__ __forceinline__ bool pt_halo_slot(int t, int& hx, int& hy) {
    if (t < TX) { hx = t; hy = -1; return true; }
    if (t < 2 * TX) { hx = t - TX; hy = TY; return true; }
    if (t < 2 * TX + TY) { hx = -1; hy = t - 2 * TX; return true; }
    if (t < 2 * TX + 2 * TY) { hx = TX; hy = t - 2 * TX - TY; return true; }
    hx = hy = 0;
    return false;
}

// Index in the shared plane of the tile cell (x, y), x in [-1, TX], y in [-1, TY].
__device__ __forceinline__ int pt_index(int x, int y) { return (y + 1) * PT_W + x + 1; }

// Whether the staged kernels serve a grid: whole tiles along x (every x neighbour of an active
// cell is in its tile or its halo) and no periodic wrap.
inline bool plane_tiles_fit(const Dims& d) { return d.nx % TX == 0 && !(d.walls & PERIODIC_X); }

// ------------------------------------------------------------------ 2x2 cells per thread
// The quad kernels (k_cg_a_q in kernels.cu; k_mg_cg_b_q, k_mg_restrict_q, k_mg_smooth_q in
// mg.cu) march QX x QY tiles of a plane with TX x TY threads, each thread owning the 2 x 2 cells
// (2 tx + {0, 1}, 2 ty + {0, 1}) of every plane of its z-chunk: loads and stores of a row pair are
// float2, the face between two cells of a thread is formed once for both, and the z face between
// planes k and k+1 is carried to plane k+1.  Rounding is that of the single-cell kernels (a face
// is rcp(eta_a + eta_b), and the addition commutes).  Shared planes have a row stride of QS floats
// and the tile's first cell at column 2, so a thread's row pair is 8-byte aligned.
constexpr int QX = 2 * TX, QY = 2 * TY, QS = QX + 4, QN = QS * (QY + 2);

// Index in a quad shared plane of the tile cell (x, y), x in [-1, QX], y in [-1, QY].
__device__ __forceinline__ int q_index(int x, int y) { return (y + 1) * QS + x + 2; }

// Halo slot of thread t = threadIdx.x + TX threadIdx.y: a pair of the row below the tile
// (t < TX: cells x = 2t, 2t + 1, y = -1), a pair of the row above (next TX: y = QY), one cell of
// the column to the left (next QY: x = -1) or to the right (next QY: x = QX).
__device__ __forceinline__ int q_halo_slot(int t, int& hx, int& hy) {
    if (t < TX) { hx = 2 * t; hy = -1; return 2; }
    if (t < 2 * TX) { hx = 2 * (t - TX); hy = QY; return 2; }
    if (t < 2 * TX + QY) { hx = -1; hy = t - 2 * TX; return 1; }
    if (t < 2 * TX + 2 * QY) { hx = QX; hy = t - 2 * TX - QY; return 1; }
    hx = hy = 0;
    return 0;
}

// Whether the quad kernels serve a grid: whole tiles along x and whole row pairs (and, for the
// V-cycle's passes, aggregates of 2 x 2 cells in x-y, which these imply, periodic x included).
inline bool quad_tiles_fit(const Dims& d) { return d.nx % QX == 0 && d.ny % 2 == 0; }

// z-chunk of the quad kernels: even (a coarse plane of the restriction never straddles two
// chunks), at most 64 planes, chosen for the fewest block-waves (blocks_per_sm resident) times
// the planes a block walks.
int quad_kc(const Dims& d, int blocks_per_sm);

inline dim3 quad_grid(const Dims& d, int kc) {
    return dim3(d.nx / QX, (d.ny + QY - 1) / QY, (d.nz + kc - 1) / kc);
}

template <typename E>
__device__ __forceinline__ float2 eta_load2(const E* p, int c);
template <>
__device__ __forceinline__ float2 eta_load2<float>(const float* p, int c) {
    return __ldg(reinterpret_cast<const float2*>(p + c));
}
template <>
__device__ __forceinline__ float2 eta_load2<__nv_bfloat16>(const __nv_bfloat16* p, int c) {
    return __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(p + c));
}

__device__ __forceinline__ float2 ld2(const float* p, int c) {
    return *reinterpret_cast<const float2*>(p + c);
}
__device__ __forceinline__ void st2(float* p, int c, float a, float b) {
    *reinterpret_cast<float2*>(p + c) = make_float2(a, b);
}

// One plane of a thread's 2 x 2 cells: values [r][q] at (x0 + q, y0 + r).
struct Quad {
    float v[2][2];
};

// A u and the diagonal D on the thread's 2 x 2 cells of plane k of the rho/2 operator.  u, e:
// the cells' values and rho/2 on plane k; um, up: u on planes k - 1 and k + 1; ep: rho/2 on plane
// k + 1; U, Es: the shared planes of u and rho/2 (k), si = q_index of cell (0, 0); fzd: in, the z
// faces below plane k (used when k > 0), out, the faces above it.  xlo/xhi/ylo/yhi: the block's
// outer x/y neighbours exist (else a wall or nothing, as `walls` says).  Per cell the weights,
// the diagonal and the neighbour sum are formed as in eta_stencil / the single-cell kernels.
__device__ __forceinline__ void quad_apply(const Dims& d, int k, bool xlo, bool xhi, bool ylo,
                                           bool yhi, const Quad& u, const Quad& e, const Quad& um,
                                           const Quad& up, const Quad& ep, const float* U,
                                           const float* Es, int si, Quad& fzd, Quad& q, Quad& D) {
    const float2 ub = *reinterpret_cast<const float2*>(U + si - QS);
    const float2 ua = *reinterpret_cast<const float2*>(U + si + 2 * QS);
    const float2 eb = *reinterpret_cast<const float2*>(Es + si - QS);
    const float2 ea = *reinterpret_cast<const float2*>(Es + si + 2 * QS);
    const float ul[2] = {U[si - 1], U[si + QS - 1]}, ur[2] = {U[si + 2], U[si + QS + 2]};
    const float el[2] = {Es[si - 1], Es[si + QS - 1]}, er[2] = {Es[si + 2], Es[si + QS + 2]};
    const float ubq[2] = {ub.x, ub.y}, uaq[2] = {ua.x, ua.y};
    const float ebq[2] = {eb.x, eb.y}, eaq[2] = {ea.x, ea.y};
    const bool zlo = k > 0, top = k + 1 == d.nz;
    // the y faces between the thread's two rows
    const float fym[2] = {rcp_approx(e.v[0][0] + e.v[1][0]), rcp_approx(e.v[0][1] + e.v[1][1])};
#pragma unroll
    for (int r = 0; r < 2; ++r) {
        const float fxm = rcp_approx(e.v[r][0] + e.v[r][1]);  // between the row's two cells
#pragma unroll
        for (int c = 0; c < 2; ++c) {
            const float ec = e.v[r][c];
            const float ew = rcp_approx(ec);
            float xm, xp, ym, yp;
            bool hxm, hxp, hym, hyp;
            if (c == 0) {
                hxm = xlo;
                xm = xlo ? rcp_approx(ec + el[r]) : ((d.walls & 1) ? ew : 0.f);
                hxp = true;
                xp = fxm;
            } else {
                hxm = true;
                xm = fxm;
                hxp = xhi;
                xp = xhi ? rcp_approx(ec + er[r]) : ((d.walls & 2) ? ew : 0.f);
            }
            if (r == 0) {
                hym = ylo;
                ym = ylo ? rcp_approx(ec + ebq[c]) : ((d.walls & 4) ? ew : 0.f);
                hyp = true;
                yp = fym[c];
            } else {
                hym = true;
                ym = fym[c];
                hyp = yhi;
                yp = yhi ? rcp_approx(ec + eaq[c]) : ((d.walls & 8) ? ew : 0.f);
            }
            const float zm = zlo ? fzd.v[r][c] : ((d.walls & 16) ? ew : 0.f);
            const float fzu = rcp_approx(ec + ep.v[r][c]);
            const float wzp = top ? ew : fzu;
            const float zp = top ? 0.f : wzp;
            fzd.v[r][c] = fzu;
            D.v[r][c] = xm + xp + ym + yp + zm + wzp;
            const float uxm = c == 0 ? ul[r] : u.v[r][0];
            const float uxp = c == 0 ? u.v[r][1] : ur[r];
            const float uym = r == 0 ? ubq[c] : u.v[0][c];
            const float uyp = r == 0 ? u.v[1][c] : uaq[c];
            float s = 0.f;
            if (hxm) s += xm * uxm;
            if (hxp) s += xp * uxp;
            if (hym) s += ym * uym;
            if (hyp) s += yp * uyp;
            if (zlo) s += zm * um.v[r][c];
            if (!top) s += zp * up.v[r][c];
            q.v[r][c] = D.v[r][c] * u.v[r][c] - s;
        }
    }
}


// Planes of look-ahead of the quad kernels' loads: the stencil field and rho/2 are loaded
// QUAD_DEPTH planes ahead of the plane being computed, the per-cell inputs and the halo
// QUAD_DEPTH - 1 planes ahead.
// resident blocks per SM of each quad kernel (its register budget)
constexpr int QB_CG_A = 3, QB_CG_B = 3, QB_RESTRICT = 3, QB_SMOOTH = 3;
// ... and of the quad kernels on FP32 faces
constexpr int QB_FACES = 2;
constexpr int QUAD_DEPTH = 2;

// Stencil fields of the quad kernels: u = v, and u = a + beta b (CG phase A: p = z + beta p).
// A field is loaded in up to two raw parts, a and b (raw(), raw1()), and formed by comb()
// only when its plane is next needed, so that the arithmetic does not wait for loads still in
// flight: the own cells of a plane loaded two planes ahead are formed after the next plane's
// barrier, the halo when it is stored.  FieldPlain: u = a; FieldSum: u = a + beta b.
struct FieldPlain {
    const float* v;
    __device__ __forceinline__ void raw(int c, int, int, int, float2& a, float2& b) const {
        a = ld2(v, c);
        b = make_float2(0.f, 0.f);
    }
    __device__ __forceinline__ void raw1(int c, int, int, int, float& a, float& b) const {
        a = v[c];
        b = 0.f;
    }
    __device__ __forceinline__ float comb(float a, float) const { return a; }
};
struct FieldSum {
    const float* a;
    const float* b;
    float beta;
    __device__ __forceinline__ void raw(int c, int, int, int, float2& p, float2& q) const {
        p = ld2(a, c);
        q = ld2(b, c);
    }
    __device__ __forceinline__ void raw1(int c, int, int, int, float& p, float& q) const {
        p = a[c];
        q = b[c];
    }
    __device__ __forceinline__ float comb(float p, float q) const { return p + beta * q; }
};

// u of the thread's 2 x 2 cells from its raw parts A, B
template <typename Field>
__device__ __forceinline__ void quad_comb(const Field& F, Quad& A, const Quad& B) {
#pragma unroll
    for (int r = 0; r < 2; ++r)
#pragma unroll
        for (int q = 0; q < 2; ++q) A.v[r][q] = F.comb(A.v[r][q], B.v[r][q]);
}

// The quad kernels' march over one block's tile and z-chunk.  F gives the stencil field u at a
// cell pair (float2) or one cell; Body has NX per-cell inputs in[] (loaded as row pairs) and
// cell(c, x0, y0, k, u, A u, D, inputs) for the thread's 2 x 2 cells of plane k.  The block's
// threads publish plane k (their own cells and the halo) in a shared plane, one barrier per plane
// (two buffers); planes k - 1 and k + 1 of the own cells stay in registers.
template <typename E, typename Field, typename Body>
__device__ __forceinline__ void quad_march(const Dims& d, const E* eta, int kc, const Field& F,
                                           Body& B) {
    constexpr int D = QUAD_DEPTH;
    constexpr int NX = Body::NX > 0 ? Body::NX : 1;
    __shared__ __align__(16) float Us[2][QN];
    __shared__ __align__(16) float Ess[2][QN];
    const int x0 = blockIdx.x * QX + 2 * threadIdx.x, y0 = blockIdx.y * QY + 2 * threadIdx.y;
    const int k0 = blockIdx.z * kc;
    const int k1 = min(d.nz, k0 + kc);
    const bool act = y0 < d.ny;
    const int si = q_index(2 * threadIdx.x, 2 * threadIdx.y);
    int hx, hy;
    const int hk = q_halo_slot(threadIdx.x + TX * threadIdx.y, hx, hy);
    // periodic x: the halo columns hold the other end of their rows
    const bool per = d.walls & PERIODIC_X;
    int gx = blockIdx.x * QX + hx;
    if (per && hk == 1) gx = (gx + d.nx) % d.nx;
    const int gy = blockIdx.y * QY + hy;
    const bool hv = hk && gx >= 0 && gx < d.nx && gy >= 0 && gy < d.ny;
    const int hi = hk ? q_index(hx, hy) : 0;
    const bool xlo = x0 > 0 || per, xhi = x0 + 2 < d.nx || per, ylo = y0 > 0, yhi = y0 + 2 < d.ny;
    static_assert(QUAD_DEPTH == 2, "the deferred field forming assumes two planes of look-ahead");
    // the field's raw parts (U, Ub) and rho/2 of the own cells of plane k
    auto ldq = [&](Quad& U, Quad& Ub, Quad& Et, int e, int k) {
        float2 a, b, a1, b1;
        F.raw(e, x0, y0, k, a, b);
        F.raw(e + d.nx, x0, y0 + 1, k, a1, b1);
        const float2 ea = eta_load2(eta, e), eb = eta_load2(eta, e + d.nx);
        U.v[0][0] = a.x; U.v[0][1] = a.y; U.v[1][0] = a1.x; U.v[1][1] = a1.y;
        Ub.v[0][0] = b.x; Ub.v[0][1] = b.y; Ub.v[1][0] = b1.x; Ub.v[1][1] = b1.y;
        Et.v[0][0] = ea.x; Et.v[0][1] = ea.y; Et.v[1][0] = eb.x; Et.v[1][1] = eb.y;
    };
    auto ldx = [&](Quad (&X)[NX][D], int t, int e) {
#pragma unroll
        for (int q = 0; q < Body::NX; ++q) {
            const float2 a = ld2(B.in[q], e), b = ld2(B.in[q], e + d.nx);
            X[q][t].v[0][0] = a.x; X[q][t].v[0][1] = a.y;
            X[q][t].v[1][0] = b.x; X[q][t].v[1][1] = b.y;
        }
    };
    // the halo cell's raw parts (hu, hb) and rho/2
    auto ldh = [&](float2& hu, float2& hb, float2& he, int e, int k) {
        if (hk == 2) {
            F.raw(e, gx, gy, k, hu, hb);
            he = eta_load2(eta, e);
        } else {
            F.raw1(e, gx, gy, k, hu.x, hb.x);
            he.x = eta_load(eta, e);
        }
    };
    int c = x0 + d.nx * (y0 + d.ny * k0);
    int h = gx + d.nx * (gy + d.ny * k0);
    // U[s], Et[s]: planes k - 1 + s (s = 0 .. D + 1), U[D + 1] raw (its second part in Ub) and
    // U[D] raw until formed after the barrier (its second part in Ubq); X[.][t], HU/HB/HE[t]:
    // planes k + t (the halo raw until stored)
    Quad U[D + 2], Et[D + 2], X[NX][D], fzd{}, Ub{}, Ubq{};
    float2 HU[D], HB[D], HE[D];
    bool pend = false;  // U[D] is raw
#pragma unroll
    for (int s2 = 0; s2 < D + 2; ++s2) { U[s2] = Quad{}; Et[s2] = Quad{}; }
#pragma unroll
    for (int t = 0; t < D; ++t) {
        HU[t] = make_float2(0.f, 0.f);
        HB[t] = HU[t];
        HE[t] = HU[t];
#pragma unroll
        for (int q = 0; q < NX; ++q) X[q][t] = Quad{};
    }
    if (act) {
#pragma unroll
        for (int s2 = 0; s2 <= D; ++s2) {
            const int m = k0 - 1 + s2;
            if (m >= 0 && m < d.nz && m <= k1) {
                Quad b2;
                ldq(U[s2], b2, Et[s2], c + (s2 - 1) * d.sxy, m);
                quad_comb(F, U[s2], b2);
            }
        }
#pragma unroll
        for (int t = 0; t + 1 < D; ++t)
            if (k0 + t < k1) ldx(X, t, c + t * d.sxy);
        if (k0 > 0)
#pragma unroll
            for (int r = 0; r < 2; ++r)
#pragma unroll
                for (int q = 0; q < 2; ++q) fzd.v[r][q] = rcp_approx(Et[1].v[r][q] + Et[0].v[r][q]);
    }
    if (hv)
#pragma unroll
        for (int t = 0; t + 1 < D; ++t)
            if (k0 + t < k1) ldh(HU[t], HB[t], HE[t], h + t * d.sxy, k0 + t);
    for (int k = k0; k < k1; ++k, c += d.sxy, h += d.sxy) {
        const int b = (k - k0) & 1;
        float* Up = Us[b];
        float* Es = Ess[b];
        st2(Up, si, U[1].v[0][0], U[1].v[0][1]);
        st2(Up, si + QS, U[1].v[1][0], U[1].v[1][1]);
        st2(Es, si, Et[1].v[0][0], Et[1].v[0][1]);
        st2(Es, si + QS, Et[1].v[1][0], Et[1].v[1][1]);
        if (hk == 2) {
            st2(Up, hi, F.comb(HU[0].x, HB[0].x), F.comb(HU[0].y, HB[0].y));
            st2(Es, hi, HE[0].x, HE[0].y);
        } else if (hk == 1) {
            Up[hi] = F.comb(HU[0].x, HB[0].x);
            Es[hi] = HE[0].x;
        }
        bool loaded = false;
        if (act) {
            if (k + D <= k1 && k + D < d.nz) {
                ldq(U[D + 1], Ub, Et[D + 1], c + D * d.sxy, k + D);
                loaded = true;
            }
            if (k + D - 1 < k1) ldx(X, D - 1, c + (D - 1) * d.sxy);
        }
        if (hv && k + D - 1 < k1)
            ldh(HU[D - 1], HB[D - 1], HE[D - 1], h + (D - 1) * d.sxy, k + D - 1);
        __syncthreads();
        if (act) {
            if (pend) quad_comb(F, U[D], Ubq);  // plane k + 1, loaded an iteration ago
            Quad q, Dg, Xc[NX];
#pragma unroll
            for (int t = 0; t < NX; ++t) Xc[t] = X[t][0];
            quad_apply(d, k, xlo, xhi, ylo, yhi, U[1], Et[1], U[0], U[2], Et[2], Up, Es, si, fzd,
                       q, Dg);
            B.cell(c, x0, y0, k, U[1], q, Dg, Xc);
        }
#pragma unroll
        for (int s2 = 0; s2 < D + 1; ++s2) { U[s2] = U[s2 + 1]; Et[s2] = Et[s2 + 1]; }
        Ubq = Ub;
        pend = loaded;
#pragma unroll
        for (int t = 0; t + 1 < D; ++t) {
            HU[t] = HU[t + 1];
            HB[t] = HB[t + 1];
            HE[t] = HE[t + 1];
#pragma unroll
            for (int q = 0; q < NX; ++q) X[q][t] = X[q][t + 1];
        }
    }
}


// quad_march on an operator stored as FP32 faces (CoefFaces32: cut-cell handles and the V-cycle's
// coarse levels).  Per cell: xm = bx[c], xp = bx[c + 1] (0 past the last cell), ym = by[c],
// yp = by[c + nx], zm = bz[c], zp = bz[c + sxy], D = diag[c], as CoefFaces32::weights, and the
// neighbour sum in nb_sum's order.  Shared planes: u with the one-cell halo, bx with the column
// right of the tile, by with the row above it; bz and diag stay in registers (bz of plane k + 1 is
// plane k's zp: loaded two planes ahead, the other coefficients one plane ahead).
template <typename Field, typename Body>
__device__ __forceinline__ void quad_march_faces(const Dims& d, const CoefFaces32& cf, int kc,
                                                 const Field& F, Body& B) {
    constexpr int NX = Body::NX > 0 ? Body::NX : 1;
    __shared__ __align__(16) float Us[2][QN];
    __shared__ __align__(16) float Bxs[2][QN];
    __shared__ __align__(16) float Bys[2][QN];
    const int x0 = blockIdx.x * QX + 2 * threadIdx.x, y0 = blockIdx.y * QY + 2 * threadIdx.y;
    const int k0 = blockIdx.z * kc;
    const int k1 = min(d.nz, k0 + kc);
    const bool act = y0 < d.ny;
    const int si = q_index(2 * threadIdx.x, 2 * threadIdx.y);
    int hx, hy;
    const int hk = q_halo_slot(threadIdx.x + TX * threadIdx.y, hx, hy);
    // periodic x: the halo columns hold the other end of their rows
    const bool per = d.walls & PERIODIC_X;
    int gx = blockIdx.x * QX + hx;
    if (per && hk == 1) gx = (gx + d.nx) % d.nx;
    const int gy = blockIdx.y * QY + hy;
    const bool hv = hk && gx >= 0 && gx < d.nx && gy >= 0 && gy < d.ny;
    const int hi = hk ? q_index(hx, hy) : 0;
    const bool hbx = hk == 1 && hx == QX;  // the slot's cell is right of the tile: its bx
    const bool hby = hk == 2 && hy == QY;  // above the tile: its by (a pair)
    const bool xlo = x0 > 0 || per, xhi = x0 + 2 < d.nx || per, ylo = y0 > 0, yhi = y0 + 2 < d.ny;
    auto quad_ld = [&](const float* a, int e, Quad& Q) {
        const float2 p = ld2(a, e), q = ld2(a, e + d.nx);
        Q.v[0][0] = p.x; Q.v[0][1] = p.y; Q.v[1][0] = q.x; Q.v[1][1] = q.y;
    };
    // the field's raw parts of the own cells (U, Ub) and of the halo cell (hu, hb); formed later
    // (see quad_march)
    auto ldu = [&](Quad& U, Quad& Ub, int e, int k) {
        float2 a, b, a1, b1;
        F.raw(e, x0, y0, k, a, b);
        F.raw(e + d.nx, x0, y0 + 1, k, a1, b1);
        U.v[0][0] = a.x; U.v[0][1] = a.y; U.v[1][0] = a1.x; U.v[1][1] = a1.y;
        Ub.v[0][0] = b.x; Ub.v[0][1] = b.y; Ub.v[1][0] = b1.x; Ub.v[1][1] = b1.y;
    };
    auto ldh = [&](float2& hu, float2& hb, float2& hc, int e, int k) {
        if (hk == 2) {
            F.raw(e, gx, gy, k, hu, hb);
            if (hby) hc = ld2(cf.by, e);
        } else {
            F.raw1(e, gx, gy, k, hu.x, hb.x);
            if (hbx) hc.x = cf.bx[e];
        }
    };
    int c = x0 + d.nx * (y0 + d.ny * k0);
    int h = gx + d.nx * (gy + d.ny * k0);
    // U[s]: planes k - 1 + s; BZ[s]: planes k + s; BX, BY, DG, X, HU, HC: planes k, k + 1
    Quad U[4], BZ[3], BX[2], BY[2], DG[2], X[NX][2], Ub{}, Ubq{};
    bool pend = false;  // U[2] is raw (its second part in Ubq)
#pragma unroll
    for (int s2 = 0; s2 < 4; ++s2) U[s2] = Quad{};
#pragma unroll
    for (int s2 = 0; s2 < 3; ++s2) BZ[s2] = Quad{};
#pragma unroll
    for (int t = 0; t < 2; ++t) {
        BX[t] = Quad{}; BY[t] = Quad{}; DG[t] = Quad{};
#pragma unroll
        for (int q = 0; q < NX; ++q) X[q][t] = Quad{};
    }
    float2 HU[2] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f)}, HC[2] = {HU[0], HU[1]};
    float2 HB[2] = {HU[0], HU[1]};
    if (act) {
        Quad b2;
        if (k0 > 0) {
            ldu(U[0], b2, c - d.sxy, k0 - 1);
            quad_comb(F, U[0], b2);
        }
        ldu(U[1], b2, c, k0);
        quad_comb(F, U[1], b2);
        if (k0 + 1 < d.nz) {
            ldu(U[2], b2, c + d.sxy, k0 + 1);
            quad_comb(F, U[2], b2);
            quad_ld(cf.bz, c + d.sxy, BZ[1]);
        }
        quad_ld(cf.bz, c, BZ[0]);
        quad_ld(cf.bx, c, BX[0]);
        quad_ld(cf.by, c, BY[0]);
        quad_ld(cf.diag, c, DG[0]);
#pragma unroll
        for (int q = 0; q < Body::NX; ++q) quad_ld(B.in[q], c, X[q][0]);
    }
    if (hv) ldh(HU[0], HB[0], HC[0], h, k0);
    for (int k = k0; k < k1; ++k, c += d.sxy, h += d.sxy) {
        const int b = (k - k0) & 1;
        float* Up = Us[b];
        float* Bx = Bxs[b];
        float* By = Bys[b];
        st2(Up, si, U[1].v[0][0], U[1].v[0][1]);
        st2(Up, si + QS, U[1].v[1][0], U[1].v[1][1]);
        st2(Bx, si, BX[0].v[0][0], BX[0].v[0][1]);
        st2(Bx, si + QS, BX[0].v[1][0], BX[0].v[1][1]);
        st2(By, si, BY[0].v[0][0], BY[0].v[0][1]);
        st2(By, si + QS, BY[0].v[1][0], BY[0].v[1][1]);
        if (hk == 2) {
            st2(Up, hi, F.comb(HU[0].x, HB[0].x), F.comb(HU[0].y, HB[0].y));
            if (hby) st2(By, hi, HC[0].x, HC[0].y);
        } else if (hk == 1) {
            Up[hi] = F.comb(HU[0].x, HB[0].x);
            if (hbx) Bx[hi] = HC[0].x;
        }
        bool loaded = false;
        if (act) {
            if (k + 2 <= k1 && k + 2 < d.nz) {
                ldu(U[3], Ub, c + 2 * d.sxy, k + 2);
                quad_ld(cf.bz, c + 2 * d.sxy, BZ[2]);
                loaded = true;
            }
            if (k + 1 < k1) {
                quad_ld(cf.bx, c + d.sxy, BX[1]);
                quad_ld(cf.by, c + d.sxy, BY[1]);
                quad_ld(cf.diag, c + d.sxy, DG[1]);
#pragma unroll
                for (int q = 0; q < Body::NX; ++q) quad_ld(B.in[q], c + d.sxy, X[q][1]);
            }
        }
        if (hv && k + 1 < k1) ldh(HU[1], HB[1], HC[1], h + d.sxy, k + 1);
        __syncthreads();
        if (act) {
            if (pend) quad_comb(F, U[2], Ubq);  // plane k + 1, loaded an iteration ago
            const bool zlo = k > 0, top = k + 1 == d.nz;
            const float2 ub = *reinterpret_cast<const float2*>(Up + si - QS);
            const float2 ua = *reinterpret_cast<const float2*>(Up + si + 2 * QS);
            const float2 bya = *reinterpret_cast<const float2*>(By + si + 2 * QS);
            const float ul[2] = {Up[si - 1], Up[si + QS - 1]}, ur[2] = {Up[si + 2], Up[si + QS + 2]};
            const float bxr[2] = {Bx[si + 2], Bx[si + QS + 2]};
            const float ubq[2] = {ub.x, ub.y}, uaq[2] = {ua.x, ua.y}, byq[2] = {bya.x, bya.y};
            Quad q, Dg, Xc[NX];
#pragma unroll
            for (int r = 0; r < 2; ++r)
#pragma unroll
                for (int cc = 0; cc < 2; ++cc) {
                    const float xm = BX[0].v[r][cc];
                    const float xp = cc == 0 ? BX[0].v[r][1] : (xhi ? bxr[r] : 0.f);
                    const float ym = BY[0].v[r][cc];
                    const float yp = r == 0 ? BY[0].v[1][cc] : (yhi ? byq[cc] : 0.f);
                    const float zm = BZ[0].v[r][cc];
                    const float zp = top ? 0.f : BZ[1].v[r][cc];
                    const bool hxm = cc == 0 ? xlo : true, hxp = cc == 0 ? true : xhi;
                    const bool hym = r == 0 ? ylo : true, hyp = r == 0 ? true : yhi;
                    const float uxm = cc == 0 ? ul[r] : U[1].v[r][0];
                    const float uxp = cc == 0 ? U[1].v[r][1] : ur[r];
                    const float uym = r == 0 ? ubq[cc] : U[1].v[0][cc];
                    const float uyp = r == 0 ? U[1].v[1][cc] : uaq[cc];
                    float s = 0.f;
                    if (hxm) s += xm * uxm;
                    if (hxp) s += xp * uxp;
                    if (hym) s += ym * uym;
                    if (hyp) s += yp * uyp;
                    if (zlo) s += zm * U[0].v[r][cc];
                    if (!top) s += zp * U[2].v[r][cc];
                    Dg.v[r][cc] = DG[0].v[r][cc];
                    q.v[r][cc] = Dg.v[r][cc] * U[1].v[r][cc] - s;
                }
#pragma unroll
            for (int t = 0; t < NX; ++t) Xc[t] = X[t][0];
            B.cell(c, x0, y0, k, U[1], q, Dg, Xc);
        }
#pragma unroll
        for (int s2 = 0; s2 < 3; ++s2) U[s2] = U[s2 + 1];
        Ubq = Ub;
        pend = loaded;
        BZ[0] = BZ[1];
        BZ[1] = BZ[2];
        BX[0] = BX[1];
        BY[0] = BY[1];
        DG[0] = DG[1];
#pragma unroll
        for (int t = 0; t < NX; ++t) X[t][0] = X[t][1];
        HU[0] = HU[1];
        HB[0] = HB[1];
        HC[0] = HC[1];
    }
}

}  // namespace pcg

// march.cu -- the FP32 CG passes as 2.5-D plane-marching kernels with TMA-staged x-y planes.
//
// A CTA of 32 x TYT threads owns an x-y tile of W x HT cells (W = 32 CX, HT = TYT CY; each
// thread owns a CX x CY block of cells) and walks a chunk of z-planes.  Each plane of the inputs
// that need neighbours (p, or z and p_old; and rho/2) is copied into a ring of NS shared-memory
// stages by one TMA box load with a one-cell halo in y and an aligned halo in x (the box starts
// at x0 - 4 for FP32 and x0 - 8 for BF16 so its first coordinate stays on a 16-byte boundary);
// the z-neighbours of a cell are the previous / next plane's centre values kept in registers.
// One mbarrier per stage counts the transaction bytes; every wait is bounded.
//
//   phase A:  p = z + beta p_old, q = A p, sum p.q     (reads z, p_old, eta; writes p)
//   phase B:  q = A p, x += alpha p, r -= alpha q, z = D^{-1} r, sums r.z, r.r
//                                                        (reads p, eta, x, r; writes x, r, z)
//
// Faces are formed once per thread and shared by the cells of its block (x and y), and the face
// between planes k and k+1 is reused as the lower face of plane k+1.  The arithmetic is the
// column kernels' (kernels.cu): face 1/(eta_c + eta_n), top term 1/eta_c, D = xm + xp + ym + yp +
// zm + (zp or top), q = D p_c - sum_n w_n p_n.
#include "internal.cuh"
#include "kernels.h"
#include "march.h"
#include "tma.cuh"

#include <cudaTypedefs.h>

#include <algorithm>
#include <atomic>
#include <mutex>

namespace pcg {

constexpr int NS = 4;  // shared-memory stages (planes) in the ring

__host__ __device__ constexpr int align128(int b) { return (b + 127) & ~127; }

template <typename E>
struct EtaX {
    static constexpr int OFF = 16 / (int)sizeof(E);  // 16 bytes of halo in x
};

template <int CX, int CY, int TYT, typename E>
struct Geo {
    static constexpr int W = 32 * CX;               // tile width (cells)
    static constexpr int HT = CY * TYT;             // tile height (cells)
    static constexpr int VOFF = 4;                  // FP32 halo in x
    static constexpr int VW = W + 2 * VOFF;
    static constexpr int EOFF = EtaX<E>::OFF;
    static constexpr int EW = W + 2 * EOFF;
    static constexpr int H = HT + 2;
    static constexpr int VB = VW * H * 4;
    static constexpr int EB = EW * H * (int)sizeof(E);
    static constexpr int CB = W * HT * 4;
    // phase A stage: z | p_old | eta
    static constexpr int A_Z = 0, A_P = align128(VB), A_E = A_P + align128(VB);
    static constexpr int A_STAGE = A_E + align128(EB);
    static constexpr int A_TX = 2 * VB + EB;
    // phase B stage: p | eta | x | r
    static constexpr int B_P = 0, B_E = align128(VB), B_X = B_E + align128(EB);
    static constexpr int B_R = B_X + align128(CB);
    static constexpr int B_STAGE = B_R + align128(CB);
    static constexpr int B_TX_HALO = VB + EB;  // planes k0-1 and k1: p, eta only
    static constexpr int B_TX = VB + EB + 2 * CB;
};

// CX consecutive values of a shared-memory row (CX = 1 or 2), widened to float.
template <int CX>
__device__ __forceinline__ void ld_row(const float* p, float (&v)[CX]) {
    if constexpr (CX == 2) {
        const float2 t = *reinterpret_cast<const float2*>(p);
        v[0] = t.x;
        v[1] = t.y;
    } else {
        v[0] = *p;
    }
}
template <int CX>
__device__ __forceinline__ void ld_row(const __nv_bfloat16* p, float (&v)[CX]) {
    if constexpr (CX == 2) {
        const __nv_bfloat162 t = *reinterpret_cast<const __nv_bfloat162*>(p);
        v[0] = __low2float(t);
        v[1] = __high2float(t);
    } else {
        v[0] = __bfloat162float(*p);
    }
}
__device__ __forceinline__ float ld1(const float* p) { return *p; }
__device__ __forceinline__ float ld1(const __nv_bfloat16* p) { return __bfloat162float(*p); }

template <int CX>
__device__ __forceinline__ void st_row(float* g, const float (&v)[CX]) {
    if constexpr (CX == 2)
        *reinterpret_cast<float2*>(g) = make_float2(v[0], v[1]);
    else
        *g = v[0];
}

// Gives up on a failed wait: records the timeout, then (thread 0) waits, bounded, for the
// stages still in flight so no copy lands in shared memory after the CTA has gone.
__device__ __forceinline__ void march_abort(Scalars* sc, uint64_t* bars, int waited, int issued,
                                            int tid) {
    if (tid == 0) {
        atomicExch(&sc->done, (int)TIMEDOUT);
        for (int q = waited; q < issued; ++q) (void)mbar_wait(&bars[q % NS], (q / NS) & 1);
        __threadfence();
    }
    __syncthreads();
}

// The stencil of one plane for the CX x CY block of a thread.
//   cen: centre values of plane k (registers); vxm/vxp/vym/vyp: the block's neighbour strips in
//   plane k; vm/vp: centre values of planes k-1 and k+1; e*: the same for eta; wzl: face to
//   plane k-1 (0 on the floor).  Returns q = A v and the diagonal per cell, and moves wzl to the
//   face between k and k+1 (0 at the top layer, whose Dirichlet term goes into D).
template <int CX, int CY>
__device__ __forceinline__ void stencil(const Dims& d, int i0, int j0, int k,
                                        const float (&cen)[CY][CX], const float (&vxm)[CY],
                                        const float (&vxp)[CY], const float (&vym)[CX],
                                        const float (&vyp)[CX], const float (&vm)[CY][CX],
                                        const float (&vp)[CY][CX], const float (&ec)[CY][CX],
                                        const float (&exm)[CY], const float (&exq)[CY],
                                        const float (&eym)[CX], const float (&eyp)[CX],
                                        const float (&ep)[CY][CX], float (&wzl)[CY][CX],
                                        float (&q)[CY][CX], float (&D)[CY][CX]) {
    const bool top = (k + 1 == d.nz);
    // x faces of each row: fx[a][b] couples cells b-1 and b (b = 0: the -x neighbour)
    float fx[CY][CX + 1];
#pragma unroll
    for (int a = 0; a < CY; ++a) {
        fx[a][0] = (i0 > 0) ? rcp_approx(ec[a][0] + exm[a]) : 0.f;
#pragma unroll
        for (int b = 1; b < CX; ++b)
            fx[a][b] = (i0 + b < d.nx) ? rcp_approx(ec[a][b - 1] + ec[a][b]) : 0.f;
        fx[a][CX] = (i0 + CX < d.nx) ? rcp_approx(ec[a][CX - 1] + exq[a]) : 0.f;
    }
    float fy[CY + 1][CX];
#pragma unroll
    for (int b = 0; b < CX; ++b) {
        fy[0][b] = (j0 > 0) ? rcp_approx(ec[0][b] + eym[b]) : 0.f;
#pragma unroll
        for (int a = 1; a < CY; ++a)
            fy[a][b] = (j0 + a < d.ny) ? rcp_approx(ec[a - 1][b] + ec[a][b]) : 0.f;
        fy[CY][b] = (j0 + CY < d.ny) ? rcp_approx(ec[CY - 1][b] + eyp[b]) : 0.f;
    }
#pragma unroll
    for (int a = 0; a < CY; ++a)
#pragma unroll
        for (int b = 0; b < CX; ++b) {
            const float wzt = top ? rcp_approx(ec[a][b]) : rcp_approx(ec[a][b] + ep[a][b]);
            const float wzp = top ? 0.f : wzt;
            const float wxm = fx[a][b], wxp = fx[a][b + 1];
            const float wym = fy[a][b], wyp = fy[a + 1][b];
            D[a][b] = wxm + wxp + wym + wyp + wzl[a][b] + wzt;
            const float pxm = (b == 0) ? vxm[a] : cen[a][b > 0 ? b - 1 : 0];
            const float pxp = (b == CX - 1) ? vxp[a] : cen[a][b < CX - 1 ? b + 1 : b];
            const float pym = (a == 0) ? vym[b] : cen[a > 0 ? a - 1 : 0][b];
            const float pyp = (a == CY - 1) ? vyp[b] : cen[a < CY - 1 ? a + 1 : a][b];
            float s = wxm * pxm;
            s += wxp * pxp;
            s += wym * pym;
            s += wyp * pyp;
            s += wzl[a][b] * vm[a][b];
            s += wzp * vp[a][b];
            q[a][b] = D[a][b] * cen[a][b] - s;
            wzl[a][b] = wzp;
        }
}

// Loads the four halo strips around a thread's CX x CY block from one plane tile.
template <int CX, int CY, typename T>
__device__ __forceinline__ void load_halo(const T* t, int pitch, int r0, int c0, float (&xm)[CY],
                                          float (&xp)[CY], float (&ym)[CX], float (&yp)[CX]) {
#pragma unroll
    for (int a = 0; a < CY; ++a) {
        xm[a] = ld1(t + (r0 + a) * pitch + c0 - 1);
        xp[a] = ld1(t + (r0 + a) * pitch + c0 + CX);
    }
    ld_row<CX>(t + (r0 - 1) * pitch + c0, ym);
    ld_row<CX>(t + (r0 + CY) * pitch + c0, yp);
}

template <int CX, int CY, typename T>
__device__ __forceinline__ void load_centre(const T* t, int pitch, int r0, int c0,
                                            float (&cen)[CY][CX]) {
#pragma unroll
    for (int a = 0; a < CY; ++a) ld_row<CX>(t + (r0 + a) * pitch + c0, cen[a]);
}

template <int CX, int CY, int TYT, typename E>
__global__ void __launch_bounds__(32 * TYT) k_march_a(Dims d, int kchunk,
                                                     const __grid_constant__ CUtensorMap mz,
                                                     const __grid_constant__ CUtensorMap mp,
                                                     const __grid_constant__ CUtensorMap me,
                                                     float* __restrict__ p_out, Scalars* sc,
                                                     double* partials) {
    using G = Geo<CX, CY, TYT, E>;
    extern __shared__ __align__(128) unsigned char sm[];
    __shared__ __align__(8) uint64_t bars[NS];
    __shared__ double red[64];
    if (sc->done) return;
    const int tx = threadIdx.x, ty = threadIdx.y, tid = tx + 32 * ty;
    const int x0 = blockIdx.x * G::W, y0 = blockIdx.y * G::HT;
    const int k0 = blockIdx.z * kchunk, k1 = min(d.nz, k0 + kchunk);
    const int nplanes = k1 - k0 + 2;  // k0-1 .. k1
    const float beta = (float)sc->beta;

    if (tid == 0) {
        for (int s = 0; s < NS; ++s) mbar_init(&bars[s], 1);
        fence_mbar_init();
    }
    __syncthreads();
    auto issue = [&](int q) {
        const int s = q % NS, kk = k0 - 1 + q;
        unsigned char* st = sm + s * G::A_STAGE;
        mbar_arrive_expect_tx(&bars[s], G::A_TX);
        tma_load_3d(st + G::A_Z, &mz, &bars[s], x0 - G::VOFF, y0 - 1, kk);
        tma_load_3d(st + G::A_P, &mp, &bars[s], x0 - G::VOFF, y0 - 1, kk);
        tma_load_3d(st + G::A_E, &me, &bars[s], x0 - G::EOFF, y0 - 1, kk);
    };
    if (tid == 0)
        for (int q = 0; q < NS && q < nplanes; ++q) issue(q);
    int issued = min(NS, nplanes);

    const int r0 = 1 + CY * ty, cv = G::VOFF + CX * tx, ce = G::EOFF + CX * tx;
    const int i0 = x0 + CX * tx, j0 = y0 + CY * ty;
    auto Zs = [&](int q) { return (const float*)(sm + (q % NS) * G::A_STAGE + G::A_Z); };
    auto Ps = [&](int q) { return (const float*)(sm + (q % NS) * G::A_STAGE + G::A_P); };
    auto Es = [&](int q) { return (const E*)(sm + (q % NS) * G::A_STAGE + G::A_E); };
    // p = z + beta p_old of a centre block
    auto centre_pn = [&](int q, float (&o)[CY][CX]) {
        float zz[CY][CX], pp[CY][CX];
        load_centre<CX, CY>(Zs(q), G::VW, r0, cv, zz);
        load_centre<CX, CY>(Ps(q), G::VW, r0, cv, pp);
#pragma unroll
        for (int a = 0; a < CY; ++a)
#pragma unroll
            for (int b = 0; b < CX; ++b) o[a][b] = zz[a][b] + beta * pp[a][b];
    };

    bool ok = mbar_wait(&bars[0], 0);
    ok = ok && mbar_wait(&bars[1], 0);
    float vm[CY][CX], vc[CY][CX], em[CY][CX], ec[CY][CX], wzl[CY][CX];
    centre_pn(0, vm);
    centre_pn(1, vc);
    load_centre<CX, CY>(Es(0), G::EW, r0, ce, em);
    load_centre<CX, CY>(Es(1), G::EW, r0, ce, ec);
#pragma unroll
    for (int a = 0; a < CY; ++a)
#pragma unroll
        for (int b = 0; b < CX; ++b) wzl[a][b] = (k0 > 0) ? rcp_approx(ec[a][b] + em[a][b]) : 0.f;
    float acc = 0.f;
    int waited = 2;
    bool failed = false;
    for (int k = k0; k < k1; ++k) {
        const int q = k - k0 + 1;
        ok = ok && mbar_wait(&bars[(q + 1) % NS], ((q + 1) / NS) & 1);
        if (__syncthreads_or(!ok)) {  // also: every thread is done with plane q-1
            failed = true;
            break;
        }
        waited = q + 2;
        if (tid == 0 && q - 1 + NS < nplanes) issue(q - 1 + NS);
        if (q - 1 + NS < nplanes) issued = q + NS;
        float vp[CY][CX], ep[CY][CX];
        centre_pn(q + 1, vp);
        load_centre<CX, CY>(Es(q + 1), G::EW, r0, ce, ep);
        // neighbour strips of p = z + beta p_old in plane q
        float zxm[CY], zxp[CY], zym[CX], zyp[CX];
        float pxm[CY], pxp[CY], pym[CX], pyp[CX];
        load_halo<CX, CY>(Zs(q), G::VW, r0, cv, zxm, zxp, zym, zyp);
        load_halo<CX, CY>(Ps(q), G::VW, r0, cv, pxm, pxp, pym, pyp);
        float vxm[CY], vxp[CY], vym[CX], vyp[CX];
#pragma unroll
        for (int a = 0; a < CY; ++a) {
            vxm[a] = zxm[a] + beta * pxm[a];
            vxp[a] = zxp[a] + beta * pxp[a];
        }
#pragma unroll
        for (int b = 0; b < CX; ++b) {
            vym[b] = zym[b] + beta * pym[b];
            vyp[b] = zyp[b] + beta * pyp[b];
        }
        float exm[CY], exp_[CY], eym[CX], eyp[CX];
        load_halo<CX, CY>(Es(q), G::EW, r0, ce, exm, exp_, eym, eyp);
        float qv[CY][CX], D[CY][CX];
        stencil<CX, CY>(d, i0, j0, k, vc, vxm, vxp, vym, vyp, vm, vp, ec, exm, exp_, eym, eyp, ep,
                        wzl, qv, D);
        if (i0 < d.nx) {
#pragma unroll
            for (int a = 0; a < CY; ++a) {
                if (j0 + a < d.ny) {
#pragma unroll
                    for (int b = 0; b < CX; ++b) acc += vc[a][b] * qv[a][b];
                    st_row<CX>(p_out + (size_t)i0 + (size_t)d.nx * (j0 + a + (size_t)d.ny * k), vc[a]);
                }
            }
        }
#pragma unroll
        for (int a = 0; a < CY; ++a)
#pragma unroll
            for (int b = 0; b < CX; ++b) {
                vm[a][b] = vc[a][b];
                vc[a][b] = vp[a][b];
                ec[a][b] = ep[a][b];
            }
    }
    if (failed) march_abort(sc, bars, waited, issued, tid);
    double v[1] = {(double)acc}, tot[1];
    if (grid_sum<1>(v, partials, &sc->ticket, tot, red)) {
        if (tid == 0 && sc->done == RUNNING) {
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

template <int CX, int CY, int TYT, typename E>
__global__ void __launch_bounds__(32 * TYT) k_march_b(Dims d, int kchunk,
                                                     const __grid_constant__ CUtensorMap mp,
                                                     const __grid_constant__ CUtensorMap me,
                                                     const __grid_constant__ CUtensorMap mx,
                                                     const __grid_constant__ CUtensorMap mr,
                                                     float* __restrict__ x, float* __restrict__ r,
                                                     float* __restrict__ z, Scalars* sc,
                                                     double* partials) {
    using G = Geo<CX, CY, TYT, E>;
    extern __shared__ __align__(128) unsigned char sm[];
    __shared__ __align__(8) uint64_t bars[NS];
    __shared__ double red[64];
    if (sc->done) return;
    const int tx = threadIdx.x, ty = threadIdx.y, tid = tx + 32 * ty;
    const int x0 = blockIdx.x * G::W, y0 = blockIdx.y * G::HT;
    const int k0 = blockIdx.z * kchunk, k1 = min(d.nz, k0 + kchunk);
    const int nplanes = k1 - k0 + 2;
    const float alpha = (float)sc->alpha;

    if (tid == 0) {
        for (int s = 0; s < NS; ++s) mbar_init(&bars[s], 1);
        fence_mbar_init();
    }
    __syncthreads();
    auto issue = [&](int q) {
        const int s = q % NS, kk = k0 - 1 + q;
        unsigned char* st = sm + s * G::B_STAGE;
        const bool centre = (q > 0) && (q < nplanes - 1);
        mbar_arrive_expect_tx(&bars[s], centre ? G::B_TX : G::B_TX_HALO);
        tma_load_3d(st + G::B_P, &mp, &bars[s], x0 - G::VOFF, y0 - 1, kk);
        tma_load_3d(st + G::B_E, &me, &bars[s], x0 - G::EOFF, y0 - 1, kk);
        if (centre) {
            tma_load_3d(st + G::B_X, &mx, &bars[s], x0, y0, kk);
            tma_load_3d(st + G::B_R, &mr, &bars[s], x0, y0, kk);
        }
    };
    if (tid == 0)
        for (int q = 0; q < NS && q < nplanes; ++q) issue(q);
    int issued = min(NS, nplanes);

    const int r0 = 1 + CY * ty, cv = G::VOFF + CX * tx, ce = G::EOFF + CX * tx;
    const int cc = CX * tx;  // column in the centre boxes
    const int i0 = x0 + CX * tx, j0 = y0 + CY * ty;
    auto Ps = [&](int q) { return (const float*)(sm + (q % NS) * G::B_STAGE + G::B_P); };
    auto Es = [&](int q) { return (const E*)(sm + (q % NS) * G::B_STAGE + G::B_E); };
    auto Xs = [&](int q) { return (const float*)(sm + (q % NS) * G::B_STAGE + G::B_X); };
    auto Rs = [&](int q) { return (const float*)(sm + (q % NS) * G::B_STAGE + G::B_R); };

    bool ok = mbar_wait(&bars[0], 0);
    ok = ok && mbar_wait(&bars[1], 0);
    float vm[CY][CX], vc[CY][CX], em[CY][CX], ec[CY][CX], wzl[CY][CX];
    load_centre<CX, CY>(Ps(0), G::VW, r0, cv, vm);
    load_centre<CX, CY>(Ps(1), G::VW, r0, cv, vc);
    load_centre<CX, CY>(Es(0), G::EW, r0, ce, em);
    load_centre<CX, CY>(Es(1), G::EW, r0, ce, ec);
#pragma unroll
    for (int a = 0; a < CY; ++a)
#pragma unroll
        for (int b = 0; b < CX; ++b) wzl[a][b] = (k0 > 0) ? rcp_approx(ec[a][b] + em[a][b]) : 0.f;
    float arz = 0.f, arr = 0.f;
    int waited = 2;
    bool failed = false;
    for (int k = k0; k < k1; ++k) {
        const int q = k - k0 + 1;
        ok = ok && mbar_wait(&bars[(q + 1) % NS], ((q + 1) / NS) & 1);
        if (__syncthreads_or(!ok)) {
            failed = true;
            break;
        }
        waited = q + 2;
        if (tid == 0 && q - 1 + NS < nplanes) issue(q - 1 + NS);
        if (q - 1 + NS < nplanes) issued = q + NS;
        float vp[CY][CX], ep[CY][CX];
        load_centre<CX, CY>(Ps(q + 1), G::VW, r0, cv, vp);
        load_centre<CX, CY>(Es(q + 1), G::EW, r0, ce, ep);
        float vxm[CY], vxp[CY], vym[CX], vyp[CX];
        load_halo<CX, CY>(Ps(q), G::VW, r0, cv, vxm, vxp, vym, vyp);
        float exm[CY], exp_[CY], eym[CX], eyp[CX];
        load_halo<CX, CY>(Es(q), G::EW, r0, ce, exm, exp_, eym, eyp);
        float qv[CY][CX], D[CY][CX];
        stencil<CX, CY>(d, i0, j0, k, vc, vxm, vxp, vym, vyp, vm, vp, ec, exm, exp_, eym, eyp, ep,
                        wzl, qv, D);
        float xo[CY][CX], ro[CY][CX];
        load_centre<CX, CY>(Xs(q), G::W, CY * ty, cc, xo);
        load_centre<CX, CY>(Rs(q), G::W, CY * ty, cc, ro);
        if (i0 < d.nx) {
#pragma unroll
            for (int a = 0; a < CY; ++a) {
                if (j0 + a < d.ny) {
                    float xn[CX], rn[CX], zn[CX];
#pragma unroll
                    for (int b = 0; b < CX; ++b) {
                        xn[b] = xo[a][b] + alpha * vc[a][b];
                        rn[b] = ro[a][b] - alpha * qv[a][b];
                        zn[b] = rn[b] * rcp_approx(D[a][b]);
                        arz += rn[b] * zn[b];
                        arr += rn[b] * rn[b];
                    }
                    const size_t c = (size_t)i0 + (size_t)d.nx * (j0 + a + (size_t)d.ny * k);
                    st_row<CX>(x + c, xn);
                    st_row<CX>(r + c, rn);
                    st_row<CX>(z + c, zn);
                }
            }
        }
#pragma unroll
        for (int a = 0; a < CY; ++a)
#pragma unroll
            for (int b = 0; b < CX; ++b) {
                vm[a][b] = vc[a][b];
                vc[a][b] = vp[a][b];
                ec[a][b] = ep[a][b];
            }
    }
    if (failed) march_abort(sc, bars, waited, issued, tid);
    double v[2] = {(double)arz, (double)arr}, tot[2];
    if (grid_sum<2>(v, partials, &sc->ticket, tot, red)) {
        if (tid == 0 && sc->done == RUNNING) {
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

// ------------------------------------------------------------------ host side
static PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                             &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
        else
            cudaGetLastError();
    });
    return fn;
}

static bool encode3d(CUtensorMap* m, const void* base, CUtensorMapDataType dt, int esz,
                     const Dims& d, int bx, int by) {
    auto fn = encode_fn();
    if (!fn) return false;
    cuuint64_t dims[3] = {(cuuint64_t)d.nx, (cuuint64_t)d.ny, (cuuint64_t)d.nz};
    cuuint64_t strides[2] = {(cuuint64_t)d.nx * esz, (cuuint64_t)d.nx * d.ny * esz};
    cuuint32_t box[3] = {(cuuint32_t)bx, (cuuint32_t)by, 1};
    cuuint32_t es[3] = {1, 1, 1};
    return fn(m, dt, 3, const_cast<void*>(base), dims, strides, box, es,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
              CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

bool march_supported(const Dims& d) {
    // global strides must be multiples of 16 bytes for FP32 and BF16 rows
    return (d.nx % 8) == 0 && encode_fn() != nullptr;
}

// ------------------------------------------------------------------ variant table
// A variant is (CX, CY, TYT); its tile is 32 CX wide and CY TYT high.
struct VariantOps {
    int cx, cy, tyt;
    int smem_a32, smem_b32, smem_a16, smem_b16;
    const void *ka32, *kb32, *ka16, *kb16;
};

template <int CX, int CY, int TYT>
static VariantOps make_ops() {
    using G32 = Geo<CX, CY, TYT, float>;
    using G16 = Geo<CX, CY, TYT, __nv_bfloat16>;
    return VariantOps{CX, CY, TYT,
                      NS * G32::A_STAGE, NS * G32::B_STAGE, NS * G16::A_STAGE, NS * G16::B_STAGE,
                      (const void*)k_march_a<CX, CY, TYT, float>,
                      (const void*)k_march_b<CX, CY, TYT, float>,
                      (const void*)k_march_a<CX, CY, TYT, __nv_bfloat16>,
                      (const void*)k_march_b<CX, CY, TYT, __nv_bfloat16>};
}

static const VariantOps* variants(int* count) {
    static const VariantOps table[] = {
        make_ops<1, 1, 4>(), make_ops<1, 1, 8>(), make_ops<1, 1, 16>(),
        make_ops<2, 2, 2>(), make_ops<2, 2, 4>(), make_ops<2, 2, 8>(),
        make_ops<2, 1, 8>(), make_ops<1, 2, 8>(),
    };
    static std::once_flag once;
    std::call_once(once, [] {
        for (const auto& v : table) {
            cudaFuncSetAttribute(v.ka32, cudaFuncAttributeMaxDynamicSharedMemorySize, v.smem_a32);
            cudaFuncSetAttribute(v.kb32, cudaFuncAttributeMaxDynamicSharedMemorySize, v.smem_b32);
            cudaFuncSetAttribute(v.ka16, cudaFuncAttributeMaxDynamicSharedMemorySize, v.smem_a16);
            cudaFuncSetAttribute(v.kb16, cudaFuncAttributeMaxDynamicSharedMemorySize, v.smem_b16);
        }
        cudaGetLastError();
    });
    *count = (int)(sizeof(table) / sizeof(table[0]));
    return table;
}

int march_variant_count() {
    int n;
    variants(&n);
    return n;
}

MarchVariant march_variant(int id) {
    int n;
    const VariantOps* t = variants(&n);
    const VariantOps& v = t[id < 0 || id >= n ? 0 : id];
    return MarchVariant{id, v.cx, v.cy, v.tyt, 32 * v.cx, v.cy * v.tyt};
}

int march_find_variant(int cx, int cy, int tyt) {
    int n;
    const VariantOps* t = variants(&n);
    for (int q = 0; q < n; ++q)
        if (t[q].cx == cx && t[q].cy == cy && t[q].tyt == tyt) return q;
    return -1;
}

bool march_maps(MarchMaps* mm, const Dims& d, int variant, const float* z, const float* pa,
                const float* pb, const void* eta, bool bf16, const float* x, const float* r) {
    const MarchVariant v = march_variant(variant);
    const int eoff = bf16 ? 8 : 4;
    const CUtensorMapDataType f32 = CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
    const CUtensorMapDataType edt = bf16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : f32;
    bool ok = true;
    ok = ok && encode3d(&mm->z, z, f32, 4, d, v.width + 8, v.height + 2);
    ok = ok && encode3d(&mm->pa, pa, f32, 4, d, v.width + 8, v.height + 2);
    ok = ok && encode3d(&mm->pb, pb, f32, 4, d, v.width + 8, v.height + 2);
    ok = ok && encode3d(&mm->eta, eta, edt, bf16 ? 2 : 4, d, v.width + 2 * eoff, v.height + 2);
    ok = ok && encode3d(&mm->x, x, f32, 4, d, v.width, v.height);
    ok = ok && encode3d(&mm->r, r, f32, 4, d, v.width, v.height);
    mm->variant = variant;
    mm->bf16 = bf16;
    return ok;
}

size_t march_blocks(const Dims& d, int variant, int kchunk) {
    const MarchVariant v = march_variant(variant);
    return (size_t)((d.nx + v.width - 1) / v.width) * ((d.ny + v.height - 1) / v.height) *
           ((d.nz + kchunk - 1) / kchunk);
}

size_t march_max_blocks(const Dims& d, int kchunk) {
    size_t m = 0;
    for (int q = 0; q < march_variant_count(); ++q) m = std::max(m, march_blocks(d, q, kchunk));
    return m;
}

int march_occupancy(int variant, bool bf16) {
    int n;
    const VariantOps& v = variants(&n)[variant];
    int oa = 0, ob = 0;
    const int threads = 32 * v.tyt;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&oa, bf16 ? v.ka16 : v.ka32, threads,
                                                      bf16 ? v.smem_a16 : v.smem_a32) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&ob, bf16 ? v.kb16 : v.kb32, threads,
                                                      bf16 ? v.smem_b16 : v.smem_b32) != cudaSuccess) {
        cudaGetLastError();
        return 1;
    }
    return std::max(1, std::min(oa, ob));
}

template <int CX, int CY, int TYT, typename E>
static void launch_ab(const Dims& d, int kchunk, const MarchMaps& mm, bool a_side, bool p_is_a,
                      float* p_out, float* x, float* r, float* z, Scalars* sc, double* part,
                      cudaStream_t st) {
    using G = Geo<CX, CY, TYT, E>;
    const dim3 grid((d.nx + G::W - 1) / G::W, (d.ny + G::HT - 1) / G::HT,
                    (d.nz + kchunk - 1) / kchunk);
    const dim3 block(32, TYT);
    if (a_side)
        k_march_a<CX, CY, TYT, E><<<grid, block, NS * G::A_STAGE, st>>>(
            d, kchunk, mm.z, p_is_a ? mm.pa : mm.pb, mm.eta, p_out, sc, part);
    else
        k_march_b<CX, CY, TYT, E><<<grid, block, NS * G::B_STAGE, st>>>(
            d, kchunk, p_is_a ? mm.pa : mm.pb, mm.eta, mm.x, mm.r, x, r, z, sc, part);
    g_kernel_launches.fetch_add(1, std::memory_order_relaxed);
}

template <typename E>
static void dispatch(const Dims& d, int kchunk, const MarchMaps& mm, bool a_side, bool p_is_a,
                     float* p_out, float* x, float* r, float* z, Scalars* sc, double* part,
                     cudaStream_t st) {
    int n;
    variants(&n);  // function attributes set
    switch (mm.variant) {
#define CASE(ID, CX, CY, TYT)                                                                \
    case ID:                                                                                 \
        launch_ab<CX, CY, TYT, E>(d, kchunk, mm, a_side, p_is_a, p_out, x, r, z, sc, part, st); \
        break;
        CASE(0, 1, 1, 4)
        CASE(1, 1, 1, 8)
        CASE(2, 1, 1, 16)
        CASE(3, 2, 2, 2)
        CASE(4, 2, 2, 4)
        CASE(5, 2, 2, 8)
        CASE(6, 2, 1, 8)
        CASE(7, 1, 2, 8)
#undef CASE
        default: break;
    }
}

void launch_march_a(const Dims& d, int kchunk, const MarchMaps& mm, bool pin_is_a, float* p_out,
                    Scalars* sc, double* part, cudaStream_t st) {
    if (mm.bf16)
        dispatch<__nv_bfloat16>(d, kchunk, mm, true, pin_is_a, p_out, nullptr, nullptr, nullptr,
                                sc, part, st);
    else
        dispatch<float>(d, kchunk, mm, true, pin_is_a, p_out, nullptr, nullptr, nullptr, sc, part,
                        st);
}

void launch_march_b(const Dims& d, int kchunk, const MarchMaps& mm, bool p_is_a, float* x,
                    float* r, float* z, Scalars* sc, double* part, cudaStream_t st) {
    if (mm.bf16)
        dispatch<__nv_bfloat16>(d, kchunk, mm, false, p_is_a, nullptr, x, r, z, sc, part, st);
    else
        dispatch<float>(d, kchunk, mm, false, p_is_a, nullptr, x, r, z, sc, part, st);
}

}  // namespace pcg

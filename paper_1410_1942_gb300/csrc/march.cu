// march.cu -- the FP32 CG passes as 2.5-D plane-marching kernels with TMA-staged x-y planes.
//
// A CTA of 32 x TYT threads works on x-y tiles of W x HT cells (W = 32 CX, HT = TYT CY; each
// thread owns a CX x CY block of cells) and walks them along z.  The grid is persistent (as many
// CTAs as fit on the GPU at once) and driven by a work list of z-segments, so every CTA gets the
// same number of tile-planes whatever the grid shape, and one launch can serve many solves of
// different sizes (each segment names its solve; per-solve tensor maps, vectors and scalars
// live in device memory).  Each plane of the inputs
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
#include <vector>

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

// ------------------------------------------------------------------ work-list kernels
// The grid is persistent: CTA c walks the segments [cta_seg[c], cta_seg[c+1]) of the work list.
// A segment is one tile column of one solve over planes [k0, k1); its plane stream is k0-1 .. k1
// (one halo plane at each end).  The planes of all of a CTA's segments form one stream through
// the NS-stage ring, so the TMA lookahead runs on across segment boundaries.  Each segment
// leaves its partial sums in seg_part; the CTA that completes the last segment of a solve (the
// solve's ticket) adds that solve's partials in segment order and updates its scalars.
//
// A solve whose scalars say it is finished is skipped.  That flag only changes once every
// segment of the solve has been processed in the current launch, so every reader of a pending
// segment sees the value it had at launch.

__device__ __forceinline__ bool seg_active(const SolveDev* solves, const Seg& s) {
    return *(volatile const int*)&solves[s.solve].sc->done == RUNNING;
}

// Thread 0's issue cursor over the plane stream of this CTA.
struct Cursor {
    int seg;  // current segment
    int off;  // plane offset within it (0 .. L+1)
    int n;    // stream positions issued
};

template <int NV>
__device__ __forceinline__ bool segment_done(const SolveDev& sv, int s, double (&v)[NV],
                                             double* seg_part, double (&tot)[NV], double* red,
                                             int tid, int nthreads) {
    __shared__ int s_last;
    block_sum<NV>(v, red);
    if (tid == 0) {
#pragma unroll
        for (int q = 0; q < NV; ++q) seg_part[(size_t)s * NV + q] = v[q];
        __threadfence();
        const unsigned t = atomicAdd(&sv.sc->ticket, 1u);
        s_last = (t + 1 == (unsigned)(sv.seg_end - sv.seg_begin)) ? 1 : 0;
    }
    __syncthreads();
    if (!s_last) return false;
    __threadfence();
    double acc[NV];
#pragma unroll
    for (int q = 0; q < NV; ++q) acc[q] = 0.0;
    for (int b = sv.seg_begin + tid; b < sv.seg_end; b += nthreads)
#pragma unroll
        for (int q = 0; q < NV; ++q) acc[q] += __ldcg(&seg_part[(size_t)b * NV + q]);
    block_sum<NV>(acc, red);
    if (tid == 0) {
#pragma unroll
        for (int q = 0; q < NV; ++q) red[q] = acc[q];
        sv.sc->ticket = 0u;
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < NV; ++q) tot[q] = red[q];
    __syncthreads();
    return true;
}

template <int CX, int CY, int TYT, typename E>
__global__ void __launch_bounds__(32 * TYT) k_march_a(const SolveDev* __restrict__ solves,
                                                     const Seg* __restrict__ segs,
                                                     const int* __restrict__ cta_seg,
                                                     const CUtensorMap* __restrict__ maps,
                                                     double* seg_part, int pin_is_a) {
    using G = Geo<CX, CY, TYT, E>;
    extern __shared__ __align__(128) unsigned char sm[];
    __shared__ __align__(8) uint64_t bars[NS];
    __shared__ double red[64];
    const int sb = cta_seg[blockIdx.x], se = cta_seg[blockIdx.x + 1];
    if (sb >= se) return;
    const int tx = threadIdx.x, ty = threadIdx.y, tid = tx + 32 * ty;
    if (tid == 0) {
        for (int s = 0; s < NS; ++s) mbar_init(&bars[s], 1);
        fence_mbar_init();
    }
    __syncthreads();

    Cursor cur{sb, 0, 0};
    auto issue_next = [&]() {  // thread 0
        while (cur.seg < se && cur.off == 0 && !seg_active(solves, segs[cur.seg])) ++cur.seg;
        if (cur.seg >= se) return;
        const Seg sg = segs[cur.seg];
        const int st = cur.n % NS, kk = sg.k0 - 1 + cur.off;
        unsigned char* dst = sm + st * G::A_STAGE;
        const CUtensorMap* m = maps + 6 * sg.solve;
        const int pm = pin_is_a ? MAP_PA : MAP_PB;
        mbar_arrive_expect_tx(&bars[st], G::A_TX);
        tma_load_3d(dst + G::A_Z, m + MAP_Z, &bars[st], sg.x0 - G::VOFF, sg.y0 - 1, kk);
        tma_load_3d(dst + G::A_P, m + pm, &bars[st], sg.x0 - G::VOFF, sg.y0 - 1, kk);
        tma_load_3d(dst + G::A_E, m + MAP_ETA, &bars[st], sg.x0 - G::EOFF, sg.y0 - 1, kk);
        ++cur.n;
        if (++cur.off == sg.k1 - sg.k0 + 2) {
            cur.off = 0;
            ++cur.seg;
        }
    };
    if (tid == 0)
        for (int q = 0; q < NS; ++q) issue_next();

    int g = 0;  // next stream position to acquire
    bool ok = true, failed = false;
    auto acquire = [&]() -> bool {
        ok = ok && mbar_wait(&bars[g % NS], (g / NS) & 1);
        if (__syncthreads_or(!ok)) return false;  // also: every thread is done with plane g-2
        if (tid == 0 && g >= 2) issue_next();
        ++g;
        return true;
    };
    auto Zs = [&](int q) { return (const float*)(sm + (q % NS) * G::A_STAGE + G::A_Z); };
    auto Ps = [&](int q) { return (const float*)(sm + (q % NS) * G::A_STAGE + G::A_P); };
    auto Es = [&](int q) { return (const E*)(sm + (q % NS) * G::A_STAGE + G::A_E); };
    const int r0 = 1 + CY * ty, cv = G::VOFF + CX * tx, ce = G::EOFF + CX * tx;

    for (int s = sb; s < se; ++s) {
        const Seg sg = segs[s];
        if (!seg_active(solves, sg)) continue;
        const SolveDev& sv = solves[sg.solve];
        const Dims d = sv.d;
        const float beta = (float)sv.sc->beta;
        float* p_out = pin_is_a ? sv.pb : sv.pa;
        const int i0 = sg.x0 + CX * tx, j0 = sg.y0 + CY * ty;
        auto centre_pn = [&](int q, float (&o)[CY][CX]) {
            float zz[CY][CX], pp[CY][CX];
            load_centre<CX, CY>(Zs(q), G::VW, r0, cv, zz);
            load_centre<CX, CY>(Ps(q), G::VW, r0, cv, pp);
#pragma unroll
            for (int a = 0; a < CY; ++a)
#pragma unroll
                for (int b = 0; b < CX; ++b) o[a][b] = zz[a][b] + beta * pp[a][b];
        };
        float vm[CY][CX], vc[CY][CX], em[CY][CX], ec[CY][CX], wzl[CY][CX];
        if (!acquire()) { failed = true; break; }  // plane k0-1
        centre_pn(g - 1, vm);
        load_centre<CX, CY>(Es(g - 1), G::EW, r0, ce, em);
        if (!acquire()) { failed = true; break; }  // plane k0
        centre_pn(g - 1, vc);
        load_centre<CX, CY>(Es(g - 1), G::EW, r0, ce, ec);
#pragma unroll
        for (int a = 0; a < CY; ++a)
#pragma unroll
            for (int b = 0; b < CX; ++b)
                wzl[a][b] = (sg.k0 > 0) ? rcp_approx(ec[a][b] + em[a][b]) : 0.f;
        float acc = 0.f;
        for (int k = sg.k0; k < sg.k1; ++k) {
            if (!acquire()) { failed = true; break; }  // plane k+1 (lookahead)
            const int qc = g - 2, qn = g - 1;
            float vp[CY][CX], ep[CY][CX];
            centre_pn(qn, vp);
            load_centre<CX, CY>(Es(qn), G::EW, r0, ce, ep);
            float zxm[CY], zxp[CY], zym[CX], zyp[CX];
            float pxm[CY], pxp[CY], pym[CX], pyp[CX];
            load_halo<CX, CY>(Zs(qc), G::VW, r0, cv, zxm, zxp, zym, zyp);
            load_halo<CX, CY>(Ps(qc), G::VW, r0, cv, pxm, pxp, pym, pyp);
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
            float exm[CY], exq[CY], eym[CX], eyp[CX];
            load_halo<CX, CY>(Es(qc), G::EW, r0, ce, exm, exq, eym, eyp);
            float qv[CY][CX], D[CY][CX];
            stencil<CX, CY>(d, i0, j0, k, vc, vxm, vxp, vym, vyp, vm, vp, ec, exm, exq, eym, eyp,
                            ep, wzl, qv, D);
            if (i0 < d.nx) {
#pragma unroll
                for (int a = 0; a < CY; ++a) {
                    if (j0 + a < d.ny) {
#pragma unroll
                        for (int b = 0; b < CX; ++b) acc += vc[a][b] * qv[a][b];
                        st_row<CX>(p_out + (size_t)i0 + (size_t)d.nx * (j0 + a + (size_t)d.ny * k),
                                   vc[a]);
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
        if (failed) break;
        double v[1] = {(double)acc}, tot[1];
        if (segment_done<1>(sv, s, v, seg_part, tot, red, tid, 32 * TYT)) {
            if (tid == 0 && sv.sc->done == RUNNING) {
                const double pq = tot[0];
                if (!(pq > 0.0) || !isfinite(pq)) {
                    sv.sc->done = BREAKDOWN;
                } else {
                    sv.sc->pq = pq;
                    sv.sc->alpha = sv.sc->rz / pq;
                }
            }
        }
    }
    if (failed) {
        if (tid == 0) {
            for (int s = sb; s < se; ++s) atomicExch(&solves[segs[s].solve].sc->done, (int)TIMEDOUT);
            for (int q = g; q < cur.n; ++q) (void)mbar_wait(&bars[q % NS], (q / NS) & 1);
            __threadfence();
        }
        __syncthreads();
    }
}

template <int CX, int CY, int TYT, typename E>
__global__ void __launch_bounds__(32 * TYT) k_march_b(const SolveDev* __restrict__ solves,
                                                     const Seg* __restrict__ segs,
                                                     const int* __restrict__ cta_seg,
                                                     const CUtensorMap* __restrict__ maps,
                                                     double* seg_part, int p_is_a) {
    using G = Geo<CX, CY, TYT, E>;
    extern __shared__ __align__(128) unsigned char sm[];
    __shared__ __align__(8) uint64_t bars[NS];
    __shared__ double red[64];
    const int sb = cta_seg[blockIdx.x], se = cta_seg[blockIdx.x + 1];
    if (sb >= se) return;
    const int tx = threadIdx.x, ty = threadIdx.y, tid = tx + 32 * ty;
    if (tid == 0) {
        for (int s = 0; s < NS; ++s) mbar_init(&bars[s], 1);
        fence_mbar_init();
    }
    __syncthreads();

    Cursor cur{sb, 0, 0};
    auto issue_next = [&]() {  // thread 0
        while (cur.seg < se && cur.off == 0 && !seg_active(solves, segs[cur.seg])) ++cur.seg;
        if (cur.seg >= se) return;
        const Seg sg = segs[cur.seg];
        const int L = sg.k1 - sg.k0;
        const int st = cur.n % NS, kk = sg.k0 - 1 + cur.off;
        unsigned char* dst = sm + st * G::B_STAGE;
        const CUtensorMap* m = maps + 6 * sg.solve;
        const bool centre = cur.off > 0 && cur.off <= L;
        mbar_arrive_expect_tx(&bars[st], centre ? G::B_TX : G::B_TX_HALO);
        tma_load_3d(dst + G::B_P, m + (p_is_a ? MAP_PA : MAP_PB), &bars[st], sg.x0 - G::VOFF,
                    sg.y0 - 1, kk);
        tma_load_3d(dst + G::B_E, m + MAP_ETA, &bars[st], sg.x0 - G::EOFF, sg.y0 - 1, kk);
        if (centre) {
            tma_load_3d(dst + G::B_X, m + MAP_X, &bars[st], sg.x0, sg.y0, kk);
            tma_load_3d(dst + G::B_R, m + MAP_R, &bars[st], sg.x0, sg.y0, kk);
        }
        ++cur.n;
        if (++cur.off == L + 2) {
            cur.off = 0;
            ++cur.seg;
        }
    };
    if (tid == 0)
        for (int q = 0; q < NS; ++q) issue_next();

    int g = 0;
    bool ok = true, failed = false;
    auto acquire = [&]() -> bool {
        ok = ok && mbar_wait(&bars[g % NS], (g / NS) & 1);
        if (__syncthreads_or(!ok)) return false;
        if (tid == 0 && g >= 2) issue_next();
        ++g;
        return true;
    };
    auto Ps = [&](int q) { return (const float*)(sm + (q % NS) * G::B_STAGE + G::B_P); };
    auto Es = [&](int q) { return (const E*)(sm + (q % NS) * G::B_STAGE + G::B_E); };
    auto Xs = [&](int q) { return (const float*)(sm + (q % NS) * G::B_STAGE + G::B_X); };
    auto Rs = [&](int q) { return (const float*)(sm + (q % NS) * G::B_STAGE + G::B_R); };
    const int r0 = 1 + CY * ty, cv = G::VOFF + CX * tx, ce = G::EOFF + CX * tx;
    const int cc = CX * tx;

    for (int s = sb; s < se; ++s) {
        const Seg sg = segs[s];
        if (!seg_active(solves, sg)) continue;
        const SolveDev& sv = solves[sg.solve];
        const Dims d = sv.d;
        const float alpha = (float)sv.sc->alpha;
        float* x = sv.x;
        float* r = sv.r;
        float* z = sv.z;
        const int i0 = sg.x0 + CX * tx, j0 = sg.y0 + CY * ty;
        float vm[CY][CX], vc[CY][CX], em[CY][CX], ec[CY][CX], wzl[CY][CX];
        if (!acquire()) { failed = true; break; }
        load_centre<CX, CY>(Ps(g - 1), G::VW, r0, cv, vm);
        load_centre<CX, CY>(Es(g - 1), G::EW, r0, ce, em);
        if (!acquire()) { failed = true; break; }
        load_centre<CX, CY>(Ps(g - 1), G::VW, r0, cv, vc);
        load_centre<CX, CY>(Es(g - 1), G::EW, r0, ce, ec);
#pragma unroll
        for (int a = 0; a < CY; ++a)
#pragma unroll
            for (int b = 0; b < CX; ++b)
                wzl[a][b] = (sg.k0 > 0) ? rcp_approx(ec[a][b] + em[a][b]) : 0.f;
        float arz = 0.f, arr = 0.f;
        for (int k = sg.k0; k < sg.k1; ++k) {
            if (!acquire()) { failed = true; break; }
            const int qc = g - 2, qn = g - 1;
            float vp[CY][CX], ep[CY][CX];
            load_centre<CX, CY>(Ps(qn), G::VW, r0, cv, vp);
            load_centre<CX, CY>(Es(qn), G::EW, r0, ce, ep);
            float vxm[CY], vxp[CY], vym[CX], vyp[CX];
            load_halo<CX, CY>(Ps(qc), G::VW, r0, cv, vxm, vxp, vym, vyp);
            float exm[CY], exq[CY], eym[CX], eyp[CX];
            load_halo<CX, CY>(Es(qc), G::EW, r0, ce, exm, exq, eym, eyp);
            float qv[CY][CX], D[CY][CX];
            stencil<CX, CY>(d, i0, j0, k, vc, vxm, vxp, vym, vyp, vm, vp, ec, exm, exq, eym, eyp,
                            ep, wzl, qv, D);
            float xo[CY][CX], ro[CY][CX];
            load_centre<CX, CY>(Xs(qc), G::W, CY * ty, cc, xo);
            load_centre<CX, CY>(Rs(qc), G::W, CY * ty, cc, ro);
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
        if (failed) break;
        double v[2] = {(double)arz, (double)arr}, tot[2];
        if (segment_done<2>(sv, s, v, seg_part, tot, red, tid, 32 * TYT)) {
            Scalars* sc = sv.sc;
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
    if (failed) {
        if (tid == 0) {
            for (int s = sb; s < se; ++s) atomicExch(&solves[segs[s].solve].sc->done, (int)TIMEDOUT);
            for (int q = g; q < cur.n; ++q) (void)mbar_wait(&bars[q % NS], (q / NS) & 1);
            __threadfence();
        }
        __syncthreads();
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

#define MARCH_VARIANTS(X) X(0, 1, 1, 4) X(1, 1, 1, 8) X(2, 1, 1, 16) X(3, 2, 2, 2) \
    X(4, 2, 2, 4) X(5, 2, 2, 8) X(6, 2, 1, 8) X(7, 1, 2, 8)

static const VariantOps* variants(int* count) {
#define ROW(ID, CX, CY, TYT) make_ops<CX, CY, TYT>(),
    static const VariantOps table[] = {MARCH_VARIANTS(ROW)};
#undef ROW
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

// ------------------------------------------------------------------ plans
bool march_encode_solve(CUtensorMap (&m)[6], const MarchSolve& s, int variant, bool bf16) {
    const MarchVariant v = march_variant(variant);
    const int eoff = bf16 ? 8 : 4;
    const CUtensorMapDataType f32 = CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
    const CUtensorMapDataType edt = bf16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : f32;
    const Dims& d = s.d;
    bool ok = true;
    ok = ok && encode3d(&m[MAP_Z], s.z, f32, 4, d, v.width + 8, v.height + 2);
    ok = ok && encode3d(&m[MAP_PA], s.pa, f32, 4, d, v.width + 8, v.height + 2);
    ok = ok && encode3d(&m[MAP_PB], s.pb, f32, 4, d, v.width + 8, v.height + 2);
    ok = ok && encode3d(&m[MAP_ETA], s.eta, edt, bf16 ? 2 : 4, d, v.width + 2 * eoff, v.height + 2);
    ok = ok && encode3d(&m[MAP_X], s.x, f32, 4, d, v.width, v.height);
    ok = ok && encode3d(&m[MAP_R], s.r, f32, 4, d, v.width, v.height);
    return ok;
}

void march_plan_free(MarchPlan* p) {
    void* ptrs[] = {p->solves, p->segs, p->cta_seg, p->maps, p->seg_part};
    for (void* q : ptrs)
        if (q) cudaFree(q);
    *p = MarchPlan{};
}

// Splits the solves' tile columns into segments and gives every CTA an equal share of the
// linearised (solve, tile, plane) space: CTA c owns planes [c W / G, (c + 1) W / G), cut into
// one segment per tile column it touches.  Segments come out ordered by solve.
int march_plan_build(MarchPlan* p, const MarchSolve* solves, int nsolves, int variant, bool bf16,
                     int nctas, cudaStream_t st) {
    march_plan_free(p);
    const MarchVariant v = march_variant(variant);
    std::vector<long long> base(nsolves + 1, 0);  // first plane unit of each solve
    std::vector<int> tiles_x(nsolves), tiles_y(nsolves);
    for (int s = 0; s < nsolves; ++s) {
        tiles_x[s] = (solves[s].d.nx + v.width - 1) / v.width;
        tiles_y[s] = (solves[s].d.ny + v.height - 1) / v.height;
        base[s + 1] = base[s] + (long long)tiles_x[s] * tiles_y[s] * solves[s].d.nz;
    }
    const long long W = base[nsolves];
    if (W <= 0) return -1;
    if (nctas > W) nctas = (int)W;
    std::vector<Seg> segs;
    std::vector<int> cta_seg(nctas + 1, 0);
    std::vector<SolveDev> sd(nsolves);
    int sol = 0;
    for (int c = 0; c < nctas; ++c) {
        cta_seg[c] = (int)segs.size();
        long long u = W * c / nctas;
        const long long u1 = W * (c + 1) / nctas;
        while (u < u1) {
            while (base[sol + 1] <= u) ++sol;
            const Dims& d = solves[sol].d;
            const long long local = u - base[sol];
            const int tile = (int)(local / d.nz);
            const int k0 = (int)(local % d.nz);
            const int k1 = (int)std::min<long long>(d.nz, k0 + (u1 - u));
            Seg g{};
            g.solve = sol;
            g.x0 = (tile % tiles_x[sol]) * v.width;
            g.y0 = (tile / tiles_x[sol]) * v.height;
            g.k0 = k0;
            g.k1 = k1;
            segs.push_back(g);
            u += k1 - k0;
        }
    }
    cta_seg[nctas] = (int)segs.size();
    for (int s = 0; s < nsolves; ++s) {
        sd[s].d = solves[s].d;
        sd[s].x = solves[s].x;
        sd[s].r = solves[s].r;
        sd[s].z = solves[s].z;
        sd[s].pa = solves[s].pa;
        sd[s].pb = solves[s].pb;
        sd[s].sc = solves[s].sc;
        sd[s].seg_begin = (int)segs.size();
        sd[s].seg_end = 0;
    }
    for (int q = 0; q < (int)segs.size(); ++q) {
        SolveDev& t = sd[segs[q].solve];
        t.seg_begin = std::min(t.seg_begin, q);
        t.seg_end = std::max(t.seg_end, q + 1);
    }
    std::vector<CUtensorMap> maps(6 * (size_t)nsolves);
    for (int s = 0; s < nsolves; ++s) {
        CUtensorMap m[6];
        if (!march_encode_solve(m, solves[s], variant, bf16)) return -1;
        for (int q = 0; q < 6; ++q) maps[6 * (size_t)s + q] = m[q];
    }
    p->variant = variant;
    p->bf16 = bf16;
    p->nctas = nctas;
    p->nsolves = nsolves;
    p->nsegs = (int)segs.size();
    auto up = [&](void** dst, const void* src, size_t bytes) -> bool {
        if (cudaMalloc(dst, bytes) != cudaSuccess) {
            cudaGetLastError();
            *dst = nullptr;
            return false;
        }
        return cudaMemcpyAsync(*dst, src, bytes, cudaMemcpyHostToDevice, st) == cudaSuccess;
    };
    bool ok = up((void**)&p->solves, sd.data(), sizeof(SolveDev) * sd.size()) &&
              up((void**)&p->segs, segs.data(), sizeof(Seg) * segs.size()) &&
              up((void**)&p->cta_seg, cta_seg.data(), sizeof(int) * cta_seg.size()) &&
              up((void**)&p->maps, maps.data(), sizeof(CUtensorMap) * maps.size());
    if (ok && cudaMalloc((void**)&p->seg_part, sizeof(double) * 2 * segs.size()) != cudaSuccess) {
        cudaGetLastError();
        ok = false;
    }
    if (ok) ok = cudaStreamSynchronize(st) == cudaSuccess;  // host vectors go out of scope
    if (!ok) {
        march_plan_free(p);
        return -2;
    }
    return 0;
}

template <int CX, int CY, int TYT, typename E>
static void launch_ab(const MarchPlan& p, bool a_side, int flag, cudaStream_t st) {
    using G = Geo<CX, CY, TYT, E>;
    const dim3 block(32, TYT);
    if (a_side)
        k_march_a<CX, CY, TYT, E><<<p.nctas, block, NS * G::A_STAGE, st>>>(
            p.solves, p.segs, p.cta_seg, p.maps, p.seg_part, flag);
    else
        k_march_b<CX, CY, TYT, E><<<p.nctas, block, NS * G::B_STAGE, st>>>(
            p.solves, p.segs, p.cta_seg, p.maps, p.seg_part, flag);
    g_kernel_launches.fetch_add(1, std::memory_order_relaxed);
}

template <typename E>
static void dispatch(const MarchPlan& p, bool a_side, int flag, cudaStream_t st) {
    int n;
    variants(&n);  // function attributes set
    switch (p.variant) {
#define CASE(ID, CX, CY, TYT) \
    case ID: launch_ab<CX, CY, TYT, E>(p, a_side, flag, st); break;
        MARCH_VARIANTS(CASE)
#undef CASE
        default: break;
    }
}

void launch_march_a(const MarchPlan& p, bool pin_is_a, cudaStream_t st) {
    if (p.bf16)
        dispatch<__nv_bfloat16>(p, true, pin_is_a ? 1 : 0, st);
    else
        dispatch<float>(p, true, pin_is_a ? 1 : 0, st);
}

void launch_march_b(const MarchPlan& p, bool p_is_a, cudaStream_t st) {
    if (p.bf16)
        dispatch<__nv_bfloat16>(p, false, p_is_a ? 1 : 0, st);
    else
        dispatch<float>(p, false, p_is_a ? 1 : 0, st);
}

}  // namespace pcg

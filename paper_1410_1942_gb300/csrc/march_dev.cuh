// march_dev.cuh -- device helpers shared by the plane-marching CG kernels (march.cu, march1.cu):
// shared-memory stage geometry, row loads and stores, the 7-point stencil of a CX x CY block,
// grid barriers with bounded waits, and fixed-order reductions of per-segment partial sums.
#pragma once

#include "internal.cuh"
#include "march.h"
#include "tma.cuh"

namespace pcg {

// Shared-memory stages (planes) in a kernel's ring: a template parameter of each kernel
// (3, 4 or 6 in the variant table).

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
    static constexpr int STAGE = A_STAGE > B_STAGE ? A_STAGE : B_STAGE;
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

// Which faces of a thread's CX x CY block at the block's edges are open (have a coefficient):
// bit 0 the -x faces (column i0), bit 1 the +x faces (after column i0+CX-1), bit 2 the -y faces
// (row j0), bit 2+a the faces between rows j0+a-1 and j0+a for a = 1..CY (a = CY: the +y faces).
// Open means inside the grid or on a Dirichlet wall (Dims::walls): a Dirichlet wall's face has
// the coefficient 1/eta_c, which the shared expression gives because the zero-filled halo beyond
// the grid holds eta = 0 and value 0.  Interior x faces of the block are always open (nx is a
// multiple of 8 for these kernels).  Computed once per segment.
template <int CX, int CY>
__device__ __forceinline__ unsigned block_edges(const Dims& d, int i0, int j0) {
    unsigned e = 0;
    if (i0 > 0 || (d.walls & (1 | PERIODIC_X))) e |= 1u;
    if (i0 + CX < d.nx || (d.walls & (2 | PERIODIC_X))) e |= 2u;
    if (j0 > 0 || (d.walls & 4)) e |= 4u;
#pragma unroll
    for (int a = 1; a <= CY; ++a)
        if (j0 + a < d.ny || (d.walls & 8)) e |= 4u << a;
    return e;
}

// The stencil of one plane for the CX x CY block of a thread.
//   cen: centre values of plane k (registers); vxm/vxp/vym/vyp: the block's neighbour strips in
//   plane k; vm/vp: centre values of planes k-1 and k+1; e*: the same for eta; wzl: face to
//   plane k-1 (0 on the floor).  Returns q = A v and the diagonal per cell, and moves wzl to the
//   face between k and k+1 (0 at the top layer, whose Dirichlet term goes into D).
template <int CX, int CY>
__device__ __forceinline__ void stencil(const Dims& d, unsigned edges, int k,
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
        fx[a][0] = (edges & 1u) ? rcp_approx(ec[a][0] + exm[a]) : 0.f;
#pragma unroll
        for (int b = 1; b < CX; ++b) fx[a][b] = rcp_approx(ec[a][b - 1] + ec[a][b]);
        fx[a][CX] = (edges & 2u) ? rcp_approx(ec[a][CX - 1] + exq[a]) : 0.f;
    }
    float fy[CY + 1][CX];
#pragma unroll
    for (int b = 0; b < CX; ++b) {
        fy[0][b] = (edges & 4u) ? rcp_approx(ec[0][b] + eym[b]) : 0.f;
#pragma unroll
        for (int a = 1; a < CY; ++a)
            fy[a][b] = (edges & (4u << a)) ? rcp_approx(ec[a - 1][b] + ec[a][b]) : 0.f;
        fy[CY][b] = (edges & (4u << CY)) ? rcp_approx(ec[CY - 1][b] + eyp[b]) : 0.f;
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


constexpr int MAXSEG = 16;                                           // segments per CTA
constexpr unsigned long long BAR_NS = 1000ull * 1000ull * 1000ull;   // 1 s per barrier

__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Arrival at grid barrier m (thread 0): CTA 0 clears the count slot of barrier m + 1, the CTA adds
// its unfinished owned solves to the slot of barrier m, then the arrival itself.
__device__ __forceinline__ void barrier_arrive(MarchCtl* ctl, unsigned m, int add) {
    if (blockIdx.x == 0) *(volatile int*)&ctl->alive[(m + 1) % 3] = 0;
    if (add) atomicAdd(&ctl->alive[m % 3], add);
    __threadfence();
}

// Thread 0's bounded wait for `target` arrivals; false after a timeout or another CTA's error.
__device__ __forceinline__ bool barrier_spin(MarchCtl* ctl, unsigned target) {
    unsigned long long t0 = 0;
    while (ld_acquire(&ctl->bar) < target) {
        if (*(volatile int*)&ctl->error) return false;
        const unsigned long long t = globaltimer();
        if (!t0) t0 = t;
        else if (t - t0 > BAR_NS) {
            atomicExch(&ctl->error, 1);
            return false;
        }
    }
    return true;
}

// Grid barrier m (target = m * nctas arrivals).  add: this CTA's unfinished owned solves; *alive
// (every thread): the unfinished solves of the whole launch as of this barrier.
// Tracing (stamp): the last CTA to arrive stamps the time, and a thread passing imb/rel adds its
// wait for the last arrival and the release latency after it (ns).
__device__ __forceinline__ bool grid_barrier(MarchCtl* ctl, unsigned m, unsigned target, int tid,
                                             int add, int* alive, bool stamp = false,
                                             unsigned long long* imb = nullptr,
                                             unsigned long long* rel = nullptr) {
    __shared__ int s_ok, s_alive;
    // generic-proxy stores of this phase must be ordered before the next phase's TMA reads
    asm volatile("fence.proxy.async.global;" ::: "memory");
    __syncthreads();
    if (tid == 0) {
        barrier_arrive(ctl, m, add);
        const unsigned long long t_arr = imb ? globaltimer() : 0;
        const unsigned old = atomicAdd(&ctl->bar, 1u);
        if (stamp && old + 1 == target) *(volatile unsigned long long*)&ctl->t_last = globaltimer();
        const int ok = barrier_spin(ctl, target) ? 1 : 0;
        if (imb) {
            // (a stamp older than this CTA's arrival is the previous barrier's: not counted)
            const unsigned long long tl = *(volatile unsigned long long*)&ctl->t_last;
            const unsigned long long tn = globaltimer();
            if (tl >= t_arr && tn >= tl) {
                *imb += tl - t_arr;
                *rel += tn - tl;
            }
        }
        __threadfence();
        asm volatile("fence.proxy.async.global;" ::: "memory");
        s_alive = *(volatile int*)&ctl->alive[m % 3];
        s_ok = ok;
    }
    __syncthreads();
    *alive = s_alive;
    return s_ok != 0;
}

// Split-phase form of grid_barrier: arrive (after the CTA's stores), do independent work, wait.
// With a trace, the last CTA to arrive stamps the time of its arrival.
__device__ __forceinline__ void grid_arrive(MarchCtl* ctl, int tid, unsigned m, unsigned target,
                                            int add, bool stamp = false) {
    asm volatile("fence.proxy.async.global;" ::: "memory");
    __syncthreads();
    if (tid == 0) {
        barrier_arrive(ctl, m, add);
        const unsigned old = atomicAdd(&ctl->bar, 1u);
        if (stamp && old + 1 == target) *(volatile unsigned long long*)&ctl->t_last = globaltimer();
    }
}

__device__ __forceinline__ bool grid_wait(MarchCtl* ctl, unsigned m, unsigned target, int tid,
                                          int* alive) {
    __shared__ int s_ok2, s_alive2;
    if (tid == 0) {
        const int ok = barrier_spin(ctl, target) ? 1 : 0;
        __threadfence();
        asm volatile("fence.proxy.async.global;" ::: "memory");
        s_alive2 = *(volatile int*)&ctl->alive[m % 3];
        s_ok2 = ok;
    }
    __syncthreads();
    *alive = s_alive2;
    return s_ok2 != 0;
}

// ------------------------------------------------------------------ float-float sums
// FP64 arithmetic on this GPU runs at a small fraction of the FP32 rate (a warp-wide FP64 add
// occupies an SM's FP64 pipe for many cycles), so the per-iteration reductions of the
// persistent kernels add in "float-float": a value is hi + lo with |lo| <= ulp(hi) / 2, and an
// addition is Knuth's TwoSum of the high parts, the low parts added to its error term, and
// Dekker's Fast2Sum to renormalise -- about 2^-44 relative error per addition, all on the FP32
// pipe.  TwoSum's error term is exact for either operand order, so ff_add is commutative bit for
// bit and a butterfly warp sum leaves the same value in every lane.
struct ff {
    float hi, lo;
};

__device__ __forceinline__ ff ff_add(ff a, ff b) {
    const float s = __fadd_rn(a.hi, b.hi);
    const float bv = __fsub_rn(s, a.hi);
    const float av = __fsub_rn(s, bv);
    const float e = __fadd_rn(__fsub_rn(a.hi, av), __fsub_rn(b.hi, bv));
    const float t = __fadd_rn(__fadd_rn(a.lo, b.lo), e);
    const float hi = __fadd_rn(s, t);
    return ff{hi, __fsub_rn(t, __fsub_rn(hi, s))};
}

__device__ __forceinline__ ff ff_warp_sum(ff v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        ff w;
        w.hi = __shfl_xor_sync(0xffffffffu, v.hi, o);
        w.lo = __shfl_xor_sync(0xffffffffu, v.lo, o);
        v = ff_add(v, w);
    }
    return v;
}

__device__ __forceinline__ double ff_value(ff v) { return (double)v.hi + (double)v.lo; }

// Sum over segments [b, e) of part[seg * NV + q], in a fixed order (the result is the same in
// every CTA); valid in all threads.  Each thread issues all its loads (U per round) before
// adding, so one round trip to L2 covers U * nthreads segments; the warp totals are then added
// by every thread in warp order.  red: at least NV * nwarps entries.
template <int NV>
__device__ __forceinline__ void range_sum(const float2* part, int b, int e, double (&out)[NV],
                                          ff* red, int tid, int nthreads, int bar_id = 0) {
    // threads [0, nthreads) take part; bar_id 0: the whole CTA (__syncthreads), else that named
    // barrier over nthreads threads
    constexpr int U = 4;
    ff acc[NV];
#pragma unroll
    for (int q = 0; q < NV; ++q) acc[q] = ff{0.f, 0.f};
    for (int s0 = b; s0 < e; s0 += U * nthreads) {
        ff v[U][NV];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int s = s0 + u * nthreads + tid;
#pragma unroll
            for (int q = 0; q < NV; ++q) {
                if (s < e) {
                    const float2 t = __ldcg(part + (size_t)s * NV + q);
                    v[u][q] = ff{t.x, t.y};
                } else {
                    v[u][q] = ff{0.f, 0.f};
                }
            }
        }
#pragma unroll
        for (int u = 0; u < U; ++u)
#pragma unroll
            for (int q = 0; q < NV; ++q) acc[q] = ff_add(acc[q], v[u][q]);
    }
#pragma unroll
    for (int q = 0; q < NV; ++q) acc[q] = ff_warp_sum(acc[q]);
    const int nw = (nthreads + 31) >> 5;
    if ((tid & 31) == 0)
#pragma unroll
        for (int q = 0; q < NV; ++q) red[(tid >> 5) * NV + q] = acc[q];
    if (bar_id) named_sync(bar_id, nthreads); else __syncthreads();
#pragma unroll
    for (int q = 0; q < NV; ++q) {
        ff t{0.f, 0.f};
        for (int w = 0; w < nw; ++w) t = ff_add(t, red[w * NV + q]);
        out[q] = ff_value(t);
    }
    if (bar_id) named_sync(bar_id, nthreads); else __syncthreads();
}

// The same sum by one warp (valid in every lane).
template <int NV>
__device__ __forceinline__ void warp_range_sum(const float2* part, int b, int e, int lane,
                                               double (&out)[NV]) {
    constexpr int U = 8;  // loads in flight per lane
    ff acc[NV];
#pragma unroll
    for (int q = 0; q < NV; ++q) acc[q] = ff{0.f, 0.f};
    for (int s0 = b; s0 < e; s0 += 32 * U) {
        ff v[U][NV];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int s = s0 + 32 * u + lane;
#pragma unroll
            for (int q = 0; q < NV; ++q) {
                if (s < e) {
                    const float2 t = __ldcg(part + (size_t)s * NV + q);
                    v[u][q] = ff{t.x, t.y};
                } else {
                    v[u][q] = ff{0.f, 0.f};
                }
            }
        }
#pragma unroll
        for (int u = 0; u < U; ++u)
#pragma unroll
            for (int q = 0; q < NV; ++q) acc[q] = ff_add(acc[q], v[u][q]);
    }
#pragma unroll
    for (int q = 0; q < NV; ++q) out[q] = ff_value(ff_warp_sum(acc[q]));
}

// Partial sums of one segment: the FP32 per-thread sums v[0..NV) of the nthr threads [0, nthr)
// (whole warps) added in float-float, warp totals in warp order; thread 0 stores them to
// part[0..NV).  All nthr threads must call it; bar_id / nthr name the barrier they share.
template <int NV>
__device__ __forceinline__ void segment_partials(const float (&v)[NV], float2* part, ff* red, int tid,
                                                 int nthr, int bar_id) {
    const int lane = tid & 31, warp = tid >> 5, nw = nthr >> 5;
#pragma unroll
    for (int q = 0; q < NV; ++q) {
        const ff t = ff_warp_sum(ff{v[q], 0.f});
        if (lane == 0) red[warp * NV + q] = t;
    }
    named_sync(bar_id, nthr);
    if (tid == 0) {
#pragma unroll
        for (int q = 0; q < NV; ++q) {
            ff t{0.f, 0.f};
            for (int w = 0; w < nw; ++w) t = ff_add(t, red[w * NV + q]);
            part[q] = make_float2(t.hi, t.lo);
        }
    }
    named_sync(bar_id, nthr);
}

struct LocalSolve {
    Dims d;
    float *x, *r, *z, *pa, *pb;
    Scalars* sc;
    int seg_begin, seg_end;
    double rz, alpha, beta, rr, stop2;
    int done, iter, max_iter, finished, owner;
};

// Kernels of the one-sweep family (march1.cu): (CX, CY, TYT, NS) of each instantiation.
#define CG1_CONFIGS(X) X(2, 2, 4, 4) X(2, 2, 4, 3) X(2, 2, 8, 3)
struct Cg1Kernel {
    const void *k32, *k16;
    int smem32, smem16;
    const void *k32p = nullptr, *k16p = nullptr;  // periodic-x instantiations (one-sweep family)
};
Cg1Kernel cg1_kernel(int cx, int cy, int tyt, int ns);  // null kernels if not instantiated
// Kernels of the one-sweep family with A p formed in the sweep (march2.cu).
#define CG2_CONFIGS(X) X(2, 2, 4, 4) X(2, 2, 4, 5) X(2, 2, 8, 4)
Cg1Kernel cg2_kernel(int cx, int cy, int tyt, int ns);  // null kernels if not instantiated

template <int TYT>
struct WsMinBlocks {
    static constexpr int value = TYT >= 8 ? 2 : (TYT >= 4 ? 3 : 4);
};

}  // namespace pcg

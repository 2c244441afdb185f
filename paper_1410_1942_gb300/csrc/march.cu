// march.cu -- the FP32 CG passes as 2.5-D plane-marching kernels with TMA-staged x-y planes.
//
// A CTA owns an x-y tile of 32 x TY cells and walks a chunk of z-planes.  Each plane of the
// inputs that need neighbours (p or z/p_old, and rho/2) is copied into a ring of NS shared-memory
// stages by one TMA box load with a one-cell halo in y and an aligned halo in x (the box starts
// at x0 - 4 for FP32 and x0 - 8 for BF16 so its first coordinate stays on a 16-byte boundary);
// the z-neighbours of a cell are the previous / next plane's centre values kept in registers.
// One mbarrier per stage counts the transaction bytes; every wait is bounded.
//
//   phase A:  p = z + beta p_old, q = A p, sum p.q     (reads z, p_old, eta; writes p)
//   phase B:  q = A p, x += alpha p, r -= alpha q, z = D^{-1} r, sums r.z, r.r
//                                                        (reads p, eta, x, r; writes x, r, z)
//
// The stencil arithmetic is the column kernels' (kernels.cu), term for term: faces
// 1/(eta_c + eta_n), top term 1/eta_c, D = sum of faces, q = D p_c - sum_n w_n p_n.
#include "internal.cuh"
#include "kernels.h"
#include "march.h"
#include "tma.cuh"

#include <cudaTypedefs.h>

#include <atomic>
#include <map>
#include <mutex>

namespace pcg {

constexpr int MTX = 32;  // tile width in x (one warp per row)
constexpr int NS = 4;    // shared-memory stages (planes) in the ring

__host__ __device__ constexpr int align128(int b) { return (b + 127) & ~127; }

template <typename E>
struct EtaX;
template <>
struct EtaX<float> {
    static constexpr int OFF = 4;  // 16 bytes of FP32
};
template <>
struct EtaX<__nv_bfloat16> {
    static constexpr int OFF = 8;  // 16 bytes of BF16
};

template <int TY, typename E>
struct Geo {
    static constexpr int VW = MTX + 8;              // FP32 halo row (x0-4 .. x0+35)
    static constexpr int EOFF = EtaX<E>::OFF;
    static constexpr int EW = MTX + 2 * EOFF;       // eta halo row
    static constexpr int H = TY + 2;                // rows (y0-1 .. y0+TY)
    static constexpr int VB = VW * H * 4;           // bytes of one FP32 halo box
    static constexpr int EB = EW * H * (int)sizeof(E);
    static constexpr int CB = MTX * TY * 4;         // bytes of one FP32 centre box
    // phase A stage: z | p_old | eta
    static constexpr int A_Z = 0, A_P = align128(VB), A_E = A_P + align128(VB);
    static constexpr int A_STAGE = A_E + align128(EB);
    static constexpr int A_TX = 2 * VB + EB;
    // phase B stage: p | eta | x | r
    static constexpr int B_P = 0, B_E = align128(VB), B_X = B_E + align128(EB);
    static constexpr int B_R = B_X + align128(CB);
    static constexpr int B_STAGE = B_R + align128(CB);
    static constexpr int B_TX_HALO = VB + EB;        // planes k0-1 and k1: p, eta only
    static constexpr int B_TX = VB + EB + 2 * CB;
};

__device__ __forceinline__ float to_f(float v) { return v; }
__device__ __forceinline__ float to_f(__nv_bfloat16 v) { return __bfloat162float(v); }

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

template <int TY, typename E>
__global__ void __launch_bounds__(MTX * TY) k_march_a(Dims d, int kchunk,
                                                     const __grid_constant__ CUtensorMap mz,
                                                     const __grid_constant__ CUtensorMap mp,
                                                     const __grid_constant__ CUtensorMap me,
                                                     float* __restrict__ p_out, Scalars* sc,
                                                     double* partials) {
    using G = Geo<TY, E>;
    extern __shared__ __align__(128) unsigned char sm[];
    __shared__ __align__(8) uint64_t bars[NS];
    __shared__ double red[64];
    if (sc->done) return;
    const int tx = threadIdx.x, ty = threadIdx.y, tid = tx + MTX * ty;
    const int x0 = blockIdx.x * MTX, y0 = blockIdx.y * TY;
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
        tma_load_3d(st + G::A_Z, &mz, &bars[s], x0 - 4, y0 - 1, kk);
        tma_load_3d(st + G::A_P, &mp, &bars[s], x0 - 4, y0 - 1, kk);
        tma_load_3d(st + G::A_E, &me, &bars[s], x0 - G::EOFF, y0 - 1, kk);
    };
    if (tid == 0) {
        for (int q = 0; q < NS && q < nplanes; ++q) issue(q);
    }
    int issued = min(NS, nplanes);

    const int hx = tx + 4, he = tx + G::EOFF, hy = ty + 1;
    const int i = x0 + tx, j = y0 + ty;
    const bool valid = (i < d.nx) && (j < d.ny);
    auto Z = [&](int q) { return (const float*)(sm + (q % NS) * G::A_STAGE + G::A_Z); };
    auto P = [&](int q) { return (const float*)(sm + (q % NS) * G::A_STAGE + G::A_P); };
    auto Ev = [&](int q) { return (const E*)(sm + (q % NS) * G::A_STAGE + G::A_E); };

    bool ok = mbar_wait(&bars[0], 0);
    ok = ok && mbar_wait(&bars[1 % NS], (1 / NS) & 1);
    float pm = Z(0)[hy * G::VW + hx] + beta * P(0)[hy * G::VW + hx];
    float em = to_f(Ev(0)[hy * G::EW + he]);
    float pc = Z(1)[hy * G::VW + hx] + beta * P(1)[hy * G::VW + hx];
    float ec = to_f(Ev(1)[hy * G::EW + he]);
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
        const float* Zs = Z(q);
        const float* Ps = P(q);
        const E* Es = Ev(q);
        const float* Z1 = Z(q + 1);
        const float* P1 = P(q + 1);
        const float pp = Z1[hy * G::VW + hx] + beta * P1[hy * G::VW + hx];
        const float ep = to_f(Ev(q + 1)[hy * G::EW + he]);
        auto pn = [&](int o) { return Zs[o] + beta * Ps[o]; };
        const int o = hy * G::VW + hx, oe = hy * G::EW + he;
        const float wxm = (i > 0) ? rcp_approx(ec + to_f(Es[oe - 1])) : 0.f;
        const float wxp = (i + 1 < d.nx) ? rcp_approx(ec + to_f(Es[oe + 1])) : 0.f;
        const float wym = (j > 0) ? rcp_approx(ec + to_f(Es[oe - G::EW])) : 0.f;
        const float wyp = (j + 1 < d.ny) ? rcp_approx(ec + to_f(Es[oe + G::EW])) : 0.f;
        const float wzm = (k > 0) ? rcp_approx(ec + em) : 0.f;
        const bool top = (k + 1 == d.nz);
        const float wzt = top ? rcp_approx(ec) : rcp_approx(ec + ep);
        const float wzp = top ? 0.f : wzt;
        const float D = wxm + wxp + wym + wyp + wzm + wzt;
        float s = 0.f;
        if (i > 0) s += wxm * pn(o - 1);
        if (i + 1 < d.nx) s += wxp * pn(o + 1);
        if (j > 0) s += wym * pn(o - G::VW);
        if (j + 1 < d.ny) s += wyp * pn(o + G::VW);
        if (k > 0) s += wzm * pm;
        if (!top) s += wzp * pp;
        const float qv = D * pc - s;
        if (valid) {
            acc += pc * qv;
            p_out[i + d.nx * (j + d.ny * k)] = pc;
        }
        pm = pc;
        pc = pp;
        em = ec;
        ec = ep;
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

template <int TY, typename E>
__global__ void __launch_bounds__(MTX * TY) k_march_b(Dims d, int kchunk,
                                                     const __grid_constant__ CUtensorMap mp,
                                                     const __grid_constant__ CUtensorMap me,
                                                     const __grid_constant__ CUtensorMap mx,
                                                     const __grid_constant__ CUtensorMap mr,
                                                     float* __restrict__ x, float* __restrict__ r,
                                                     float* __restrict__ z, Scalars* sc,
                                                     double* partials) {
    using G = Geo<TY, E>;
    extern __shared__ __align__(128) unsigned char sm[];
    __shared__ __align__(8) uint64_t bars[NS];
    __shared__ double red[64];
    if (sc->done) return;
    const int tx = threadIdx.x, ty = threadIdx.y, tid = tx + MTX * ty;
    const int x0 = blockIdx.x * MTX, y0 = blockIdx.y * TY;
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
        tma_load_3d(st + G::B_P, &mp, &bars[s], x0 - 4, y0 - 1, kk);
        tma_load_3d(st + G::B_E, &me, &bars[s], x0 - G::EOFF, y0 - 1, kk);
        if (centre) {
            tma_load_3d(st + G::B_X, &mx, &bars[s], x0, y0, kk);
            tma_load_3d(st + G::B_R, &mr, &bars[s], x0, y0, kk);
        }
    };
    if (tid == 0) {
        for (int q = 0; q < NS && q < nplanes; ++q) issue(q);
    }
    int issued = min(NS, nplanes);

    const int hx = tx + 4, he = tx + G::EOFF, hy = ty + 1;
    const int i = x0 + tx, j = y0 + ty;
    const bool valid = (i < d.nx) && (j < d.ny);
    auto P = [&](int q) { return (const float*)(sm + (q % NS) * G::B_STAGE + G::B_P); };
    auto Ev = [&](int q) { return (const E*)(sm + (q % NS) * G::B_STAGE + G::B_E); };
    auto X = [&](int q) { return (const float*)(sm + (q % NS) * G::B_STAGE + G::B_X); };
    auto R = [&](int q) { return (const float*)(sm + (q % NS) * G::B_STAGE + G::B_R); };

    bool ok = mbar_wait(&bars[0], 0);
    ok = ok && mbar_wait(&bars[1 % NS], (1 / NS) & 1);
    float pm = P(0)[hy * G::VW + hx];
    float em = to_f(Ev(0)[hy * G::EW + he]);
    float pc = P(1)[hy * G::VW + hx];
    float ec = to_f(Ev(1)[hy * G::EW + he]);
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
        const float* Ps = P(q);
        const E* Es = Ev(q);
        const float pp = P(q + 1)[hy * G::VW + hx];
        const float ep = to_f(Ev(q + 1)[hy * G::EW + he]);
        const int o = hy * G::VW + hx, oe = hy * G::EW + he;
        const float wxm = (i > 0) ? rcp_approx(ec + to_f(Es[oe - 1])) : 0.f;
        const float wxp = (i + 1 < d.nx) ? rcp_approx(ec + to_f(Es[oe + 1])) : 0.f;
        const float wym = (j > 0) ? rcp_approx(ec + to_f(Es[oe - G::EW])) : 0.f;
        const float wyp = (j + 1 < d.ny) ? rcp_approx(ec + to_f(Es[oe + G::EW])) : 0.f;
        const float wzm = (k > 0) ? rcp_approx(ec + em) : 0.f;
        const bool top = (k + 1 == d.nz);
        const float wzt = top ? rcp_approx(ec) : rcp_approx(ec + ep);
        const float wzp = top ? 0.f : wzt;
        const float D = wxm + wxp + wym + wyp + wzm + wzt;
        float s = 0.f;
        if (i > 0) s += wxm * Ps[o - 1];
        if (i + 1 < d.nx) s += wxp * Ps[o + 1];
        if (j > 0) s += wym * Ps[o - G::VW];
        if (j + 1 < d.ny) s += wyp * Ps[o + G::VW];
        if (k > 0) s += wzm * pm;
        if (!top) s += wzp * pp;
        const float qv = D * pc - s;
        const int oc = ty * MTX + tx;
        const float xn = X(q)[oc] + alpha * pc;
        const float rn = R(q)[oc] - alpha * qv;
        const float zn = rn * rcp_approx(D);
        if (valid) {
            const int c = i + d.nx * (j + d.ny * k);
            x[c] = xn;
            r[c] = rn;
            z[c] = zn;
            arz += rn * zn;
            arr += rn * rn;
        }
        pm = pc;
        pc = pp;
        em = ec;
        ec = ep;
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

int march_smem_a(int ty, bool bf16) {
    switch (ty) {
        case 4: return NS * (bf16 ? Geo<4, __nv_bfloat16>::A_STAGE : Geo<4, float>::A_STAGE);
        case 8: return NS * (bf16 ? Geo<8, __nv_bfloat16>::A_STAGE : Geo<8, float>::A_STAGE);
        default: return NS * (bf16 ? Geo<16, __nv_bfloat16>::A_STAGE : Geo<16, float>::A_STAGE);
    }
}

int march_smem_b(int ty, bool bf16) {
    switch (ty) {
        case 4: return NS * (bf16 ? Geo<4, __nv_bfloat16>::B_STAGE : Geo<4, float>::B_STAGE);
        case 8: return NS * (bf16 ? Geo<8, __nv_bfloat16>::B_STAGE : Geo<8, float>::B_STAGE);
        default: return NS * (bf16 ? Geo<16, __nv_bfloat16>::B_STAGE : Geo<16, float>::B_STAGE);
    }
}

bool march_maps(MarchMaps* mm, const Dims& d, int ty, const float* z, const float* pa,
                const float* pb, const void* eta, bool bf16, const float* x, const float* r) {
    const int eoff = bf16 ? 8 : 4;
    const CUtensorMapDataType edt =
        bf16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
    bool ok = true;
    ok = ok && encode3d(&mm->z, z, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, d, MTX + 8, ty + 2);
    ok = ok && encode3d(&mm->pa, pa, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, d, MTX + 8, ty + 2);
    ok = ok && encode3d(&mm->pb, pb, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, d, MTX + 8, ty + 2);
    ok = ok && encode3d(&mm->eta, eta, edt, bf16 ? 2 : 4, d, MTX + 2 * eoff, ty + 2);
    ok = ok && encode3d(&mm->x, x, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, d, MTX, ty);
    ok = ok && encode3d(&mm->r, r, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, d, MTX, ty);
    mm->ty = ty;
    mm->bf16 = bf16;
    return ok;
}

template <int TY, typename E>
static void set_smem_attrs() {
    static std::once_flag once;
    std::call_once(once, [] {
        cudaFuncSetAttribute(k_march_a<TY, E>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             NS * Geo<TY, E>::A_STAGE);
        cudaFuncSetAttribute(k_march_b<TY, E>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             NS * Geo<TY, E>::B_STAGE);
    });
}

template <int TY, typename E>
static void launch_ab(const Dims& d, int kchunk, const MarchMaps& mm, bool a_side, bool p_is_a,
                      float* p_out, float* x, float* r, float* z, Scalars* sc, double* part,
                      cudaStream_t st) {
    set_smem_attrs<TY, E>();
    const dim3 grid((d.nx + MTX - 1) / MTX, (d.ny + TY - 1) / TY, (d.nz + kchunk - 1) / kchunk);
    const dim3 block(MTX, TY);
    if (a_side) {
        k_march_a<TY, E><<<grid, block, NS * Geo<TY, E>::A_STAGE, st>>>(
            d, kchunk, mm.z, p_is_a ? mm.pa : mm.pb, mm.eta, p_out, sc, part);
    } else {
        k_march_b<TY, E><<<grid, block, NS * Geo<TY, E>::B_STAGE, st>>>(
            d, kchunk, p_is_a ? mm.pa : mm.pb, mm.eta, mm.x, mm.r, x, r, z, sc, part);
    }
    g_kernel_launches.fetch_add(1, std::memory_order_relaxed);
}

template <typename E>
static void dispatch(const Dims& d, int kchunk, const MarchMaps& mm, bool a_side, bool p_is_a,
                     float* p_out, float* x, float* r, float* z, Scalars* sc, double* part,
                     cudaStream_t st) {
    switch (mm.ty) {
        case 4: launch_ab<4, E>(d, kchunk, mm, a_side, p_is_a, p_out, x, r, z, sc, part, st); break;
        case 8: launch_ab<8, E>(d, kchunk, mm, a_side, p_is_a, p_out, x, r, z, sc, part, st); break;
        default: launch_ab<16, E>(d, kchunk, mm, a_side, p_is_a, p_out, x, r, z, sc, part, st); break;
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

size_t march_blocks(const Dims& d, int ty, int kchunk) {
    return (size_t)((d.nx + MTX - 1) / MTX) * ((d.ny + ty - 1) / ty) * ((d.nz + kchunk - 1) / kchunk);
}

int march_occupancy(int ty, bool bf16, bool a_side) {
    int n = 0;
    const int smem = a_side ? march_smem_a(ty, bf16) : march_smem_b(ty, bf16);
    const void* f = nullptr;
#define PICK(T)                                                                         \
    if (ty == T) {                                                                      \
        if (bf16) {                                                                     \
            set_smem_attrs<T, __nv_bfloat16>();                                        \
            f = a_side ? (const void*)k_march_a<T, __nv_bfloat16>                       \
                       : (const void*)k_march_b<T, __nv_bfloat16>;                      \
        } else {                                                                        \
            set_smem_attrs<T, float>();                                                 \
            f = a_side ? (const void*)k_march_a<T, float> : (const void*)k_march_b<T, float>; \
        }                                                                               \
    }
    PICK(4) PICK(8) PICK(16)
#undef PICK
    if (!f || cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, f, MTX * ty, smem) != cudaSuccess) {
        cudaGetLastError();
        return 1;
    }
    return n > 0 ? n : 1;
}

}  // namespace pcg

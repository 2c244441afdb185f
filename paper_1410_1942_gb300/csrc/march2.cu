// march2.cu -- the FP32 inner PCG in one sweep per iteration with BOTH matrix products formed in
// the sweep: A p directly (instead of the recurrence s^ = w^ + beta s^) and A u'.  Only u, p, x
// and eta live in memory, so a sweep moves 24 bytes per cell on average.
//
// The scalar recurrences are those of the Chronopoulos-Gear form (march1.cu): with M = D,
//   p   = u + beta p                    s^ = D^-1 A p       (formed, not stored)
//   x  += alpha p                       u' = u - alpha s^
//   gamma' = (D u', u'),  delta' = (A u', u'),  rho' = |D u'|^2     (one reduction)
//   beta'  = gamma' / gamma,  alpha' = gamma' / (delta' - beta' gamma' / alpha)
// A sweep reads u, p (2-cell halo boxes), eta (2-cell halo) and writes u', p: 20 B per cell, plus
// x read and written every other iteration (4 B on average; an odd iteration stores
// x_{i+1} = x_{i-1} + alpha_{i-1} p_{i-1} + alpha_i p_i).  u and p are double buffered.
//
// Per plane the kernel runs two staggered stencils.  Stage 1 at plane m: p = u + beta p_old on the
// tile and a 2-cell ring (pointwise from the boxes), A p and D on the tile and its 1-cell ring,
// u' = u - alpha (A p) / D there; u' of the plane goes to a shared-memory plane buffer (three
// buffers in rotation).  Stage 2 at plane m - 1: A u' on the tile, from the buffer (in-plane
// neighbours) and the thread's own u' of planes m - 2, m - 1, m (registers).  A segment over
// planes [k0, k1) streams planes k0 - 2 .. k1 + 1.  A ring cell's u' is computed by the CTA that
// needs it with the same per-cell arithmetic (explicit FMAs, one order) as by the CTA that owns
// it, so every CTA sees the same u'.  Cells outside the grid (ragged tiles, planes below 0 or at
// nz and above) get u' = 0 and face coefficient 0.
//
// The first sweep of a launch runs with alpha = beta = 0 (u = D^-1 r from the init kernel, p = 0):
// it forms A u for the first delta.  Work list, roles (TMA producer warp + TYT consumer warps),
// bounded waits, float-float reductions and the finishing protocol are those of march1.cu.
#include "march_dev.cuh"

#include <cudaTypedefs.h>

namespace pcg {

template <int CX, int CY, int TYT, typename E>
struct Geo2 {
    static constexpr int W = 32 * CX;
    static constexpr int HT = CY * TYT;
    static constexpr int VOFF = 4;               // FP32 halo in x (16 bytes; >= 2 cells)
    static constexpr int VW = W + 2 * VOFF;
    static constexpr int EOFF = EtaX<E>::OFF;
    static constexpr int EW = W + 2 * EOFF;
    static constexpr int H2 = HT + 4;            // 2-cell halo in y
    static constexpr int VB = VW * H2 * 4;
    static constexpr int EB = EW * H2 * (int)sizeof(E);
    static constexpr int CB = W * HT * 4;
    // stage: u | p_old (2-halo boxes) | eta (2-halo box) | x (centre box, odd iterations)
    static constexpr int U = 0, P = align128(VB), ETA = 2 * align128(VB);
    static constexpr int X = ETA + align128(EB);
    static constexpr int STAGE = X + align128(CB);
    static constexpr int TX_NOX = 2 * VB + EB;
    static constexpr int TX_X = TX_NOX + CB;
    // u' plane buffers: the tile and its 1-cell ring
    static constexpr int BW = W + 2, BH = HT + 2, BN = BW * BH;
    static constexpr int RING = 2 * W + 2 * HT;  // ring cells that touch the tile through a face
};

struct LocalSolve2 {
    Dims d;
    float *x, *u[2], *p[2];
    Scalars* sc;
    int seg_begin, seg_end;
    double gamma, alpha, beta, rr, stop2, alpha_prev;
    int done, iter, max_iter, finished, owner, first, xfix;
};

__device__ __forceinline__ bool x_sweep2(const LocalSolve2& L) { return !L.first && (L.iter & 1); }

// Face coefficients of one cell and its diagonal.  zt is the z+ term of the diagonal: the
// Dirichlet top term 1/eta_c on the last layer, else the z+ face.
struct Faces {
    float xm, xp, ym, yp, zm, zp, zt;
};

__device__ __forceinline__ float diag_of(const Faces& f) {
    return __fadd_rn(__fadd_rn(__fadd_rn(__fadd_rn(__fadd_rn(f.xm, f.xp), f.ym), f.yp), f.zm), f.zt);
}

// (A v)_c = D v_c - sum_f w_f v_f, accumulated in one fixed order
__device__ __forceinline__ float apply_cell(const Faces& f, float D, float c, float xm, float xp,
                                            float ym, float yp, float zm, float zp) {
    float s = __fmul_rn(f.xm, xm);
    s = __fmaf_rn(f.xp, xp, s);
    s = __fmaf_rn(f.ym, ym, s);
    s = __fmaf_rn(f.yp, yp, s);
    s = __fmaf_rn(f.zm, zm, s);
    s = __fmaf_rn(f.zp, zp, s);
    return __fmaf_rn(D, c, -s);
}

__device__ __forceinline__ float face(bool open, float a, float b) {
    return open ? rcp_approx(__fadd_rn(a, b)) : 0.f;
}

template <int CX, int CY, int TYT, typename E, int NS>
__global__ void __launch_bounds__(32 * (TYT + 1), WsMinBlocks<TYT>::value) k_cg2_ws(PcgArgs a) {
    using G = Geo2<CX, CY, TYT, E>;
    constexpr int NT = 32 * (TYT + 1);
    constexpr int NC = 32 * TYT;
    extern __shared__ __align__(128) unsigned char sm[];
    __shared__ __align__(8) uint64_t full[NS];
    __shared__ __align__(8) uint64_t empty[NS];
    __shared__ double red[64];
    __shared__ Seg s_seg[MAXSEG];
    __shared__ LocalSolve2 s_sol[MAXSEG];
    __shared__ int s_member[MAXSEG];
    __shared__ volatile int s_fail;
    __shared__ float ubuf[3][G::BN];
    const int tx = threadIdx.x, ty = threadIdx.y, tid = tx + 32 * ty;
    const bool producer = (ty == TYT);
    const int sb = a.cta_seg[blockIdx.x];
    const int nseg = min(MAXSEG, a.cta_seg[blockIdx.x + 1] - sb);
    if (tid < nseg) s_seg[tid] = a.segs[sb + tid];
    if (tid == 0) {
        for (int s = 0; s < NS; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], TYT);
        }
        fence_mbar_init();
        s_fail = 0;
    }
    __syncthreads();
    const int first = nseg ? s_seg[0].solve : 0;
    const int nloc = nseg ? s_seg[nseg - 1].solve - first + 1 : 0;
    if (tid < nloc) {
        const SolveDev& sv = a.solves[first + tid];
        LocalSolve2& L = s_sol[tid];
        L.d = sv.d;
        L.x = sv.x;
        L.u[0] = sv.z;
        L.u[1] = sv.sa;
        L.p[0] = sv.pa;
        L.p[1] = sv.pb;
        L.sc = sv.sc;
        L.seg_begin = sv.seg_begin;
        L.seg_end = sv.seg_end;
        L.gamma = sv.sc->rz;
        L.rr = sv.sc->rr;
        L.stop2 = sv.sc->stop2;
        L.alpha = 0.0;
        L.alpha_prev = 0.0;
        L.beta = 0.0;
        L.done = sv.sc->done;
        L.iter = 0;
        L.max_iter = sv.sc->max_iter;
        L.finished = 0;
        L.first = 1;
        L.xfix = 0;
        L.owner = 0;
        for (int q = 0; q < nseg; ++q)
            if (s_seg[q].slot == sv.seg_begin) L.owner = 1;
        s_member[tid] = (L.done == RUNNING);
    }
    __syncthreads();

    const int warp = ty, lane = tx;
    auto stage = [&](int q) { return sm + (q % NS) * G::STAGE; };
    int np = 0;  // planes issued (producer lane 0)
    int nc = 0;  // planes acquired (each consumer warp)

    // in: the buffer (0 or 1) of u and p read by this sweep
    auto produce = [&](int in) {
        for (int ls = 0; ls < nseg; ++ls) {
            const Seg& sg = s_seg[ls];
            if (!s_member[sg.solve - first]) continue;
            const int L = sg.k1 - sg.k0;
            const CUtensorMap* m = a.maps + MAPS_PER_SOLVE * sg.solve;
            const bool xs = x_sweep2(s_sol[sg.solve - first]);
            for (int off = 0; off < L + 4; ++off) {
                if (s_fail) return;
                const int st = np % NS, kk = sg.k0 - 2 + off;
                if (np >= NS && !mbar_wait_or(&empty[st], ((np / NS) - 1) & 1, &s_fail)) {
                    s_fail = 1;
                    return;
                }
                unsigned char* dst = sm + st * G::STAGE;
                const bool centre = kk >= sg.k0 && kk < sg.k1;
                uint64_t* bar = &full[st];
                mbar_arrive_expect_tx(bar, (centre && xs) ? G::TX_X : G::TX_NOX);
                tma_load_3d(dst + G::U, m + MAP2_U0 + in, bar, sg.x0 - G::VOFF, sg.y0 - 2, kk);
                tma_load_3d(dst + G::P, m + MAP2_P0 + in, bar, sg.x0 - G::VOFF, sg.y0 - 2, kk);
                tma_load_3d(dst + G::ETA, m + MAP2_ETA, bar, sg.x0 - G::EOFF, sg.y0 - 2, kk);
                if (centre && xs) tma_load_3d(dst + G::X, m + MAP2_X, bar, sg.x0, sg.y0, kk);
                ++np;
            }
        }
    };

    auto consume = [&](int in) {
        auto acquire = [&]() -> bool {
            const int q = nc++;
            if (s_fail) return false;
            if (!mbar_wait_or(&full[q % NS], (q / NS) & 1, &s_fail)) {
                s_fail = 1;
                return false;
            }
            return true;
        };
        auto release = [&](int q) {
            __syncwarp();
            if (lane == 0) mbar_arrive(&empty[q % NS]);
        };
        const int out = in ^ 1;
        for (int ls = 0; ls < nseg; ++ls) {
            const Seg sg = s_seg[ls];
            const int l = sg.solve - first;
            if (!s_member[l]) continue;
            const bool work = s_sol[l].done == RUNNING;
            const Dims d = s_sol[l].d;
            const float al = (float)s_sol[l].alpha, be = (float)s_sol[l].beta;
            const float alp = (float)s_sol[l].alpha_prev;
            const bool xs = x_sweep2(s_sol[l]);
            const int p0 = nc;  // stream position of plane k0 - 2
            // tile coordinates -> shared-memory offsets of a stage
            auto vidx = [&](int xx, int yy) { return (yy + 2) * G::VW + xx + G::VOFF; };
            auto eidx = [&](int xx, int yy) { return (yy + 2) * G::EW + xx + G::EOFF; };
            auto U_of = [&](int q) { return (const float*)(stage(q) + G::U); };
            auto P_of = [&](int q) { return (const float*)(stage(q) + G::P); };
            auto E_of = [&](int q) { return (const E*)(stage(q) + G::ETA); };
            // p_i = u + beta p_old at tile coordinates of stream position q
            auto pv = [&](int q, int xx, int yy) {
                const int o = vidx(xx, yy);
                return __fmaf_rn(be, P_of(q)[o], U_of(q)[o]);
            };
            auto ev = [&](int q, int xx, int yy) { return ld1(E_of(q) + eidx(xx, yy)); };
            auto inside = [&](int xx, int yy, int k) {
                const int i = sg.x0 + xx, j = sg.y0 + yy;
                return i >= 0 && i < d.nx && j >= 0 && j < d.ny && k >= 0 && k < d.nz;
            };
            // Stage 1 for one cell at tile coordinates (xx, yy) of plane m (stream position q,
            // planes m-1, m+1 at q-1, q+1): u' = u - alpha (A p)/D, and D.  0 outside the grid.
            auto unew_cell = [&](int q, int m, int xx, int yy, float* Dout) -> float {
                if (!inside(xx, yy, m)) {
                    if (Dout) *Dout = 0.f;
                    return 0.f;
                }
                const int i = sg.x0 + xx, j = sg.y0 + yy;
                const float ec = ev(q, xx, yy);
                Faces f;
                // a Dirichlet wall's face: the halo beyond the grid is zero-filled (eta = 0)
                f.xm = face(i > 0 || (d.walls & 1), ec, ev(q, xx - 1, yy));
                f.xp = face(i + 1 < d.nx || (d.walls & 2), ec, ev(q, xx + 1, yy));
                f.ym = face(j > 0 || (d.walls & 4), ec, ev(q, xx, yy - 1));
                f.yp = face(j + 1 < d.ny || (d.walls & 8), ec, ev(q, xx, yy + 1));
                f.zm = face(m > 0 || (d.walls & 16), ec, ev(q - 1, xx, yy));
                f.zp = face(m + 1 < d.nz, ec, ev(q + 1, xx, yy));
                f.zt = (m + 1 == d.nz) ? rcp_approx(ec) : f.zp;
                const float D = diag_of(f);
                const float Ap = apply_cell(f, D, pv(q, xx, yy), pv(q, xx - 1, yy), pv(q, xx + 1, yy),
                                            pv(q, xx, yy - 1), pv(q, xx, yy + 1), pv(q - 1, xx, yy),
                                            pv(q + 1, xx, yy));
                if (Dout) *Dout = D;
                return __fmaf_rn(-al, __fmul_rn(Ap, rcp_approx(D)), U_of(q)[vidx(xx, yy)]);
            };
            // the thread's own cells and its share of the ring
            const int ox = CX * tx, oy = CY * warp;
            auto ring_xy = [&](int e, int& xx, int& yy) {
                if (e < G::W) { xx = e; yy = -1; }
                else if (e < 2 * G::W) { xx = e - G::W; yy = G::HT; }
                else if (e < 2 * G::W + G::HT) { xx = -1; yy = e - 2 * G::W; }
                else { xx = G::W; yy = e - 2 * G::W - G::HT; }
            };
            auto bidx = [&](int xx, int yy) { return (yy + 1) * G::BW + xx + 1; };
            // Stage 1 at plane m (stream position q): own u' into uo and the plane buffer of m,
            // then the thread's ring cells into the buffer.
            auto stage1 = [&](int q, int m, float (&uo)[CY][CX]) {
                float* B = ubuf[(m + 3) % 3];
#pragma unroll
                for (int y = 0; y < CY; ++y)
#pragma unroll
                    for (int x = 0; x < CX; ++x) {
                        uo[y][x] = unew_cell(q, m, ox + x, oy + y, nullptr);
                        B[bidx(ox + x, oy + y)] = uo[y][x];
                    }
                for (int e = tid; e < G::RING; e += NC) {
                    int xx, yy;
                    ring_xy(e, xx, yy);
                    B[bidx(xx, yy)] = unew_cell(q, m, xx, yy, nullptr);
                }
            };
            float ukm1[CY][CX], uk[CY][CX], ukp1[CY][CX];  // own u' of planes k-1, k, k+1
            float wzl[CY][CX];                             // own faces to plane k-1 (stage 2)
            float ag = 0.f, ad = 0.f, ar = 0.f;
            // Stage 2 at plane k (stream position q; plane k+1 at q+1): A u' on the own cells,
            // the partial sums, and the stores of p, u' (and x on odd iterations) at plane k.
            auto stage2 = [&](int q, int k) {
                const float* B = ubuf[(k + 3) % 3];
#pragma unroll
                for (int y = 0; y < CY; ++y) {
                    const int j = sg.y0 + oy + y;
                    float pn[CX], uo[CX], xn[CX];
#pragma unroll
                    for (int x = 0; x < CX; ++x) {
                        const int xx = ox + x, yy = oy + y;
                        const int i = sg.x0 + xx;
                        const float ec = ev(q, xx, yy);
                        Faces f;
                        f.xm = face(i > 0 || (d.walls & 1), ec, ev(q, xx - 1, yy));
                        f.xp = face(i + 1 < d.nx || (d.walls & 2), ec, ev(q, xx + 1, yy));
                        f.ym = face(j > 0 || (d.walls & 4), ec, ev(q, xx, yy - 1));
                        f.yp = face(j + 1 < d.ny || (d.walls & 8), ec, ev(q, xx, yy + 1));
                        f.zm = wzl[y][x];
                        f.zp = face(k + 1 < d.nz, ec, ev(q + 1, xx, yy));
                        f.zt = (k + 1 == d.nz) ? rcp_approx(ec) : f.zp;
                        wzl[y][x] = f.zp;
                        const float D = diag_of(f);
                        const float c = uk[y][x];
                        const float Au = apply_cell(f, D, c, B[bidx(xx - 1, yy)], B[bidx(xx + 1, yy)],
                                                    B[bidx(xx, yy - 1)], B[bidx(xx, yy + 1)],
                                                    ukm1[y][x], ukp1[y][x]);
                        const int o = vidx(xx, yy);
                        const float pold = P_of(q)[o];
                        pn[x] = __fmaf_rn(be, pold, U_of(q)[o]);
                        uo[x] = c;
                        if (xs) {
                            const float xo = ((const float*)(stage(q) + G::X))[yy * G::W + xx];
                            xn[x] = __fmaf_rn(al, pn[x], __fmaf_rn(alp, pold, xo));
                        }
                        if (i < d.nx && j < d.ny) {
                            const float du = __fmul_rn(D, c);
                            ag = __fmaf_rn(du, c, ag);
                            ad = __fmaf_rn(Au, c, ad);
                            ar = __fmaf_rn(du, du, ar);
                        }
                    }
                    if (j < d.ny && sg.x0 + ox < d.nx) {
                        const size_t cidx =
                            (size_t)(sg.x0 + ox) + (size_t)d.nx * ((size_t)j + (size_t)d.ny * k);
                        st_row<CX>(s_sol[l].p[out] + cidx, pn);
                        st_row<CX>(s_sol[l].u[out] + cidx, uo);
                        if (xs) st_row<CX>(s_sol[l].x + cidx, xn);
                    }
                }
            };

            // planes k0-2, k0-1, k0 in; stage 1 at k0-1 (its planes k0-2 .. k0)
            bool ok = acquire();
            ok = acquire() && ok;
            ok = acquire() && ok;
            if (ok && work) stage1(p0 + 1, sg.k0 - 1, uk);
            release(p0);  // plane k0-2
            for (int m = sg.k0; m <= sg.k1; ++m) {
                const int q = p0 + (m - sg.k0) + 2;  // stream position of plane m
                ok = acquire() && ok;                // plane m+1
                if (ok && work) {
                    if (m == sg.k0) {
                        // own faces between planes k0-1 and k0 for the first stage 2
#pragma unroll
                        for (int y = 0; y < CY; ++y)
#pragma unroll
                            for (int x = 0; x < CX; ++x)
                                wzl[y][x] = face(sg.k0 > 0 || (d.walls & 16), ev(q, ox + x, oy + y),
                                                 ev(q - 1, ox + x, oy + y));
                    }
                    stage1(q, m, ukp1);
                }
                named_sync(1, NC);  // the plane buffer of m is complete (and m-2's is free)
                if (ok && work) {
                    if (m > sg.k0) stage2(q - 1, m - 1);
#pragma unroll
                    for (int y = 0; y < CY; ++y)
#pragma unroll
                        for (int x = 0; x < CX; ++x) {
                            ukm1[y][x] = uk[y][x];
                            uk[y][x] = ukp1[y][x];
                        }
                }
                release(q - 1);  // plane m-1
            }
            release(p0 + (sg.k1 - sg.k0) + 2);  // plane k1
            release(p0 + (sg.k1 - sg.k0) + 3);  // plane k1+1
            // the segment's partial sums (gamma, delta, rho), over the consumer warps
            const float v[3] = {ag, ad, ar};
            segment_partials<3>(v, a.part_b + 3 * (size_t)s_seg[ls].slot, reinterpret_cast<ff*>(red),
                                tid, NC, 1);
        }
    };

    unsigned nbar = 0;
    int alive = 0;  // unfinished solves of the launch as of the last grid barrier
    // unfinished solves this CTA owns (thread 0 adds them at every grid barrier)
    auto owned_running = [&]() {
        int c = 0;
        for (int l = 0; l < nloc; ++l) c += (s_sol[l].owner && s_sol[l].done == RUNNING) ? 1 : 0;
        return c;
    };
    int in = 0;
    bool failed = false;
    const bool tr = a.trace && blockIdx.x == 0 && tid == 0;
    unsigned long long tt[TRACE_PARTS] = {};
    unsigned long long tprev = tr ? globaltimer() : 0;
    auto mark = [&](int part) {
        if (tr) {
            const unsigned long long t = globaltimer();
            tt[part] += t - tprev;
            tprev = t;
        }
    };
    for (;;) {
        if (producer) {
            if (lane == 0) produce(in);
            __syncwarp();
        } else {
            consume(in);
        }
        __syncthreads();
        mark(TR_A);
        if (s_fail) { failed = true; break; }
        ++nbar;
        if (!grid_barrier(a.ctl, nbar, nbar * (unsigned)a.nctas, tid, owned_running(), &alive)) {
            failed = true;
            break;
        }
        mark(TR_BAR1);
        if (alive == 0) break;
        for (int l = 0; l < nloc; ++l) {
            if (s_sol[l].done != RUNNING) continue;
            double t[3];
            // SM cycles (the globaltimer's granularity is too coarse for these parts)
            const long long t_s0 = tr ? clock64() : 0;
            range_sum<3>(a.part_b, s_sol[l].seg_begin, s_sol[l].seg_end, t, reinterpret_cast<ff*>(red),
                         tid, NT);
            const long long t_s1 = tr ? clock64() : 0;
            if (tid == 0) {
                LocalSolve2& L = s_sol[l];
                const double gn = t[0], dn = t[1], rn = t[2];
                L.rr = rn;
                if (!isfinite(gn) || !isfinite(dn) || !isfinite(rn) || gn < 0.0) {
                    L.done = BREAKDOWN;
                } else if (L.first) {
                    // the start-up sweep: A u formed, no iterate changed
                    L.first = 0;
                    L.gamma = gn;
                    if (rn <= L.stop2) L.done = CONVERGED;
                    else if (!(dn > 0.0)) L.done = BREAKDOWN;
                    else {
                        L.alpha = gn / dn;
                        L.beta = 0.0;
                    }
                } else {
                    const bool x_updated = (L.iter & 1) != 0;  // this sweep wrote x_{i+1}
                    L.iter += 1;
                    if (rn <= L.stop2) {
                        L.done = CONVERGED;
                    } else if (L.iter >= L.max_iter) {
                        L.done = CAPPED;
                    } else {
                        const double be = gn / L.gamma;
                        const double den = dn - be * gn / L.alpha;
                        if (!(den > 0.0) || !isfinite(den)) {
                            L.done = BREAKDOWN;
                        } else {
                            L.beta = be;
                            L.alpha_prev = L.alpha;
                            L.alpha = gn / den;
                            L.gamma = gn;
                        }
                    }
                    if (L.done != RUNNING && !x_updated) L.xfix = 1;
                }
                if (L.done != RUNNING) L.finished = 1;
            }
            if (tr) {
                const long long t_s2 = clock64();
                tt[TR_SUM] += (unsigned long long)(t_s1 - t_s0);
                tt[TR_DECIDE] += (unsigned long long)(t_s2 - t_s1);
            }
            __syncthreads();
        }
        // Solves that stopped after an even iteration: x_{i+1} = x_i + alpha_i p_i over this CTA's
        // cells of the solve (p_i is what this CTA stored in the sweep just done).
        bool any_fix = false;
        for (int l = 0; l < nloc; ++l) any_fix = any_fix || s_sol[l].xfix;
        if (any_fix) {
            for (int ls = 0; ls < nseg; ++ls) {
                const Seg sg = s_seg[ls];
                const LocalSolve2& L = s_sol[sg.solve - first];
                if (!L.xfix) continue;
                const int nx = L.d.nx, ny = L.d.ny;
                const int wd = min(G::W, nx - sg.x0), ht = min(G::HT, ny - sg.y0);
                const int per = wd * ht;
                const long long cnt = (long long)per * (sg.k1 - sg.k0);
                const float al = (float)L.alpha;
                const float* pw = L.p[in ^ 1];
                for (long long q = tid; q < cnt; q += NT) {
                    const int k = sg.k0 + (int)(q / per), r = (int)(q % per);
                    const size_t c = (size_t)(sg.x0 + r % wd) +
                                     (size_t)nx * ((size_t)(sg.y0 + r / wd) + (size_t)ny * k);
                    L.x[c] = __fmaf_rn(al, pw[c], L.x[c]);
                }
            }
            __syncthreads();
            if (tid < nloc) s_sol[tid].xfix = 0;
        }
        mark(TR_ALPHA);
        if (tid < nloc) {
            LocalSolve2& L = s_sol[tid];
            if (L.finished) {
                L.finished = 0;
                if (L.owner) {
                    L.sc->iter = L.iter;
                    L.sc->rr = L.rr;
                    L.sc->rz = L.gamma;
                    L.sc->done = L.done;
                    __threadfence();
                }
            }
            s_member[tid] = (L.done == RUNNING);
        }
        __syncthreads();
        mark(TR_BETA);
        if (tr) tt[TR_ITERS] += 1;
        in ^= 1;
    }
    if (tr)
        for (int q = 0; q < TRACE_PARTS; ++q) a.trace[q] += tt[q];
    if (failed) {
        if (tid == 0) {
            atomicExch(&a.ctl->error, 1);
            for (int l = 0; l < nloc; ++l) {
                s_sol[l].sc->iter = s_sol[l].iter;
                atomicExch(&s_sol[l].sc->done, (int)TIMEDOUT);
            }
        }
        if (producer && lane == 0) {
            // only the last NS planes can still be in flight
            for (int q = max(0, np - NS); q < np; ++q) (void)mbar_wait(&full[q % NS], (q / NS) & 1);
        }
        __threadfence();
        __syncthreads();
    }
}

template <int CX, int CY, int TYT, int NS>
static Cg1Kernel cg2_of() {
    return Cg1Kernel{(const void*)k_cg2_ws<CX, CY, TYT, float, NS>,
                     (const void*)k_cg2_ws<CX, CY, TYT, __nv_bfloat16, NS>,
                     NS * Geo2<CX, CY, TYT, float>::STAGE,
                     NS * Geo2<CX, CY, TYT, __nv_bfloat16>::STAGE};
}

Cg1Kernel cg2_kernel(int cx, int cy, int tyt, int ns) {
#define CG2_ROW(CX, CY, TYT, NS) \
    if (cx == CX && cy == CY && tyt == TYT && ns == NS) return cg2_of<CX, CY, TYT, NS>();
    CG2_CONFIGS(CG2_ROW)
#undef CG2_ROW
    return Cg1Kernel{nullptr, nullptr, 0, 0};
}

}  // namespace pcg

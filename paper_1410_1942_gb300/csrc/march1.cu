// march1.cu -- the FP32 inner PCG with ONE sweep over the grid and ONE grid barrier per
// iteration: the Chronopoulos-Gear form of Jacobi-preconditioned CG, as a persistent TMA
// plane-marching kernel.
//
// Standard PCG (Section 3.2's pressure solve) needs two global reductions per iteration, p.Ap
// before the update of x and r and r.z after it, and so two passes over the grid with a grid
// barrier after each (march.cu).  The Chronopoulos-Gear recurrences reach the same iterates in
// exact arithmetic with both inner products taken in the same pass.  With M = D (Jacobi), keep
// the preconditioned vectors u = M^-1 r, s^ = M^-1 A p and w^ = M^-1 A u instead of r, A p, A u:
//
//   p     = u + beta p             s^ = w^ + beta s^
//   x    += alpha p                u' = u - alpha s^        (= M^-1 (r - alpha A p))
//   w^'   = M^-1 A u'
//   gamma' = (D u', u'),  delta' = (A u', u'),  rho' = |D u'|^2     (one reduction)
//   beta'  = gamma' / gamma,  alpha' = gamma' / (delta' - beta' gamma' / alpha)
//
// A sweep reads p, u, s^, w^ and eta and writes p, u', s^, w^' (36 bytes per cell); x is read
// and written every other iteration only: an even iteration i leaves x_i in memory and an odd one
// stores x_{i+1} = x_{i-1} + alpha_{i-1} p_{i-1} + alpha_i p_i from the p it reads and the p it
// forms, so x costs 4 bytes per cell-iteration and a sweep 40 on average (44 for the two passes
// of the standard form).  A solve that stops after an even iteration adds alpha_i p_i to x in a
// short pass over its own cells.  The neighbours of a cell's u' are
// formed from the neighbours' u, s^, w^ (halo boxes of the plane), so u, s^ and w^ are double
// buffered (a CTA writes u' while its neighbours still read u).  The first sweep of a launch has
// alpha = beta = 0 (u = M^-1 r from the init kernel, s^ = w^ = p = 0): it only forms w^ = M^-1 A u
// and the first gamma and delta.  Each cell's u' is evaluated with explicit fused multiply-adds
// in the same order wherever it is needed, so every CTA sees the same u'.
//
// Work list, CTA roles (a TMA producer warp and TYT consumer warps), bounded waits, fixed-order
// reductions and the finishing protocol are those of k_pcg_ws (march.cu).
#include "march_dev.cuh"

#include <cudaTypedefs.h>

namespace pcg {

template <int CX, int CY, int TYT, typename E>
struct Geo1 {
    static constexpr int W = 32 * CX;
    static constexpr int HT = CY * TYT;
    static constexpr int VOFF = 4;
    static constexpr int VW = W + 2 * VOFF;
    static constexpr int EOFF = EtaX<E>::OFF;
    static constexpr int EW = W + 2 * EOFF;
    static constexpr int H = HT + 2;
    static constexpr int VB = VW * H * 4;
    static constexpr int EB = EW * H * (int)sizeof(E);
    static constexpr int CB = W * HT * 4;
    // stage: u | s^ | w^ (halo boxes) | eta (halo box) | x | p (centre boxes)
    static constexpr int U = 0, S = align128(VB), WV = 2 * align128(VB), ETA = 3 * align128(VB);
    static constexpr int X = ETA + align128(EB), P = X + align128(CB);
    static constexpr int STAGE = P + align128(CB);
    static constexpr int TX_HALO = 3 * VB + EB;  // planes k0-1 and k1: no x, p
    static constexpr int TX = TX_HALO + 2 * CB;
};

struct LocalSolve1 {
    Dims d;
    float *x, *p, *u[2], *s[2], *w[2];
    Scalars* sc;
    int seg_begin, seg_end;
    double gamma, alpha, beta, rr, stop2;
    double alpha_prev;  // alpha of the previous iteration (odd iterations update x with it)
    double den;         // delta - beta gamma / alpha of the last iteration: (p, A p)
    int per;            // periodic x: u, s^, w^ and eta live in padded rows with ghost columns
    int nxp;            // row length of u, s^, w^ (nx + 2 PAD_V when periodic)
    double ginv[2];     // 1/gamma, by the parity of the grid barrier it was formed at
    int done, iter, max_iter, finished, owner, first;
    int xfix;           // stopped after an even iteration: x still lacks alpha p
};

// u' = u - alpha (w^ + beta s^), rounded the same way everywhere
__device__ __forceinline__ float u_next(float u, float s, float w, float al, float be) {
    return __fmaf_rn(-al, __fmaf_rn(be, s, w), u);
}

// Whether the coming sweep updates x: odd iterations (the start-up sweep and even iterations
// leave x as it is).
__device__ __forceinline__ bool x_sweep(const LocalSolve1& L) { return !L.first && (L.iter & 1); }

// PER: the solves have periodic x (padded rows with ghost columns); a separate instantiation so
// that the plain kernel carries none of it.
template <int CX, int CY, int TYT, typename E, int NS, bool PER>
__global__ void __launch_bounds__(32 * (TYT + 1), WsMinBlocks<TYT>::value) k_cg1_ws(PcgArgs a) {
    using G = Geo1<CX, CY, TYT, E>;
    constexpr int NT = 32 * (TYT + 1);
    constexpr int NC = 32 * TYT;
    extern __shared__ __align__(128) unsigned char sm[];
    __shared__ __align__(8) uint64_t full[NS];
    __shared__ __align__(8) uint64_t empty[NS];
    __shared__ double red[64];
    __shared__ Seg s_seg[MAXSEG];
    __shared__ LocalSolve1 s_sol[MAXSEG];
    __shared__ int s_member[MAXSEG];  // solve streamed in the coming sweep
    __shared__ int s_nextxs[MAXSEG];  // the coming sweep updates x (producer's copy)
    __shared__ volatile int s_fail;
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
        LocalSolve1& L = s_sol[tid];
        L.d = sv.d;
        L.x = sv.x;
        L.p = sv.pa;
        L.u[0] = sv.z;
        L.u[1] = sv.pb;
        L.s[0] = sv.sa;
        L.s[1] = sv.sb;
        L.w[0] = sv.wa;
        L.w[1] = sv.wb;
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
        L.per = (sv.d.walls & PERIODIC_X) ? 1 : 0;
        L.nxp = sv.d.nx + (L.per ? 2 * PAD_V : 0);
        L.owner = 0;
        for (int q = 0; q < nseg; ++q)
            if (s_seg[q].slot == sv.seg_begin) L.owner = 1;
        s_member[tid] = (L.done == RUNNING);
        s_nextxs[tid] = 0;  // the start-up sweep leaves x alone
    }
    __syncthreads();

    const int r0 = 1 + CY * ty, cv = G::VOFF + CX * tx, ce = G::EOFF + CX * tx, cc = CX * tx;
    const int warp = ty, lane = tx;
    auto stage = [&](int q) { return sm + (q % NS) * G::STAGE; };
    int np = 0;  // planes issued (producer lane 0)
    int nc = 0;  // planes acquired (each consumer warp)

    // in: the buffer (0 or 1) of u, s^, w^ read by this sweep
    auto produce = [&](int in) {
        for (int ls = 0; ls < nseg; ++ls) {
            const Seg& sg = s_seg[ls];
            if (!s_member[sg.solve - first]) continue;
            const int L = sg.k1 - sg.k0;
            const CUtensorMap* m = a.maps + MAPS_PER_SOLVE * sg.solve;
            const bool xs = s_nextxs[sg.solve - first] != 0;
            // periodic x: the padded rows start PAD_V (eta: EOFF) columns before x = 0
            constexpr bool per = PER;
            const int xv = sg.x0 - G::VOFF + (per ? PAD_V : 0), xe = sg.x0 - G::EOFF + (per ? G::EOFF : 0);
            for (int off = 0; off < L + 2; ++off) {
                if (s_fail) return;
                const int st = np % NS, kk = sg.k0 - 1 + off;
                if (np >= NS && !mbar_wait_or(&empty[st], ((np / NS) - 1) & 1, &s_fail)) {
                    s_fail = 1;
                    return;
                }
                unsigned char* dst = sm + st * G::STAGE;
                const bool centre = off > 0 && off <= L;
                uint64_t* bar = &full[st];
                mbar_arrive_expect_tx(bar, centre ? (xs ? G::TX : G::TX - G::CB) : G::TX_HALO);
                tma_load_3d(dst + G::U, m + MAP1_U0 + in, bar, xv, sg.y0 - 1, kk);
                tma_load_3d(dst + G::S, m + MAP1_S0 + in, bar, xv, sg.y0 - 1, kk);
                tma_load_3d(dst + G::WV, m + MAP1_W0 + in, bar, xv, sg.y0 - 1, kk);
                tma_load_3d(dst + G::ETA, m + MAP1_ETA, bar, xe, sg.y0 - 1, kk);
                if (centre) {
                    if (xs) tma_load_3d(dst + G::X, m + MAP1_X, bar, sg.x0, sg.y0, kk);
                    tma_load_3d(dst + G::P, m + MAP1_P, bar, sg.x0, sg.y0, kk);
                }
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
            const bool xs = x_sweep(s_sol[l]);
            const int i0 = sg.x0 + CX * tx, j0 = sg.y0 + CY * warp;
            const unsigned edges = block_edges<CX, CY>(d, i0, j0);
            // u' of the thread's own block in plane q
            auto u_centre = [&](int q, float (&o)[CY][CX]) {
                const unsigned char* S = stage(q);
                float uu[CY][CX], ss[CY][CX], ww[CY][CX];
                load_centre<CX, CY>((const float*)(S + G::U), G::VW, r0, cv, uu);
                load_centre<CX, CY>((const float*)(S + G::S), G::VW, r0, cv, ss);
                load_centre<CX, CY>((const float*)(S + G::WV), G::VW, r0, cv, ww);
#pragma unroll
                for (int y = 0; y < CY; ++y)
#pragma unroll
                    for (int x = 0; x < CX; ++x) o[y][x] = u_next(uu[y][x], ss[y][x], ww[y][x], al, be);
            };
            auto eta_of = [&](int q) { return (const E*)(stage(q) + G::ETA); };
            float um[CY][CX], uc[CY][CX], em[CY][CX], ec[CY][CX], wzl[CY][CX];
            const int p0 = nc;
            bool ok = acquire();  // plane k0-1
            if (ok && work) {
                u_centre(p0, um);
                load_centre<CX, CY>(eta_of(p0), G::EW, r0, ce, em);
            }
            release(p0);
            ok = acquire();  // plane k0
            if (ok && work) {
                u_centre(p0 + 1, uc);
                load_centre<CX, CY>(eta_of(p0 + 1), G::EW, r0, ce, ec);
#pragma unroll
                for (int y = 0; y < CY; ++y)
#pragma unroll
                    for (int x = 0; x < CX; ++x)
                        wzl[y][x] = (sg.k0 > 0 || (d.walls & 16)) ? rcp_approx(ec[y][x] + em[y][x]) : 0.f;
            }
            float ag = 0.f, ad = 0.f, ar = 0.f;
            for (int k = sg.k0; k < sg.k1; ++k) {
                const int qc = p0 + 1 + (k - sg.k0), qn = qc + 1;
                ok = acquire();  // plane k+1
                if (ok && work) {
                    const unsigned char* S = stage(qc);
                    float up[CY][CX], ep[CY][CX];
                    u_centre(qn, up);
                    load_centre<CX, CY>(eta_of(qn), G::EW, r0, ce, ep);
                    // u' of the four neighbour strips in plane k
                    float vxm[CY], vxp[CY], vym[CX], vyp[CX];
                    {
                        float sxm[CY], sxp[CY], sym[CX], syp[CX];
                        float wxm[CY], wxp[CY], wym[CX], wyp[CX];
                        load_halo<CX, CY>((const float*)(S + G::U), G::VW, r0, cv, vxm, vxp, vym, vyp);
                        load_halo<CX, CY>((const float*)(S + G::S), G::VW, r0, cv, sxm, sxp, sym, syp);
                        load_halo<CX, CY>((const float*)(S + G::WV), G::VW, r0, cv, wxm, wxp, wym, wyp);
#pragma unroll
                        for (int y = 0; y < CY; ++y) {
                            vxm[y] = u_next(vxm[y], sxm[y], wxm[y], al, be);
                            vxp[y] = u_next(vxp[y], sxp[y], wxp[y], al, be);
                        }
#pragma unroll
                        for (int x = 0; x < CX; ++x) {
                            vym[x] = u_next(vym[x], sym[x], wym[x], al, be);
                            vyp[x] = u_next(vyp[x], syp[x], wyp[x], al, be);
                        }
                    }
                    float exm[CY], exq[CY], eym[CX], eyp[CX];
                    load_halo<CX, CY>(eta_of(qc), G::EW, r0, ce, exm, exq, eym, eyp);
                    float qv[CY][CX], D[CY][CX];
                    stencil<CX, CY>(d, edges, k, uc, vxm, vxp, vym, vyp, um, up, ec, exm, exq, eym,
                                    eyp, ep, wzl, qv, D);
                    if (i0 < d.nx) {
                        float u0[CY][CX], s0[CY][CX], w0[CY][CX], xo[CY][CX], po[CY][CX];
                        load_centre<CX, CY>((const float*)(S + G::U), G::VW, r0, cv, u0);
                        load_centre<CX, CY>((const float*)(S + G::S), G::VW, r0, cv, s0);
                        load_centre<CX, CY>((const float*)(S + G::WV), G::VW, r0, cv, w0);
                        if (xs) load_centre<CX, CY>((const float*)(S + G::X), G::W, CY * warp, cc, xo);
                        load_centre<CX, CY>((const float*)(S + G::P), G::W, CY * warp, cc, po);
#pragma unroll
                        for (int y = 0; y < CY; ++y) {
                            if (j0 + y < d.ny) {
                                float pn[CX], xn[CX], sn[CX], wn[CX];
#pragma unroll
                                for (int x = 0; x < CX; ++x) {
                                    pn[x] = __fmaf_rn(be, po[y][x], u0[y][x]);
                                    sn[x] = __fmaf_rn(be, s0[y][x], w0[y][x]);
                                    if (xs)
                                        xn[x] = __fmaf_rn(al, pn[x], __fmaf_rn(alp, po[y][x], xo[y][x]));
                                    wn[x] = qv[y][x] * rcp_approx(D[y][x]);
                                    const float du = D[y][x] * uc[y][x];
                                    ag += du * uc[y][x];
                                    ad += qv[y][x] * uc[y][x];
                                    ar += du * du;
                                }
                                const size_t c =
                                    (size_t)i0 + (size_t)d.nx * (j0 + y + (size_t)d.ny * k);
                                if (xs) st_row<CX>(s_sol[l].x + c, xn);
                                st_row<CX>(s_sol[l].p + c, pn);
                                const LocalSolve1& Ls = s_sol[l];
                                const size_t row = (size_t)(PER ? Ls.nxp : d.nx) *
                                                   (j0 + y + (size_t)d.ny * k);
                                const size_t cp = row + i0 + (PER ? PAD_V : 0);
                                st_row<CX>(Ls.u[out] + cp, uc[y]);
                                st_row<CX>(Ls.s[out] + cp, sn);
                                st_row<CX>(Ls.w[out] + cp, wn);
                                if (PER && (i0 < PAD_V || i0 >= d.nx - PAD_V)) {
                                    // the ghost copy at the other end of the padded row
                                    const long long cg = (long long)row + i0 + PAD_V +
                                                         (i0 < PAD_V ? d.nx : -d.nx);
                                    st_row<CX>(Ls.u[out] + cg, uc[y]);
                                    st_row<CX>(Ls.s[out] + cg, sn);
                                    st_row<CX>(Ls.w[out] + cg, wn);
                                }
                            }
                        }
                    }
#pragma unroll
                    for (int y = 0; y < CY; ++y)
#pragma unroll
                        for (int x = 0; x < CX; ++x) {
                            um[y][x] = uc[y][x];
                            uc[y][x] = up[y][x];
                            ec[y][x] = ep[y][x];
                        }
                }
                release(qc);
                if (k + 1 == sg.k1) release(qn);
            }
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
    // The producer streams the next sweep as soon as a grid barrier has passed, while the
    // consumers add the partial sums and decide; the next sweep's membership and x parity are
    // therefore fixed just before the barrier (a solve that stops at the coming decisions is
    // walked once more without arithmetic).
    if (producer && lane == 0) produce(in);
    for (;;) {
        if (!producer) consume(in);
        __syncthreads();  // the sweep is issued and consumed
        mark(TR_A);
        if (s_fail) { failed = true; break; }
        if (tid < nloc) {
            const LocalSolve1& L = s_sol[tid];
            s_member[tid] = (L.done == RUNNING);
            s_nextxs[tid] = L.first ? 0 : ((L.iter + 1) & 1);
        }
        ++nbar;
        if (!grid_barrier(a.ctl, nbar, nbar * (unsigned)a.nctas, tid, owned_running(), &alive,
                          a.trace != nullptr, tr ? &tt[TR_IMB] : nullptr,
                          tr ? &tt[TR_REL] : nullptr)) {
            failed = true;
            break;
        }
        mark(TR_BAR1);
        if (alive == 0) break;
        if (producer) {
            if (lane == 0) produce(in ^ 1);
            __syncwarp();
            in ^= 1;
            continue;
        }
        // consumers only from here on (named barrier 1 over NC threads)
        for (int l = 0; l < nloc; ++l) {
            if (s_sol[l].done != RUNNING) continue;
            double t[3];
            // SM cycles (the globaltimer's granularity is too coarse for these parts)
            const long long t_s0 = tr ? clock64() : 0;
            range_sum<3>(a.part_b, s_sol[l].seg_begin, s_sol[l].seg_end, t, reinterpret_cast<ff*>(red),
                         tid, NC, 1);
            const long long t_s1 = tr ? clock64() : 0;
            // 1/gamma for the next decision, off thread 0's path (another warp)
            if (tid == 32) s_sol[l].ginv[nbar & 1] = 1.0 / t[0];
            if (tid == 0) {
                LocalSolve1& L = s_sol[l];
                const double gn = t[0], dn = t[1], rn = t[2];
                L.rr = rn;
                if (!isfinite(gn) || !isfinite(dn) || !isfinite(rn) || gn < 0.0) {
                    L.done = BREAKDOWN;
                } else if (L.first) {
                    // the start-up sweep: w^ = M^-1 A u formed, no iterate changed
                    L.first = 0;
                    L.gamma = gn;
                    if (rn <= L.stop2) L.done = CONVERGED;
                    else if (!(dn > 0.0)) L.done = BREAKDOWN;
                    else {
                        L.den = dn;
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
                        // beta = gamma'/gamma; delta' - beta gamma'/alpha = delta' - beta^2 den
                        // (alpha = gamma/den): one division on this thread's path
                        const double be = gn * L.ginv[(nbar - 1) & 1];
                        const double den = fma(-be * be, L.den, dn);
                        if (!(den > 0.0) || !isfinite(den)) {
                            L.done = BREAKDOWN;
                        } else {
                            L.beta = be;
                            L.alpha_prev = L.alpha;
                            L.alpha = gn / den;
                            L.gamma = gn;
                            L.den = den;
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
            named_sync(1, NC);
        }
        // Solves that stopped after an even iteration: x_{i+1} = x_i + alpha_i p_i over this CTA's
        // cells of the solve (p_i is what this CTA stored in the sweep just done).
        bool any_fix = false;
        for (int l = 0; l < nloc; ++l) any_fix = any_fix || s_sol[l].xfix;
        if (any_fix) {
            for (int ls = 0; ls < nseg; ++ls) {
                const Seg sg = s_seg[ls];
                const LocalSolve1& L = s_sol[sg.solve - first];
                if (!L.xfix) continue;
                const int nx = L.d.nx, ny = L.d.ny;
                const int wd = min(G::W, nx - sg.x0), ht = min(G::HT, ny - sg.y0);
                const int per = wd * ht;
                const long long cnt = (long long)per * (sg.k1 - sg.k0);
                const float al = (float)L.alpha;
                for (long long q = tid; q < cnt; q += NC) {
                    const int k = sg.k0 + (int)(q / per), r = (int)(q % per);
                    const size_t c = (size_t)(sg.x0 + r % wd) +
                                     (size_t)nx * ((size_t)(sg.y0 + r / wd) + (size_t)ny * k);
                    L.x[c] = __fmaf_rn(al, L.p[c], L.x[c]);
                }
            }
            named_sync(1, NC);
            if (tid < nloc) s_sol[tid].xfix = 0;
        }
        mark(TR_ALPHA);
        if (tid < nloc) {
            LocalSolve1& L = s_sol[tid];
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
        }
        named_sync(1, NC);
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
static Cg1Kernel cg1_of() {
    return Cg1Kernel{(const void*)k_cg1_ws<CX, CY, TYT, float, NS, false>,
                     (const void*)k_cg1_ws<CX, CY, TYT, __nv_bfloat16, NS, false>,
                     NS * Geo1<CX, CY, TYT, float>::STAGE,
                     NS * Geo1<CX, CY, TYT, __nv_bfloat16>::STAGE,
                     (const void*)k_cg1_ws<CX, CY, TYT, float, NS, true>,
                     (const void*)k_cg1_ws<CX, CY, TYT, __nv_bfloat16, NS, true>};
}

Cg1Kernel cg1_kernel(int cx, int cy, int tyt, int ns) {
#define CG1_ROW(CX, CY, TYT, NS) \
    if (cx == CX && cy == CY && tyt == TYT && ns == NS) return cg1_of<CX, CY, TYT, NS>();
    CG1_CONFIGS(CG1_ROW)
#undef CG1_ROW
    return Cg1Kernel{nullptr, nullptr, 0, 0};
}

}  // namespace pcg

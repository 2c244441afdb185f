// march_rb.cu -- red-black SSOR (omega = 1) PCG as ONE persistent TMA plane-marching sweep and
// ONE grid barrier per iteration, on half the vector traffic of the Jacobi kernels.
//
// In red-black order (red = (i + j + k) even) the FP32 inner operator is
//     A = [ D_R  -C ]          (C: the face coefficients between red rows and black columns;
//         [ -C^T D_B ]          every neighbour of a red cell is black and vice versa)
// and the symmetric Gauss-Seidel preconditioner (SSOR with omega = 1, red first) is
// M = (D - L) D^-1 (D - L^T), L = [0 0; C^T 0].  Then M = A + [0 0; 0 C^T D_R^-1 C], and from a
// start whose red equations hold (r_R = 0) every PCG iterate keeps r_R = 0: with z = M^-1 r,
// z_B = D_B^-1 r_B and z_R = D_R^-1 C z_B, so each search direction p has (A p)_R = 0 and
// (A p)_B = S p_B with the Schur complement S = D_B - C^T D_R^-1 C; r.z = r_B.D_B^-1 r_B and
// p.Ap = p_B.S p_B.  The black parts of the SSOR-PCG iterates are therefore exactly the iterates
// of Jacobi-preconditioned CG on S x_B = b_B + C^T D_R^-1 b_R (Eisenstat's observation for
// red-black orderings), and the red parts follow as x_R = D_R^-1 (b_R + C x_B).  This file runs
// that CG:
//   k_rb_init   red relaxation d_R = r_R / D_R from d = 0, reduced right side
//               r^_B = r_B + C d_R, u = D_B^-1 r^_B, the other black vectors zeroed, |r|^2;
//   k_rb_ws     the persistent kernel: Chronopoulos-Gear CG on S with M_B = D_B (the form of
//               march1.cu, one reduction per iteration), vectors stored for black cells only;
//   k_rb_finish d_B = x_B, d_R = D_R^-1 (r_R + C x_B) into the full-size correction.
//
// Black vectors are compressed: row (j, k) holds its nx/2 black cells, black cell (i, j, k) at
// m = i / 2 (i = 2 m + ((j + k + 1) & 1)), index m + (nx/2) (j + ny k).  A sweep reads u, s^, w^,
// p and x (black only) and rho/2 of every cell, and writes u', s^, w^', p and x: per cell of the
// grid 10 half-cells of FP32 vectors plus eta, 24 bytes (22 with BF16 eta) against 40 for the
// Jacobi one-sweep kernel, at about half its iteration count.
//
// The consumer warps (TYT; a producer warp streams planes by TMA) do three steps per arriving
// plane q, each over the whole tile from shared memory, skewed by two planes so that one barrier
// per plane separates every write from its reads:
//   1. u' = u - alpha (w^ + beta s^) of plane q on the black cells of the tile and two rings;
//   2. t = D_r^-1 sum_faces beta u' of plane q-2 on the red cells of the tile and one ring;
//   3. S u' = D_b u' - sum_faces beta t of plane q-4 on the tile's black cells, then
//      p = u + beta p, s^ = w^ + beta s^, x += alpha p, w^' = D_b^-1 S u' and the three sums.
// u' and t live in shared memory compressed like the black vectors (a red cell (i, j, k) at
// m = i / 2 as well), so a warp's lanes, one per m, read neighbours at consecutive addresses: the
// x neighbours of a cell of parity bit c (i = 2m + c) sit at m - 1 + c and m + c of the other
// colour, its y and z neighbours at m.  Rings of 5 u' planes and 4 t planes; a segment of planes
// [k0, k1) streams planes k0-2 .. k1+1 and runs two more steps without a new plane.  Tiles whose
// cells and rings lie inside the grid in x and y take a stencil without boundary tests.  The
// faces are 1/(eta_c + eta_n) (eta = rho/2) formed on the fly as in the Jacobi kernels, so S is
// the Schur complement of the same inner operator.  Work list, producer/consumer roles, bounded
// waits, fixed-order float-float reductions and the finishing protocol are those of march1.cu.
#include "march_rb.h"

#include <cudaTypedefs.h>

#include "kernels.h"

namespace pcg {

template <int CX, int CY, int TYT, typename E>
struct GeoRB {
    static constexpr int W = 32 * CX;    // tile width (cells)
    static constexpr int WB = W / 2;     // black (and red) cells per tile row: one per lane
    static constexpr int HT = CY * TYT;  // tile height (rows)
    static constexpr int VOFF = 4;       // halo of the compressed boxes in x (16 bytes)
    static constexpr int VW = WB + 2 * VOFF;
    static constexpr int H = HT + 4;     // rows of the halo boxes: two each side
    static constexpr int EOFF = EtaX<E>::OFF;
    static constexpr int EW = W + 2 * EOFF;
    static constexpr int VB = VW * H * 4;
    static constexpr int EB = EW * H * (int)sizeof(E);
    static constexpr int CB = WB * HT * 4;
    // stage: u | s^ | w^ (compressed halo boxes) | eta (halo box) | x | p (compressed centre)
    static constexpr int U = 0, S = align128(VB), WV = 2 * align128(VB), ETA = 3 * align128(VB);
    static constexpr int X = ETA + align128(EB), P = X + align128(CB);
    static constexpr int STAGE = P + align128(CB);
    static constexpr int TX_HALO = 3 * VB + EB;  // planes outside [k0, k1): no x, p
    static constexpr int TX_P = TX_HALO + CB;    // a centre plane without x (start-up sweep)
    static constexpr int TX = TX_HALO + 2 * CB;
    // compressed on-chip planes: u' at m = x0/2 - 2 .. x0/2 + WB + 1 on rows y0 - 2 .. y0 + HT + 1;
    // t at m = x0/2 - 1 .. x0/2 + WB on rows y0 - 1 .. y0 + HT
    static constexpr int UC = WB + 4, UR = HT + 4, UPL = UC * UR, RINGU = 5;
    static constexpr int TC = WB + 2, TR = HT + 2, TPL = TC * TR, RINGT = 4;
    static constexpr int ON_CHIP = (RINGU * UPL + RINGT * TPL) * 4;
};

struct LocalSolveRB {
    Dims d;
    float *x, *p, *u[2], *s[2], *w[2];
    Scalars* sc;
    int seg_begin, seg_end;
    double gamma, alpha, beta, rr, stop2;
    double den;      // delta - beta gamma / alpha of the last iteration: (p, S p)
    double ginv[2];  // 1/gamma, by the parity of the grid barrier it was formed at
    int done, iter, max_iter, finished, owner, first;
};

__device__ __forceinline__ float u_next_rb(float u, float s, float w, float al, float be) {
    return __fmaf_rn(-al, __fmaf_rn(be, s, w), u);
}

__device__ __forceinline__ int ring(int k, int n) { return (k + 4 * n) % n; }

// The faces and diagonal of a cell whose x and y neighbours are all inside the grid (the
// expressions of eta_stencil with its x and y tests dropped; the z tests are uniform per plane).
__device__ __forceinline__ void eta_stencil_inner(const Dims& d, int k, float ec, float exm,
                                                  float exp_, float eym, float eyp, float ezm,
                                                  float ezp, Stencil<float>& w) {
    w.xm = rcp_approx(ec + exm);
    w.xp = rcp_approx(ec + exp_);
    w.ym = rcp_approx(ec + eym);
    w.yp = rcp_approx(ec + eyp);
    w.zm = (k > 0) ? rcp_approx(ec + ezm) : ((d.walls & 16) ? rcp_approx(ec) : 0.f);
    const bool top = (k + 1 == d.nz);
    const float wzt = top ? rcp_approx(ec) : rcp_approx(ec + ezp);
    w.zp = top ? 0.f : wzt;
    w.D = w.xm + w.xp + w.ym + w.yp + w.zm + wzt;
}

template <int CX, int CY, int TYT, typename E, int NS>
__global__ void __launch_bounds__(32 * (TYT + 1), 2) k_rb_ws(PcgArgs a) {
    using G = GeoRB<CX, CY, TYT, E>;
    static_assert(G::WB == 32, "one lane per compressed column of the tile");
    static_assert(NS >= 7, "six stages are held while a seventh is filled");
    constexpr int NC = 32 * TYT;
    extern __shared__ __align__(128) unsigned char sm[];
    float* const Ur = reinterpret_cast<float*>(sm + NS * G::STAGE);  // RINGU planes of u'
    float* const Tr = Ur + G::RINGU * G::UPL;                        // RINGT planes of t
    __shared__ __align__(8) uint64_t full[NS];
    __shared__ __align__(8) uint64_t empty[NS];
    __shared__ double red[64];
    __shared__ Seg s_seg[MAXSEG];
    __shared__ LocalSolveRB s_sol[MAXSEG];
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
        LocalSolveRB& L = s_sol[tid];
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
        L.beta = 0.0;
        L.done = sv.sc->done;
        L.iter = 0;
        L.max_iter = sv.sc->max_iter;
        L.finished = 0;
        L.first = 1;
        L.owner = 0;
        for (int q = 0; q < nseg; ++q)
            if (s_seg[q].slot == sv.seg_begin) L.owner = 1;
        s_member[tid] = (L.done == RUNNING);
        s_nextxs[tid] = 0;  // the start-up sweep leaves x alone
    }
    __syncthreads();

    const int lane = tx, warp = ty;
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
            const int xb = sg.x0 / 2 - G::VOFF, xe = sg.x0 - G::EOFF;
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
                mbar_arrive_expect_tx(bar, centre ? (xs ? G::TX : G::TX_P) : G::TX_HALO);
                tma_load_3d(dst + G::U, m + MAP1_U0 + in, bar, xb, sg.y0 - 2, kk);
                tma_load_3d(dst + G::S, m + MAP1_S0 + in, bar, xb, sg.y0 - 2, kk);
                tma_load_3d(dst + G::WV, m + MAP1_W0 + in, bar, xb, sg.y0 - 2, kk);
                tma_load_3d(dst + G::ETA, m + MAP1_ETA, bar, xe, sg.y0 - 2, kk);
                if (centre) {
                    if (xs) tma_load_3d(dst + G::X, m + MAP1_X, bar, sg.x0 / 2, sg.y0, kk);
                    tma_load_3d(dst + G::P, m + MAP1_P, bar, sg.x0 / 2, sg.y0, kk);
                }
                ++np;
            }
        }
    };

    // step 1 on plane q: u' at compressed column jc (m = x0/2 - 2 + jc) of on-chip row r
    auto step1 = [&](const unsigned char* S, float* Uq, float al, float be, int r, int jc) {
        const int si = r * G::VW + G::VOFF - 2 + jc;
        const float* Su = (const float*)(S + G::U);
        const float* Ss = (const float*)(S + G::S);
        const float* Sw = (const float*)(S + G::WV);
        Uq[r * G::UC + jc] = u_next_rb(Su[si], Ss[si], Sw[si], al, be);
    };

    // step 2 on plane kt: t of the red cell at compressed column jt (m = x0/2 - 1 + jt) of
    // on-chip row rt (y = y0 - 1 + rt); 0 outside the grid
    auto step2 = [&](const Dims& d, const Seg& sg, bool inner, int kt, const E* Em, const E* Ec,
                     const E* Ep, const float* Um, const float* Uc, const float* Up, float* Tt,
                     int rt, int jt) {
        const int y = sg.y0 - 1 + rt;
        const int pr = (y + kt) & 1;  // red: i + j + k even, i = 2m + pr
        const int x = sg.x0 - 2 + 2 * jt + pr;
        float t = 0.f;
        if (inner || (x >= 0 && x < d.nx && y >= 0 && y < d.ny)) {
            const int ei = (rt + 1) * G::EW + 2 * jt - 2 + pr + G::EOFF;
            Stencil<float> w;
            if (inner)
                eta_stencil_inner(d, kt, ld1(Ec + ei), ld1(Ec + ei - 1), ld1(Ec + ei + 1),
                                  ld1(Ec + ei - G::EW), ld1(Ec + ei + G::EW), ld1(Em + ei),
                                  ld1(Ep + ei), w);
            else
                eta_stencil(d, x, y, kt, ld1(Ec + ei), ld1(Ec + ei - 1), ld1(Ec + ei + 1),
                            ld1(Ec + ei - G::EW), ld1(Ec + ei + G::EW), ld1(Em + ei), ld1(Ep + ei),
                            w);
            const int ui = (rt + 1) * G::UC + jt;  // u' column of m - 1
            float s = w.xm * Uc[ui + pr];
            s += w.xp * Uc[ui + 1 + pr];
            s += w.ym * Uc[ui + 1 - G::UC];
            s += w.yp * Uc[ui + 1 + G::UC];
            s += w.zm * Um[ui + 1];
            s += w.zp * Up[ui + 1];
            t = s * rcp_approx(w.D);
        }
        Tt[rt * G::TC + jt] = t;
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
            const LocalSolveRB& Ls = s_sol[l];
            const int nxh = d.nx >> 1;
            const float al = (float)Ls.alpha, be = (float)Ls.beta;
            const bool xs = !Ls.first;
            const int L = sg.k1 - sg.k0;
            // the tile, its two rings of u' and the neighbours of its ring of t inside the grid
            const bool inner = sg.x0 >= 4 && sg.x0 + G::W + 4 <= d.nx && sg.y0 >= 3 &&
                               sg.y0 + G::HT + 3 <= d.ny;
            const int p0 = nc;  // sequence number of plane k0 - 2
            float ag = 0.f, ad = 0.f, ar = 0.f;
            for (int off = 0; off < L + 6; ++off) {
                const int q = sg.k0 - 2 + off, qs = p0 + off;
                const bool arrives = off < L + 4;
                const bool ok = arrives ? acquire() : !s_fail;
                if (ok && work) {
                    // Steps 1 and 2 are spread over all consumer threads by flat element index
                    // (consecutive threads on consecutive columns); step 2 from the first thread
                    // and step 1 from the last, so the threads left with one t fewer take the
                    // extra u' values.
                    if (arrives) {
                        // step 1: u' of plane q on the tile and two rings
                        const unsigned char* S = stage(qs);
                        float* Uq = Ur + ring(q, G::RINGU) * G::UPL;
                        for (int e = NC - 1 - tid; e < G::UPL; e += NC) {
                            const int r = e / G::UC;
                            step1(S, Uq, al, be, r, e - r * G::UC);
                        }
                    }
                    const int kt = q - 2;
                    if (off >= 3 && off <= L + 4) {
                        // step 2: t of plane kt = q - 2 on the red cells of the tile and one ring
                        float* Tt = Tr + ring(kt, G::RINGT) * G::TPL;
                        if (kt < 0 || kt >= d.nz) {
                            for (int e = tid; e < G::TPL; e += NC) Tt[e] = 0.f;
                        } else {
                            const float* Um = Ur + ring(kt - 1, G::RINGU) * G::UPL;
                            const float* Uc = Ur + ring(kt, G::RINGU) * G::UPL;
                            const float* Up = Ur + ring(kt + 1, G::RINGU) * G::UPL;
                            const E* Em = (const E*)(stage(qs - 3) + G::ETA);
                            const E* Ec = (const E*)(stage(qs - 2) + G::ETA);
                            const E* Ep = (const E*)(stage(qs - 1) + G::ETA);
                            for (int e = tid; e < G::TPL; e += NC) {
                                const int rt = e / G::TC;
                                step2(d, sg, inner, kt, Em, Ec, Ep, Um, Uc, Up, Tt, rt,
                                      e - rt * G::TC);
                            }
                        }
                    }
                    const int k = q - 4;
                    if (off >= 6) {
                        // step 3: S u' of plane k = q - 4 on the tile's black cells and updates
                        const unsigned char* S = stage(qs - 4);
                        const float* Su = (const float*)(S + G::U);
                        const float* Ss = (const float*)(S + G::S);
                        const float* Sw = (const float*)(S + G::WV);
                        const float* Sx = (const float*)(S + G::X);
                        const float* Sp = (const float*)(S + G::P);
                        const E* Em = (const E*)(stage(qs - 5) + G::ETA);
                        const E* Ec = (const E*)(S + G::ETA);
                        const E* Ep = (const E*)(stage(qs - 3) + G::ETA);
                        const float* Tm = Tr + ring(k - 1, G::RINGT) * G::TPL;
                        const float* Tc = Tr + ring(k, G::RINGT) * G::TPL;
                        const float* Tp = Tr + ring(k + 1, G::RINGT) * G::TPL;
                        const float* Uc = Ur + ring(k, G::RINGU) * G::UPL;
                        const int m = sg.x0 / 2 + lane;
                        for (int r = warp; r < G::HT; r += TYT) {
                            const int y = sg.y0 + r;
                            if (!inner && (y >= d.ny || m >= nxh)) continue;
                            const int pb = (y + k + 1) & 1;  // black: i = 2m + pb
                            const int ei = (r + 2) * G::EW + 2 * lane + pb + G::EOFF;
                            Stencil<float> w;
                            if (inner)
                                eta_stencil_inner(d, k, ld1(Ec + ei), ld1(Ec + ei - 1),
                                                  ld1(Ec + ei + 1), ld1(Ec + ei - G::EW),
                                                  ld1(Ec + ei + G::EW), ld1(Em + ei),
                                                  ld1(Ep + ei), w);
                            else
                                eta_stencil(d, sg.x0 + 2 * lane + pb, y, k, ld1(Ec + ei),
                                            ld1(Ec + ei - 1), ld1(Ec + ei + 1),
                                            ld1(Ec + ei - G::EW), ld1(Ec + ei + G::EW),
                                            ld1(Em + ei), ld1(Ep + ei), w);
                            const int ti = (r + 1) * G::TC + lane;  // t column of m - 1
                            float s = w.xm * Tc[ti + pb];
                            s += w.xp * Tc[ti + 1 + pb];
                            s += w.ym * Tc[ti + 1 - G::TC];
                            s += w.yp * Tc[ti + 1 + G::TC];
                            s += w.zm * Tm[ti + 1];
                            s += w.zp * Tp[ti + 1];
                            const float ub = Uc[(r + 2) * G::UC + lane + 2];
                            const float su = w.D * ub - s;
                            const int si = (r + 2) * G::VW + G::VOFF + lane;
                            const float pn = __fmaf_rn(be, Sp[r * G::WB + lane], Su[si]);
                            const float sn = __fmaf_rn(be, Ss[si], Sw[si]);
                            const float wn = su * rcp_approx(w.D);
                            const size_t cb = (size_t)m + (size_t)nxh * (y + (size_t)d.ny * k);
                            if (xs) Ls.x[cb] = __fmaf_rn(al, pn, Sx[r * G::WB + lane]);
                            Ls.p[cb] = pn;
                            Ls.u[out][cb] = ub;
                            Ls.s[out][cb] = sn;
                            Ls.w[out][cb] = wn;
                            const float du = w.D * ub;
                            ag += du * ub;
                            ad += su * ub;
                            ar += du * du;
                        }
                    }
                }
                named_sync(1, NC);
                if (off >= 5) release(qs - 5);
            }
            release(p0 + L + 1);
            release(p0 + L + 2);
            release(p0 + L + 3);
            // the segment's partial sums (gamma, delta, rho), over the consumer warps
            const float v[3] = {ag, ad, ar};
            segment_partials<3>(v, a.part_b + 3 * (size_t)s_seg[ls].slot, reinterpret_cast<ff*>(red),
                                tid, NC, 1);
        }
    };

    unsigned nbar = 0;
    int alive = 0;  // unfinished solves of the launch as of the last grid barrier
    auto owned_running = [&]() {
        int c = 0;
        for (int l = 0; l < nloc; ++l) c += (s_sol[l].owner && s_sol[l].done == RUNNING) ? 1 : 0;
        return c;
    };
    int in = 0;
    bool failed = false;
    // The producer streams the next sweep as soon as a grid barrier has passed, while the
    // consumers add the partial sums and decide (membership is fixed just before the barrier; a
    // solve that stops at the coming decision is walked once more without arithmetic).
    if (producer && lane == 0) produce(in);
    for (;;) {
        if (!producer) consume(in);
        __syncthreads();
        if (s_fail) { failed = true; break; }
        if (tid < nloc) {
            s_member[tid] = (s_sol[tid].done == RUNNING);
            s_nextxs[tid] = 1;  // every sweep after the start-up sweep updates x
        }
        ++nbar;
        if (!grid_barrier(a.ctl, nbar, nbar * (unsigned)a.nctas, tid, owned_running(), &alive)) {
            failed = true;
            break;
        }
        if (alive == 0) break;
        if (producer) {
            if (lane == 0) produce(in ^ 1);
            __syncwarp();
            in ^= 1;
            continue;
        }
        for (int l = 0; l < nloc; ++l) {
            if (s_sol[l].done != RUNNING) continue;
            double t[3];
            range_sum<3>(a.part_b, s_sol[l].seg_begin, s_sol[l].seg_end, t,
                         reinterpret_cast<ff*>(red), tid, NC, 1);
            if (tid == 32) s_sol[l].ginv[nbar & 1] = 1.0 / t[0];
            if (tid == 0) {
                LocalSolveRB& L = s_sol[l];
                const double gn = t[0], dn = t[1], rn = t[2];
                L.rr = rn;
                if (!isfinite(gn) || !isfinite(dn) || !isfinite(rn) || gn < 0.0) {
                    L.done = BREAKDOWN;
                } else if (L.first) {
                    // the start-up sweep: w^ = D_B^-1 S u formed, no iterate changed
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
                    L.iter += 1;
                    if (rn <= L.stop2) {
                        L.done = CONVERGED;
                    } else if (L.iter >= L.max_iter) {
                        L.done = CAPPED;
                    } else {
                        // beta = gamma'/gamma; delta' - beta gamma'/alpha = delta' - beta^2 den
                        const double be = gn * L.ginv[(nbar - 1) & 1];
                        const double den = fma(-be * be, L.den, dn);
                        if (!(den > 0.0) || !isfinite(den)) {
                            L.done = BREAKDOWN;
                        } else {
                            L.beta = be;
                            L.alpha = gn / den;
                            L.gamma = gn;
                            L.den = den;
                        }
                    }
                }
                if (L.done != RUNNING) L.finished = 1;
            }
            named_sync(1, NC);
        }
        if (tid < nloc) {
            LocalSolveRB& L = s_sol[tid];
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
        in ^= 1;
    }
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
static Cg1Kernel rb_of() {
    using G32 = GeoRB<CX, CY, TYT, float>;
    using G16 = GeoRB<CX, CY, TYT, __nv_bfloat16>;
    return Cg1Kernel{(const void*)k_rb_ws<CX, CY, TYT, float, NS>,
                     (const void*)k_rb_ws<CX, CY, TYT, __nv_bfloat16, NS>,
                     NS * G32::STAGE + G32::ON_CHIP, NS * G16::STAGE + G16::ON_CHIP};
}

Cg1Kernel rb_kernel(int cx, int cy, int tyt, int ns) {
#define RB_ROW(CX, CY, TYT, NS) \
    if (cx == CX && cy == CY && tyt == TYT && ns == NS) return rb_of<CX, CY, TYT, NS>();
    RB_CONFIGS(RB_ROW)
#undef RB_ROW
    return Cg1Kernel{nullptr, nullptr, 0, 0};
}

// ------------------------------------------------------------------ start and finish
constexpr int RB_T = 256;

// The compressed index e of a black cell: (m, j, k) -> cell (2m + ((j + k + 1) & 1), j, k).
__device__ __forceinline__ void rb_black_cell(const Dims& d, long long e, int& i, int& j, int& k) {
    const int nxh = d.nx >> 1;
    const int m = (int)(e % nxh);
    const long long rest = e / nxh;
    j = (int)(rest % d.ny);
    k = (int)(rest / d.ny);
    i = 2 * m + ((j + k + 1) & 1);
}

template <typename E>
__global__ void __launch_bounds__(RB_T) k_rb_init(Dims d, const E* __restrict__ eta,
                                                  const float* __restrict__ r, float* __restrict__ u,
                                                  float* __restrict__ s, float* __restrict__ w,
                                                  float* __restrict__ p, float* __restrict__ x,
                                                  Scalars* sc, double* partials, double tol2,
                                                  int max_iter) {
    __shared__ double smem[64];
    const CoefEta<E> coef{eta};
    const long long nb = (long long)d.n / 2;
    double rr = 0.0;
    // d_R = r_R / D_R of the red neighbour at c (inside the grid)
    auto dr = [&](int c, int i, int j, int k) {
        Stencil<float> ws;
        coef.weights(d, c, i, j, k, ws);
        return r[c] * rcp_approx(ws.D);
    };
    for (long long e = blockIdx.x * (long long)RB_T + threadIdx.x; e < nb;
         e += (long long)gridDim.x * RB_T) {
        int i, j, k;
        rb_black_cell(d, e, i, j, k);
        const int c = i + d.nx * (j + d.ny * k);
        Stencil<float> wb;
        coef.weights(d, c, i, j, k, wb);
        float acc = 0.f;
        if (i > 0) acc += wb.xm * dr(c - 1, i - 1, j, k);
        if (i + 1 < d.nx) acc += wb.xp * dr(c + 1, i + 1, j, k);
        if (j > 0) acc += wb.ym * dr(c - d.nx, i, j - 1, k);
        if (j + 1 < d.ny) acc += wb.yp * dr(c + d.nx, i, j + 1, k);
        if (k > 0) acc += wb.zm * dr(c - d.sxy, i, j, k - 1);
        if (k + 1 < d.nz) acc += wb.zp * dr(c + d.sxy, i, j, k + 1);
        u[e] = (r[c] + acc) * rcp_approx(wb.D);
        s[e] = 0.f;
        w[e] = 0.f;
        p[e] = 0.f;
        x[e] = 0.f;
        const float rp = r[(i & 1) ? c - 1 : c + 1];  // the other cell of the pair (2m, 2m+1)
        rr += (double)r[c] * r[c] + (double)rp * rp;
    }
    double v[1] = {rr}, tot[1];
    if (grid_sum<1>(v, partials, &sc->ticket, tot, smem)) {
        if (threadIdx.x == 0) {
            sc->rr = tot[0];
            sc->rr0 = tot[0];
            sc->rz = 0.0;
            sc->beta = 0.0;
            sc->alpha = 0.0;
            sc->iter = 0;
            sc->max_iter = max_iter;
            sc->stop2 = tol2 * tot[0];
            sc->done = (tot[0] <= sc->stop2) ? CONVERGED : RUNNING;
            if (!isfinite(tot[0])) sc->done = BREAKDOWN;
        }
    }
}

template <typename E>
__global__ void __launch_bounds__(RB_T) k_rb_finish(Dims d, const E* __restrict__ eta,
                                                    const float* __restrict__ r,
                                                    const float* __restrict__ xb,
                                                    float* __restrict__ out) {
    const CoefEta<E> coef{eta};
    const int nxh = d.nx >> 1;
    auto xat = [&](int i, int j, int k) { return xb[(i >> 1) + (size_t)nxh * (j + (size_t)d.ny * k)]; };
    for (long long t = blockIdx.x * (long long)RB_T + threadIdx.x; t < d.n;
         t += (long long)gridDim.x * RB_T) {
        const int c = (int)t;
        const int i = c % d.nx, j = (c / d.nx) % d.ny, k = c / d.sxy;
        if ((i + j + k) & 1) {
            out[c] = xat(i, j, k);
            continue;
        }
        Stencil<float> w;
        coef.weights(d, c, i, j, k, w);
        float acc = 0.f;
        if (i > 0) acc += w.xm * xat(i - 1, j, k);
        if (i + 1 < d.nx) acc += w.xp * xat(i + 1, j, k);
        if (j > 0) acc += w.ym * xat(i, j - 1, k);
        if (j + 1 < d.ny) acc += w.yp * xat(i, j + 1, k);
        if (k > 0) acc += w.zm * xat(i, j, k - 1);
        if (k + 1 < d.nz) acc += w.zp * xat(i, j, k + 1);
        out[c] = (r[c] + acc) * rcp_approx(w.D);
    }
}

static unsigned rb_blocks(long long n) {
    long long b = (n + RB_T - 1) / RB_T;
    return (unsigned)(b < 1 ? 1 : (b > 2048 ? 2048 : b));
}

template <typename E>
void launch_rb_init(const Dims& d, const E* eta, const float* r, float* u, float* s, float* w,
                    float* p, float* x, Scalars* sc, double* part, double tol2, int max_iter,
                    cudaStream_t st) {
    k_rb_init<E><<<rb_blocks((long long)d.n / 2), RB_T, 0, st>>>(d, eta, r, u, s, w, p, x, sc, part,
                                                                  tol2, max_iter);
    g_kernel_launches.fetch_add(1, std::memory_order_relaxed);
}

template <typename E>
void launch_rb_finish(const Dims& d, const E* eta, const float* r, const float* xb, float* out,
                      cudaStream_t st) {
    k_rb_finish<E><<<rb_blocks(d.n), RB_T, 0, st>>>(d, eta, r, xb, out);
    g_kernel_launches.fetch_add(1, std::memory_order_relaxed);
}

template void launch_rb_init<float>(const Dims&, const float*, const float*, float*, float*,
                                    float*, float*, float*, Scalars*, double*, double, int,
                                    cudaStream_t);
template void launch_rb_init<__nv_bfloat16>(const Dims&, const __nv_bfloat16*, const float*,
                                            float*, float*, float*, float*, float*, Scalars*,
                                            double*, double, int, cudaStream_t);
template void launch_rb_finish<float>(const Dims&, const float*, const float*, const float*,
                                      float*, cudaStream_t);
template void launch_rb_finish<__nv_bfloat16>(const Dims&, const __nv_bfloat16*, const float*,
                                              const float*, float*, cudaStream_t);

}  // namespace pcg

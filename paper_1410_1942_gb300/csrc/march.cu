// march.cu -- the FP32 CG passes as 2.5-D plane-marching kernels with TMA-staged x-y planes.
//
// A CTA of 32 x TYT threads works on x-y tiles of W x HT cells (W = 32 CX, HT = TYT CY; each
// thread owns a CX x CY block of cells) and walks them along z.  The grid is persistent (as many
// CTAs as fit on the GPU at once, launched cooperatively) and runs every CG iteration of the
// inner solve; it is driven by a work list of z-segments, so every CTA gets the same number of
// tile-planes whatever the grid shape, and one launch serves many solves of different sizes
// (each segment names its solve; per-solve tensor maps, vectors and scalars live in device
// memory).  Each plane of the inputs
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
#include "alloc.h"
#include "internal.cuh"
#include "kernels.h"
#include "march.h"
#include "march_dev.cuh"
#include "march_rb.h"
#include "tma.cuh"

#include <cudaTypedefs.h>

#include <algorithm>
#include <cstdlib>
#include <atomic>
#include <mutex>
#include <vector>

namespace pcg {

// ------------------------------------------------------------------ persistent PCG kernel
// One cooperative launch runs the whole FP32 inner PCG of one or many solves.  CTA c walks the
// segments [cta_seg[c], cta_seg[c+1]) of the work list (a segment is one tile column of one
// solve over planes [k0, k1); its plane stream is k0-1 .. k1), phase A then phase B, with a grid
// barrier after each phase.  Each segment leaves its partial sums in part_a / part_b; after the
// barrier every CTA adds, in segment order, the partials of the solves it works on and derives
// alpha, beta and the stopping decision itself -- the same numbers in every CTA.  The CTA that
// owns a solve's first segment publishes its final state; at every grid barrier each CTA adds
// the unfinished solves it owns to the barrier's count (MarchCtl::alive), and the loop ends, in
// every CTA at once, when a barrier's count is zero.
//
// Barrier waits spin on a global counter with a deadline (BAR_NS); a wait that runs out sets
// ctl->error, marks the CTA's solves TIMEDOUT, waits (bounded) for its TMA copies in flight
// and leaves the loop.

// Stream membership: the planes of a solve's segments are streamed in a phase iff s_member was
// set for it when the phase's stream began (right after the preceding grid barrier, before that
// barrier's decisions), so the first planes of a phase are already in flight while the partial
// sums of the previous one are being added.  A solve that finished at that barrier is walked
// once more without arithmetic (its work flag is off).
template <int CX, int CY, int TYT, typename E, int NS>
__global__ void __launch_bounds__(32 * TYT) k_pcg(PcgArgs a) {
    using G = Geo<CX, CY, TYT, E>;
    extern __shared__ __align__(128) unsigned char sm[];
    __shared__ __align__(8) uint64_t bars[NS];
    __shared__ double red[64];
    __shared__ Seg s_seg[MAXSEG];
    __shared__ LocalSolve s_sol[MAXSEG];
    __shared__ int s_member[MAXSEG];
    const int tx = threadIdx.x, ty = threadIdx.y, tid = tx + 32 * ty;
    const int sb = a.cta_seg[blockIdx.x];
    const int nseg = min(MAXSEG, a.cta_seg[blockIdx.x + 1] - sb);
    if (tid < nseg) s_seg[tid] = a.segs[sb + tid];
    if (tid == 0) {
        for (int s = 0; s < NS; ++s) mbar_init(&bars[s], 1);
        fence_mbar_init();
    }
    __syncthreads();
    const int first = nseg ? s_seg[0].solve : 0;
    const int nloc = nseg ? s_seg[nseg - 1].solve - first + 1 : 0;
    if (tid < nloc) {
        const SolveDev& sv = a.solves[first + tid];
        LocalSolve& L = s_sol[tid];
        L.d = sv.d;
        L.x = sv.x; L.r = sv.r; L.z = sv.z; L.pa = sv.pa; L.pb = sv.pb;
        L.sc = sv.sc;
        L.seg_begin = sv.seg_begin;
        L.seg_end = sv.seg_end;
        L.rz = sv.sc->rz;
        L.rr = sv.sc->rr;
        L.stop2 = sv.sc->stop2;
        L.alpha = 0.0;
        L.beta = 0.0;
        L.done = sv.sc->done;
        L.iter = 0;
        L.max_iter = sv.sc->max_iter;
        L.finished = 0;
        L.owner = 0;
        for (int q = 0; q < nseg; ++q)
            if (s_seg[q].slot == sv.seg_begin) L.owner = 1;
        s_member[tid] = (L.done == RUNNING);
    }
    __syncthreads();

    const int r0 = 1 + CY * ty, cv = G::VOFF + CX * tx, ce = G::EOFF + CX * tx, cc = CX * tx;
    const int lane = tx, warp = ty;
    auto stage = [&](int q) { return sm + (q % NS) * G::STAGE; };
    int g = 0;        // stream positions acquired (all threads)
    int nissued = 0;  // stream positions issued (thread 0)
    int g0 = 0;       // first position of the current phase
    bool ok = true;

    // ---------------------------------------------------------------- the plane stream (thread 0)
    int cs = 0, coff = 0;           // issue cursor
    bool st_a = true, st_pa = true;  // phase of the stream being issued, p_in is pa
    // Planes whose independent boxes went out before a grid barrier, waiting for the rest.
    int pend_n = 0, pend_seg[NS], pend_off[NS], pend_st[NS];
    // part: 0 = the whole plane, 1 = boxes not written by other CTAs since the last barrier
    // (eta; x and r; p_in of phase A), with the plane's full byte count expected but no
    // arrival, 2 = the remaining box (p of phase B, z of phase A) and the arrival.
    auto issue_boxes = [&](int seg, int off, int st, int part) {
        const Seg& sg = s_seg[seg];
        const int L = sg.k1 - sg.k0, kk = sg.k0 - 1 + off;
        unsigned char* dst = sm + st * G::STAGE;
        const CUtensorMap* m = a.maps + MAPS_PER_SOLVE * sg.solve;
        uint64_t* bar = &bars[st];
        if (st_a) {
            if (part == 0) mbar_arrive_expect_tx(bar, G::A_TX);
            if (part == 1) mbar_expect_tx(bar, G::A_TX);
            if (part != 2) {
                tma_load_3d(dst + G::A_P, m + (st_pa ? MAP_PA : MAP_PB), bar, sg.x0 - G::VOFF,
                            sg.y0 - 1, kk);
                tma_load_3d(dst + G::A_E, m + MAP_ETA, bar, sg.x0 - G::EOFF, sg.y0 - 1, kk);
            }
            if (part != 1)
                tma_load_3d(dst + G::A_Z, m + MAP_Z, bar, sg.x0 - G::VOFF, sg.y0 - 1, kk);
        } else {
            const bool centre = off > 0 && off <= L;
            const uint32_t tx = centre ? G::B_TX : G::B_TX_HALO;
            if (part == 0) mbar_arrive_expect_tx(bar, tx);
            if (part == 1) mbar_expect_tx(bar, tx);
            if (part != 2) {
                tma_load_3d(dst + G::B_E, m + MAP_ETA, bar, sg.x0 - G::EOFF, sg.y0 - 1, kk);
                if (centre) {
                    tma_load_3d(dst + G::B_X, m + MAP_X, bar, sg.x0, sg.y0, kk);
                    tma_load_3d(dst + G::B_R, m + MAP_R, bar, sg.x0, sg.y0, kk);
                }
            }
            if (part != 1)
                tma_load_3d(dst + G::B_P, m + (st_pa ? MAP_PB : MAP_PA), bar, sg.x0 - G::VOFF,
                            sg.y0 - 1, kk);
        }
        if (part == 2) mbar_arrive(bar);
    };
    // Issues the next plane of the stream (or, with pre, only its independent boxes).
    auto issue_next = [&](bool pre = false) {
        while (cs < nseg && coff == 0 && !s_member[s_seg[cs].solve - first]) ++cs;
        if (cs >= nseg) return;
        const int st = nissued % NS;
        if (pre) {
            issue_boxes(cs, coff, st, 1);
            pend_seg[pend_n] = cs;
            pend_off[pend_n] = coff;
            pend_st[pend_n] = st;
            ++pend_n;
        } else {
            issue_boxes(cs, coff, st, 0);
        }
        ++nissued;
        if (++coff == s_seg[cs].k1 - s_seg[cs].k0 + 2) {
            coff = 0;
            ++cs;
        }
    };
    // Starts the stream of a phase.  With pre, only the first NS planes' independent boxes go
    // out (before a grid barrier completes); finish_stream() then adds the rest.
    auto begin_stream = [&](bool a_side, bool p_in_a, bool pre) {
        g0 = g;
        if (tid == 0) {
            cs = 0;
            coff = 0;
            st_a = a_side;
            st_pa = p_in_a;
            pend_n = 0;
            for (int q = 0; q < NS; ++q) issue_next(pre);
        }
    };
    auto finish_stream = [&]() {
        if (tid == 0) {
            for (int q = 0; q < pend_n; ++q) issue_boxes(pend_seg[q], pend_off[q], pend_st[q], 2);
            pend_n = 0;
        }
    };
    auto acquire = [&]() -> bool {
        ok = ok && mbar_wait(&bars[g % NS], (g / NS) & 1);
        if (__syncthreads_or(!ok)) return false;  // also: every thread is done with g-2
        if (tid == 0 && g - g0 >= 2) issue_next();
        ++g;
        return true;
    };

    // ---------------------------------------------------------------- one phase over the segments
    auto run_phase = [&](bool a_side, bool p_in_a) -> bool {
        for (int ls = 0; ls < nseg; ++ls) {
            const Seg sg = s_seg[ls];
            const int l = sg.solve - first;
            if (!s_member[l]) continue;
            const bool work = s_sol[l].done == RUNNING;
            const Dims d = s_sol[l].d;
            const float coefv = (float)(a_side ? s_sol[l].beta : s_sol[l].alpha);
            const int i0 = sg.x0 + CX * tx, j0 = sg.y0 + CY * ty;
            const unsigned edges = block_edges<CX, CY>(d, i0, j0);
            auto centre = [&](int q, float (&o)[CY][CX]) {
                const unsigned char* S = stage(q);
                if (a_side) {
                    float zz[CY][CX];
                    load_centre<CX, CY>((const float*)(S + G::A_Z), G::VW, r0, cv, zz);
                    load_centre<CX, CY>((const float*)(S + G::A_P), G::VW, r0, cv, o);
#pragma unroll
                    for (int y = 0; y < CY; ++y)
#pragma unroll
                        for (int x = 0; x < CX; ++x) o[y][x] = zz[y][x] + coefv * o[y][x];
                } else {
                    load_centre<CX, CY>((const float*)(S + G::B_P), G::VW, r0, cv, o);
                }
            };
            auto eta_of = [&](int q) { return (const E*)(stage(q) + (a_side ? G::A_E : G::B_E)); };
            float vm[CY][CX], vc[CY][CX], em[CY][CX], ec[CY][CX], wzl[CY][CX];
            if (!acquire()) return false;  // plane k0-1
            if (work) {
                centre(g - 1, vm);
                load_centre<CX, CY>(eta_of(g - 1), G::EW, r0, ce, em);
            }
            if (!acquire()) return false;  // plane k0
            if (work) {
                centre(g - 1, vc);
                load_centre<CX, CY>(eta_of(g - 1), G::EW, r0, ce, ec);
#pragma unroll
                for (int y = 0; y < CY; ++y)
#pragma unroll
                    for (int x = 0; x < CX; ++x)
                        wzl[y][x] = (sg.k0 > 0 || (d.walls & 16)) ? rcp_approx(ec[y][x] + em[y][x]) : 0.f;
            }
            float acc0 = 0.f, acc1 = 0.f;
            for (int k = sg.k0; k < sg.k1; ++k) {
                if (!acquire()) return false;  // plane k+1
                if (!work) continue;
                const int qc = g - 2, qn = g - 1;
                const unsigned char* S = stage(qc);
                float vp[CY][CX], ep[CY][CX];
                centre(qn, vp);
                load_centre<CX, CY>(eta_of(qn), G::EW, r0, ce, ep);
                float vxm[CY], vxp[CY], vym[CX], vyp[CX];
                if (a_side) {
                    float zxm[CY], zxp[CY], zym[CX], zyp[CX];
                    load_halo<CX, CY>((const float*)(S + G::A_Z), G::VW, r0, cv, zxm, zxp, zym, zyp);
                    load_halo<CX, CY>((const float*)(S + G::A_P), G::VW, r0, cv, vxm, vxp, vym, vyp);
#pragma unroll
                    for (int y = 0; y < CY; ++y) {
                        vxm[y] = zxm[y] + coefv * vxm[y];
                        vxp[y] = zxp[y] + coefv * vxp[y];
                    }
#pragma unroll
                    for (int x = 0; x < CX; ++x) {
                        vym[x] = zym[x] + coefv * vym[x];
                        vyp[x] = zyp[x] + coefv * vyp[x];
                    }
                } else {
                    load_halo<CX, CY>((const float*)(S + G::B_P), G::VW, r0, cv, vxm, vxp, vym, vyp);
                }
                float exm[CY], exq[CY], eym[CX], eyp[CX];
                load_halo<CX, CY>(eta_of(qc), G::EW, r0, ce, exm, exq, eym, eyp);
                float qv[CY][CX], D[CY][CX];
                stencil<CX, CY>(d, edges, k, vc, vxm, vxp, vym, vyp, vm, vp, ec, exm, exq, eym,
                                eyp, ep, wzl, qv, D);
                if (a_side) {
                    float* p_out = p_in_a ? s_sol[l].pb : s_sol[l].pa;
                    if (i0 < d.nx) {
#pragma unroll
                        for (int y = 0; y < CY; ++y) {
                            if (j0 + y < d.ny) {
#pragma unroll
                                for (int x = 0; x < CX; ++x) acc0 += vc[y][x] * qv[y][x];
                                st_row<CX>(p_out + (size_t)i0 +
                                               (size_t)d.nx * (j0 + y + (size_t)d.ny * k), vc[y]);
                            }
                        }
                    }
                } else {
                    float xo[CY][CX], ro[CY][CX];
                    load_centre<CX, CY>((const float*)(S + G::B_X), G::W, CY * ty, cc, xo);
                    load_centre<CX, CY>((const float*)(S + G::B_R), G::W, CY * ty, cc, ro);
                    if (i0 < d.nx) {
#pragma unroll
                        for (int y = 0; y < CY; ++y) {
                            if (j0 + y < d.ny) {
                                float xn[CX], rn[CX], zn[CX];
#pragma unroll
                                for (int x = 0; x < CX; ++x) {
                                    xn[x] = xo[y][x] + coefv * vc[y][x];
                                    rn[x] = ro[y][x] - coefv * qv[y][x];
                                    zn[x] = rn[x] * rcp_approx(D[y][x]);
                                    acc0 += rn[x] * zn[x];
                                    acc1 += rn[x] * rn[x];
                                }
                                const size_t c =
                                    (size_t)i0 + (size_t)d.nx * (j0 + y + (size_t)d.ny * k);
                                st_row<CX>(s_sol[l].x + c, xn);
                                st_row<CX>(s_sol[l].r + c, rn);
                                st_row<CX>(s_sol[l].z + c, zn);
                            }
                        }
                    }
                }
#pragma unroll
                for (int y = 0; y < CY; ++y)
#pragma unroll
                    for (int x = 0; x < CX; ++x) {
                        vm[y][x] = vc[y][x];
                        vc[y][x] = vp[y][x];
                        ec[y][x] = ep[y][x];
                    }
            }
            // the segment's partial sums
            if (a_side) {
                const float v[1] = {acc0};
                segment_partials<1>(v, a.part_a + s_seg[ls].slot, reinterpret_cast<ff*>(red), tid,
                                    32 * TYT, 1);
            } else {
                const float v[2] = {acc0, acc1};
                segment_partials<2>(v, a.part_b + 2 * (size_t)s_seg[ls].slot,
                                    reinterpret_cast<ff*>(red), tid, 32 * TYT, 1);
            }
        }
        return true;
    };

    unsigned nbar = 0;
    int alive = 0;  // unfinished solves of the launch as of the last grid barrier
    // unfinished solves this CTA owns (thread 0 adds them at every grid barrier)
    auto owned_running = [&]() {
        int c = 0;
        for (int l = 0; l < nloc; ++l) c += (s_sol[l].owner && s_sol[l].done == RUNNING) ? 1 : 0;
        return c;
    };
    bool p_in_a = true;
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
    auto snapshot_members = [&]() {
        if (tid < nloc) s_member[tid] = (s_sol[tid].done == RUNNING);
        __syncthreads();
    };
    begin_stream(true, p_in_a, false);
    for (;;) {
        if (!run_phase(true, p_in_a)) { failed = true; break; }
        mark(TR_A);
        snapshot_members();
        ++nbar;
        grid_arrive(a.ctl, tid, nbar, nbar * (unsigned)a.nctas, owned_running(), a.trace != nullptr);
        const unsigned long long t_arr1 = tr ? globaltimer() : 0;
        begin_stream(false, p_in_a, true);
        if (!grid_wait(a.ctl, nbar, nbar * (unsigned)a.nctas, tid, &alive)) { failed = true; break; }
        if (tr) {
            const unsigned long long tl = *(volatile unsigned long long*)&a.ctl->t_last;
            const unsigned long long tn = globaltimer();
            if (tl > t_arr1) tt[TR_IMB] += tl - t_arr1;
            if (tn > tl) tt[TR_REL] += tn - tl;
        }
        finish_stream();
        mark(TR_BAR1);
        if (alive == 0) break;
        if (warp == 0) {
            for (int l = 0; l < nloc; ++l) {
                if (s_sol[l].done != RUNNING) continue;
                double t[1];
                warp_range_sum<1>(a.part_a, s_sol[l].seg_begin, s_sol[l].seg_end, lane, t);
                if (lane == 0) {
                    if (!(t[0] > 0.0) || !isfinite(t[0])) {
                        s_sol[l].done = BREAKDOWN;
                        s_sol[l].finished = 1;
                    } else {
                        s_sol[l].alpha = s_sol[l].rz / t[0];
                    }
                }
                __syncwarp();
            }
        }
        __syncthreads();
        mark(TR_ALPHA);
        if (!run_phase(false, p_in_a)) { failed = true; break; }
        mark(TR_B);
        snapshot_members();
        ++nbar;
        grid_arrive(a.ctl, tid, nbar, nbar * (unsigned)a.nctas, owned_running(), a.trace != nullptr);
        const unsigned long long t_arr2 = tr ? globaltimer() : 0;
        begin_stream(true, !p_in_a, true);
        if (!grid_wait(a.ctl, nbar, nbar * (unsigned)a.nctas, tid, &alive)) { failed = true; break; }
        if (tr) {
            const unsigned long long tl = *(volatile unsigned long long*)&a.ctl->t_last;
            const unsigned long long tn = globaltimer();
            if (tl > t_arr2) tt[TR_IMB] += tl - t_arr2;
            if (tn > tl) tt[TR_REL] += tn - tl;
        }
        finish_stream();
        mark(TR_BAR2);
        if (warp == 0) {
            for (int l = 0; l < nloc; ++l) {
                if (s_sol[l].done != RUNNING) continue;
                double t[2];
                warp_range_sum<2>(a.part_b, s_sol[l].seg_begin, s_sol[l].seg_end, lane, t);
                if (lane == 0) {
                    LocalSolve& L = s_sol[l];
                    L.iter += 1;
                    L.rr = t[1];
                    if (!isfinite(t[0]) || !isfinite(t[1]) || t[0] < 0.0) {
                        L.done = BREAKDOWN;
                    } else if (t[1] <= L.stop2) {
                        L.done = CONVERGED;
                    } else if (L.iter >= L.max_iter) {
                        L.done = CAPPED;
                    } else {
                        L.beta = t[0] / L.rz;
                        L.rz = t[0];
                    }
                    if (L.done != RUNNING) L.finished = 1;
                }
                __syncwarp();
            }
            // owners publish the solves that finished in this iteration (counted out at the next
            // phase-A barrier)
            if (lane < nloc) {
                LocalSolve& L = s_sol[lane];
                if (L.finished) {
                    L.finished = 0;
                    if (L.owner) {
                        L.sc->iter = L.iter;
                        L.sc->rr = L.rr;
                        L.sc->rz = L.rz;
                        L.sc->done = L.done;
                        __threadfence();
                    }
                }
            }
        }
        __syncthreads();
        mark(TR_BETA);
        if (tr) tt[TR_ITERS] += 1;
        p_in_a = !p_in_a;
    }
    if (tr)
        for (int q = 0; q < TRACE_PARTS; ++q) a.trace[q] += tt[q];
    // Planes issued but not consumed (the stream begun at the last barrier, or the rest of a
    // failed phase): complete any half-issued plane, then wait for them so no copy lands after
    // the CTA has gone.
    finish_stream();
    if (tid == 0) {
        if (failed) {
            atomicExch(&a.ctl->error, 1);
            for (int l = 0; l < nloc; ++l) {
                s_sol[l].sc->iter = s_sol[l].iter;
                atomicExch(&s_sol[l].sc->done, (int)TIMEDOUT);
            }
        }
        for (int q = g; q < nissued; ++q) (void)mbar_wait(&bars[q % NS], (q / NS) & 1);
        __threadfence();
    }
    __syncthreads();
}

// ------------------------------------------------------------------ warp-specialised variant
// Same work list, phases, grid barriers and reductions as k_pcg, but with a producer warp: its
// lane 0 walks the plane stream issuing TMA loads into the NS-stage ring, waiting on an "empty"
// mbarrier per stage (one arrival per consumer warp) before refilling it.  The TYT consumer
// warps wait on the "full" barriers, compute, and release each plane after its last use, so no
// block-wide barrier is taken per plane.  A timed-out wait sets s_fail; from then on every wait
// returns at once, so all warps still pass the same named barriers and leave together.

template <int CX, int CY, int TYT, typename E, int NS>
__global__ void __launch_bounds__(32 * (TYT + 1), WsMinBlocks<TYT>::value) k_pcg_ws(PcgArgs a) {
    using G = Geo<CX, CY, TYT, E>;
    constexpr int NT = 32 * (TYT + 1);  // all threads
    constexpr int NC = 32 * TYT;        // consumer threads
    extern __shared__ __align__(128) unsigned char sm[];
    __shared__ __align__(8) uint64_t full[NS];
    __shared__ __align__(8) uint64_t empty[NS];
    __shared__ double red[64];
    __shared__ Seg s_seg[MAXSEG];
    __shared__ LocalSolve s_sol[MAXSEG];
    __shared__ int s_member[MAXSEG];  // solve streamed in this iteration
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
        LocalSolve& L = s_sol[tid];
        L.d = sv.d;
        L.x = sv.x; L.r = sv.r; L.z = sv.z; L.pa = sv.pa; L.pb = sv.pb;
        L.sc = sv.sc;
        L.seg_begin = sv.seg_begin;
        L.seg_end = sv.seg_end;
        L.rz = sv.sc->rz;
        L.rr = sv.sc->rr;
        L.stop2 = sv.sc->stop2;
        L.alpha = 0.0;
        L.beta = 0.0;
        L.done = sv.sc->done;
        L.iter = 0;
        L.max_iter = sv.sc->max_iter;
        L.finished = 0;
        L.owner = 0;
        for (int q = 0; q < nseg; ++q)
            if (s_seg[q].slot == sv.seg_begin) L.owner = 1;
        s_member[tid] = (L.done == RUNNING);
    }
    __syncthreads();

    const int r0 = 1 + CY * ty, cv = G::VOFF + CX * tx, ce = G::EOFF + CX * tx, cc = CX * tx;
    const int warp = ty, lane = tx;
    auto stage = [&](int q) { return sm + (q % NS) * G::STAGE; };
    int np = 0;  // planes issued (producer lane 0)
    int nc = 0;  // planes acquired (each consumer warp)

    auto produce = [&](bool a_side, bool p_in_a) {
        for (int ls = 0; ls < nseg; ++ls) {
            const Seg& sg = s_seg[ls];
            if (!s_member[sg.solve - first]) continue;
            const int L = sg.k1 - sg.k0;
            const CUtensorMap* m = a.maps + MAPS_PER_SOLVE * sg.solve;
            for (int off = 0; off < L + 2; ++off) {
                if (s_fail) return;
                const int st = np % NS, kk = sg.k0 - 1 + off;
                if (np >= NS && !mbar_wait_or(&empty[st], ((np / NS) - 1) & 1, &s_fail)) {
                    s_fail = 1;
                    return;
                }
                unsigned char* dst = sm + st * G::STAGE;
                if (a_side) {
                    mbar_arrive_expect_tx(&full[st], G::A_TX);
                    tma_load_3d(dst + G::A_Z, m + MAP_Z, &full[st], sg.x0 - G::VOFF, sg.y0 - 1, kk);
                    tma_load_3d(dst + G::A_P, m + (p_in_a ? MAP_PA : MAP_PB), &full[st],
                                sg.x0 - G::VOFF, sg.y0 - 1, kk);
                    tma_load_3d(dst + G::A_E, m + MAP_ETA, &full[st], sg.x0 - G::EOFF, sg.y0 - 1, kk);
                } else {
                    const bool centre = off > 0 && off <= L;
                    mbar_arrive_expect_tx(&full[st], centre ? G::B_TX : G::B_TX_HALO);
                    tma_load_3d(dst + G::B_P, m + (p_in_a ? MAP_PB : MAP_PA), &full[st],
                                sg.x0 - G::VOFF, sg.y0 - 1, kk);
                    tma_load_3d(dst + G::B_E, m + MAP_ETA, &full[st], sg.x0 - G::EOFF, sg.y0 - 1, kk);
                    if (centre) {
                        tma_load_3d(dst + G::B_X, m + MAP_X, &full[st], sg.x0, sg.y0, kk);
                        tma_load_3d(dst + G::B_R, m + MAP_R, &full[st], sg.x0, sg.y0, kk);
                    }
                }
                ++np;
            }
        }
    };

    auto consume = [&](bool a_side, bool p_in_a) {
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
        for (int ls = 0; ls < nseg; ++ls) {
            const Seg sg = s_seg[ls];
            const int l = sg.solve - first;
            if (!s_member[l]) continue;
            const bool work = s_sol[l].done == RUNNING;
            const Dims d = s_sol[l].d;
            const float coefv = (float)(a_side ? s_sol[l].beta : s_sol[l].alpha);
            const int i0 = sg.x0 + CX * tx, j0 = sg.y0 + CY * warp;
            const unsigned edges = block_edges<CX, CY>(d, i0, j0);
            auto centre = [&](int q, float (&o)[CY][CX]) {
                const unsigned char* S = stage(q);
                if (a_side) {
                    float zz[CY][CX];
                    load_centre<CX, CY>((const float*)(S + G::A_Z), G::VW, r0, cv, zz);
                    load_centre<CX, CY>((const float*)(S + G::A_P), G::VW, r0, cv, o);
#pragma unroll
                    for (int y = 0; y < CY; ++y)
#pragma unroll
                        for (int x = 0; x < CX; ++x) o[y][x] = zz[y][x] + coefv * o[y][x];
                } else {
                    load_centre<CX, CY>((const float*)(S + G::B_P), G::VW, r0, cv, o);
                }
            };
            auto eta_of = [&](int q) { return (const E*)(stage(q) + (a_side ? G::A_E : G::B_E)); };
            float vm[CY][CX], vc[CY][CX], em[CY][CX], ec[CY][CX], wzl[CY][CX];
            const int p0 = nc;
            bool ok = acquire();  // plane k0-1
            if (ok && work) {
                centre(p0, vm);
                load_centre<CX, CY>(eta_of(p0), G::EW, r0, ce, em);
            }
            release(p0);
            ok = acquire();  // plane k0
            if (ok && work) {
                centre(p0 + 1, vc);
                load_centre<CX, CY>(eta_of(p0 + 1), G::EW, r0, ce, ec);
#pragma unroll
                for (int y = 0; y < CY; ++y)
#pragma unroll
                    for (int x = 0; x < CX; ++x)
                        wzl[y][x] = (sg.k0 > 0 || (d.walls & 16)) ? rcp_approx(ec[y][x] + em[y][x]) : 0.f;
            }
            float acc0 = 0.f, acc1 = 0.f;
            for (int k = sg.k0; k < sg.k1; ++k) {
                const int qc = p0 + 1 + (k - sg.k0), qn = qc + 1;
                ok = acquire();  // plane k+1
                if (ok && work) {
                    const unsigned char* S = stage(qc);
                    float vp[CY][CX], ep[CY][CX];
                    centre(qn, vp);
                    load_centre<CX, CY>(eta_of(qn), G::EW, r0, ce, ep);
                    float vxm[CY], vxp[CY], vym[CX], vyp[CX];
                    if (a_side) {
                        float zxm[CY], zxp[CY], zym[CX], zyp[CX];
                        load_halo<CX, CY>((const float*)(S + G::A_Z), G::VW, r0, cv, zxm, zxp, zym, zyp);
                        load_halo<CX, CY>((const float*)(S + G::A_P), G::VW, r0, cv, vxm, vxp, vym, vyp);
#pragma unroll
                        for (int y = 0; y < CY; ++y) {
                            vxm[y] = zxm[y] + coefv * vxm[y];
                            vxp[y] = zxp[y] + coefv * vxp[y];
                        }
#pragma unroll
                        for (int x = 0; x < CX; ++x) {
                            vym[x] = zym[x] + coefv * vym[x];
                            vyp[x] = zyp[x] + coefv * vyp[x];
                        }
                    } else {
                        load_halo<CX, CY>((const float*)(S + G::B_P), G::VW, r0, cv, vxm, vxp, vym, vyp);
                    }
                    float exm[CY], exq[CY], eym[CX], eyp[CX];
                    load_halo<CX, CY>(eta_of(qc), G::EW, r0, ce, exm, exq, eym, eyp);
                    float qv[CY][CX], D[CY][CX];
                    stencil<CX, CY>(d, edges, k, vc, vxm, vxp, vym, vyp, vm, vp, ec, exm, exq, eym,
                                    eyp, ep, wzl, qv, D);
                    if (a_side) {
                        float* p_out = p_in_a ? s_sol[l].pb : s_sol[l].pa;
                        if (i0 < d.nx) {
#pragma unroll
                            for (int y = 0; y < CY; ++y) {
                                if (j0 + y < d.ny) {
#pragma unroll
                                    for (int x = 0; x < CX; ++x) acc0 += vc[y][x] * qv[y][x];
                                    st_row<CX>(p_out + (size_t)i0 +
                                                   (size_t)d.nx * (j0 + y + (size_t)d.ny * k), vc[y]);
                                }
                            }
                        }
                    } else {
                        float xo[CY][CX], ro[CY][CX];
                        load_centre<CX, CY>((const float*)(S + G::B_X), G::W, CY * warp, cc, xo);
                        load_centre<CX, CY>((const float*)(S + G::B_R), G::W, CY * warp, cc, ro);
                        if (i0 < d.nx) {
#pragma unroll
                            for (int y = 0; y < CY; ++y) {
                                if (j0 + y < d.ny) {
                                    float xn[CX], rn[CX], zn[CX];
#pragma unroll
                                    for (int x = 0; x < CX; ++x) {
                                        xn[x] = xo[y][x] + coefv * vc[y][x];
                                        rn[x] = ro[y][x] - coefv * qv[y][x];
                                        zn[x] = rn[x] * rcp_approx(D[y][x]);
                                        acc0 += rn[x] * zn[x];
                                        acc1 += rn[x] * rn[x];
                                    }
                                    const size_t c =
                                        (size_t)i0 + (size_t)d.nx * (j0 + y + (size_t)d.ny * k);
                                    st_row<CX>(s_sol[l].x + c, xn);
                                    st_row<CX>(s_sol[l].r + c, rn);
                                    st_row<CX>(s_sol[l].z + c, zn);
                                }
                            }
                        }
                    }
#pragma unroll
                    for (int y = 0; y < CY; ++y)
#pragma unroll
                        for (int x = 0; x < CX; ++x) {
                            vm[y][x] = vc[y][x];
                            vc[y][x] = vp[y][x];
                            ec[y][x] = ep[y][x];
                        }
                }
                release(qc);
                if (k + 1 == sg.k1) release(qn);
            }
            // the segment's partial sums, over the consumer warps
            if (a_side) {
                const float v[1] = {acc0};
                segment_partials<1>(v, a.part_a + s_seg[ls].slot, reinterpret_cast<ff*>(red), tid,
                                    NC, 1);
            } else {
                const float v[2] = {acc0, acc1};
                segment_partials<2>(v, a.part_b + 2 * (size_t)s_seg[ls].slot,
                                    reinterpret_cast<ff*>(red), tid, NC, 1);
            }
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
    bool p_in_a = true;
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
            if (lane == 0) produce(true, p_in_a);
            __syncwarp();
        } else {
            consume(true, p_in_a);
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
            double t[1];
            range_sum<1>(a.part_a, s_sol[l].seg_begin, s_sol[l].seg_end, t, reinterpret_cast<ff*>(red),
                         tid, NT);
            if (tid == 0) {
                if (!(t[0] > 0.0) || !isfinite(t[0])) {
                    s_sol[l].done = BREAKDOWN;
                    s_sol[l].finished = 1;
                } else {
                    s_sol[l].alpha = s_sol[l].rz / t[0];
                }
            }
            __syncthreads();
        }
        mark(TR_ALPHA);
        if (producer) {
            if (lane == 0) produce(false, p_in_a);
            __syncwarp();
        } else {
            consume(false, p_in_a);
        }
        __syncthreads();
        mark(TR_B);
        if (s_fail) { failed = true; break; }
        ++nbar;
        if (!grid_barrier(a.ctl, nbar, nbar * (unsigned)a.nctas, tid, owned_running(), &alive)) {
            failed = true;
            break;
        }
        mark(TR_BAR2);
        for (int l = 0; l < nloc; ++l) {
            if (s_sol[l].done != RUNNING) continue;
            double t[2];
            range_sum<2>(a.part_b, s_sol[l].seg_begin, s_sol[l].seg_end, t, reinterpret_cast<ff*>(red),
                         tid, NT);
            if (tid == 0) {
                LocalSolve& L = s_sol[l];
                L.iter += 1;
                L.rr = t[1];
                if (!isfinite(t[0]) || !isfinite(t[1]) || t[0] < 0.0) {
                    L.done = BREAKDOWN;
                } else if (t[1] <= L.stop2) {
                    L.done = CONVERGED;
                } else if (L.iter >= L.max_iter) {
                    L.done = CAPPED;
                } else {
                    L.beta = t[0] / L.rz;
                    L.rz = t[0];
                }
                if (L.done != RUNNING) L.finished = 1;
            }
            __syncthreads();
        }
        if (tid < nloc) {
            LocalSolve& L = s_sol[tid];
            if (L.finished) {
                L.finished = 0;
                if (L.owner) {
                    L.sc->iter = L.iter;
                    L.sc->rr = L.rr;
                    L.sc->rz = L.rz;
                    L.sc->done = L.done;
                    __threadfence();
                }
            }
            s_member[tid] = (L.done == RUNNING);
        }
        __syncthreads();
        mark(TR_BETA);
        if (tr) tt[TR_ITERS] += 1;
        p_in_a = !p_in_a;
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
    // (periodic x: the tiles' TMA halo boxes do not wrap; the column kernels serve it)
    // (cut cells: the faces carry open fractions the kernels cannot form from rho/2; periodic x
    // runs on the one-sweep kernels with padded rows)
    return (d.nx % 8) == 0 && !(d.walls & CUT_CELLS) && encode_fn() != nullptr;
}

// ------------------------------------------------------------------ variant table
// A variant is (CX, CY, TYT); its tile is 32 CX wide and CY TYT high.
struct VariantOps {
    int cx, cy, tyt, ws, ns;
    int smem32, smem16;
    const void *k32, *k16;
    int family;
    const void *k32p = nullptr, *k16p = nullptr;  // periodic-x instantiations (family 1)
};

template <int CX, int CY, int TYT, int WS, int NS, int F>
static VariantOps make_ops() {
    if constexpr (F == 3) {
        static_assert(WS == 1, "the red-black kernels have a producer warp");
        const Cg1Kernel k = rb_kernel(CX, CY, TYT, NS);
        return VariantOps{CX, CY, TYT, 1, NS, k.smem32, k.smem16, k.k32, k.k16, F};
    } else if constexpr (F == 1 || F == 2) {
        static_assert(WS == 1, "the one-sweep kernels have a producer warp");
        const Cg1Kernel k = F == 1 ? cg1_kernel(CX, CY, TYT, NS) : cg2_kernel(CX, CY, TYT, NS);
        return VariantOps{CX, CY, TYT, 1, NS, k.smem32, k.smem16, k.k32, k.k16, F, k.k32p, k.k16p};
    } else if constexpr (WS)
        return VariantOps{CX, CY, TYT, 1, NS, NS * Geo<CX, CY, TYT, float>::STAGE,
                          NS * Geo<CX, CY, TYT, __nv_bfloat16>::STAGE,
                          (const void*)k_pcg_ws<CX, CY, TYT, float, NS>,
                          (const void*)k_pcg_ws<CX, CY, TYT, __nv_bfloat16, NS>, 0};
    else
        return VariantOps{CX, CY, TYT, 0, NS, NS * Geo<CX, CY, TYT, float>::STAGE,
                          NS * Geo<CX, CY, TYT, __nv_bfloat16>::STAGE,
                          (const void*)k_pcg<CX, CY, TYT, float, NS>,
                          (const void*)k_pcg<CX, CY, TYT, __nv_bfloat16, NS>, 0};
}

// (CX, CY, TYT, warp-specialised, ring stages, family); family 1, 2 and 3 rows must be in
// CG1_CONFIGS, CG2_CONFIGS and RB_CONFIGS
#define MARCH_VARIANTS(X)                                                                       \
    X(1, 1, 8, 0, 4, 0) X(2, 2, 4, 0, 4, 0) X(2, 2, 8, 0, 4, 0) X(2, 2, 4, 1, 4, 0)             \
    X(2, 2, 8, 1, 4, 0) X(2, 2, 4, 0, 3, 0) X(2, 2, 8, 0, 3, 0) X(2, 2, 8, 1, 3, 0)             \
    X(2, 2, 4, 0, 6, 0) X(2, 2, 8, 1, 6, 0) X(2, 2, 4, 1, 4, 1) X(2, 2, 4, 1, 3, 1)             \
    X(2, 2, 8, 1, 3, 1) X(2, 2, 4, 1, 4, 2) X(2, 2, 4, 1, 5, 2) X(2, 2, 8, 1, 4, 2)             \
    X(2, 2, 4, 1, 8, 3) X(2, 2, 4, 1, 7, 3) X(2, 1, 8, 1, 8, 3) X(2, 2, 8, 1, 7, 3)

static const VariantOps* variants(int* count) {
#define ROW(CX, CY, TYT, WS, NS, F) make_ops<CX, CY, TYT, WS, NS, F>(),
    static const VariantOps table[] = {MARCH_VARIANTS(ROW)};
#undef ROW
    static std::once_flag once;
    std::call_once(once, [] {
        for (const auto& v : table) {
            cudaFuncSetAttribute(v.k32, cudaFuncAttributeMaxDynamicSharedMemorySize, v.smem32);
            cudaFuncSetAttribute(v.k16, cudaFuncAttributeMaxDynamicSharedMemorySize, v.smem16);
            if (v.k32p)
                cudaFuncSetAttribute(v.k32p, cudaFuncAttributeMaxDynamicSharedMemorySize, v.smem32);
            if (v.k16p)
                cudaFuncSetAttribute(v.k16p, cudaFuncAttributeMaxDynamicSharedMemorySize, v.smem16);
        }
        cudaGetLastError();
    });
    *count = (int)(sizeof(table) / sizeof(table[0]));
    return table;
}

static int threads_of(const VariantOps& v) { return 32 * (v.tyt + v.ws); }

int march_variant_count() {
    int n;
    variants(&n);
    return n;
}

MarchVariant march_variant(int id) {
    int n;
    const VariantOps* t = variants(&n);
    const VariantOps& v = t[id < 0 || id >= n ? 0 : id];
    return MarchVariant{id, v.cx, v.cy, v.tyt, v.ws, v.ns, 32 * v.cx, v.cy * v.tyt, v.family};
}

int march_find_variant(int cx, int cy, int tyt, int ws, int ns, int family) {
    int n;
    const VariantOps* t = variants(&n);
    for (int q = 0; q < n; ++q)
        if (t[q].cx == cx && t[q].cy == cy && t[q].tyt == tyt && t[q].ws == ws && t[q].ns == ns &&
            t[q].family == family && t[q].k32)
            return q;
    return -1;
}

int march_variant_of_tile(int tile) {
    if (tile < 0 || tile / 10000000 > 3 || (tile / 1000000) % 10 >= MARCH_SPLITS) return -1;
    const int family = tile / 10000000;
    tile %= 1000000;
    const int ns = tile / 100000 ? tile / 100000 : 4;
    return march_find_variant((tile / 1000) % 10, (tile / 100) % 10, tile % 100,
                              (tile / 10000) % 10, ns, family);
}

int march_split_of_tile(int tile) { return (tile / 1000000) % 10; }

int march_tile_of(int variant) {
    const MarchVariant v = march_variant(variant);
    return 10000000 * v.family + (v.ns == 4 ? 0 : 100000 * v.ns) + 10000 * v.ws + 1000 * v.cx +
           100 * v.cy + v.tyt;
}

int march_occupancy(int variant, bool bf16) {
    int n;
    const VariantOps& v = variants(&n)[variant];
    int o = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, bf16 ? v.k16 : v.k32, threads_of(v),
                                                      bf16 ? v.smem16 : v.smem32) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    // a plan sized here may launch the periodic instantiation: take the smaller residency
    const void* kp = bf16 ? v.k16p : v.k32p;
    int op = o;
    if (kp && cudaOccupancyMaxActiveBlocksPerMultiprocessor(&op, kp, threads_of(v),
                                                            bf16 ? v.smem16 : v.smem32) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return o < op ? o : op;
}

// ------------------------------------------------------------------ plans
bool march_encode_solve(CUtensorMap (&m)[MAPS_PER_SOLVE], const MarchSolve& s, int variant,
                        bool bf16) {
    const MarchVariant v = march_variant(variant);
    const int eoff = bf16 ? 8 : 4;
    const CUtensorMapDataType f32 = CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
    const CUtensorMapDataType edt = bf16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : f32;
    const Dims& d = s.d;
    bool ok = true;
    if ((d.walls & PERIODIC_X) && v.family != 1) return false;  // no wrapped halos there
    if (v.family == 3) {
        // compressed black vectors (nx/2 per row) with 2-row halo boxes; eta at full size
        Dims db = d;
        db.nx = d.nx / 2;
        db.sxy = db.nx * d.ny;
        db.n = d.n / 2;
        const int wb = v.width / 2, bw = wb + 8, bh = v.height + 4;
        ok = ok && s.sa && s.sb && s.wa && s.wb && (d.nx % 8) == 0;
        ok = ok && encode3d(&m[MAP1_U0], s.z, f32, 4, db, bw, bh);
        ok = ok && encode3d(&m[MAP1_U1], s.pb, f32, 4, db, bw, bh);
        ok = ok && encode3d(&m[MAP1_S0], s.sa, f32, 4, db, bw, bh);
        ok = ok && encode3d(&m[MAP1_S1], s.sb, f32, 4, db, bw, bh);
        ok = ok && encode3d(&m[MAP1_W0], s.wa, f32, 4, db, bw, bh);
        ok = ok && encode3d(&m[MAP1_W1], s.wb, f32, 4, db, bw, bh);
        ok = ok && encode3d(&m[MAP1_ETA], s.eta, edt, bf16 ? 2 : 4, d, v.width + 2 * eoff, bh);
        ok = ok && encode3d(&m[MAP1_X], s.x, f32, 4, db, wb, v.height);
        ok = ok && encode3d(&m[MAP1_P], s.pa, f32, 4, db, wb, v.height);
        return ok;
    }
    if (v.family == 2) {
        const int bw = v.width + 8, bh = v.height + 4;
        ok = ok && s.sa;
        ok = ok && encode3d(&m[MAP2_U0], s.z, f32, 4, d, bw, bh);
        ok = ok && encode3d(&m[MAP2_U1], s.sa, f32, 4, d, bw, bh);
        ok = ok && encode3d(&m[MAP2_P0], s.pa, f32, 4, d, bw, bh);
        ok = ok && encode3d(&m[MAP2_P1], s.pb, f32, 4, d, bw, bh);
        ok = ok && encode3d(&m[MAP2_ETA], s.eta, edt, bf16 ? 2 : 4, d, v.width + 2 * eoff, bh);
        ok = ok && encode3d(&m[MAP2_X], s.x, f32, 4, d, v.width, v.height);
        return ok;
    }
    if (v.family == 1) {
        const int bw = v.width + 8, bh = v.height + 2;
        // periodic x: u, s^, w^ and eta in rows padded with ghost columns
        const bool per = d.walls & PERIODIC_X;
        Dims dv = d, de = d;
        if (per) {
            dv.nx = d.nx + 2 * PAD_V;
            de.nx = d.nx + 2 * eoff;
        }
        ok = ok && s.sa && s.sb && s.wa && s.wb;
        ok = ok && encode3d(&m[MAP1_U0], s.z, f32, 4, dv, bw, bh);
        ok = ok && encode3d(&m[MAP1_U1], s.pb, f32, 4, dv, bw, bh);
        ok = ok && encode3d(&m[MAP1_S0], s.sa, f32, 4, dv, bw, bh);
        ok = ok && encode3d(&m[MAP1_S1], s.sb, f32, 4, dv, bw, bh);
        ok = ok && encode3d(&m[MAP1_W0], s.wa, f32, 4, dv, bw, bh);
        ok = ok && encode3d(&m[MAP1_W1], s.wb, f32, 4, dv, bw, bh);
        ok = ok && encode3d(&m[MAP1_ETA], s.eta, edt, bf16 ? 2 : 4, de, v.width + 2 * eoff, bh);
        ok = ok && encode3d(&m[MAP1_X], s.x, f32, 4, d, v.width, v.height);
        ok = ok && encode3d(&m[MAP1_P], s.pa, f32, 4, d, v.width, v.height);
        return ok;
    }
    ok = ok && encode3d(&m[MAP_Z], s.z, f32, 4, d, v.width + 8, v.height + 2);
    ok = ok && encode3d(&m[MAP_PA], s.pa, f32, 4, d, v.width + 8, v.height + 2);
    ok = ok && encode3d(&m[MAP_PB], s.pb, f32, 4, d, v.width + 8, v.height + 2);
    ok = ok && encode3d(&m[MAP_ETA], s.eta, edt, bf16 ? 2 : 4, d, v.width + 2 * eoff, v.height + 2);
    ok = ok && encode3d(&m[MAP_X], s.x, f32, 4, d, v.width, v.height);
    ok = ok && encode3d(&m[MAP_R], s.r, f32, 4, d, v.width, v.height);
    return ok;
}

void march_plan_free(MarchPlan* p) {
    void* ptrs[] = {p->solves, p->segs, p->cta_seg, p->maps, p->part_a, p->part_b, p->ctl,
                    p->trace};
    for (void* q : ptrs)
        if (q) lib_free(q);
    *p = MarchPlan{};
}

// Device buffer of at least `bytes`, reallocated only when it must grow.
static bool plan_buffer(void** buf, size_t* cap, size_t bytes) {
    if (*buf && *cap >= bytes) return true;
    if (*buf) lib_free(*buf);
    *buf = nullptr;
    *cap = 0;
    if (lib_malloc(buf, bytes) != cudaSuccess) {
        cudaGetLastError();
        *buf = nullptr;
        return false;
    }
    *cap = bytes;
    return true;
}

// Splits the solves' tile columns into z-segments and packs them into at most nctas CTAs:
// EQUAL and BALANCED make the largest per-CTA cost (planes + a fixed cost per segment) as
// small as possible, LOCKSTEP keeps neighbouring tiles on the same planes.  A CTA's segments
// come out ordered by solve.  Fails (-1) if a CTA would hold more than MAXSEG segments or span
// more than MAXSEG solves, or a tensor map cannot be encoded.
int march_plan_build(MarchPlan* p, const MarchSolve* solves, int nsolves, int variant, bool bf16,
                     int nctas, int strategy, cudaStream_t st) {
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
    std::vector<int> cta_seg;
    long long ntiles = 0;
    for (int s = 0; s < nsolves; ++s) ntiles += (long long)tiles_x[s] * tiles_y[s];
    if (strategy == MARCH_SPLIT_LOCKSTEP_FILL && ntiles > nctas && ntiles % nctas != 0) {
        // One round of whole columns in lockstep (CTA c: tiles c, c + nctas, ... for ntiles /
        // nctas rounds), then the columns left over as one pool of planes cut into nctas equal
        // ranges in (solve, tile, plane) order: CTA c takes range c after its whole columns.
        std::vector<std::pair<int, int>> tl;  // (solve, tile)
        for (int s = 0; s < nsolves; ++s)
            for (int t = 0; t < tiles_x[s] * tiles_y[s]; ++t) tl.push_back({s, t});
        const long long rounds = ntiles / nctas, first_left = rounds * nctas;
        std::vector<long long> lbase(1, 0);  // first pool plane of each leftover column
        for (long long t = first_left; t < ntiles; ++t)
            lbase.push_back(lbase.back() + solves[tl[t].first].d.nz);
        const long long pool = lbase.back();
        auto seg_of = [&](long long t, int k0, int k1) {
            Seg g{};
            g.solve = tl[t].first;
            g.x0 = (tl[t].second % tiles_x[g.solve]) * v.width;
            g.y0 = (tl[t].second / tiles_x[g.solve]) * v.height;
            g.k0 = k0;
            g.k1 = k1;
            return g;
        };
        for (int c = 0; c < nctas; ++c) {
            cta_seg.push_back((int)segs.size());
            std::vector<Seg> mine;
            for (long long r = 0; r < rounds; ++r) {
                const long long t = c + r * nctas;
                mine.push_back(seg_of(t, 0, solves[tl[t].first].d.nz));
            }
            const long long a = pool * c / nctas, b = pool * (c + 1) / nctas;
            for (long long t = first_left; t < ntiles && a < b; ++t) {
                const long long lo = lbase[t - first_left], hi = lbase[t - first_left + 1];
                const long long s0 = std::max(a, lo), s1 = std::min(b, hi);
                if (s0 < s1) mine.push_back(seg_of(t, (int)(s0 - lo), (int)(s1 - lo)));
            }
            // a CTA's segments ordered by solve (the kernel's local records)
            std::stable_sort(mine.begin(), mine.end(),
                             [](const Seg& x, const Seg& y) { return x.solve < y.solve; });
            for (const Seg& g : mine) segs.push_back(g);
        }
        cta_seg.push_back((int)segs.size());
        // partial-sum slots contiguous per solve
        std::vector<int> per(nsolves + 1, 0);
        for (const Seg& g : segs) ++per[g.solve + 1];
        for (int q = 0; q < nsolves; ++q) per[q + 1] += per[q];
        for (Seg& g : segs) g.slot = per[g.solve]++;
    } else if (strategy == MARCH_SPLIT_LOCKSTEP || strategy == MARCH_SPLIT_LOCKSTEP_FILL) {
        // Whole columns dealt round-robin when there are at least as many tile columns as CTAs
        // (CTA c: tiles c, c + G, c + 2G, ... of the (solve, tile) list); otherwise every column
        // is cut into q equal z-chunks and CTA c * ntiles + t takes chunk c of tile t.  Either
        // way the CTAs holding neighbouring tiles march the same planes at the same time.
        if (ntiles < 1) return -1;
        std::vector<std::pair<int, int>> tl;  // (solve, tile)
        for (int s = 0; s < nsolves; ++s)
            for (int t = 0; t < tiles_x[s] * tiles_y[s]; ++t) tl.push_back({s, t});
        auto seg_of = [&](long long t, int k0, int k1, int slot) {
            Seg g{};
            g.solve = tl[t].first;
            g.x0 = (tl[t].second % tiles_x[g.solve]) * v.width;
            g.y0 = (tl[t].second / tiles_x[g.solve]) * v.height;
            g.k0 = k0;
            g.k1 = k1;
            g.slot = slot;
            return g;
        };
        if (ntiles >= nctas) {
            const long long m = (ntiles + nctas - 1) / nctas;
            const int G = (int)((ntiles + m - 1) / m);
            for (int c = 0; c < G; ++c) {
                cta_seg.push_back((int)segs.size());
                for (long long t = c; t < ntiles; t += G) {
                    const int nz = solves[tl[t].first].d.nz;
                    segs.push_back(seg_of(t, 0, nz, (int)t));  // slots in (solve, tile) order
                }
            }
            nctas = G;
        } else {
            int q = (int)(nctas / ntiles);
            for (int s = 0; s < nsolves; ++s) q = std::min(q, solves[s].d.nz);
            for (int c = 0; c < q; ++c)
                for (long long t = 0; t < ntiles; ++t) {
                    const int nz = solves[tl[t].first].d.nz;
                    cta_seg.push_back((int)segs.size());
                    // slots in (solve, tile, chunk) order
                    segs.push_back(seg_of(t, (int)((long long)c * nz / q),
                                          (int)((long long)(c + 1) * nz / q), (int)(t * q + c)));
                }
            nctas = (int)cta_seg.size();
        }
        cta_seg.push_back((int)segs.size());
    } else {
        // A CTA's cost is its planes plus SEG_COST per segment (the two halo planes of a
        // segment and its pipeline start; 0 for the plain equal-planes split).  The smallest
        // capacity T for which a greedy walk over the tile columns (in solve, tile order) fits
        // in nctas CTAs is found by bisection; the walk then cuts the work list, taking a new
        // segment only when the current CTA has room for at least MIN_PLANES more planes.
        const double SEG_COST = strategy == MARCH_SPLIT_BALANCED ? 2.0 : 0.0;
        const int MIN_PLANES = strategy == MARCH_SPLIT_BALANCED ? 2 : 1;
        struct Col { int solve, tile, nz; };
        std::vector<Col> cols;
        for (int s = 0; s < nsolves; ++s)
            for (int t = 0; t < tiles_x[s] * tiles_y[s]; ++t) cols.push_back({s, t, solves[s].d.nz});
        auto walk = [&](double T, bool emit) -> long long {
            long long ctas = 1;
            double cost = 0.0;
            if (emit) cta_seg.push_back(0);
            for (const Col& c : cols) {
                int k = 0;
                while (k < c.nz) {
                    int room = (int)(T - cost - SEG_COST + 1e-9);
                    if (room < MIN_PLANES && cost > 0.0) {
                        ++ctas;
                        cost = 0.0;
                        if (emit) cta_seg.push_back((int)segs.size());
                        continue;
                    }
                    if (room < 1) room = 1;
                    const int take = std::min(room, c.nz - k);
                    if (emit) {
                        Seg g{};
                        g.solve = c.solve;
                        g.x0 = (c.tile % tiles_x[c.solve]) * v.width;
                        g.y0 = (c.tile / tiles_x[c.solve]) * v.height;
                        g.k0 = k;
                        g.k1 = k + take;
                        g.slot = (int)segs.size();
                        segs.push_back(g);
                    }
                    cost += SEG_COST + take;
                    k += take;
                }
            }
            return ctas;
        };
        double lo = (double)W / nctas + SEG_COST - 1.0, hi = (double)W / nctas * 2.0 + 4.0 * SEG_COST;
        while (walk(hi, false) > nctas) hi *= 2.0;
        for (int it = 0; it < 40; ++it) {
            const double mid = 0.5 * (lo + hi);
            if (walk(mid, false) <= nctas) hi = mid; else lo = mid;
        }
        walk(hi, true);
        nctas = (int)cta_seg.size();
        cta_seg.push_back((int)segs.size());
    }
    std::vector<SolveDev> sd(nsolves);
    for (int c = 0; c < nctas; ++c) {
        const int b = cta_seg[c], e = cta_seg[c + 1];
        if (e - b > MAXSEG) return -1;
        // the kernel keeps one local record per solve from the CTA's first to its last
        if (e > b && segs[e - 1].solve - segs[b].solve + 1 > MAXSEG) return -1;
    }
    for (int s = 0; s < nsolves; ++s) {
        sd[s].d = solves[s].d;
        sd[s].x = solves[s].x;
        sd[s].r = solves[s].r;
        sd[s].z = solves[s].z;
        sd[s].pa = solves[s].pa;
        sd[s].pb = solves[s].pb;
        sd[s].sc = solves[s].sc;
        sd[s].sa = solves[s].sa;
        sd[s].sb = solves[s].sb;
        sd[s].wa = solves[s].wa;
        sd[s].wb = solves[s].wb;
        sd[s].seg_begin = (int)segs.size();
        sd[s].seg_end = 0;
    }
    for (int q = 0; q < (int)segs.size(); ++q) {
        SolveDev& t = sd[segs[q].solve];
        t.seg_begin = std::min(t.seg_begin, segs[q].slot);
        t.seg_end = std::max(t.seg_end, segs[q].slot + 1);
    }
    std::vector<CUtensorMap> maps(MAPS_PER_SOLVE * (size_t)nsolves);
    for (int s = 0; s < nsolves; ++s) {
        CUtensorMap m[MAPS_PER_SOLVE] = {};
        if (!march_encode_solve(m, solves[s], variant, bf16)) return -1;
        for (int q = 0; q < MAPS_PER_SOLVE; ++q) maps[MAPS_PER_SOLVE * (size_t)s + q] = m[q];
    }
    int nper = 0;
    for (int s = 0; s < nsolves; ++s) nper += (solves[s].d.walls & PERIODIC_X) ? 1 : 0;
    if (nper != 0 && nper != nsolves) return -1;  // one instantiation per launch
    p->variant = variant;
    p->strategy = strategy;
    p->bf16 = bf16;
    p->periodic = nper > 0;
    p->nctas = nctas;
    p->nsolves = nsolves;
    p->nsegs = (int)segs.size();
    auto up = [&](void** dst, size_t* cap, const void* src, size_t bytes) -> bool {
        return plan_buffer(dst, cap, bytes) &&
               cudaMemcpyAsync(*dst, src, bytes, cudaMemcpyHostToDevice, st) == cudaSuccess;
    };
    bool ok = up((void**)&p->solves, &p->cap_solves, sd.data(), sizeof(SolveDev) * sd.size()) &&
              up((void**)&p->segs, &p->cap_segs, segs.data(), sizeof(Seg) * segs.size()) &&
              up((void**)&p->cta_seg, &p->cap_cta, cta_seg.data(), sizeof(int) * cta_seg.size()) &&
              up((void**)&p->maps, &p->cap_maps, maps.data(), sizeof(CUtensorMap) * maps.size());
    ok = ok && plan_buffer((void**)&p->part_a, &p->cap_pa, sizeof(float2) * segs.size()) &&
         plan_buffer((void**)&p->part_b, &p->cap_pb, sizeof(float2) * 3 * segs.size()) &&
         plan_buffer((void**)&p->ctl, &p->cap_ctl, sizeof(MarchCtl));
    if (ok && getenv("POISSON_TRACE") && !p->trace) {
        if (lib_malloc((void**)&p->trace, sizeof(unsigned long long) * TRACE_PARTS) != cudaSuccess ||
            cudaMemsetAsync(p->trace, 0, sizeof(unsigned long long) * TRACE_PARTS, st) != cudaSuccess) {
            cudaGetLastError();
            lib_free(p->trace);
            p->trace = nullptr;
        }
    }
    if (ok) ok = cudaStreamSynchronize(st) == cudaSuccess;  // host vectors go out of scope
    if (!ok) {
        march_plan_free(p);
        return -2;
    }
    return 0;
}

int launch_march_pcg(const MarchPlan& p, cudaStream_t st) {
    int n;
    const VariantOps& v = variants(&n)[p.variant];
    PcgArgs args{p.solves, p.segs, p.cta_seg, p.maps, p.part_a,         p.part_b,
                 p.ctl,    p.nctas + p.barrier_extra,          p.trace};
    void* params[] = {&args};
    const void* k = p.periodic ? (p.bf16 ? v.k16p : v.k32p) : (p.bf16 ? v.k16 : v.k32);
    if (!k) return -1;
    const cudaError_t e = cudaLaunchCooperativeKernel(k, dim3(p.nctas),
                                                      dim3(32, v.tyt + v.ws), params,
                                                      (size_t)(p.bf16 ? v.smem16 : v.smem32), st);
    g_kernel_launches.fetch_add(1, std::memory_order_relaxed);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return -1;
    }
    return 0;
}

}  // namespace pcg

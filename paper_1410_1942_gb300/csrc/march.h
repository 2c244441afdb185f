// march.h -- host interface of the TMA plane-marching CG kernels (march.cu).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include "internal.cuh"

namespace pcg {

// One kernel variant: 32 x tyt compute threads, each owning cx x cy cells, plus one TMA
// producer warp when ws, an ns-stage plane ring; tile width x height cells.  family 0: two
// sweeps (and two grid barriers) per CG iteration; family 1: one sweep per iteration (the
// Chronopoulos-Gear recurrences, march1.cu); family 2: one sweep per iteration with A p formed
// in the sweep (march2.cu).
struct MarchVariant {
    int id, cx, cy, tyt, ws, ns, width, height, family;
};

// Tensor maps of one solve, in this order: halo boxes (width+8) x (height+2) x 1 for z and both
// p buffers, (width+8, or +16 for BF16) x (height+2) for eta, centre boxes width x height x 1
// for x and r.
enum { MAP_Z = 0, MAP_PA = 1, MAP_PB = 2, MAP_ETA = 3, MAP_X = 4, MAP_R = 5 };
// Family 1: halo boxes for both buffers of u (z, pb), s-hat (sa, sb) and w-hat (wa, wb), eta as
// above, centre boxes for x and p (pa).
enum { MAP1_U0 = 0, MAP1_U1 = 1, MAP1_S0 = 2, MAP1_S1 = 3, MAP1_W0 = 4, MAP1_W1 = 5,
       MAP1_ETA = 6, MAP1_X = 7, MAP1_P = 8 };
// Family 2: 2-cell halo boxes for both buffers of u (z, sa) and p (pa, pb) and for eta, a centre
// box for x.
enum { MAP2_U0 = 0, MAP2_U1 = 1, MAP2_P0 = 2, MAP2_P1 = 3, MAP2_ETA = 4, MAP2_X = 5 };
constexpr int MAPS_PER_SOLVE = 9;

// Periodic x in the one-sweep kernels: u, s^, w^ live in rows padded with PAD_V ghost columns on
// each side (eta with its halo width: 4 FP32 / 8 BF16 columns), the ghosts holding the other end
// of the row, so the TMA halo boxes read wrapped values; the CTAs writing the first and last
// PAD_V columns of a row also write their ghost copies.
constexpr int PAD_V = 4;

// One solve of a plan as the host describes it.
struct MarchSolve {
    Dims d;
    float *x, *r, *z, *pa, *pb;
    const void* eta;  // float or bf16, rho/2 per cell
    Scalars* sc;
    float *sa, *sb, *wa, *wb;  // family 1 only
};

// Device-side copy: the partial-sum slots [seg_begin, seg_end) of the solve.
struct SolveDev {
    Dims d;
    int seg_begin, seg_end;
    float *x, *r, *z, *pa, *pb;
    Scalars* sc;
    float *sa, *sb, *wa, *wb;
};

// One tile column of one solve over planes [k0, k1); its partial sums go to slot `slot` of the
// partial arrays (slots are contiguous per solve, in solve order).
struct Seg {
    int solve, x0, y0, k0, k1, slot, pad1, pad2;
};

// Control words of one persistent launch (set by the host before the launch).
// alive[m % 3]: at grid barrier m every CTA adds, before it arrives, the number of unfinished
// solves it owns; once the barrier is passed the sum is complete and no CTA changes it until all
// have left, so every CTA reads the same count and takes the same decision to stop.  CTA 0
// clears alive[(m + 1) % 3] before it arrives at barrier m (its readers left at barrier m - 1,
// its writers come after barrier m).
struct MarchCtl {
    unsigned bar;  // grid-barrier arrivals (0 at launch)
    int running;   // solves at launch (informational)
    int error;     // 1 once a wait has timed out
    int pad;
    unsigned long long t_last;  // trace only: global time of the last arrival at a barrier
    int alive[3];  // 0 at launch
    int pad2;
};

// Work-split strategies of march_plan_build.
// LOCKSTEP deals whole tile columns round-robin (CTA c: tiles c, c + G, ...) so that all CTAs
// march the same planes at the same time (halo rows of neighbouring tiles stay in L2).
// LOCKSTEP_FILL deals one round of whole columns to every CTA in lockstep and cuts the columns
// left over into equal plane counts over all CTAs, so that every CTA of the launch has work
// when the columns do not divide evenly.
enum { MARCH_SPLIT_EQUAL = 0, MARCH_SPLIT_BALANCED = 1, MARCH_SPLIT_LOCKSTEP = 2,
       MARCH_SPLIT_LOCKSTEP_FILL = 3, MARCH_SPLITS = 4 };

// A persistent launch: nctas CTAs, CTA c owns segments [cta_seg[c], cta_seg[c+1]).
struct MarchPlan {
    int variant = 0;
    int strategy = 0;
    bool bf16 = false;
    bool periodic = false;  // the solves have periodic x (the kernel's periodic instantiation)
    int nctas = 0, nsolves = 0, nsegs = 0;
    SolveDev* solves = nullptr;
    Seg* segs = nullptr;
    int* cta_seg = nullptr;
    CUtensorMap* maps = nullptr;
    // per-segment partial sums as float-float pairs (hi, lo)
    float2* part_a = nullptr;  // per segment: p.Ap
    float2* part_b = nullptr;  // per segment: r.z, r.r (family 1: gamma, delta, r.r)
    MarchCtl* ctl = nullptr;
    unsigned long long* trace = nullptr;  // TRACE_PARTS counters when tracing is on
    // testing aid (poisson_test_unreachable_barrier): the grid barriers wait for this many CTAs
    // beyond the nctas launched, so the first one can only end by its deadline
    int barrier_extra = 0;
    // allocated bytes of the buffers above (a rebuild reuses them when they suffice)
    size_t cap_solves = 0, cap_segs = 0, cap_cta = 0, cap_maps = 0, cap_pa = 0, cap_pb = 0,
           cap_ctl = 0;
};

// Kernel parameters of the persistent PCG launch.
struct PcgArgs {
    const SolveDev* solves;
    const Seg* segs;
    const int* cta_seg;
    const CUtensorMap* maps;
    float2* part_a;
    float2* part_b;
    MarchCtl* ctl;
    int nctas;
    unsigned long long* trace;  // optional: CTA 0 adds its per-part times (ns), TRACE_PARTS slots
};

// Parts of a persistent-PCG iteration timed by the optional trace (CTA 0's view).
// TR_IMB: CTA 0's arrival to the last CTA's arrival; TR_REL: last arrival to CTA 0's release.
// One-sweep kernels: TR_SUM the cross-CTA sums, TR_DECIDE the scalar recurrences (both inside
// TR_ALPHA; in SM cycles, not ns).
enum { TR_A = 0, TR_BAR1, TR_ALPHA, TR_B, TR_BAR2, TR_BETA, TR_ITERS, TR_IMB, TR_REL, TR_SUM,
       TR_DECIDE, TRACE_PARTS };

bool march_supported(const Dims& d);
int march_variant_count();
MarchVariant march_variant(int id);
int march_find_variant(int cx, int cy, int tyt, int ws, int ns, int family = 0);  // -1: none
// poisson_opts.tile codes: 10000000 family + 1000000 split + 100000 NS (omitted for NS = 4) +
// 10000 WS + 1000 CX + 100 CY + T
int march_variant_of_tile(int tile);  // -1 if there is none
int march_tile_of(int variant);
int march_split_of_tile(int tile);  // the 1000000s digit: the split strategy
int march_occupancy(int variant, bool bf16);       // resident CTAs per SM (0 if unknown)

// Builds a plan (device arrays allocated, or reused when large enough, copied on st,
// synchronised) / frees it.  0 on success, -1 if a tensor map cannot be encoded or a CTA would
// hold too many segments, -2 on allocation failure.
// strategy: MARCH_SPLIT_EQUAL (equal planes per CTA) or MARCH_SPLIT_BALANCED (planes plus a
// per-segment cost).
int march_plan_build(MarchPlan* p, const MarchSolve* solves, int nsolves, int variant, bool bf16,
                     int nctas, int strategy, cudaStream_t st);
void march_plan_free(MarchPlan* p);

// Cooperative launch of the persistent PCG over the plan (every solve's r, z, scalars
// initialised, pa zeroed, *ctl set).  0 on success, -1 if the launch was refused.
int launch_march_pcg(const MarchPlan& p, cudaStream_t st);

}  // namespace pcg

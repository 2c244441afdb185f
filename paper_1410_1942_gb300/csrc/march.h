// march.h -- host interface of the TMA plane-marching CG kernels (march.cu).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include "internal.cuh"

namespace pcg {

// One kernel variant: 32 x tyt threads, each owning cx x cy cells; tile width x height cells.
struct MarchVariant {
    int id, cx, cy, tyt, width, height;
};

// Tensor maps of one solve, in this order: halo boxes (width+8) x (height+2) x 1 for z and both
// p buffers, (width+8, or +16 for BF16) x (height+2) for eta, centre boxes width x height x 1
// for x and r.
enum { MAP_Z = 0, MAP_PA = 1, MAP_PB = 2, MAP_ETA = 3, MAP_X = 4, MAP_R = 5 };

// One solve of a plan as the host describes it.
struct MarchSolve {
    Dims d;
    float *x, *r, *z, *pa, *pb;
    const void* eta;  // float or bf16, rho/2 per cell
    Scalars* sc;
};

// Device-side copy: the segment range [seg_begin, seg_end) of the solve in the work list.
struct SolveDev {
    Dims d;
    int seg_begin, seg_end;
    float *x, *r, *z, *pa, *pb;
    Scalars* sc;
};

// One tile column of one solve over planes [k0, k1).
struct Seg {
    int solve, x0, y0, k0, k1, pad0, pad1, pad2;
};

// A persistent launch: nctas CTAs, CTA c owns segments [cta_seg[c], cta_seg[c+1]).
struct MarchPlan {
    int variant = 0;
    bool bf16 = false;
    int nctas = 0, nsolves = 0, nsegs = 0;
    SolveDev* solves = nullptr;
    Seg* segs = nullptr;
    int* cta_seg = nullptr;
    CUtensorMap* maps = nullptr;
    double* seg_part = nullptr;
};

bool march_supported(const Dims& d);
int march_variant_count();
MarchVariant march_variant(int id);
int march_find_variant(int cx, int cy, int tyt);  // -1 if there is none
int march_occupancy(int variant, bool bf16);       // resident CTAs per SM (min of both phases)

// Builds (device arrays allocated, copied on st, synchronised) / frees a plan.  0 on success,
// -1 if a tensor map cannot be encoded, -2 on allocation failure.
int march_plan_build(MarchPlan* p, const MarchSolve* solves, int nsolves, int variant, bool bf16,
                     int nctas, cudaStream_t st);
void march_plan_free(MarchPlan* p);

// phase A: p = z + beta p_in (p_in = pa if pin_is_a else pb; p written to the other buffer).
void launch_march_a(const MarchPlan& p, bool pin_is_a, cudaStream_t st);
// phase B: reads p (pa if p_is_a else pb), eta, x, r; writes x, r, z.
void launch_march_b(const MarchPlan& p, bool p_is_a, cudaStream_t st);

}  // namespace pcg

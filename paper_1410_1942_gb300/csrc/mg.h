// mg.h -- multigrid V-cycle preconditioner for the column-kernel PCG (POISSON_MG).
//
// The paper leaves its PCG preconditioner open (Introduction); this one is the standard stronger
// choice for the variable-coefficient pressure equation:
//   * hierarchy: level l+1 aggregates cells of level l in blocks of fx x fy x fz (2 along every
//     axis with more than one cell; along a periodic x axis only while nx is even and >= 4) and
//     carries the Galerkin operator A_{l+1} = P^T A_l P of the 0/1 aggregation P: a symmetric
//     7-point stencil (coarse face = sum of the fine faces across it, diagonal = sum of the
//     block's diagonals minus twice its internal faces).  Level 1 is formed from the FP64 faces;
//     coarsening stops at MG_COARSE_MAX cells or when no axis can be coarsened (level 0 is always
//     coarsened once).
//   * V-cycle y = V_l(r): x = w D^-1 r; e = V_{l+1}(P^T (r - A x)); x += a P e;
//     y = x + w D^-1 (r - A x); on the coarsest level MG_COARSE_SWEEPS damped Jacobi sweeps
//     from zero.  Symmetric and positive definite (0 < w < 1), so PCG keeps its theory.
//
// Kernels per V-cycle: one restriction per level pair down to the bottom levels (the fine one
// reads r and the pre-smoothed x), one single-block kernel for the levels of at most 2048 cells
// and the coarsest sweeps, one prolongation + post-smoothing per level above them; the fine
// post-smoothing writes z and reduces (r, z) into the CG scalars.
#pragma once

#include "internal.cuh"

namespace pcg {

constexpr int MG_MAX_LEVELS = 32;
constexpr double MG_OMEGA = 0.9;   // Jacobi smoother damping
constexpr double MG_ALPHA = 1.5;   // coarse-correction scaling
constexpr int MG_COARSE_MAX = 512;
constexpr int MG_COARSE_SWEEPS = 16;

struct MgHier {
    int nlev = 0;     // levels, the fine one included (>= 2 once planned)
    bool dbl = false;  // level arrays in FP64 (FP64 handles) or FP32
    Dims d[MG_MAX_LEVELS] = {};
    int f[MG_MAX_LEVELS][3] = {};  // aggregation factors from level l to l + 1
    // levels >= 1: Galerkin faces (low side) and diagonal; r, the pre-smoothed x, the output y
    void *bx[MG_MAX_LEVELS] = {}, *by[MG_MAX_LEVELS] = {}, *bz[MG_MAX_LEVELS] = {},
         *diag[MG_MAX_LEVELS] = {};
    void *r[MG_MAX_LEVELS] = {}, *x[MG_MAX_LEVELS] = {}, *y[MG_MAX_LEVELS] = {};
    // x[0]: the fine level's pre-smoothed vector (n values)
};

// Level shapes and factors for a fine grid; returns the number of levels (< 2: no hierarchy).
int mg_plan(const Dims& fine, MgHier* m);
// Device arrays of the planned hierarchy (FP64 when dbl); POISSON_OK or POISSON_ENOMEM.
int mg_alloc(MgHier* m, bool dbl);
void mg_free(MgHier* m);
// Galerkin operators of levels 1.. from the FP64 fine faces.
void mg_setup(MgHier* m, const double* bx, const double* by, const double* bz,
              const double* diag, cudaStream_t st);

// PCG passes with the V-cycle (the fine operator is `coef`, z the CG's preconditioned vector):
// start (x0 = w D^-1 r, scalars set as by k_cg_init, then z = V(r) and rz), phase B (x, r
// updates, x0, r.r, then z = V(r), r.z and the beta / stopping update), and the checking apply
// (z = V(r), no scalars).
template <typename V, typename Coef>
void mg_init(MgHier* m, const Dims& d, int kc, const Coef& coef, const V* r, V* z, Scalars* sc,
             double* part, double tol2, int rel_to_b, int max_iter, cudaStream_t st);
template <typename V, typename Coef>
void mg_cg_b(MgHier* m, const Dims& d, int kc, const Coef& coef, const V* p, V* x, V* r, V* z,
             Scalars* sc, double* part, cudaStream_t st);
template <typename V, typename Coef>
void mg_apply(MgHier* m, const Dims& d, int kc, const Coef& coef, const V* r, V* z,
              cudaStream_t st);

}  // namespace pcg

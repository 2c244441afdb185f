/*
 * poisson.h -- C ABI of libpoisson, a GB300 (sm_103a) solver for the variable-coefficient pressure
 * Poisson equation of a Cartesian-grid two-phase ship-wave method.
 *
 * The equation (Formulation, eq. (pois); the two stage solves of Numerical Time Integration) is
 *
 *     div( (1/rho) grad p ) = s,        s = div(u*) / dt,
 *
 * on a uniform grid of nx x ny x nz cells of spacing h, cell-centred p, with
 *   rho = rho_air + F (rho_water - rho_air)        (eq. (density); F = water fraction of the cell)
 *   face coefficient = 2 / (rho_c + rho_n)          (harmonic mean of 1/rho over the two cells)
 *   zero normal gradient on the walls x = 0, x = nx h, y = 0, y = ny h, z = 0;
 *   p = 0 on the top face z = nz h (second order: ghost value -p_c).
 * The Introduction states that this second-order variable-coefficient Poisson equation is solved by
 * preconditioned conjugate gradients; the preconditioner is Jacobi or red-black SSOR (the paper
 * names neither), or a multigrid V-cycle (POISSON_MG, beyond the paper, below).
 *
 * Conventions for every call:
 *   - 3-D arrays are float64, nx*ny*nz elements, x fastest: element (i, j, k) at i + nx*(j + ny*k).
 *   - A pointer argument may be host memory or device memory of the current CUDA device; the
 *     library tells them apart with cudaPointerGetAttributes (pageable, pinned and device memory
 *     are all accepted).  The caller owns every array it passes; the library never frees them.
 *     A host array of at least 1 MiB in pinned memory (mapped into the device's address space,
 *     as cudaHostAlloc and cudaHostRegister memory is) is read or written by a copy kernel
 *     through that mapping, which stays fast when the host pages' translations have gone cold;
 *     other host arrays go through cudaMemcpyAsync.
 *   - Device pointers are read or written on the handle's stream (poisson_opts.stream); calls that
 *     return results on the host synchronise that stream before returning.
 *   - Every call returns POISSON_OK (0) or a negative status; poisson_strerror names it.
 *   - A handle is not thread-safe: do not call into one handle from two threads at once.
 */
#ifndef POISSON_H
#define POISSON_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------------ status codes */
/* Walls of poisson_opts.dirichlet_walls */
#define POISSON_WALL_XM 1   /* x = 0  */
#define POISSON_WALL_XP 2   /* x = Lx */
#define POISSON_WALL_YM 4   /* y = 0  */
#define POISSON_WALL_YP 8   /* y = Ly */
#define POISSON_WALL_ZM 16  /* z = 0 (the bottom) */
#define POISSON_WALLS_ALL 31

#define POISSON_OK 0
#define POISSON_PENDING 1            /* poisson_poll: solve still running */
#define POISSON_EINVAL (-1)          /* bad argument: size <= 0, h <= 0, tol <= 0, NULL, ...  */
#define POISSON_ENOMEM (-2)          /* device or host allocation failed */
#define POISSON_ENOTCONV (-3)        /* iteration cap reached; p holds the best iterate */
#define POISSON_EBREAKDOWN (-4)      /* CG breakdown: p.Ap <= 0 or a non-finite scalar */
#define POISSON_ETIMEOUT (-5)        /* a device-side wait exceeded its deadline */
#define POISSON_ENOTREADY (-6)       /* solve before set_density */
#define POISSON_ECUDA (-7)           /* a CUDA runtime call failed */
#define POISSON_ENOMEM_BUDGET (-8)   /* poisson_required_bytes: over the device-memory budget */
#define POISSON_ENOTICKET (-9)       /* poisson_poll: unknown or already collected ticket */
#define POISSON_ETOOLARGE (-10)      /* poisson_residual_noalloc: grid beyond its static scratch */

/* ------------------------------------------------------------------ options */
#define POISSON_FP64 0           /* plain FP64 PCG on the GPU */
#define POISSON_FP32 1           /* FP32 inner PCG inside FP64 iterative refinement */
#define POISSON_FP32_BF16COEF 2  /* as POISSON_FP32, inner densities stored as bfloat16 */

#define POISSON_JACOBI 0
#define POISSON_RBSSOR 1
/* Multigrid V-cycle (column kernels, any precision).  Level l+1 aggregates the cells of level l
 * in 2x2x2 blocks (an axis of one cell is not coarsened; a periodic x axis only while nx is even
 * and >= 4; the last block of an odd axis has one cell) and carries the Galerkin operator
 * P^T A P of that aggregation; levels stop at 512 cells.  One cycle: x = 0.9 D^-1 r;
 * e = V(P^T (r - A x)) on the next level; x += 1.5 P e; z = x + 0.9 D^-1 (r - A x); 16 damped
 * Jacobi sweeps (0.9) from zero on the coarsest level.  Symmetric positive definite.  The
 * coarse levels are built from the FP64 operator by poisson_set_density and stored in FP64
 * (POISSON_FP64 handles) or FP32.  poisson_create returns EINVAL when the grid has no coarser
 * level (every axis of one cell, or periodic x of odd nx with ny = nz = 1).  With FP32 inner
 * solves an inner_tol of 1e-5 takes one refinement step fewer than the default 1e-4 on the
 * strut and wedge workloads. */
#define POISSON_MG 2

#define POISSON_MEM_HOST 0
#define POISSON_MEM_DEVICE 1

typedef struct poisson_s poisson_t; /* opaque; the library owns all device state of a handle */

typedef struct {
    int precision;     /* POISSON_FP64 | POISSON_FP32 | POISSON_FP32_BF16COEF (default FP32)     */
    int precond;       /* POISSON_JACOBI | POISSON_RBSSOR | POISSON_MG (default JACOBI)           */
    double omega;      /* SSOR relaxation factor in (0, 2) (default 1.0)                           */
    int max_iters;     /* cap on total CG iterations of one solve (default 20000)                  */
    double inner_tol;  /* FP32 inner solve: relative residual reduction per refinement step
                          (default 1e-4; ignored by POISSON_FP64)                                  */
    int tile;          /* FP32 inner-solve kernels.  0 = TMA plane-marching kernels, variant and
                          z-chunk autotuned per shape (when nx % 8 == 0, else the column
                          kernels); -1 = column kernels (plain loads); 10000000 F + 1000000 P +
                          100000 S + 10000 WS + 1000 CX + 100 CY + T = persistent marching
                          kernel with T rows of 32 threads, each owning CX x CY cells (tile
                          32 CX x CY T), a TMA producer warp when WS = 1 and an S-stage plane
                          ring (S omitted = 4).  F = 0, two sweeps per CG iteration: 1108, 2204,
                          2208, 12204, 12208, 302204, 302208, 312208, 602204, 612208; F = 1, one
                          sweep per iteration (Chronopoulos-Gear recurrences): 12204, 312204,
                          312208 (plus 10000000); F = 2, one sweep with A p formed in it (2-cell
                          halos, u, p, x and eta in memory): 12204, 512204, 12208 (plus
                          20000000); F = 3, red-black SSOR in reduced form (RBSSOR handles
                          only): 812204, 712204, 812108, 712208.  P = split of the tile columns
                          over the CTAs: 0 equal planes per CTA, 1 balanced (segment start cost
                          counted), 2 lockstep (neighbouring tiles on the same planes), 3 lockstep
                          then the leftover columns cut evenly over all CTAs (default 0)        */
    void* stream;      /* cudaStream_t to run on; NULL = the legacy default stream                 */
    int dirichlet_walls; /* side/bottom walls with p = 0 on the wall face instead of a zero normal
                          gradient: a bitmask of POISSON_WALL_* (default 0, the paper's walls);
                          the top face z = Lz always has p = 0.  Each such wall adds 2/rho_c to
                          the diagonal of the cells that touch it and, in poisson_project, its
                          face is corrected with 1/rho_c over the half cell.                    */
    int periodic_x;    /* 1: x periodic (the cells i = 0 and i = nx-1 of a row are neighbours
                          through the face x = 0 = Lx, as in the paper's strut run); no x walls
                          then (EINVAL with POISSON_WALL_XM/XP), red-black SSOR needs an even nx,
                          and the inner solve runs on the column kernels.  Face arrays of
                          poisson_divergence / poisson_project keep nx+1 x-faces; faces 0 and nx
                          are the same face (poisson_project writes both).  Default 0.         */
} poisson_opts;

typedef struct {
    int outer_iters;      /* FP64 refinement steps (1 for POISSON_FP64)                           */
    int inner_iters;      /* CG iterations in total                                                */
    double rel_residual;  /* ||b - A p||_2 / ||b||_2 of the returned p, in FP64 on the device      */
    double seconds;       /* wall time of the call                                                 */
} poisson_stats;

/* Fill *opts with the defaults above. */
void poisson_default_opts(poisson_opts* opts);

/* Create a handle for an nx x ny x nz grid of spacing h (Formulation; uniform grid).  opts may be
 * NULL (defaults).  Allocates the handle's device state.  Errors: EINVAL (a size <= 0, h <= 0,
 * bad option), ENOMEM, ECUDA.  *out is set only on success. */
int poisson_create(int nx, int ny, int nz, double h, const poisson_opts* opts, poisson_t** out);

/* Release the handle and its device memory (after synchronising its stream).  NULL is a no-op.
 * Errors: EINVAL while the handle is in a batch job that poisson_poll has not reported (the
 * handle is left as it was). */
int poisson_destroy(poisson_t* h);

/* ------------------------------------------------------------------ device-memory budget
 * For admission by a device-memory budget (a served request loop creates handles as memory
 * frees up).  poisson_required_bytes: the device bytes a handle of this grid and these options
 * (NULL = defaults) holds once poisson_create has returned -- its arrays, its multigrid hierarchy
 * (POISSON_MG), and an upper bound on its persistent-launch plan -- counted from the same list of
 * arrays that poisson_create allocates; the caller's own arrays are not included.  budget > 0:
 * returns POISSON_ENOMEM_BUDGET when the bytes exceed it (*bytes is still set); budget 0: no
 * check.  No device memory is touched.  Errors: EINVAL (NULL bytes, bad sizes or options as for
 * poisson_create). */
int poisson_required_bytes(int nx, int ny, int nz, const poisson_opts* opts, uint64_t budget,
                           uint64_t* bytes);

/* The device bytes the handle holds now: the arrays of poisson_required_bytes (its plan at its
 * actual size) plus what later calls added (cut-cell fractions, staging buffers of the checking
 * entry points given host arrays).  Errors: EINVAL. */
int poisson_handle_bytes(poisson_t* h, uint64_t* bytes);

/* Set the density from the water fraction F (eq. (density), rho = rho_air + F (rho_water -
 * rho_air)) and build the operator: face coefficients (harmonic means), diagonal, and the
 * reduced-precision copies.  F: nx*ny*nz doubles; mem = POISSON_MEM_HOST or POISSON_MEM_DEVICE
 * says where F lives (checked against the pointer).  F is read during the call only.
 * Errors: EINVAL (NULL, rho <= 0, mem mismatch; or some cell's density is not a positive finite
 * number -- F non-finite, or far enough outside [0, 1] -- in which case the handle is left not
 * ready and solves return ENOTREADY until a valid density is set), ECUDA. */
int poisson_set_density(poisson_t* h, const double* F, double rho_air, double rho_water, int mem);

/* Solve div((1/rho) grad p) = rhs (eq. (pois)) to relative residual ||b - A p|| / ||b|| <= tol,
 * where A is the FP64 operator and b = -h^2 rhs.  rhs: the source s = div(u*)/dt, nx*ny*nz
 * doubles.  p: on entry the initial guess (warm start; zeros for none), on exit the solution.
 * stats may be NULL.  An all-zero rhs returns p = 0 and OK.  Errors: ENOTREADY (no density set),
 * EINVAL (NULL, tol <= 0), ENOTCONV (cap reached: p = best iterate, stats = its residual),
 * EBREAKDOWN (also for a non-finite rhs or initial guess: the first residual norm is then not
 * finite; p is unspecified), ECUDA.  The handle stays usable after any of these. */
int poisson_solve(poisson_t* h, const double* rhs, double* p, double tol, poisson_stats* stats);

/* y = A x with the handle's operator at the given precision (A = -h^2 div_h((1/rho) grad_h)).
 * POISSON_FP64 uses the FP64 face coefficients; POISSON_FP32 / _BF16COEF apply the inner
 * reduced-precision operator with FP32 vectors (x is rounded to float, y widened back).
 * x, y: nx*ny*nz doubles, distinct.  Errors: ENOTREADY, EINVAL, ECUDA. */
int poisson_apply(poisson_t* h, const double* x, double* y, int precision);

/* z = M^{-1} r for the preconditioner kind (POISSON_JACOBI, POISSON_RBSSOR with the handle's
 * omega, POISSON_MG) at the given precision, with M built from the operator of that precision:
 * Jacobi M = D; SSOR M = (D - wE) D^{-1} (D - wE^T) / (w (2 - w)) in red-black order (red =
 * (i+j+k) even first, A = D - E - E^T); MG one V-cycle of the handle's hierarchy (only on a
 * POISSON_MG handle and at its own precision, else EINVAL; the FP32 cycle uses the handle's
 * inner FP32 vectors as scratch).  Errors: ENOTREADY, EINVAL, ECUDA. */
int poisson_precond_apply(poisson_t* h, const double* r, double* z, int kind, int precision);

/* Copy out the FP64 operator: low-side face coefficients bx, by, bz (bx[c] couples cell c with
 * its -x neighbour, 0 on the wall) and the diagonal.  Any pointer may be NULL to skip it.
 * Errors: ENOTREADY, ECUDA. */
int poisson_get_operator(poisson_t* h, double* bx, double* by, double* bz, double* diag);

/* ------------------------------------------------------------------ batched solves
 * Many independent solves of uneven size driven together.  Every FP64 refinement step of the
 * batch is one batched residual kernel, one batched CG start and ONE cooperative persistent
 * PCG launch over all unfinished solves (captured in CUDA graphs, rebuilt when the batch
 * changes).  Solves submitted while a batch runs join it at its next refinement step
 * (continuous batching).  Handles with POISSON_FP64, POISSON_RBSSOR or nx % 8 != 0 are solved
 * one by one with poisson_solve when polled.
 * poisson_batch_submit enqueues n solves (handles[i] with its density already set, rhs[i],
 * p[i] in/out as in poisson_solve, tol[i]) and returns a ticket per solve.  The arrays must stay
 * valid, and the handles must not be used or destroyed, until poisson_poll reports the ticket.
 * A handle may belong to one unreported ticket at a time.  Errors: EINVAL, ENOTREADY. */
int poisson_batch_submit(poisson_t* const* handles, const double* const* rhs, double* const* p,
                         const double* tol, int n, uint64_t* tickets);

/* POISSON_PENDING while the ticket's solve runs; then its final status (OK, ENOTCONV, ...),
 * with *stats filled (may be NULL); a finished ticket is forgotten after it is reported once.
 * Polling drives the batch: a poll of an unfinished ticket runs one refinement step of its
 * batch (or, for a one-by-one solve, the solve) before it returns. */
int poisson_poll(uint64_t ticket, poisson_stats* stats);

/* ------------------------------------------------------------------ instrumentation */
/* Kernel classes timed by poisson_profile (indices into poisson_kernel_times). */
#define POISSON_K_CG_A 0      /* CG phase A: p = z + beta p, sum p.Ap                      */
#define POISSON_K_CG_B 1      /* CG phase B: x, r, z updates, sums r.z and r.r             */
#define POISSON_K_RESIDUAL 2  /* FP64 residual b - A x and its norm                        */
#define POISSON_K_OTHER 3     /* set-up, scaling, refinement update, CG init               */
#define POISSON_K_PCG 4       /* persistent PCG: every iteration of one inner solve         */
#define POISSON_K_CLASSES 5

typedef struct {
    long long launches[POISSON_K_CLASSES]; /* kernel launches per class                     */
    double ms[POISSON_K_CLASSES];          /* summed CUDA-event time per class, ms           */
} poisson_kernel_times;

/* Total CUDA kernel launches issued by this library (all handles) since it was loaded. */
uint64_t poisson_kernel_launches(void);

/* enable != 0: record a CUDA event pair on the handle's stream around every CG phase and
 * residual kernel of later solves, and zero the accumulated times; 0 turns recording off.
 * The events add no device work; their host-side cost is a few microseconds per launch. */
int poisson_profile(poisson_t* h, int enable);

/* Copy out the accumulated per-class launch counts and event times (since poisson_profile). */
int poisson_profile_read(poisson_t* h, poisson_kernel_times* out);

/* ------------------------------------------------------------------ cut cells
 * Free-slip bodies as cut cells (Enforcement of Body Boundary Conditions: area and volume
 * fractions enter the Poisson equation and the projection, which sets the velocity normal to the
 * hull to zero).  ax, ay, az: open fractions in [0, 1] of the MAC faces (the shapes of the face
 * arrays of poisson_divergence: (nx+1) x ny x nz, nx x (ny+1) x nz, nx x ny x (nz+1), x fastest);
 * vol: fluid fractions in [0, 1] of the cells (nx*ny*nz).  Every face coefficient (interior, top,
 * Dirichlet wall) is scaled by its face's open fraction; a face of a cell with vol = 0 is closed
 * and such a cell is inactive (its pressure comes out 0); the solve's right side becomes
 * -h^2 vol rhs, poisson_divergence returns the open-fraction-weighted flux difference over
 * (h dt vol), and poisson_project corrects each open face with the face's own coefficient.  The
 * arrays are copied (host or device, as mem says; the caller keeps ownership).  Call before
 * poisson_set_density (a later call needs set_density again: ENOTREADY until then); all four
 * NULL returns to the plain operator.  With cut cells the inner FP32 solve runs on the column
 * kernels with FP32 copies of the cut faces (also for POISSON_FP32_BF16COEF).
 * Errors: EINVAL (some NULL, mem mismatch), ENOMEM, ECUDA. */
int poisson_set_apertures(poisson_t* h, const double* ax, const double* ay, const double* az,
                          const double* vol, int mem);

/* ------------------------------------------------------------------ projection
 * Numerical Time Integration: each stage forms a provisional velocity u* on the cell faces
 * (MAC grid), solves div((1/rho) grad p) = div(u*)/dt, and corrects u = u* - dt (1/rho) grad p.
 * Face arrays are doubles, x fastest:
 *   u: (nx+1) x ny x nz -- u[i + (nx+1)(j + ny k)] is on the face between cells i-1 and i;
 *      faces i = 0 and i = nx are the walls x = 0, x = Lx;
 *   v: nx x (ny+1) x nz, likewise in y (walls at j = 0, ny);
 *   w: nx x ny x (nz+1), likewise in z; the bottom k = 0 is a wall, k = nz the top boundary.
 * Host or device pointers (each detected; host arrays are staged through temporary device
 * buffers); the caller owns them.  Both calls wait for the handle's stream before returning. */

/* s_c = [(u_{i+1} - u_i) + (v_{j+1} - v_j) + (w_{k+1} - w_k)] / (h dt), in that order: the
 * source of the pressure equation for poisson_solve.  s: nx*ny*nz doubles.  Needs only the
 * handle's grid.  Errors: EINVAL (NULL, dt <= 0 or not finite), ENOMEM, ECUDA. */
int poisson_divergence(poisson_t* h, const double* u, const double* v, const double* w,
                       double dt, double* s);

/* In place, on every face: u_f <- u_f - dt (beta_f ((p_n - p_c) / h)) with the face coefficients
 * of the last poisson_set_density (beta_f = 2/(rho_c + rho_n); (p_n - p_c) across the face in
 * the +axis direction); on the top face, where p = 0, u_f <- u_f - dt ((2/rho_c)((0 - p_c)/h)),
 * i.e. 1/rho_c times the gradient over the half cell, and the same on the faces of the handle's
 * Dirichlet walls (poisson_opts.dirichlet_walls); zero-gradient wall faces are left as they are.
 * Then
 * div_h(u)/dt = div_h(u*)/dt - div_h((1/rho) grad_h p): with p from poisson_solve for
 * s = div(u*)/dt, the divergence left is the solve's residual, (A p - b)/h^2.  p: nx*ny*nz
 * doubles.  Errors: EINVAL, ENOTREADY (before set_density), ENOMEM, ECUDA. */
int poisson_project(poisson_t* h, double* u, double* v, double* w, const double* p, double dt);

/* Reduced pressure (Entrance and Exit Boundary Conditions, hydrostatic-pressure method).  Solving
 * for P_r = P - rho g (z - z_o), z_o the static free-surface height, puts the force
 * -(z - z_o) (1/rho) d(rho g)/dx_i into the momentum equations -- in the paper's units
 * (rho = lambda + (1 - lambda) H) -(z - z_o)(1 - lambda) g (1/rho) dH/dx_i -- which gives P_r a
 * jump of (z - z_o)(1 - lambda) g across the interface.  The force is a term of the provisional
 * velocity: this call adds dt f to the face velocities u, v, w in place (shapes as for
 * poisson_divergence), after which poisson_divergence gives the source for P_r and
 * poisson_project removes the force's gradient part.  On the face between cells c and n (n on the
 * +axis side): f = -(z_f - z_o) g (2/(rho_c + rho_n)) (rho_n - rho_c) / h, rho from F as in
 * poisson_set_density, z_f the face's height ((k + 1/2) h on the x and y faces of layer k, k h
 * on the z face below layer k; the grid's z = 0 is the bottom); no force on the walls and the
 * top face (H continued beyond the boundary without change along its normal); with periodic x
 * the wrap face is written to faces 0 and nx.  g is the coefficient as the paper writes it: the
 * gravity term this replaces is +g in the z momentum equation (g < 0 for z pointing up).  At rest
 * (u* = 0, a layered density) the projected velocity vanishes and P_r is the column with those
 * jumps and P_r = 0 in the top layer.  F: nx*ny*nz doubles; host or device pointers (host arrays
 * are staged through temporary device buffers); the call waits for the handle's stream.
 * Errors: EINVAL (NULL, rho <= 0, a non-finite argument), ENOMEM, ECUDA. */
int poisson_hydrostatic_force(poisson_t* h, const double* F, double rho_air, double rho_water,
                              double g, double z_o, double dt, double* u, double* v, double* w);

/* ------------------------------------------------------------------ allocation-free check
 * The paper has no counterpart to this entry point.  It is for callers that cannot allocate
 * device memory when they check a pressure field: a step loop that must not pay cudaMalloc's
 * latency or cudaFree's implicit device synchronisation, a process whose device memory belongs
 * to another allocator under a fixed budget, or code that forbids dynamic allocation after
 * initialisation.  Without any handle and without allocating, it computes the FP64 relative
 * residual ||b - A p||_2 / ||b||_2 with b = -h^2 rhs and A the operator of the paper's
 * configuration built on the fly from F: rho = rho_air + F (rho_water - rho_air), interior face
 * coefficients 2/(rho_c + rho_n), zero normal gradient on the side and bottom walls, and p = 0
 * on the top face, which adds 2/rho_c to the diagonal.  For a handle created with
 * dirichlet_walls = 0, periodic_x = 0 and no cut-cell geometry this is the figure poisson_solve
 * reports in stats->rel_residual; for other handles the two figures differ.  Its only scratch is
 * a 64 KiB static device array of the library, which every GPU that loads the library holds
 * until the process exits.
 *   F, rhs, p: device arrays of nx*ny*nz doubles (x fastest); host arrays give EINVAL.
 *   rho_air, rho_water: finite and > 0, else EINVAL.
 *   rel_residual: one double, host or device memory (a device output is written on the stream
 *     without waiting; a host output waits for the stream).  0 for an all-zero rhs.
 *   stream: cudaStream_t to run on (NULL = legacy default stream).
 * Limit: the x-y plane may span at most 4096 tiles of 32 x 8 cells (e.g. 2048 x 512 cells);
 * larger grids give POISSON_ETOOLARGE.  The first call on a device looks up the array's device
 * address (with that device current); make that first call before any stream capture.  All
 * calls on a device share the array: calls that overlap on the GPU (other streams, other
 * threads) race and must be serialised by the caller.  Errors: EINVAL, ETOOLARGE, ECUDA. */
int poisson_residual_noalloc(int nx, int ny, int nz, double h, const double* F, double rho_air,
                             double rho_water, const double* rhs, const double* p,
                             double* rel_residual, void* stream);

/* ------------------------------------------------------------------ failure-path test aid
 * A testing aid with no counterpart in the paper.  extra > 0 makes the grid barriers of the
 * handle's persistent FP32 PCG launches wait for `extra` more CTAs than are launched, so the
 * first barrier of the next solve can never complete: every CTA gives up when the barrier's
 * deadline (1 s of the GPU's global timer) runs out, lets its TMA copies in flight land and
 * leaves, and poisson_solve returns POISSON_ETIMEOUT with p holding the iterate reached.  The
 * CUDA context stays usable; extra = 0 restores normal launches.  It exists so that tests can
 * exercise the bounded-wait failure path without faulting or hanging the GPU.
 * Errors: EINVAL (NULL, extra < 0 or > 1024, or a handle whose inner solve does not use a
 * persistent launch: POISSON_FP64, RBSSOR, MG, cut cells, nx % 8 != 0, tile = -1). */
int poisson_test_unreachable_barrier(poisson_t* h, int extra);

/* Testing aids for the allocation error paths (the failure is injected on the host; nothing
 * faults on the GPU).  poisson_test_fail_alloc(n): the n-th device or pinned-host allocation the
 * library makes from now on, in any thread, fails as if memory were exhausted, and the call that
 * made it returns POISSON_ENOMEM after releasing what it had allocated (n = 0: no failure;
 * process-wide; EINVAL for n < 0).  poisson_test_live_allocations: the number of the library's
 * device and pinned-host allocations made and not yet released (every handle, plan, staging
 * buffer and batch table counts).  Errors: EINVAL (NULL). */
int poisson_test_fail_alloc(int n);
int poisson_test_live_allocations(long long* out);

/* Write a one-line description of the handle's kernel choice (family, tile, z-chunk) into buf
 * (NUL-terminated, at most len bytes). */
int poisson_describe(poisson_t* h, char* buf, int len);

/* Human-readable name of a status code. */
const char* poisson_strerror(int status);

/* Library version string. */
const char* poisson_version(void);

#ifdef __cplusplus
}
#endif

#endif /* POISSON_H */

/*
 * poisson_oracle.c -- plain FP64 CPU oracle for the pressure Poisson solve.
 *
 * TEST INFRASTRUCTURE.  Only the test suite, the smoke check and the benchmark's CPU-baseline leg
 * may load this code.  It shares nothing with the CUDA library: it is written from the paper's
 * statement of the problem, as plain loops, for a reader to check by eye.
 *
 * What it computes (Formulation, eqs. (density) and (pois); Introduction: "second-order,
 * variable-coefficient Poisson equation ... preconditioned conjugate-gradient method"):
 *
 *   rho_c  = rho_air + F_c (rho_water - rho_air)                 density from the water fraction
 *   beta_f = 2 / (rho_c + rho_n)                                 face coefficient: harmonic mean
 *                                                                of 1/rho_c and 1/rho_n
 *   walls x = 0, Lx, y = 0, Ly, z = 0: beta_f = 0                (zero normal gradient)
 *   top   z = Lz: p = 0 on the face; ghost value -p_c, so the face contributes 2 (1/rho_c) p_c
 *
 *   (A p)_c = D_c p_c - sum_{faces f of c} beta_f p_{n(f)},    D_c = sum_f beta_f + 2/rho_c [top]
 *
 * A = -h^2 L with L p = div_h(beta grad_h p); A is symmetric positive definite.  The solve of
 * div((1/rho) grad p) = s is A p = b with b = -h^2 s.
 *
 * Array layout: x fastest, linear index c = i + nx (j + ny k).  The face arrays hold the face on
 * the LOW side of each cell: bx[c] couples (i-1, j, k) and (i, j, k) and is 0 for i = 0; by[c]
 * and bz[c] likewise.  The high face of cell c is the low face of its +x/+y/+z neighbour (0 at
 * the last cell except the top, whose Dirichlet term lives in D).
 *
 * Preconditioners (the paper names none; Jacobi and red-black SSOR are the two readings used):
 *   Jacobi:  z = D^{-1} r.
 *   SSOR(w): with A = D - E - E^T in red-black order (red = (i+j+k) even, first),
 *            M = (D - wE) D^{-1} (D - wE^T) / (w (2 - w)); z = M^{-1} r is
 *              y_R = r_R / D_R
 *              y_B = (r_B + w sum_{red nbrs} beta y) / D_B
 *              t_R = y_R + w (sum_{black nbrs} beta y) / D_R        (t_B = y_B)
 *              z   = w (2 - w) t.
 *
 * PCG (textbook preconditioned conjugate gradients): r = b - A x; z = M^{-1} r; p = z; loop
 * { q = A p; alpha = (r.z)/(p.q); x += alpha p; r -= alpha q; stop when ||r||/||b|| <= tol and the
 * recomputed residual b - A x confirms it; z = M^{-1} r; beta = (r.z)_new/(r.z)_old; p = z + beta p }.
 * Floating-point contraction is disabled at build time so results do not depend on the host ISA.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_OK 0
#define OR_EINVAL -1
#define OR_ENOMEM -2
#define OR_ENOTCONV -3
#define OR_EBREAKDOWN -4

#define OR_JACOBI 0
#define OR_SSOR 1

#define OR_MEAN_HARMONIC 0   /* beta_f = 2/(rho_c + rho_n): harmonic mean of 1/rho */
#define OR_MEAN_ARITHMETIC 1 /* beta_f = (1/rho_c + 1/rho_n)/2: rejected reading, kept for tests */

typedef int64_t idx_t;

int oracle_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void oracle_set_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

/* ---------------------------------------------------------------------------- operator setup */
/* walls: bitmask of the side and bottom walls that carry p = 0 instead of a zero normal gradient
 * (1 x = 0, 2 x = Lx, 4 y = 0, 8 y = Ly, 16 z = 0); like the top face, such a wall adds
 * 2 (1/rho_c) to the diagonal of the cells that touch it and couples them to nothing. */
#define OR_WALL_XM 1
#define OR_WALL_XP 2
#define OR_WALL_YM 4
#define OR_WALL_YP 8
#define OR_WALL_ZM 16
/* periodic x: the low face of cell (0, j, k) couples it to (nx-1, j, k); no x walls.  The
 * operator functions recognise it by that face's nonzero coefficient (it is 0 without
 * periodicity). */
#define OR_PERIODIC_X 32

/* Cut cells (free-slip bodies, Enforcement of Body Boundary Conditions): ax, ay, az are the open
 * fractions of the faces on the MAC face arrays ((nx+1) x ny x nz, nx x (ny+1) x nz,
 * nx x ny x (nz+1), x fastest) and vol the fluid fraction of each cell.  Every face coefficient
 * (interior, top, Dirichlet wall) is multiplied by its face's open fraction; a face of a cell with
 * vol = 0 counts as closed; a cell with vol = 0 is inactive: diagonal 1, no coupling (its pressure
 * is 0 for a zero right side).  NULL apertures: all faces open, all cells active. */
static double face_open(const double* a, idx_t f) { return a ? a[f] : 1.0; }

int oracle_faces_cut(int nx, int ny, int nz, const double* F, double rho_air, double rho_water,
                     int mean, int walls, const double* ax, const double* ay, const double* az,
                     const double* vol, double* bx, double* by, double* bz, double* diag) {
    if (nx <= 0 || ny <= 0 || nz <= 0 || !F || !bx || !by || !bz || !diag) return OR_EINVAL;
    const idx_t n = (idx_t)nx * ny * nz;
    double* rho = (double*)malloc(sizeof(double) * (size_t)n);
    if (!rho) return OR_ENOMEM;
    for (idx_t c = 0; c < n; ++c) rho[c] = rho_air + F[c] * (rho_water - rho_air);

#pragma omp parallel for schedule(static)
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                idx_t c = i + (idx_t)nx * (j + (idx_t)ny * k);
                double rc = rho[c];
                double fx = 0.0, fy = 0.0, fz = 0.0;
                if (i > 0 || (walls & OR_PERIODIC_X)) {
                    double rn = rho[i > 0 ? c - 1 : c + nx - 1];
                    fx = (mean == OR_MEAN_HARMONIC) ? 2.0 / (rc + rn) : 0.5 * (1.0 / rc + 1.0 / rn);
                }
                if (j > 0) {
                    double rn = rho[c - nx];
                    fy = (mean == OR_MEAN_HARMONIC) ? 2.0 / (rc + rn) : 0.5 * (1.0 / rc + 1.0 / rn);
                }
                if (k > 0) {
                    double rn = rho[c - (idx_t)nx * ny];
                    fz = (mean == OR_MEAN_HARMONIC) ? 2.0 / (rc + rn) : 0.5 * (1.0 / rc + 1.0 / rn);
                }
                if (ax) {
                    const idx_t fu = (idx_t)i + (idx_t)(nx + 1) * ((idx_t)j + (idx_t)ny * k);
                    const idx_t fv = (idx_t)i + (idx_t)nx * ((idx_t)j + (idx_t)(ny + 1) * k);
                    const int act = vol[c] > 0.0;
                    const idx_t cxm = i > 0 ? c - 1 : c + nx - 1;
                    fx = (act && vol[cxm] > 0.0) ? ax[fu] * fx : 0.0;
                    fy = (act && j > 0 && vol[c - nx] > 0.0) ? ay[fv] * fy : 0.0;
                    fz = (act && k > 0 && vol[c - (idx_t)nx * ny] > 0.0) ? az[c] * fz : 0.0;
                }
                bx[c] = fx;
                by[c] = fy;
                bz[c] = fz;
            }

    /* diagonal: the six faces of the cell plus the Dirichlet top term */
#pragma omp parallel for schedule(static)
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                idx_t c = i + (idx_t)nx * (j + (idx_t)ny * k);
                if (vol && !(vol[c] > 0.0)) {
                    diag[c] = 1.0; /* inactive cell */
                    continue;
                }
                const idx_t fu = (idx_t)i + (idx_t)(nx + 1) * ((idx_t)j + (idx_t)ny * k);
                const idx_t fv = (idx_t)i + (idx_t)nx * ((idx_t)j + (idx_t)(ny + 1) * k);
                const idx_t sxy = (idx_t)nx * ny;
                double d = bx[c] + by[c] + bz[c];
                if (i + 1 < nx) d += bx[c + 1];
                else if (walls & OR_PERIODIC_X) d += bx[c + 1 - nx];
                if (j + 1 < ny) d += by[c + nx];
                if (k + 1 < nz) d += bz[c + sxy];
                else d += face_open(az, c + sxy) * (2.0 / rho[c]);
                if ((walls & OR_WALL_XM) && i == 0) d += face_open(ax, fu) * (2.0 / rho[c]);
                if ((walls & OR_WALL_XP) && i == nx - 1) d += face_open(ax, fu + 1) * (2.0 / rho[c]);
                if ((walls & OR_WALL_YM) && j == 0) d += face_open(ay, fv) * (2.0 / rho[c]);
                if ((walls & OR_WALL_YP) && j == ny - 1) d += face_open(ay, fv + nx) * (2.0 / rho[c]);
                if ((walls & OR_WALL_ZM) && k == 0) d += face_open(az, c) * (2.0 / rho[c]);
                diag[c] = d;
            }
    free(rho);
    return OR_OK;
}

int oracle_faces_bc(int nx, int ny, int nz, const double* F, double rho_air, double rho_water,
                    int mean, int walls, double* bx, double* by, double* bz, double* diag) {
    return oracle_faces_cut(nx, ny, nz, F, rho_air, rho_water, mean, walls, NULL, NULL, NULL, NULL,
                            bx, by, bz, diag);
}

int oracle_faces(int nx, int ny, int nz, const double* F, double rho_air, double rho_water,
                 int mean, double* bx, double* by, double* bz, double* diag) {
    return oracle_faces_bc(nx, ny, nz, F, rho_air, rho_water, mean, 0, bx, by, bz, diag);
}

/* ---------------------------------------------------------------------------- y = A x */
void oracle_apply(int nx, int ny, int nz, const double* bx, const double* by, const double* bz,
                  const double* diag, const double* x, double* y) {
    const idx_t sx = 1, sy = nx, sz = (idx_t)nx * ny;
#pragma omp parallel for schedule(static)
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                idx_t c = i + (idx_t)nx * (j + (idx_t)ny * k);
                double v = diag[c] * x[c];
                if (i > 0) v -= bx[c] * x[c - sx];
                else if (bx[c] != 0.0) v -= bx[c] * x[c + nx - 1];            /* periodic x */
                if (i + 1 < nx) v -= bx[c + sx] * x[c + sx];
                else if (bx[c + 1 - nx] != 0.0) v -= bx[c + 1 - nx] * x[c + 1 - nx];
                if (j > 0) v -= by[c] * x[c - sy];
                if (j + 1 < ny) v -= by[c + sy] * x[c + sy];
                if (k > 0) v -= bz[c] * x[c - sz];
                if (k + 1 < nz) v -= bz[c + sz] * x[c + sz];
                y[c] = v;
            }
}

/* Sum over the six neighbours of c of beta_f * v_n.  Every neighbour of a red cell is black and
 * vice versa, so for a black cell this reads red entries only (and the converse). */
static double nb_sum(int nx, int ny, int nz, const double* bx, const double* by, const double* bz,
                     const double* v, int i, int j, int k) {
    const idx_t sx = 1, sy = nx, sz = (idx_t)nx * ny;
    idx_t c = i + (idx_t)nx * (j + (idx_t)ny * k);
    double s = 0.0;
    if (i > 0) s += bx[c] * v[c - sx];
    else if (bx[c] != 0.0) s += bx[c] * v[c + nx - 1];                      /* periodic x */
    if (i + 1 < nx) s += bx[c + sx] * v[c + sx];
    else if (bx[c + 1 - nx] != 0.0) s += bx[c + 1 - nx] * v[c + 1 - nx];
    if (j > 0) s += by[c] * v[c - sy];
    if (j + 1 < ny) s += by[c + sy] * v[c + sy];
    if (k > 0) s += bz[c] * v[c - sz];
    if (k + 1 < nz) s += bz[c + sz] * v[c + sz];
    return s;
}

/* ---------------------------------------------------------------------------- z = M^{-1} r */
void oracle_precond(int nx, int ny, int nz, const double* bx, const double* by, const double* bz,
                    const double* diag, int kind, double omega, const double* r, double* z) {
    const idx_t n = (idx_t)nx * ny * nz;
    if (kind == OR_JACOBI) {
#pragma omp parallel for schedule(static)
        for (idx_t c = 0; c < n; ++c) z[c] = r[c] / diag[c];
        return;
    }
    /* red-black SSOR: forward sweep (red then black), backward sweep (red), scale */
    const double w = omega;
    /* y_R = r_R / D_R ; z holds y, black entries are written next */
#pragma omp parallel for schedule(static)
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                idx_t c = i + (idx_t)nx * (j + (idx_t)ny * k);
                if (((i + j + k) & 1) == 0) z[c] = r[c] / diag[c];
            }
    /* y_B = (r_B + w sum_red beta y) / D_B */
#pragma omp parallel for schedule(static)
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                idx_t c = i + (idx_t)nx * (j + (idx_t)ny * k);
                if (((i + j + k) & 1) == 1)
                    z[c] = (r[c] + w * nb_sum(nx, ny, nz, bx, by, bz, z, i, j, k)) / diag[c];
            }
    /* t_R = y_R + w (sum_black beta y) / D_R */
#pragma omp parallel for schedule(static)
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                idx_t c = i + (idx_t)nx * (j + (idx_t)ny * k);
                if (((i + j + k) & 1) == 0)
                    z[c] = z[c] + w * nb_sum(nx, ny, nz, bx, by, bz, z, i, j, k) / diag[c];
            }
    const double scale = w * (2.0 - w);
#pragma omp parallel for schedule(static)
    for (idx_t c = 0; c < n; ++c) z[c] *= scale;
}

/* ---------------------------------------------------------------------------- vector helpers */
static double dot(idx_t n, const double* a, const double* b) {
    double s = 0.0;
#pragma omp parallel for reduction(+ : s) schedule(static)
    for (idx_t c = 0; c < n; ++c) s += a[c] * b[c];
    return s;
}

/* r = b - A x; returns ||r||_2 */
double oracle_residual(int nx, int ny, int nz, const double* bx, const double* by,
                       const double* bz, const double* diag, const double* b, const double* x,
                       double* r) {
    const idx_t n = (idx_t)nx * ny * nz;
    oracle_apply(nx, ny, nz, bx, by, bz, diag, x, r);
#pragma omp parallel for schedule(static)
    for (idx_t c = 0; c < n; ++c) r[c] = b[c] - r[c];
    return sqrt(dot(n, r, r));
}

double oracle_norm2(idx_t n, const double* v) { return sqrt(dot(n, v, v)); }

/* ---------------------------------------------------------------------------- PCG
 * x: in = initial guess, out = solution.  On return iters = PCG iterations taken and
 * relres = ||b - A x||_2 / ||b||_2 recomputed from x.  tol <= 0 runs exactly max_iters
 * iterations (used to time a fixed window).  history (may be NULL) receives the recurrence
 * residual norm ||r||/||b|| after every iteration, up to max_iters entries. */
int oracle_pcg(int nx, int ny, int nz, const double* bx, const double* by, const double* bz,
               const double* diag, const double* b, double* x, double tol, int kind, double omega,
               int max_iters, int* iters_out, double* relres_out, double* history) {
    if (nx <= 0 || ny <= 0 || nz <= 0 || !b || !x || max_iters < 0) return OR_EINVAL;
    const idx_t n = (idx_t)nx * ny * nz;
    double* r = (double*)malloc(sizeof(double) * (size_t)n);
    double* z = (double*)malloc(sizeof(double) * (size_t)n);
    double* p = (double*)malloc(sizeof(double) * (size_t)n);
    double* q = (double*)malloc(sizeof(double) * (size_t)n);
    if (!r || !z || !p || !q) {
        free(r); free(z); free(p); free(q);
        return OR_ENOMEM;
    }
    int status = OR_ENOTCONV;
    int it = 0;
    const double bnorm = oracle_norm2(n, b);
    if (bnorm == 0.0) {
        memset(x, 0, sizeof(double) * (size_t)n);
        if (iters_out) *iters_out = 0;
        if (relres_out) *relres_out = 0.0;
        free(r); free(z); free(p); free(q);
        return OR_OK;
    }

    double rnorm = oracle_residual(nx, ny, nz, bx, by, bz, diag, b, x, r);
    if (tol > 0.0 && rnorm / bnorm <= tol) { status = OR_OK; goto done; }
    oracle_precond(nx, ny, nz, bx, by, bz, diag, kind, omega, r, z);
    memcpy(p, z, sizeof(double) * (size_t)n);
    double rz = dot(n, r, z);

    while (it < max_iters) {
        oracle_apply(nx, ny, nz, bx, by, bz, diag, p, q);
        const double pq = dot(n, p, q);
        if (!(pq > 0.0) || !isfinite(pq)) { status = OR_EBREAKDOWN; break; }
        const double alpha = rz / pq;
#pragma omp parallel for schedule(static)
        for (idx_t c = 0; c < n; ++c) {
            x[c] += alpha * p[c];
            r[c] -= alpha * q[c];
        }
        ++it;
        rnorm = oracle_norm2(n, r);
        if (history) history[it - 1] = rnorm / bnorm;
        if (tol > 0.0 && rnorm / bnorm <= tol) {
            /* confirm with the recomputed residual; if the recurrence drifted, restart from it */
            rnorm = oracle_residual(nx, ny, nz, bx, by, bz, diag, b, x, r);
            if (rnorm / bnorm <= tol) { status = OR_OK; break; }
            oracle_precond(nx, ny, nz, bx, by, bz, diag, kind, omega, r, z);
            memcpy(p, z, sizeof(double) * (size_t)n);
            rz = dot(n, r, z);
            continue;
        }
        oracle_precond(nx, ny, nz, bx, by, bz, diag, kind, omega, r, z);
        const double rz_new = dot(n, r, z);
        const double beta = rz_new / rz;
        rz = rz_new;
#pragma omp parallel for schedule(static)
        for (idx_t c = 0; c < n; ++c) p[c] = z[c] + beta * p[c];
    }
done:
    rnorm = oracle_residual(nx, ny, nz, bx, by, bz, diag, b, x, r);
    if (iters_out) *iters_out = it;
    if (relres_out) *relres_out = rnorm / bnorm;
    if (status == OR_ENOTCONV && tol <= 0.0) status = OR_OK;
    free(r); free(z); free(p); free(q);
    return status;
}

/*
 * The projection around the solve (Numerical Time Integration: each stage forms a provisional
 * velocity u*, solves the pressure Poisson equation whose source is div(u*)/dt, and corrects the
 * velocity by the pressure gradient divided by the density).  Velocities live on the faces of the
 * cells (MAC grid), x fastest:
 *   u: (nx+1) x ny x nz, u[i + (nx+1)(j + ny k)] on the face between cells i-1 and i
 *      (i = 0 and i = nx are the walls x = 0, x = Lx);
 *   v: nx x (ny+1) x nz, likewise in y;  w: nx x ny x (nz+1), w at k = nz on the top boundary.
 *
 * Divergence:  s_c = ((u_{i+1} - u_i) + (v_{j+1} - v_j) + (w_{k+1} - w_k)) / (h dt).
 *
 * Correction:  u_f <- u_f - dt (beta_f ((p_n - p_c) / h)) on every interior face, with the face
 * coefficient beta_f = 2/(rho_c + rho_n) of the operator (bx, by, bz); on the top face, where
 * p = 0, the gradient is (0 - p_c)/(h/2) and the coefficient 1/rho_c, written as
 * (2/rho_c) ((0 - p_c)/h); wall faces keep their value (beta = 0 there).  With these faces
 * div_h(u_new)/dt = div_h(u*)/dt - L p, i.e. divergence(u_new) = (A p - b) / h^2 for b = -h^2 s.
 */
/* With cut cells: s_c = (((a u)_{i+1} - (a u)_i + ... ) / (h dt)) / vol_c, 0 for inactive cells,
 * so that -h^2 vol s is the right side of the cut operator. */
void oracle_divergence_cut(int nx, int ny, int nz, double h, double dt, const double* u,
                           const double* v, const double* w, const double* ax, const double* ay,
                           const double* az, const double* vol, double* s) {
    const double hd = h * dt;
#pragma omp parallel for schedule(static)
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                const idx_t fu = (idx_t)i + (idx_t)(nx + 1) * ((idx_t)j + (idx_t)ny * k);
                const idx_t fv = (idx_t)i + (idx_t)nx * ((idx_t)j + (idx_t)(ny + 1) * k);
                const idx_t fw = (idx_t)i + (idx_t)nx * ((idx_t)j + (idx_t)ny * k);
                const idx_t up = fw + (idx_t)nx * ny;
                if (!(vol[fw] > 0.0)) {
                    s[fw] = 0.0;
                    continue;
                }
                const double du = ax[fu + 1] * u[fu + 1] - ax[fu] * u[fu];
                const double dv = ay[fv + nx] * v[fv + nx] - ay[fv] * v[fv];
                const double dw = az[up] * w[up] - az[fw] * w[fw];
                s[fw] = (((du + dv) + dw) / hd) / vol[fw];
            }
}

void oracle_divergence(int nx, int ny, int nz, double h, double dt, const double* u,
                       const double* v, const double* w, double* s) {
    const double hd = h * dt;
#pragma omp parallel for schedule(static)
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                const idx_t fu = (idx_t)i + (idx_t)(nx + 1) * ((idx_t)j + (idx_t)ny * k);
                const idx_t fv = (idx_t)i + (idx_t)nx * ((idx_t)j + (idx_t)(ny + 1) * k);
                const idx_t fw = (idx_t)i + (idx_t)nx * ((idx_t)j + (idx_t)ny * k);
                const double du = u[fu + 1] - u[fu];
                const double dv = v[fv + nx] - v[fv];
                const double dw = w[fw + (idx_t)nx * ny] - w[fw];
                s[fw] = ((du + dv) + dw) / hd;
            }
}

/* With cut cells (ax non-NULL; bx, by, bz the cut operator's faces): an open face of two active
 * cells is corrected with its own coefficient, the cut face coefficient over the open fraction
 * (bx / a); a top or Dirichlet wall face of an active cell with a > 0 with 2/rho_c; every other
 * face keeps its value.  Then the flux divergence sum_f a_f u_f of the corrected field is that of
 * u* minus dt (L p) h: the cut operator's residual again. */
static double cut_beta(const double* a, idx_t f, double b) { return a ? (b != 0.0 ? b / a[f] : 0.0) : b; }

void oracle_project_cut(int nx, int ny, int nz, double h, double dt, const double* F,
                        double rho_air, double rho_water, int walls, const double* ax,
                        const double* ay, const double* az, const double* vol, const double* bx,
                        const double* by, const double* bz, const double* p, double* u,
                        double* v, double* w);

void oracle_project_bc(int nx, int ny, int nz, double h, double dt, const double* F,
                       double rho_air, double rho_water, int walls, const double* bx,
                       const double* by, const double* bz, const double* p, double* u, double* v,
                       double* w) {
    oracle_project_cut(nx, ny, nz, h, dt, F, rho_air, rho_water, walls, NULL, NULL, NULL, NULL, bx,
                       by, bz, p, u, v, w);
}

void oracle_project_cut(int nx, int ny, int nz, double h, double dt, const double* F,
                        double rho_air, double rho_water, int walls, const double* ax,
                        const double* ay, const double* az, const double* vol, const double* bx,
                        const double* by, const double* bz, const double* p, double* u,
                        double* v, double* w) {
#pragma omp parallel for schedule(static)
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                const idx_t c = (idx_t)i + (idx_t)nx * ((idx_t)j + (idx_t)ny * k);
                const idx_t sxy = (idx_t)nx * ny;
                const idx_t fu = (idx_t)i + (idx_t)(nx + 1) * ((idx_t)j + (idx_t)ny * k);
                const idx_t fv = (idx_t)i + (idx_t)nx * ((idx_t)j + (idx_t)(ny + 1) * k);
                if (i > 0) {
                    const double b = cut_beta(ax, fu, bx[c]);
                    u[fu] = u[fu] - dt * (b * ((p[c] - p[c - 1]) / h));
                } else if (walls & OR_PERIODIC_X) {
                    /* faces 0 and nx are one face: corrected from face 0, written to both */
                    const double b = cut_beta(ax, fu, bx[c]);
                    u[fu] = u[fu] - dt * (b * ((p[c] - p[c + nx - 1]) / h));
                    u[fu + nx] = u[fu];
                }
                if (j > 0) {
                    const double b = cut_beta(ay, fv, by[c]);
                    v[fv] = v[fv] - dt * (b * ((p[c] - p[c - nx]) / h));
                }
                if (k > 0) {
                    const double b = cut_beta(az, c, bz[c]);
                    w[c] = w[c] - dt * (b * ((p[c] - p[c - sxy]) / h));
                }
                if (vol && !(vol[c] > 0.0)) continue; /* inactive: no boundary faces */
                const double rho = rho_air + F[c] * (rho_water - rho_air);
                if (k == nz - 1 && face_open(az, c + sxy) > 0.0) {
                    const idx_t f = c + sxy;
                    w[f] = w[f] - dt * ((2.0 / rho) * ((0.0 - p[c]) / h));
                }
                /* Dirichlet walls: p = 0 on the wall face, half a cell from the centre */
                if ((walls & OR_WALL_XM) && i == 0 && face_open(ax, fu) > 0.0)
                    u[fu] = u[fu] - dt * ((2.0 / rho) * ((p[c] - 0.0) / h));
                if ((walls & OR_WALL_XP) && i == nx - 1 && face_open(ax, fu + 1) > 0.0)
                    u[fu + 1] = u[fu + 1] - dt * ((2.0 / rho) * ((0.0 - p[c]) / h));
                if ((walls & OR_WALL_YM) && j == 0 && face_open(ay, fv) > 0.0)
                    v[fv] = v[fv] - dt * ((2.0 / rho) * ((p[c] - 0.0) / h));
                if ((walls & OR_WALL_YP) && j == ny - 1 && face_open(ay, fv + nx) > 0.0)
                    v[fv + nx] = v[fv + nx] - dt * ((2.0 / rho) * ((0.0 - p[c]) / h));
                if ((walls & OR_WALL_ZM) && k == 0 && face_open(az, c) > 0.0)
                    w[c] = w[c] - dt * ((2.0 / rho) * ((p[c] - 0.0) / h));
            }
}

void oracle_project(int nx, int ny, int nz, double h, double dt, const double* F, double rho_air,
                    double rho_water, const double* bx, const double* by, const double* bz,
                    const double* p, double* u, double* v, double* w) {
    oracle_project_bc(nx, ny, nz, h, dt, F, rho_air, rho_water, 0, bx, by, bz, p, u, v, w);
}

/* ---------------------------------------------------------------------------- reduced pressure
 * Hydrostatic-pressure method (Entrance and Exit Boundary Conditions).  The solve is for the
 * reduced pressure P_r = P - rho g (z - z_o), z_o the static free-surface height.  The momentum
 * equations then carry the force -(z - z_o) (1/rho) d(rho g)/dx_i, which in the paper's units
 * (rho = lambda + (1 - lambda) H) is -(z - z_o)(1 - lambda) g (1/rho) dH/dx_i and which makes P_r
 * jump by (z - z_o)(1 - lambda) g across the interface.  The force is one of the terms R_i of the
 * provisional velocity, so its divergence joins the source of the pressure equation and the
 * projection removes its gradient part.
 *
 * Reading on the MAC faces (the paper leaves the discretisation to a cited scheme): for the face
 * between cells c and n, n on the +axis side,
 *     f = -(z_f - z_o) g beta_f (rho_n - rho_c) / h,     beta_f = 2 / (rho_c + rho_n),
 * with rho from F as for the operator and z_f the face's height: (k + 1/2) h on the x and y faces
 * of layer k, k h on the z face below layer k.  beta_f is the operator's face coefficient, so on
 * every interior face f = -beta_f (Psi_n - Psi_c)/h + g [z face], Psi_c = rho_c g (z_c - z_o):
 * the reduced form of the face-centred gravity g e_z and the total pressure P = P_r + Psi.
 * Every boundary face (walls of either kind, the top) gets no force: H is continued beyond the
 * boundary without change along its normal.  With periodic x the wrap face (cells nx-1 and 0)
 * carries its force on faces 0 and nx.  The call adds dt f to the face velocities u, v, w (shapes
 * as in oracle_divergence): u_f <- u_f + dt f.  g is the coefficient as the paper writes it. */
static double reduced_force(double rc, double rn, double zf, double z_o, double g, double h) {
    const double a = (zf - z_o) * g;
    const double b = (2.0 / (rc + rn)) * (rn - rc);
    return -(a * b) / h;
}

void oracle_hydrostatic_force(int nx, int ny, int nz, double h, const double* F, double rho_air,
                              double rho_water, double g, double z_o, int walls, double dt,
                              double* u, double* v, double* w) {
#pragma omp parallel for schedule(static)
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                const idx_t c = (idx_t)i + (idx_t)nx * ((idx_t)j + (idx_t)ny * k);
                const idx_t sxy = (idx_t)nx * ny;
                const idx_t fu = (idx_t)i + (idx_t)(nx + 1) * ((idx_t)j + (idx_t)ny * k);
                const idx_t fv = (idx_t)i + (idx_t)nx * ((idx_t)j + (idx_t)(ny + 1) * k);
                const double rc = rho_air + F[c] * (rho_water - rho_air);
                const double zc = ((double)k + 0.5) * h; /* height of the layer's x, y faces */
                if (i > 0) {
                    const double rn = rho_air + F[c - 1] * (rho_water - rho_air);
                    /* face between c - 1 (low side) and c (high side) */
                    u[fu] = u[fu] + dt * reduced_force(rn, rc, zc, z_o, g, h);
                } else if (walls & OR_PERIODIC_X) {
                    const double rn = rho_air + F[c + nx - 1] * (rho_water - rho_air);
                    u[fu] = u[fu] + dt * reduced_force(rn, rc, zc, z_o, g, h);
                    u[fu + nx] = u[fu];
                }
                if (j > 0) {
                    const double rn = rho_air + F[c - nx] * (rho_water - rho_air);
                    v[fv] = v[fv] + dt * reduced_force(rn, rc, zc, z_o, g, h);
                }
                if (k > 0) {
                    const double rn = rho_air + F[c - sxy] * (rho_water - rho_air);
                    w[c] = w[c] + dt * reduced_force(rn, rc, (double)k * h, z_o, g, h);
                }
            }
}

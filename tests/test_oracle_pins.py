"""Pins of the FP64 CPU oracle against what the mathematics fixes, independently of the oracle.

Each test checks the oracle against a closed form, a library routine (dense LU, banded solve), an
exact layered solution or a convergence rate -- never against a retyped copy of its own loops --
chosen so that a plausible slip (dropped face, wrong sign or index, transposed operand, the other
mean, a misplaced Dirichlet boundary) fails at least one of them.
"""
import math

import numpy as np
import pytest
import scipy.linalg

import oracle
from paper_1410_1942_gb300 import inputs

RHO_A, RHO_W = 1.0, 1000.0


def _rand_F(shape, seed, sharp=False):
    rng = np.random.default_rng(seed)
    if sharp:
        return (rng.random(shape) < 0.5).astype(np.float64)
    F = rng.random(shape)
    F[rng.random(shape) < 0.3] = 0.0
    F[rng.random(shape) < 0.3] = 1.0
    return F


def _dense(op):
    """Dense A from the stencil apply on unit vectors (column j = A e_j)."""
    n = op.nx * op.ny * op.nz
    A = np.empty((n, n))
    e = np.zeros(n)
    for j in range(n):
        e[j] = 1.0
        A[:, j] = oracle.apply(op, e).ravel()
        e[j] = 0.0
    return A


def _cosine_mode(nx, ny, nz, a, b, c):
    """Closed-form eigenvector of the constant-coefficient operator with Neumann x/y/bottom walls
    and a Dirichlet top face: cos(pi a (i+1/2)/nx) cos(pi b (j+1/2)/ny) cos(pi (c+1/2)(k+1/2)/nz),
    eigenvalue 4[sin^2(pi a/2nx) + sin^2(pi b/2ny) + sin^2(pi (2c+1)/4nz)] (times beta)."""
    i = np.arange(nx) + 0.5
    j = np.arange(ny) + 0.5
    k = np.arange(nz) + 0.5
    v = (np.cos(math.pi * (c + 0.5) * k / nz)[:, None, None]
         * np.cos(math.pi * b * j / ny)[None, :, None]
         * np.cos(math.pi * a * i / nx)[None, None, :])
    lam = 4.0 * (math.sin(math.pi * a / (2 * nx)) ** 2 + math.sin(math.pi * b / (2 * ny)) ** 2
                 + math.sin(math.pi * (2 * c + 1) / (4 * nz)) ** 2)
    return v, lam


# ------------------------------------------------------------------------------- the operator
@pytest.mark.parametrize("shape", [(5, 6, 7), (4, 4, 4), (1, 3, 8), (9, 2, 3)])
def test_symmetry_and_positivity(shape):
    F = _rand_F(shape, 1)
    op = oracle.operator(F, RHO_A, RHO_W)
    rng = np.random.default_rng(2)
    x, y = rng.standard_normal(shape), rng.standard_normal(shape)
    xay = np.vdot(x, oracle.apply(op, y))
    yax = np.vdot(y, oracle.apply(op, x))
    assert abs(xay - yax) <= 1e-14 * max(abs(xay), 1.0) * 10
    assert np.vdot(x, oracle.apply(op, x)) > 0.0
    A = _dense(op)
    assert np.array_equal(A, A.T)
    assert np.linalg.eigvalsh(A).min() > 0.0


@pytest.mark.parametrize("shape", [(5, 6, 7), (3, 3, 3)])
def test_row_sums_are_the_dirichlet_leak(shape):
    """Conservation: every face flux cancels between its two cells, so A applied to a constant
    leaves only the top-face Dirichlet term 2/rho in the top layer and exactly 0 elsewhere."""
    F = _rand_F(shape, 3)
    op = oracle.operator(F, RHO_A, RHO_W)
    s = oracle.apply(op, np.ones(shape))
    rho = RHO_A + F * (RHO_W - RHO_A)
    assert np.max(np.abs(s[:-1])) <= 1e-15
    np.testing.assert_allclose(s[-1], 2.0 / rho[-1], rtol=1e-13)


@pytest.mark.parametrize("F0,beta", [(0.0, 1.0), (1.0, 1.0 / 1000.0)])
@pytest.mark.parametrize("shape,modes", [((8, 8, 8), [(0, 0, 0), (1, 2, 3), (7, 7, 7)]),
                                         ((6, 10, 5), [(0, 3, 0), (5, 0, 4), (2, 9, 1)])])
def test_constant_coefficient_eigenvectors(F0, beta, shape, modes):
    nx, ny, nz = shape
    op = oracle.operator(np.full((nz, ny, nx), F0), RHO_A, RHO_W)
    for a, b, c in modes:
        v, lam = _cosine_mode(nx, ny, nz, a, b, c)
        np.testing.assert_allclose(oracle.apply(op, v), beta * lam * v, rtol=0,
                                   atol=1e-13 * beta * lam * np.abs(v).max() + 1e-16)


@pytest.mark.parametrize("precond", ["jacobi", "ssor"])
def test_eigenvector_source_gives_exact_discrete_solution(precond):
    nx, ny, nz = 12, 10, 14
    op = oracle.operator(np.zeros((nz, ny, nx)), RHO_A, RHO_W)
    v, lam = _cosine_mode(nx, ny, nz, 3, 1, 2)
    res = oracle.pcg(op, v, tol=1e-14, precond=precond)
    assert res.status == oracle.OK
    np.testing.assert_allclose(res.x, v / lam, rtol=0, atol=1e-11 * np.abs(v / lam).max())


@pytest.mark.parametrize("mean", ["harmonic", "arithmetic"])
def test_layered_series_resistance(mean):
    """A layered column (rho constant in each cell layer, interfaces on faces) fed by a source in
    the bottom layer carries the constant flux Q = s_0 h up to the top face p = 0, so the pressure
    at the centre of layer k is -Q (rho_k h/2 + sum_{m>k} rho_m h): resistances in series.  The
    harmonic-mean face coefficient reproduces it exactly; the arithmetic mean of 1/rho must not."""
    nx, ny, nz, h = 3, 4, 12, 1.0 / 12
    rng = np.random.default_rng(5)
    layer_F = (rng.random(nz) < 0.5).astype(float)
    layer_F[3], layer_F[4] = 0.0, 1.0  # at least one air/water jump
    F = np.broadcast_to(layer_F[:, None, None], (nz, ny, nx)).copy()
    rho_layer = np.where(layer_F > 0.5, RHO_W, RHO_A)
    s = np.zeros((nz, ny, nx))
    s[0] = 7.0
    Q = 7.0 * h
    expect = np.array([-Q * (rho_layer[k] * h / 2 + rho_layer[k + 1:].sum() * h) for k in range(nz)])
    op = oracle.operator(F, RHO_A, RHO_W, mean=mean)
    res = oracle.pcg(op, oracle.rhs(s, h), tol=1e-10, precond="jacobi", max_iters=5000)
    got = res.x[:, 1, 2]
    if mean == "harmonic":
        assert res.status == oracle.OK
        np.testing.assert_allclose(res.x, np.broadcast_to(expect[:, None, None], res.x.shape),
                                   rtol=1e-10)
    else:
        assert np.max(np.abs(got - expect)) > 1e-3 * np.max(np.abs(expect))


def test_manufactured_second_order():
    """p = cos(pi x) cos(pi y) cos(pi z / 2) on the unit cube has zero normal derivative on the
    x, y and bottom walls and p = 0 on the top face; with rho = 1, div grad p = -(9/4) pi^2 p.
    The discrete solution must converge to it at second order under grid halving."""
    errs = []
    for n in (16, 32, 64):
        h = 1.0 / n
        c = (np.arange(n) + 0.5) * h
        p = (np.cos(math.pi * c)[None, None, :] * np.cos(math.pi * c)[None, :, None]
             * np.cos(0.5 * math.pi * c)[:, None, None])
        s = -2.25 * math.pi ** 2 * p
        res, _ = oracle.solve(np.zeros((n, n, n)), s, h, tol=1e-13)
        assert res.status == oracle.OK
        errs.append(np.sqrt(np.mean((res.x - p) ** 2)))
    orders = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert all(1.8 <= o <= 2.2 for o in orders), orders


@pytest.mark.parametrize("shape,sharp", [((4, 4, 4), False), ((5, 5, 5), True), ((6, 6, 6), False),
                                         ((3, 5, 4), True)])
@pytest.mark.parametrize("precond", ["jacobi", "ssor"])
def test_pcg_matches_dense_lu(shape, sharp, precond):
    F = _rand_F(shape, 11, sharp)
    op = oracle.operator(F, RHO_A, RHO_W)
    b = np.random.default_rng(12).standard_normal(shape)
    ref = scipy.linalg.solve(_dense(op), b.ravel(), assume_a="sym").reshape(shape)
    res = oracle.pcg(op, b, tol=1e-14, precond=precond)
    assert res.status == oracle.OK
    err = np.linalg.norm(res.x - ref) / np.linalg.norm(ref)
    assert err <= 1e-11, err


def test_dense_operator_structure():
    """Brute force on a tiny grid: the dense matrix has exactly the 7-point sparsity of the
    cell adjacency, negative off-diagonals equal to the face coefficient shared by both cells, and
    a positive diagonal.  A transposed or shifted index would break the adjacency pattern."""
    nx, ny, nz = 3, 4, 5
    F = _rand_F((nz, ny, nx), 13)
    A = _dense(oracle.operator(F, RHO_A, RHO_W))
    rho = (RHO_A + F * (RHO_W - RHO_A)).ravel()
    idx = lambda i, j, k: i + nx * (j + ny * k)
    for k in range(nz):
        for j in range(ny):
            for i in range(nx):
                c = idx(i, j, k)
                nbrs = set()
                for di, dj, dk in ((1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1)):
                    ii, jj, kk = i + di, j + dj, k + dk
                    if 0 <= ii < nx and 0 <= jj < ny and 0 <= kk < nz:
                        nbrs.add(idx(ii, jj, kk))
                row = A[c]
                assert set(np.flatnonzero(row)) == nbrs | {c}
                for m in nbrs:
                    # series conductance of two half cells of conductivity 1/rho
                    g = 1.0 / (0.5 * rho[c] + 0.5 * rho[m])
                    assert abs(row[m] + g) <= 1e-15 * g * 4
                assert row[c] > 0


# ------------------------------------------------------------------------------- separable pin
def test_separable_layered_density_reduces_to_tridiagonal():
    """F = F(z) (flat two-phase surface, ratio 1000) with a source cos(pi a (i+1/2)/nx)
    cos(pi b (j+1/2)/ny) g_k: the solution is the same cosines times a z-profile solving a
    tridiagonal system.  In each layer the horizontal faces join equal densities (coefficient
    1/rho_k); the vertical faces are the series conductances of two half layers.  The profile is
    solved by a banded LU (Thomas algorithm) from scipy."""
    nx, ny, nz = 10, 8, 24
    h = 1.0 / nz
    zc = (np.arange(nz) + 0.5) * h
    Fz = inputs.smoothed_step(0.5 - zc, 1.5 * h)
    F = np.broadcast_to(Fz[:, None, None], (nz, ny, nx)).copy()
    rho = RHO_A + Fz * (RHO_W - RHO_A)
    a, b = 3, 2
    lam_xy = 4.0 * (math.sin(math.pi * a / (2 * nx)) ** 2 + math.sin(math.pi * b / (2 * ny)) ** 2)
    g = np.random.default_rng(21).standard_normal(nz)
    cx = np.cos(math.pi * a * (np.arange(nx) + 0.5) / nx)
    cy = np.cos(math.pi * b * (np.arange(ny) + 0.5) / ny)
    rhs = g[:, None, None] * cy[None, :, None] * cx[None, None, :]
    # vertical conductances between layer k-1 and k, k = 1..nz-1; top face: half layer to p = 0
    gz = 1.0 / (0.5 * rho[:-1] + 0.5 * rho[1:])
    ab = np.zeros((3, nz))
    main = lam_xy / rho
    main[:-1] += gz
    main[1:] += gz
    main[-1] += 1.0 / (0.5 * rho[-1])
    ab[1] = main
    ab[0, 1:] = -gz
    ab[2, :-1] = -gz
    prof = scipy.linalg.solve_banded((1, 1), ab, g)
    expect = prof[:, None, None] * cy[None, :, None] * cx[None, None, :]
    op = oracle.operator(F, RHO_A, RHO_W)
    for pc in ("jacobi", "ssor"):
        res = oracle.pcg(op, rhs, tol=1e-14, precond=pc)
        assert res.status == oracle.OK
        np.testing.assert_allclose(res.x, expect, rtol=0, atol=1e-10 * np.abs(expect).max())


# ------------------------------------------------------------------------------- preconditioners
def test_jacobi_is_diagonal_inverse():
    shape = (5, 4, 6)
    op = oracle.operator(_rand_F(shape, 31), RHO_A, RHO_W)
    A = _dense(op)
    r = np.random.default_rng(32).standard_normal(shape)
    np.testing.assert_allclose(oracle.precond(op, r, "jacobi").ravel(), r.ravel() / np.diag(A),
                               rtol=1e-15)


@pytest.mark.parametrize("shape", [(4, 4, 4), (5, 5, 5), (6, 6, 6), (3, 5, 4)])
@pytest.mark.parametrize("omega", [1.0, 1.3])
def test_ssor_matches_literal_splitting(shape, omega):
    """Dense SSOR preconditioner from its definition: order the unknowns red ((i+j+k) even)
    first, split A = D - E - E^T with E strictly lower, M = (D - wE) D^{-1} (D - wE^T)/(w(2-w)),
    and solve M z = r with dense LU."""
    nz, ny, nx = shape[2], shape[1], shape[0]
    F = _rand_F((nz, ny, nx), 41)
    op = oracle.operator(F, RHO_A, RHO_W)
    A = _dense(op)
    kk, jj, ii = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    colour = ((ii + jj + kk) % 2).ravel()
    perm = np.concatenate([np.flatnonzero(colour == 0), np.flatnonzero(colour == 1)])
    Ap = A[np.ix_(perm, perm)]
    D = np.diag(np.diag(Ap))
    E = -np.tril(Ap, -1)
    M = (D - omega * E) @ np.linalg.inv(D) @ (D - omega * E.T) / (omega * (2.0 - omega))
    r = np.random.default_rng(42).standard_normal((nz, ny, nx))
    zp = np.linalg.solve(M, r.ravel()[perm])
    expect = np.empty_like(zp)
    expect[perm] = zp
    got = oracle.precond(op, r, "ssor", omega).ravel()
    np.testing.assert_allclose(got, expect, rtol=1e-12, atol=1e-14 * np.abs(expect).max())


@pytest.mark.parametrize("kind", ["jacobi", "ssor"])
def test_preconditioner_symmetric_positive(kind):
    shape = (7, 6, 5)
    op = oracle.operator(_rand_F(shape, 51), RHO_A, RHO_W)
    rng = np.random.default_rng(52)
    x, y = rng.standard_normal(shape), rng.standard_normal(shape)
    a = np.vdot(x, oracle.precond(op, y, kind))
    b = np.vdot(y, oracle.precond(op, x, kind))
    assert abs(a - b) <= 1e-13 * max(abs(a), 1.0)
    assert np.vdot(x, oracle.precond(op, x, kind)) > 0


# ------------------------------------------------------------------------------- PCG itself
@pytest.mark.parametrize("precond", ["jacobi", "ssor"])
def test_pcg_error_decreases_in_energy_norm(precond):
    shape = (5, 5, 5)
    op = oracle.operator(_rand_F(shape, 61), RHO_A, RHO_W)
    A = _dense(op)
    b = np.random.default_rng(62).standard_normal(shape)
    xs = scipy.linalg.solve(A, b.ravel(), assume_a="sym")
    errs = []
    for it in range(1, 40):
        res = oracle.pcg(op, b, tol=0.0, precond=precond, max_iters=it)
        e = res.x.ravel() - xs
        errs.append(float(e @ A @ e))
    errs = np.array(errs)
    assert np.all(np.diff(errs) <= 1e-12 * errs[0])


def test_pcg_iterations_bounded_by_dimension_and_recurrence_tracks_truth():
    shape = (3, 3, 3)
    op = oracle.operator(_rand_F(shape, 71), RHO_A, RHO_W)
    b = np.random.default_rng(72).standard_normal(shape)
    res = oracle.pcg(op, b, tol=1e-12, precond="jacobi", history=True)
    assert res.status == oracle.OK
    assert res.iters <= 27 + 5
    assert res.rel_residual <= 1e-12
    assert abs(res.history[-1] - res.rel_residual) <= 1e-12


def test_zero_source_gives_zero_solution():
    op = oracle.operator(_rand_F((4, 5, 6), 81), RHO_A, RHO_W)
    res = oracle.pcg(op, np.zeros((4, 5, 6)), x0=np.ones((4, 5, 6)), tol=1e-10)
    assert res.status == oracle.OK and res.iters == 0 and not res.x.any()


def test_warm_start_from_solution_takes_no_iterations():
    c = inputs.flat_case(8, 8, 8, seed=3)
    res, op = oracle.solve(c.F, c.s, c.grid.h, tol=1e-12)
    again = oracle.pcg(op, oracle.rhs(c.s, c.grid.h), x0=res.x, tol=1e-11)
    assert again.iters == 0


# ------------------------------------------------------------------------------- wall variants
def _mode_1d(n, a, low_dirichlet, high_dirichlet):
    """Closed-form eigenvector of the 1-D cell-centred second difference with the given wall
    conditions (p = 0 on a Dirichlet wall face, zero gradient on the others) and its eigenvalue:
    N-N cos(pi a (i+1/2)/n), lambda 4 sin^2(pi a/2n); N-D cos(pi (a+1/2)(i+1/2)/n) and D-N
    sin(pi (a+1/2)(i+1/2)/n), lambda 4 sin^2(pi (2a+1)/4n); D-D sin(pi (a+1)(i+1/2)/n),
    lambda 4 sin^2(pi (a+1)/2n)."""
    i = np.arange(n) + 0.5
    if not low_dirichlet and not high_dirichlet:
        th = math.pi * a / n
        return np.cos(th * i), 4 * math.sin(th / 2) ** 2
    if low_dirichlet and high_dirichlet:
        th = math.pi * (a + 1) / n
        return np.sin(th * i), 4 * math.sin(th / 2) ** 2
    th = math.pi * (a + 0.5) / n
    return (np.sin(th * i) if low_dirichlet else np.cos(th * i)), 4 * math.sin(th / 2) ** 2


@pytest.mark.parametrize("walls", [1, 2, 3, 4 | 8, 16, 1 | 8 | 16, 31])
@pytest.mark.parametrize("shape,modes", [((6, 5, 7), (1, 2, 0)), ((4, 8, 3), (0, 3, 2))])
def test_dirichlet_wall_eigenvectors(walls, shape, modes):
    """At constant density every wall mask has separable closed-form eigenvectors: products of
    the 1-D modes of each axis under its pair of wall conditions (the top face is always
    Dirichlet).  A v = lambda v to rounding pins each wall's diagonal term."""
    nz, ny, nx = shape
    vx, lx = _mode_1d(nx, modes[0], walls & 1, walls & 2)
    vy, ly = _mode_1d(ny, modes[1], walls & 4, walls & 8)
    vz, lz = _mode_1d(nz, modes[2], walls & 16, True)
    v = vz[:, None, None] * vy[None, :, None] * vx[None, None, :]
    op = oracle.operator(np.zeros(shape), RHO_A, RHO_W, walls=walls)
    lam = lx + ly + lz
    assert np.abs(oracle.apply(op, v) - lam * v).max() <= 1e-12 * max(1.0, lam)


@pytest.mark.parametrize("walls", [3, 16, 31])
def test_dirichlet_walls_pcg_matches_dense_lu(walls):
    shape = (5, 4, 6)
    op = oracle.operator(_rand_F(shape, 17), RHO_A, RHO_W, walls=walls)
    A = _dense(op)
    assert np.allclose(A, A.T, rtol=0, atol=1e-12)
    b = np.random.default_rng(18).standard_normal(shape)
    ref = scipy.linalg.solve(A, b.ravel(), assume_a="sym").reshape(shape)
    res = oracle.pcg(op, b, tol=1e-14)
    assert res.status == oracle.OK
    assert np.linalg.norm(res.x - ref) / np.linalg.norm(ref) <= 1e-11


@pytest.mark.parametrize("walls", [1, 2, 4, 8, 16, 31])
def test_projection_with_dirichlet_walls_leaves_the_residual(walls):
    shape, h, dt = (5, 6, 7), 1.0 / 8, 2e-3
    F = _rand_F(shape, 94)
    op = oracle.operator(F, RHO_A, RHO_W, walls=walls)
    u, v, w = _faces(shape, 95)
    p = np.random.default_rng(96).standard_normal(shape)
    b = oracle.rhs(oracle.divergence(u, v, w, h, dt), h)
    un, vn, wn = oracle.project(op, F, u, v, w, p, h, dt, RHO_A, RHO_W)
    r, _ = oracle.residual(op, b, p)
    div = oracle.divergence(un, vn, wn, h, dt)
    scale = (np.abs(b) + np.abs(oracle.apply(op, p))).max() / h ** 2
    assert np.abs(div + r / h ** 2).max() <= 1e-13 * scale
    # a Dirichlet wall's faces move, a zero-gradient wall's do not
    assert np.array_equal(un[:, :, 0], u[:, :, 0]) == (not walls & 1)
    assert np.array_equal(wn[0], w[0]) == (not walls & 16)


@pytest.mark.parametrize("walls", [oracle.PERIODIC_X, oracle.PERIODIC_X | 4 | 16])
@pytest.mark.parametrize("shape,a", [((5, 4, 8), 3), ((3, 6, 7), 2), ((4, 2, 1), 0)])
def test_periodic_x_eigenvectors(walls, shape, a):
    """Periodic x: cos(2 pi a (i+1/2)/nx) and sin(...) are eigenvectors of the x second difference
    with lambda 4 sin^2(pi a/nx); combined with the other axes' closed-form modes."""
    nz, ny, nx = shape
    i = np.arange(nx) + 0.5
    lx = 4 * math.sin(math.pi * a / nx) ** 2
    vy, ly = _mode_1d(ny, 1 if ny > 1 else 0, walls & 4, walls & 8)
    vz, lz = _mode_1d(nz, 1, walls & 16, True)
    op = oracle.operator(np.zeros(shape), RHO_A, RHO_W, walls=walls)
    for vx in (np.cos(2 * math.pi * a * i / nx), np.sin(2 * math.pi * a * i / nx)):
        v = vz[:, None, None] * vy[None, :, None] * vx[None, None, :]
        if not np.abs(v).max():
            continue
        lam = lx + ly + lz
        assert np.abs(oracle.apply(op, v) - lam * v).max() <= 1e-12 * max(1.0, lam)


def test_periodic_x_dense_lu_and_ssor_splitting():
    shape = (4, 3, 6)  # nx even: red-black colouring survives the wrap
    F = _rand_F(shape, 19)
    op = oracle.operator(F, RHO_A, RHO_W, walls=oracle.PERIODIC_X)
    A = _dense(op)
    assert np.allclose(A, A.T, rtol=0, atol=1e-12)
    # the wrap couples i = 0 and i = nx-1 with the harmonic face of their densities
    c0, c1 = 0, shape[2] - 1
    rho = RHO_A + F.ravel() * (RHO_W - RHO_A)
    assert A[c0, c1] == -2.0 / (rho[c0] + rho[c1])
    b = np.random.default_rng(20).standard_normal(shape)
    ref = scipy.linalg.solve(A, b.ravel(), assume_a="sym").reshape(shape)
    for pc in ("jacobi", "ssor"):
        res = oracle.pcg(op, b, tol=1e-14, precond=pc)
        assert res.status == oracle.OK
        assert np.linalg.norm(res.x - ref) / np.linalg.norm(ref) <= 1e-11
    nz, ny, nx = shape
    kk, jj, ii = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    colour = ((ii + jj + kk) % 2).ravel()
    perm = np.concatenate([np.flatnonzero(colour == 0), np.flatnonzero(colour == 1)])
    Ap = A[np.ix_(perm, perm)]
    D = np.diag(np.diag(Ap))
    E = -np.tril(Ap, -1)
    M = (D - E) @ np.linalg.inv(D) @ (D - E.T)
    r = np.random.default_rng(21).standard_normal(shape)
    zp = np.linalg.solve(M, r.ravel()[perm])
    expect = np.empty_like(zp)
    expect[perm] = zp
    got = oracle.precond(op, r, "ssor", 1.0).ravel()
    np.testing.assert_allclose(got, expect, rtol=1e-12, atol=1e-14 * np.abs(expect).max())


def test_projection_with_periodic_x_leaves_the_residual():
    shape, h, dt = (5, 6, 8), 1.0 / 8, 2e-3
    F = _rand_F(shape, 97)
    op = oracle.operator(F, RHO_A, RHO_W, walls=oracle.PERIODIC_X | 16)
    u, v, w = _faces(shape, 98)
    u[:, :, -1] = u[:, :, 0]  # faces 0 and nx are one face
    p = np.random.default_rng(99).standard_normal(shape)
    b = oracle.rhs(oracle.divergence(u, v, w, h, dt), h)
    un, vn, wn = oracle.project(op, F, u, v, w, p, h, dt, RHO_A, RHO_W)
    assert np.array_equal(un[:, :, 0], un[:, :, -1]) and not np.array_equal(un[:, :, 0], u[:, :, 0])
    r, _ = oracle.residual(op, b, p)
    div = oracle.divergence(un, vn, wn, h, dt)
    scale = (np.abs(b) + np.abs(oracle.apply(op, p))).max() / h ** 2
    assert np.abs(div + r / h ** 2).max() <= 1e-13 * scale


# ------------------------------------------------------------------------------- cut cells
def _open_apertures(shape):
    nz, ny, nx = shape
    return (np.ones((nz, ny, nx + 1)), np.ones((nz, ny + 1, nx)), np.ones((nz + 1, ny, nx)),
            np.ones(shape))


def test_cut_cells_all_open_is_the_plain_operator():
    shape = (5, 6, 7)
    F = _rand_F(shape, 101)
    for walls in (0, 31, oracle.PERIODIC_X | 16):
        a = oracle.operator(F, RHO_A, RHO_W, walls=walls)
        b = oracle.operator(F, RHO_A, RHO_W, walls=walls, apertures=_open_apertures(shape))
        for x, y in ((a.bx, b.bx), (a.by, b.by), (a.bz, b.bz), (a.diag, b.diag)):
            assert np.array_equal(x, y)


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_cut_cells_grid_aligned_body_is_a_wall_of_the_fluid_box(axis):
    """A body filling the cells beyond a grid plane (vol 0 there, the plane's faces closed)
    leaves the fluid box with a zero-gradient wall on that plane: the cut solve equals the plain
    solve on the fluid box, and the body's cells hold p = 0."""
    shape = (6, 7, 8)  # (nz, ny, nx)
    F = _rand_F(shape, 102)
    ax, ay, az, vol = _open_apertures(shape)
    cut = 4  # fluid: index < cut along the axis (x, y) or index >= cut (z: a bottom body)
    if axis == 0:
        vol[:, :, cut:] = 0
        ax[:, :, cut] = 0
        sub = (slice(None), slice(None), slice(0, cut))
    elif axis == 1:
        vol[:, cut:, :] = 0
        ay[:, cut, :] = 0
        sub = (slice(None), slice(0, cut), slice(None))
    else:
        vol[:cut - 2] = 0
        az[cut - 2] = 0
        sub = (slice(cut - 2, None), slice(None), slice(None))
    op = oracle.operator(F, RHO_A, RHO_W, apertures=(ax, ay, az, vol))
    s = np.random.default_rng(103).standard_normal(shape)
    b = oracle.rhs(s, 0.125, vol)
    res = oracle.pcg(op, b, tol=1e-13)
    assert res.status == oracle.OK
    ref = oracle.pcg(oracle.operator(np.ascontiguousarray(F[sub]), RHO_A, RHO_W),
                     oracle.rhs(np.ascontiguousarray(s[sub]), 0.125), tol=1e-13).x
    assert np.linalg.norm(res.x[sub] - ref) <= 1e-10 * np.linalg.norm(ref)
    assert not np.any(res.x[vol == 0])


def test_cut_cells_operator_symmetric_positive_and_matches_dense_lu():
    shape = (4, 5, 6)
    rng = np.random.default_rng(104)
    F = _rand_F(shape, 105)
    ax, ay, az, vol = (rng.uniform(0.05, 1.0, a.shape) for a in _open_apertures(shape))
    vol[rng.random(shape) < 0.15] = 0.0
    op = oracle.operator(F, RHO_A, RHO_W, walls=3, apertures=(ax, ay, az, vol))
    A = _dense(op)
    assert np.allclose(A, A.T, rtol=0, atol=1e-13)
    assert np.linalg.eigvalsh(A).min() > 0
    b = oracle.rhs(rng.standard_normal(shape), 0.25, vol)
    ref = scipy.linalg.solve(A, b.ravel(), assume_a="sym").reshape(shape)
    res = oracle.pcg(op, b, tol=1e-14)
    assert np.linalg.norm(res.x - ref) / np.linalg.norm(ref) <= 1e-10


@pytest.mark.parametrize("walls", [0, 16 | 1])
def test_cut_cells_projection_leaves_the_residual(walls):
    """vol s(u_new) = (A p - b)/h^2 in the active cells for any p (s the cut divergence over
    dt): the projection's open-face coefficients and boundary faces are the cut operator's."""
    shape, h, dt = (5, 6, 7), 1.0 / 8, 2e-3
    rng = np.random.default_rng(106)
    F = _rand_F(shape, 107)
    ax, ay, az, vol = (rng.uniform(0.05, 1.0, a.shape) for a in _open_apertures(shape))
    vol[rng.random(shape) < 0.15] = 0.0
    aps = (ax, ay, az, vol)
    op = oracle.operator(F, RHO_A, RHO_W, walls=walls, apertures=aps)
    u, v, w = _faces(shape, 108)
    p = rng.standard_normal(shape)
    b = oracle.rhs(oracle.divergence(u, v, w, h, dt, aps), h, vol)
    un, vn, wn = oracle.project(op, F, u, v, w, p, h, dt, RHO_A, RHO_W)
    r, _ = oracle.residual(op, b, p)
    lhs = vol * oracle.divergence(un, vn, wn, h, dt, aps)
    act = vol > 0
    scale = (np.abs(b) + np.abs(oracle.apply(op, p))).max() / h ** 2
    assert np.abs(lhs[act] + r[act] / h ** 2).max() <= 1e-12 * scale
    assert not np.any(lhs[~act])


# ------------------------------------------------------------------------------- projection
def _faces(shape, seed):
    nz, ny, nx = shape
    rng = np.random.default_rng(seed)
    return (rng.standard_normal((nz, ny, nx + 1)), rng.standard_normal((nz, ny + 1, nx)),
            rng.standard_normal((nz + 1, ny, nx)))


@pytest.mark.parametrize("shape", [(5, 6, 7), (1, 4, 9), (6, 1, 5), (3, 5, 1)])
def test_projection_leaves_the_residual_as_divergence(shape):
    """u_new = u* - dt beta grad p has div_h(u_new)/dt = s - L p, i.e. divergence(u_new) =
    (A p - b)/h^2 with b = -h^2 div(u*)/dt, for ANY p: the projection's faces, gradients and top
    boundary are those of the operator (a wrong face, sign or top factor breaks it)."""
    h, dt = 1.0 / 8, 2e-3
    F = _rand_F(shape, 91)
    op = oracle.operator(F, RHO_A, RHO_W)
    u, v, w = _faces(shape, 92)
    p = np.random.default_rng(93).standard_normal(shape)
    b = oracle.rhs(oracle.divergence(u, v, w, h, dt), h)
    un, vn, wn = oracle.project(op, F, u, v, w, p, h, dt, RHO_A, RHO_W)
    r, _ = oracle.residual(op, b, p)
    div = oracle.divergence(un, vn, wn, h, dt)
    scale = (np.abs(b) + np.abs(oracle.apply(op, p))).max() / h ** 2
    assert np.abs(div + r / h ** 2).max() <= 1e-13 * scale
    # wall faces are untouched, the others move
    assert np.array_equal(un[:, :, 0], u[:, :, 0]) and np.array_equal(un[:, :, -1], u[:, :, -1])
    assert np.array_equal(vn[:, 0, :], v[:, 0, :]) and np.array_equal(wn[0], w[0])
    assert not np.array_equal(wn[-1], w[-1])


def test_projection_removes_an_eigenmode_gradient():
    """Constant density: u* = dt grad_h v for a closed-form eigenvector v of A (Neumann walls,
    p = 0 on the top face) has divergence/dt = L v = -(lambda/h^2) v, the solve of A p = -h^2 s
    returns p = v, and the projection leaves zero velocity."""
    nx, ny, nz, h, dt = 6, 5, 4, 0.25, 1e-3
    v, lam = _cosine_mode(nx, ny, nz, 2, 1, 1)
    # gradient of v on the faces: centred differences, p = 0 on the top face (half-cell distance)
    gu = np.zeros((nz, ny, nx + 1)); gu[:, :, 1:nx] = np.diff(v, axis=2) / h
    gv = np.zeros((nz, ny + 1, nx)); gv[:, 1:ny, :] = np.diff(v, axis=1) / h
    gw = np.zeros((nz + 1, ny, nx)); gw[1:nz] = np.diff(v, axis=0) / h
    gw[nz] = (0.0 - v[-1]) / (h / 2)
    u0, v0, w0 = dt * gu, dt * gv, dt * gw
    s = oracle.divergence(u0, v0, w0, h, dt)
    assert np.abs(s + lam / h ** 2 * v).max() <= 1e-12 * lam / h ** 2
    F = np.zeros((nz, ny, nx))  # rho = rho_air = 1 everywhere
    op = oracle.operator(F, RHO_A, RHO_W)
    res = oracle.pcg(op, oracle.rhs(s, h), tol=1e-14)
    assert np.abs(res.x - v).max() <= 1e-11
    un, vn, wn = oracle.project(op, F, u0, v0, w0, res.x, h, dt, RHO_A, RHO_W)
    top = max(np.abs(u0).max(), np.abs(v0).max(), np.abs(w0).max())
    assert max(np.abs(un).max(), np.abs(vn).max(), np.abs(wn).max()) <= 1e-10 * top


def test_projection_after_a_solve_is_divergence_free_to_the_tolerance():
    c = inputs.flat_case(16, 12, 10, seed=5)
    g = c.grid
    modes = inputs.fourier_modes(np.random.default_rng(5))
    u, v, w = inputs.face_velocity(g, modes)
    op = oracle.operator(c.F)
    b = oracle.rhs(oracle.divergence(u, v, w, g.h, inputs.DT), g.h)
    res = oracle.pcg(op, b, tol=1e-12, precond="ssor")
    un, vn, wn = oracle.project(op, c.F, u, v, w, res.x, g.h, inputs.DT)
    div = oracle.divergence(un, vn, wn, g.h, inputs.DT)
    # |div(u_new)| h^2 is the residual: <= 1e-12 |b| in the 2-norm
    assert np.linalg.norm(div) * g.h ** 2 <= 1.01e-12 * np.linalg.norm(b)
    assert np.linalg.norm(div) < 1e-9 * np.linalg.norm(oracle.divergence(u, v, w, g.h, inputs.DT))


# ------------------------------------------------------------------------------- inputs
def test_source_is_discrete_divergence_of_face_velocity():
    g = inputs.Grid(12, 10, 8, 1.0 / 8)
    modes = inputs.fourier_modes(np.random.default_rng(4))
    u, v, w = inputs.face_velocity(g, modes)
    div = (np.diff(u, axis=2) + np.diff(v, axis=1) + np.diff(w, axis=0)) / (g.h * inputs.DT)
    np.testing.assert_allclose(inputs.divergence_source(g, modes, zchunk=3), div, rtol=0,
                               atol=1e-9 * np.abs(div).max())
    assert not u[:, :, 0].any() and not u[:, :, -1].any()
    assert not v[:, 0, :].any() and not v[:, -1, :].any()
    assert not w[0].any() and w[-1].any()


def test_fraction_limits_and_body():
    c = inputs.strut_case(64, 32, 32, seed=1)
    assert c.F.min() >= 0.0 and c.F.max() <= 1.0
    assert c.F[0].min() == 1.0            # bottom layer all water
    assert c.F[-1].max() > 0.5            # the strut (water density) pierces the air layer
    assert c.F[-1].mean() < 0.1           # ... and is thin


def test_oracle_reproduces_golden_fixture():
    """The stored oracle samples (written by tests/golden/make_golden.py from the oracle alone)
    are reproduced on this machine to the solve's tolerance."""
    import json
    import os
    with open(os.path.join(os.path.dirname(__file__), "golden", "flat32_seed0.json")) as f:
        g = json.load(f)
    c = inputs.flat_case(32, 32, 32, seed=0)
    res, _ = oracle.solve(c.F, c.s, c.grid.h, tol=1e-12, precond="jacobi")
    got = [res.x[k, j, i] for i, j, k in g["samples_ijk"]]
    np.testing.assert_allclose(got, g["jacobi"]["p"], rtol=1e-8)
    assert abs(res.iters - g["jacobi"]["iters"]) <= 5


def test_torch_input_twins_match_numpy():
    """The torch generators used inside the served request loop give the numpy fields."""
    torch = pytest.importorskip("torch")
    c = inputs.mixed_case((48, 32, 32), seed=7)
    grid, F, s, modes = inputs.mixed_fields_t((48, 32, 32), seed=7)
    np.testing.assert_allclose(F.numpy(), c.F, rtol=0, atol=1e-13)
    np.testing.assert_allclose(s.numpy(), c.s, rtol=0, atol=1e-9 * np.abs(c.s).max())
    drift = inputs.advect_modes(modes, grid, inputs.DT)
    np.testing.assert_allclose(inputs.divergence_source_t(grid, drift).numpy(),
                               inputs.divergence_source(grid, drift), rtol=0,
                               atol=1e-9 * np.abs(c.s).max())

"""Pins of the multigrid V-cycle oracle against definitions it does not share code with: the
Galerkin coarse operator against the dense product P^T A P of an aggregation matrix written out
from its definition, the V-cycle against its closed matrix form, symmetry and positivity, PCG
with it against a dense direct solve, and its effect on the iteration count."""
import numpy as np
import pytest

import oracle
from oracle import multigrid as mg
from paper_1410_1942_gb300 import inputs


def _rand_F(shape, seed):
    rng = np.random.default_rng(seed)
    F = rng.random(shape)
    F[rng.random(shape) < 0.3] = 0.0
    F[rng.random(shape) < 0.3] = 1.0
    return F


def _dense(op):
    """A as a dense matrix, column by column through the oracle's stencil apply."""
    n = op.nx * op.ny * op.nz
    A = np.empty((n, n))
    e = np.zeros(n)
    for q in range(n):
        e[q] = 1.0
        A[:, q] = oracle.apply(op, e).ravel()
        e[q] = 0.0
    return A


def _aggregation(shape, f):
    """P[c, I] = 1 when fine cell c = (i, j, k) lies in aggregate I = (i // fx, j // fy, k // fz)."""
    nz, ny, nx = shape
    fx, fy, fz = f
    nxc, nyc, nzc = -(-nx // fx), -(-ny // fy), -(-nz // fz)
    P = np.zeros((nx * ny * nz, nxc * nyc * nzc))
    for k in range(nz):
        for j in range(ny):
            for i in range(nx):
                I = i // fx + nxc * (j // fy + nyc * (k // fz))
                P[i + nx * (j + ny * k), I] = 1.0
    return P


def _cut_apertures(shape, seed):
    """Random open fractions with a few cells closed (vol = 0) and faces partly open."""
    nz, ny, nx = shape
    rng = np.random.default_rng(seed)
    vol = rng.uniform(0.2, 1.0, shape)
    vol[rng.random(shape) < 0.15] = 0.0
    ax = rng.uniform(0.0, 1.0, (nz, ny, nx + 1))
    ay = rng.uniform(0.0, 1.0, (nz, ny + 1, nx))
    az = rng.uniform(0.0, 1.0, (nz + 1, ny, nx))
    return ax, ay, az, vol


OPS = {
    "odd": lambda: oracle.operator(_rand_F((3, 4, 5), 1)),
    "walls": lambda: oracle.operator(_rand_F((4, 4, 6), 2), walls=31),
    "periodic": lambda: oracle.operator(_rand_F((4, 3, 8), 3),
                                        walls=oracle.PERIODIC_X | oracle.WALL_ZM),
    "periodic_odd": lambda: oracle.operator(_rand_F((4, 4, 3), 4), walls=oracle.PERIODIC_X),
    "cut": lambda: oracle.operator(_rand_F((4, 5, 6), 5), apertures=_cut_apertures((4, 5, 6), 6)),
    "flat_column": lambda: oracle.operator(_rand_F((7, 1, 1), 7)),
}


@pytest.mark.parametrize("name", list(OPS))
def test_galerkin_equals_dense_PtAP(name):
    op = OPS[name]()
    f = mg.factors(op.nx, op.ny, op.nz, bool(op.walls & oracle.PERIODIC_X))
    coarse = mg.galerkin(op, f)
    A = _dense(op)
    P = _aggregation(op.shape, f)
    assert P.shape[1] == coarse.nx * coarse.ny * coarse.nz
    want = P.T @ A @ P
    got = _dense(coarse)
    assert np.allclose(got, want, rtol=0, atol=1e-14 * np.abs(want).max())
    # the stored low faces: zero on a non-periodic x = 0 face, the wrap coupling when periodic
    if not op.walls & oracle.PERIODIC_X:
        assert np.all(coarse.bx[:, :, 0] == 0.0)


def test_factors_and_level_shapes():
    assert mg.factors(256, 128, 128, False) == (2, 2, 2)
    assert mg.factors(5, 1, 3, False) == (2, 1, 2)
    assert mg.factors(12, 4, 4, True) == (2, 2, 2)
    assert mg.factors(6, 4, 4, True) == (2, 2, 2)
    assert mg.factors(3, 4, 4, True) == (1, 2, 2)
    assert mg.factors(2, 4, 4, True) == (1, 2, 2)
    op = oracle.operator(_rand_F((16, 8, 32), 8))
    shapes = [lev.op.shape for lev in mg.hierarchy(op)]
    assert shapes == [(16, 8, 32), (8, 4, 16)]  # 512 cells: the coarsest level
    # level 0 is coarsened once even when it is small
    small = oracle.operator(_rand_F((2, 2, 2), 9))
    assert [lev.op.shape for lev in mg.hierarchy(small)] == [(2, 2, 2), (1, 1, 1)]


def _vcycle_matrix(levels, l, omega, alpha, sweeps):
    """Closed form of V_l: 2B - BAB + alpha (I - BA) P V_{l+1} P^T (I - AB), B = omega D^-1;
    on the coarsest level sum_{m < sweeps} (I - BA)^m B."""
    op = levels[l].op
    A = _dense(op)
    n = A.shape[0]
    B = np.diag(omega / op.diag.ravel())
    I = np.eye(n)
    if levels[l].f is None:
        V = np.zeros((n, n))
        T = I.copy()
        for _ in range(sweeps):
            V += T @ B
            T = T @ (I - B @ A)
        return V
    P = _aggregation(op.shape, levels[l].f)
    Vc = _vcycle_matrix(levels, l + 1, omega, alpha, sweeps)
    return 2 * B - B @ A @ B + alpha * (I - B @ A) @ P @ Vc @ P.T @ (I - A @ B)


def _vcycle_dense(levels, **kw):
    op = levels[0].op
    n = op.nx * op.ny * op.nz
    V = np.empty((n, n))
    e = np.zeros(op.shape)
    for q in range(n):
        e.flat[q] = 1.0
        V[:, q] = mg.vcycle(levels, e, **kw).ravel()
        e.flat[q] = 0.0
    return V


@pytest.mark.parametrize("name", ["odd", "walls", "periodic", "cut"])
def test_vcycle_equals_its_matrix_form(name):
    op = OPS[name]()
    levels = mg.hierarchy(op, coarse_max=4)
    assert len(levels) >= 3
    for kw in ({}, {"omega": 0.7, "alpha": 1.0, "coarse_sweeps": 3}):
        V = _vcycle_dense(levels, **kw)
        om = kw.get("omega", mg.OMEGA)
        al = kw.get("alpha", mg.ALPHA)
        sw = kw.get("coarse_sweeps", mg.COARSE_SWEEPS)
        want = _vcycle_matrix(levels, 0, om, al, sw)
        assert np.allclose(V, want, rtol=0, atol=1e-12 * np.abs(want).max())


@pytest.mark.parametrize("name", ["odd", "walls", "periodic", "cut"])
def test_vcycle_is_symmetric_positive_definite(name):
    op = OPS[name]()
    V = _vcycle_dense(mg.hierarchy(op, coarse_max=4))
    assert np.abs(V - V.T).max() <= 1e-13 * np.abs(V).max()
    assert np.linalg.eigvalsh(0.5 * (V + V.T)).min() > 0.0


@pytest.mark.parametrize("name", ["odd", "walls", "periodic", "cut"])
def test_pcg_mg_matches_dense_solve(name):
    op = OPS[name]()
    b = np.random.default_rng(11).standard_normal(op.shape)
    ref = np.linalg.solve(_dense(op), b.ravel()).reshape(op.shape)
    res = mg.pcg_mg(op, b, tol=1e-13, levels=mg.hierarchy(op, coarse_max=4))
    assert res.status == oracle.OK
    assert np.linalg.norm(res.x - ref) <= 1e-10 * np.linalg.norm(ref)


def test_mg_takes_far_fewer_iterations_than_jacobi():
    c = inputs.strut_case(64, 32, 32, seed=0)
    op = oracle.operator(c.F)
    b = oracle.rhs(c.s, c.grid.h)
    jac = oracle.pcg(op, b, tol=1e-9)
    res = mg.pcg_mg(op, b, tol=1e-9)
    assert res.status == oracle.OK and res.rel_residual <= 1e-9 * (1 + 1e-6)
    assert res.iters <= 40 and res.iters * 8 <= jac.iters, (res.iters, jac.iters)
    ref = oracle.pcg(op, b, tol=1e-12, precond="ssor")
    assert np.linalg.norm(res.x - ref.x) <= 1e-6 * np.linalg.norm(ref.x)

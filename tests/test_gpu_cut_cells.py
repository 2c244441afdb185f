"""Parity of the free-slip cut-cell operator, solve and projection with the FP64 oracle through
the C ABI: face open fractions and cell fluid fractions (bodies given by a signed distance)."""
import numpy as np
import pytest

import oracle
from paper_1410_1942_gb300 import build, capi, inputs

pytestmark = pytest.mark.gpu

L2_TOL = 1e-6


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    build.build()
    capi.load()


def _random_apertures(shape, seed):
    nz, ny, nx = shape
    rng = np.random.default_rng(seed)
    ax = rng.uniform(0.05, 1.0, (nz, ny, nx + 1))
    ay = rng.uniform(0.05, 1.0, (nz, ny + 1, nx))
    az = rng.uniform(0.05, 1.0, (nz + 1, ny, nx))
    vol = rng.uniform(0.05, 1.0, shape)
    vol[rng.random(shape) < 0.15] = 0.0
    return ax, ay, az, vol


def _strut_body(grid):
    """A full-depth elliptic strut as a free-slip body (signed distance positive in the fluid)."""
    Lx, Ly, _ = grid.lengths
    psi = lambda x, y, z: inputs.ellipse_sdf(x, y, 0.5 * Lx, 0.5 * Ly, 0.3 * Lx, 0.2 * Ly)
    return inputs.cut_apertures(grid, psi)


@pytest.mark.parametrize("walls", [0, capi.WALL_XM | capi.WALL_ZM])
def test_cut_operator_bit_exact(walls):
    c = inputs.flat_case(37, 23, 19, seed=3, tol=1e-10)
    aps = _random_apertures(c.grid.shape, 4)
    op = oracle.operator(c.F, walls=walls, apertures=aps)
    with capi.Poisson(c.grid.nx, c.grid.ny, c.grid.nz, c.grid.h, precision="fp64",
                      dirichlet_walls=walls) as s:
        s.set_apertures(*aps)
        s.set_density(c.F)
        arrs = [np.empty(c.grid.shape) for _ in range(4)]
        s.get_operator(*arrs)
        assert "cut-cells" in s.describe()
    for got, ref in zip(arrs, (op.bx, op.by, op.bz, op.diag)):
        assert np.array_equal(got, ref)


@pytest.mark.parametrize("prec,precond,shape", [
    ("fp64", "jacobi", (48, 32, 24)), ("fp64", "rbssor", (48, 32, 24)),
    ("fp32", "jacobi", (48, 32, 24)), ("fp32", "rbssor", (48, 32, 24)),
    ("bf16", "jacobi", (48, 32, 24)),
    # whole 64-cell tiles along x: the inner CG phases on the 2 x 2-cell kernels for FP32 faces
    # (ragged tile rows: 36 = 2 x 16 + 4; odd plane count)
    ("fp32", "jacobi", (128, 36, 21)), ("bf16", "jacobi", (128, 36, 21))])
def test_cut_solve_matches_oracle(prec, precond, shape):
    """A strut body through a two-phase surface: both acceptance criteria against the oracle's
    cut operator; the body's cells come out 0."""
    c = inputs.flat_case(*shape, seed=5, tol=1e-9)
    aps = _strut_body(c.grid)
    op = oracle.operator(c.F, apertures=aps)
    b = oracle.rhs(c.s, c.grid.h, aps[3])
    ref = oracle.pcg(op, b, tol=1e-12, precond="ssor")
    assert ref.status == oracle.OK
    with capi.Poisson(c.grid.nx, c.grid.ny, c.grid.nz, c.grid.h, precision=prec,
                      precond=precond) as s:
        s.set_apertures(*aps)
        s.set_density(c.F)
        p = np.zeros(c.grid.shape)
        rc, st = s.solve(c.s, p, c.tol)
    assert rc == capi.OK
    rel = oracle.rel_residual(op, b, p)
    assert rel <= c.tol * (1 + 1e-6), rel
    assert np.linalg.norm(p - ref.x) <= L2_TOL * np.linalg.norm(ref.x)
    assert not np.any(p[aps[3] == 0])


def test_cut_divergence_and_projection_bit_exact():
    nx, ny, nz = 13, 9, 7
    shape = (nz, ny, nx)
    rng = np.random.default_rng(6)
    F = rng.random(shape)
    aps = _random_apertures(shape, 7)
    u = rng.standard_normal((nz, ny, nx + 1))
    v = rng.standard_normal((nz, ny + 1, nx))
    w = rng.standard_normal((nz + 1, ny, nx))
    p = rng.standard_normal(shape)
    h, dt = 1.0 / 16, 1.3e-3
    op = oracle.operator(F, walls=capi.WALL_YP, apertures=aps)
    ref_s = oracle.divergence(u, v, w, h, dt, aps)
    ru, rv, rw = oracle.project(op, F, u, v, w, p, h, dt)
    with capi.Poisson(nx, ny, nz, h, dirichlet_walls=capi.WALL_YP) as s:
        s.set_apertures(*aps)
        s.set_density(F)
        got_s = np.empty(shape)
        s.divergence(u, v, w, dt, got_s)
        gu, gv, gw = u.copy(), v.copy(), w.copy()
        s.project(gu, gv, gw, p, dt)
    assert np.array_equal(got_s, ref_s)
    assert np.array_equal(gu, ru) and np.array_equal(gv, rv) and np.array_equal(gw, rw)


def test_cut_cells_need_set_density_again_and_can_be_removed():
    c = inputs.flat_case(32, 16, 16, seed=8, tol=1e-9)
    aps = _strut_body(c.grid)
    with capi.Poisson(c.grid.nx, c.grid.ny, c.grid.nz, c.grid.h) as s:
        s.set_density(c.F)
        march = s.describe()
        s.set_apertures(*aps)
        p = np.zeros(c.grid.shape)
        with pytest.raises(capi.PoissonError) as e:
            s.solve(c.s, p, c.tol)
        assert e.value.status == capi.ENOTREADY
        s.set_density(c.F)
        rc, _ = s.solve(c.s, p, c.tol)
        assert rc == capi.OK and "cut-cells" in s.describe()
        s.set_apertures()  # back to the plain operator and its kernels
        s.set_density(c.F)
        p2 = np.zeros(c.grid.shape)
        rc, _ = s.solve(c.s, p2, c.tol)
        assert rc == capi.OK and s.describe() == march
    op = oracle.operator(c.F)
    assert oracle.rel_residual(op, oracle.rhs(c.s, c.grid.h), p2) <= c.tol * (1 + 1e-6)

"""Parity of the projection around the solve (divergence of u*, velocity correction) with the FP64
oracle, through the C ABI: both passes bit for bit, and the full projection step (divergence,
mixed-precision solve, correction) leaving a divergence equal to the solve's residual."""
import numpy as np
import pytest

import oracle
from paper_1410_1942_gb300 import build, capi, inputs

pytestmark = pytest.mark.gpu

SHAPES = [(37, 23, 19), (64, 16, 1), (8, 9, 33), (1, 5, 7), (16, 1, 4)]


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    build.build()
    capi.load()


def _faces(shape, seed):
    nz, ny, nx = shape
    rng = np.random.default_rng(seed)
    return (rng.standard_normal((nz, ny, nx + 1)), rng.standard_normal((nz, ny + 1, nx)),
            rng.standard_normal((nz + 1, ny, nx)))


def _rand_F(shape, seed):
    rng = np.random.default_rng(seed)
    F = rng.random(shape)
    F[rng.random(shape) < 0.3] = 0.0
    F[rng.random(shape) < 0.3] = 1.0
    return F


@pytest.mark.parametrize("dev", [False, True])
@pytest.mark.parametrize("nx,ny,nz", SHAPES)
def test_divergence_bit_exact(nx, ny, nz, dev):
    import torch
    shape = (nz, ny, nx)
    u, v, w = _faces(shape, 1)
    h, dt = 1.0 / 16, 1.3e-3
    ref = oracle.divergence(u, v, w, h, dt)
    with capi.Poisson(nx, ny, nz, h) as s:
        if dev:
            ud, vd, wd = (torch.from_numpy(a).cuda() for a in (u, v, w))
            out = torch.empty(shape, dtype=torch.float64, device="cuda")
            s.divergence(ud, vd, wd, dt, out)
            got = out.cpu().numpy()
        else:
            got = np.empty(shape)
            s.divergence(u, v, w, dt, got)
    assert np.array_equal(got, ref)


@pytest.mark.parametrize("dev", [False, True])
@pytest.mark.parametrize("nx,ny,nz", SHAPES)
def test_project_bit_exact(nx, ny, nz, dev):
    import torch
    shape = (nz, ny, nx)
    F = _rand_F(shape, 2)
    u, v, w = _faces(shape, 3)
    p = np.random.default_rng(4).standard_normal(shape)
    h, dt = 1.0 / 16, 1.3e-3
    op = oracle.operator(F)
    ru, rv, rw = oracle.project(op, F, u, v, w, p, h, dt)
    with capi.Poisson(nx, ny, nz, h) as s:
        s.set_density(F)
        if dev:
            ud, vd, wd, pd = (torch.from_numpy(a.copy()).cuda() for a in (u, v, w, p))
            s.project(ud, vd, wd, pd, dt)
            gu, gv, gw = (a.cpu().numpy() for a in (ud, vd, wd))
        else:
            gu, gv, gw = u.copy(), v.copy(), w.copy()
            s.project(gu, gv, gw, p, dt)
    assert np.array_equal(gu, ru) and np.array_equal(gv, rv) and np.array_equal(gw, rw)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("case", ["flat", "strut"])
def test_projection_step_leaves_the_solve_residual(prec, case):
    """divergence -> solve -> correction on the device: div_h(u_new) h^2 is the residual of the
    solve (<= tol |b|), and the corrected velocity matches the oracle's projection of its own
    1e-12 pressure to the solve's accuracy."""
    c = (inputs.flat_case(40, 24, 20, seed=6, tol=1e-9) if case == "flat"
         else inputs.strut_case(96, 48, 40, seed=2))
    g = c.grid
    modes = inputs.fourier_modes(np.random.default_rng(7))
    u, v, w = inputs.face_velocity(g, modes)
    op = oracle.operator(c.F)
    s_ref = oracle.divergence(u, v, w, g.h, inputs.DT)
    b = oracle.rhs(s_ref, g.h)
    p = np.zeros(g.shape)
    un, vn, wn = u.copy(), v.copy(), w.copy()
    with capi.Poisson(g.nx, g.ny, g.nz, g.h, precision=prec) as s:
        s.set_density(c.F)
        rc, st = s.projection_step(un, vn, wn, inputs.DT, p, 1e-9)
    assert rc == capi.OK
    div = oracle.divergence(un, vn, wn, g.h, inputs.DT)
    r, _ = oracle.residual(op, b, p)
    scale = (np.abs(b).max() + np.abs(oracle.apply(op, p)).max()) / g.h ** 2
    assert np.abs(div + r / g.h ** 2).max() <= 1e-12 * scale
    assert np.linalg.norm(div) * g.h ** 2 <= 1e-9 * (1 + 1e-6) * np.linalg.norm(b)
    ref = oracle.pcg(op, b, tol=1e-12, precond="ssor")
    ru, rv, rw = oracle.project(op, c.F, u, v, w, ref.x, g.h, inputs.DT)
    # the correction differs by dt beta grad(p - p_ref): |p - p_ref| <= 1e-6 |p_ref| (the solve's
    # parity bound), and the CG error is smooth, so its gradient stays within a few times that
    for got, want, orig in ((un, ru, u), (vn, rv, v), (wn, rw, w)):
        assert np.linalg.norm(got - want) <= 2e-5 * np.linalg.norm(orig - want) + 1e-15


@pytest.mark.parametrize("walls", [1, 2, 4, 8, 16, 31])
def test_project_with_dirichlet_walls_bit_exact(walls):
    nx, ny, nz = 13, 9, 7
    shape = (nz, ny, nx)
    F = _rand_F(shape, 8)
    u, v, w = _faces(shape, 9)
    p = np.random.default_rng(10).standard_normal(shape)
    h, dt = 1.0 / 16, 1.3e-3
    op = oracle.operator(F, walls=walls)
    ru, rv, rw = oracle.project(op, F, u, v, w, p, h, dt)
    with capi.Poisson(nx, ny, nz, h, dirichlet_walls=walls) as s:
        s.set_density(F)
        gu, gv, gw = u.copy(), v.copy(), w.copy()
        s.project(gu, gv, gw, p, dt)
    assert np.array_equal(gu, ru) and np.array_equal(gv, rv) and np.array_equal(gw, rw)


def test_project_with_periodic_x_bit_exact():
    nx, ny, nz = 12, 9, 7
    shape = (nz, ny, nx)
    F = _rand_F(shape, 11)
    u, v, w = _faces(shape, 12)
    u[:, :, -1] = u[:, :, 0]
    p = np.random.default_rng(13).standard_normal(shape)
    h, dt = 1.0 / 16, 1.3e-3
    op = oracle.operator(F, walls=oracle.PERIODIC_X | oracle.WALL_ZM)
    ru, rv, rw = oracle.project(op, F, u, v, w, p, h, dt)
    with capi.Poisson(nx, ny, nz, h, dirichlet_walls=capi.WALL_ZM, periodic_x=True) as s:
        s.set_density(F)
        gu, gv, gw = u.copy(), v.copy(), w.copy()
        s.project(gu, gv, gw, p, dt)
    assert np.array_equal(gu, ru) and np.array_equal(gv, rv) and np.array_equal(gw, rw)


def test_projection_errors():
    c = inputs.flat_case(16, 8, 8, seed=1)
    g = c.grid
    u, v, w = _faces(g.shape, 5)
    p = np.zeros(g.shape)
    with capi.Poisson(g.nx, g.ny, g.nz, g.h) as s:
        with pytest.raises(capi.PoissonError) as e:
            s.project(u, v, w, p, 1e-3)
        assert e.value.status == capi.ENOTREADY
        s.set_density(c.F)
        with pytest.raises(capi.PoissonError) as e:
            s.project(u, v, w, p, 0.0)
        assert e.value.status == capi.EINVAL
        with pytest.raises(capi.PoissonError) as e:
            s.divergence(u, v, w, -1.0, p)
        assert e.value.status == capi.EINVAL


@pytest.mark.parametrize("precond", ["jacobi", "mg"])
def test_two_stage_projection_cycle(precond):
    """The two projections of a time step (Numerical Time Integration) on one handle: the
    density is set again between the stages (the surface moved), the second solve starts from
    the first stage's pressure, and each stage leaves the divergence its solve's residual (the
    convection and diffusion increments between the stages are not part of this library: a
    fixed smooth field stands in for them)."""
    g = inputs.Grid(48, 24, 24, 1.0 / 24)
    eta1 = lambda x, y: 0.02 * np.sin(2 * np.pi * x) * np.cos(2 * np.pi * y)
    eta2 = lambda x, y: 0.02 * np.sin(2 * np.pi * (x - 0.05)) * np.cos(2 * np.pi * y)
    F1, F2 = inputs.water_fraction(g, eta1), inputs.water_fraction(g, eta2)
    rng = np.random.default_rng(31)
    u0, v0, w0 = inputs.face_velocity(g, inputs.fourier_modes(rng))
    du, dv, dw = inputs.face_velocity(g, inputs.fourier_modes(rng), amp=0.01)
    dt, tol = inputs.DT, 1e-9
    p = np.zeros(g.shape)
    with capi.Poisson(g.nx, g.ny, g.nz, g.h, precision="fp32", precond=precond) as s:
        iters = []
        # each stage projects a provisional velocity built from the step's starting field (the
        # second with the stand-in increment), so the two pressures are close
        for F, (eu, ev, ew) in ((F1, (0.0, 0.0, 0.0)), (F2, (du, dv, dw))):
            s.set_density(F)
            u, v, w = u0 + eu, v0 + ev, w0 + ew
            b = oracle.rhs(oracle.divergence(u, v, w, g.h, dt), g.h)
            rc, st = s.projection_step(u, v, w, dt, p, tol)
            assert rc == capi.OK
            iters.append(st["inner_iters"])
            op = oracle.operator(F)
            div = oracle.divergence(u, v, w, g.h, dt)
            r, _ = oracle.residual(op, b, p)
            scale = (np.abs(b).max() + np.abs(oracle.apply(op, p)).max()) / g.h ** 2
            assert np.abs(div + r / g.h ** 2).max() <= 1e-12 * scale
            assert np.linalg.norm(div) * g.h ** 2 <= tol * (1 + 1e-6) * np.linalg.norm(b)
    # the second stage starts from the first stage's pressure: the warm start pays
    assert iters[1] < iters[0]


# ----------------------------------------------------------------------------- reduced pressure
@pytest.mark.parametrize("dev", [False, True])
@pytest.mark.parametrize("nx,ny,nz,walls", [(37, 23, 19, 0), (64, 16, 1, 0), (8, 9, 33, 31),
                                            (1, 5, 7, 0), (48, 24, 20, oracle.PERIODIC_X),
                                            (6, 4, 5, oracle.PERIODIC_X | 16)])
def test_hydrostatic_force_bit_exact(nx, ny, nz, walls, dev):
    """The reduced-pressure force added to the face velocities, bit for bit against the oracle
    (every face of random fields, boundary faces included; the periodic wrap face on faces 0
    and nx)."""
    import torch
    shape = (nz, ny, nx)
    F = _rand_F(shape, 5)
    u, v, w = _faces(shape, 6)
    h, dt, g, zo = 1.0 / nz, 1.3e-3, -9.81, 0.47
    ref = oracle.hydrostatic_force(F, u, v, w, h, g, zo, dt=dt, walls=walls)
    kw = {"dirichlet_walls": walls & 31, "periodic_x": bool(walls & oracle.PERIODIC_X)}
    with capi.Poisson(nx, ny, nz, h, **kw) as s:
        if dev:
            Fd, ud, vd, wd = (torch.from_numpy(a.copy()).cuda() for a in (F, u, v, w))
            s.hydrostatic_force(Fd, ud, vd, wd, g, zo, dt)
            got = [a.cpu().numpy() for a in (ud, vd, wd)]
        else:
            got = [u.copy(), v.copy(), w.copy()]
            s.hydrostatic_force(F, *got, g, zo, dt)
    for a, b in zip(got, ref):
        assert np.array_equal(a, b)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_hydrostatic_rest_through_the_library(prec):
    """A layered density at rest (surface above the static level, no flow): force, divergence,
    solve and projection all through the C ABI leave no velocity, and the reduced pressure is
    the column with the paper's jumps (z_f - z_o) g (rho_above - rho_below), 0 in the top layer."""
    nx, ny, nz = 32, 16, 48
    h = 1.0 / nz
    g_, zo, dt = -9.81, 0.43, 1e-3
    zc = (np.arange(nz) + 0.5) * h
    eps, zs = 1.5 * h, 0.55
    d = zs - zc
    Fz = np.where(d > eps, 1.0, np.where(d < -eps, 0.0,
                                         0.5 * (1 + d / eps + np.sin(np.pi * d / eps) / np.pi)))
    F = np.broadcast_to(Fz[:, None, None], (nz, ny, nx)).copy()
    rho = 1.0 + Fz * 999.0
    col = np.zeros(nz)
    for k in range(nz - 1, 0, -1):
        col[k - 1] = col[k] + (k * h - zo) * g_ * (rho[k] - rho[k - 1])
    u, v, w = (np.zeros(a.shape) for a in _faces((nz, ny, nx), 0))
    p = np.zeros((nz, ny, nx))
    s_ = np.empty((nz, ny, nx))
    with capi.Poisson(nx, ny, nz, h, precision=prec) as s:
        s.set_density(F)
        s.hydrostatic_force(F, u, v, w, g_, zo, dt)
        ref = np.abs(w).max()
        assert ref > 0
        s.divergence(u, v, w, dt, s_)
        rc, st = s.solve(s_, p, 1e-12)
        assert rc == capi.OK
        s.project(u, v, w, p, dt)
    assert np.abs(p - col[:, None, None]).max() <= 1e-8 * np.abs(col).max()
    for a in (u, v, w):
        assert np.abs(a).max() <= 1e-7 * ref


def test_hydrostatic_force_errors():
    with capi.Poisson(8, 8, 8, 0.125) as s:
        F = np.zeros((8, 8, 8))
        u, v, w = _faces((8, 8, 8), 0)
        for bad in ((0.0, 1000.0, -9.8, 0.5, 1e-3), (1.0, 1000.0, float("nan"), 0.5, 1e-3),
                    (1.0, 1000.0, -9.8, float("inf"), 1e-3)):
            with pytest.raises(capi.PoissonError) as e:
                s.hydrostatic_force(F, u, v, w, bad[2], bad[3], bad[4], rho_air=bad[0],
                                    rho_water=bad[1])
            assert e.value.status == capi.EINVAL

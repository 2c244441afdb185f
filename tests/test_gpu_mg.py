"""Parity of the multigrid V-cycle preconditioner (POISSON_MG) with the FP64 oracle, through the
C ABI: the hierarchy's depth, one V-cycle applied to a random vector (FP64 to rounding, FP32
within its rounding), and full MG-preconditioned solves in every precision mode, with Dirichlet
walls, periodic x and cut cells, against both acceptance criteria."""
import numpy as np
import pytest

import oracle
from oracle import multigrid as mg
from paper_1410_1942_gb300 import build, capi, inputs

pytestmark = pytest.mark.gpu

L2_TOL = 1e-6
# one V-cycle, relative L2 distance from the oracle's FP64 cycle: FP64 differs only in the order
# of the sums (a few ulp per level); FP32 carries the FP32 inner operator (rho/2 rounded to 24
# bits, approximate reciprocals: ~1e-7 per face) and FP32 rounding through some 40 chained
# sweeps and sums.
VCYCLE_TOL = {"fp64": 1e-12, "fp32": 2e-5}


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    build.build()
    capi.load()


def _rand_F(shape, seed):
    rng = np.random.default_rng(seed)
    F = rng.random(shape)
    F[rng.random(shape) < 0.3] = 0.0
    F[rng.random(shape) < 0.3] = 1.0
    return F


def _strut_apertures(grid):
    Lx, Ly = grid.nx * grid.h, grid.ny * grid.h
    psi = lambda x, y, z: inputs.ellipse_sdf(x, y, 0.5 * Lx, 0.5 * Ly, 0.3 * Lx, 0.2 * Ly)
    return inputs.cut_apertures(grid, psi)


# (shape nx, ny, nz; walls) -- several tiles, ragged tails, odd sizes, walls, periodic x
APPLY_CASES = [((37, 23, 19), 0), ((64, 16, 8), 0), ((8, 9, 33), 0), ((40, 24, 20), 31),
               ((48, 24, 20), oracle.PERIODIC_X), ((30, 12, 10), oracle.PERIODIC_X | 16),
               ((3, 1, 70), 0)]


def _walls_kw(walls):
    return dict(dirichlet_walls=walls & 31, periodic_x=bool(walls & oracle.PERIODIC_X))


@pytest.mark.parametrize("shape,walls", APPLY_CASES)
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_vcycle_apply_matches_oracle(shape, walls, prec):
    nx, ny, nz = shape
    F = _rand_F((nz, ny, nx), 1)
    op = oracle.operator(F, walls=walls)
    levels = mg.hierarchy(op)
    r = np.random.default_rng(2).standard_normal(op.shape)
    want = mg.vcycle(levels, r)
    with capi.Poisson(nx, ny, nz, 1.0 / nz, precision=prec, precond="mg", **_walls_kw(walls)) as s:
        s.set_density(F)
        assert "mg-vcycle levels=%d" % len(levels) in s.describe()
        got = np.empty_like(r)
        s.precond_apply(r, got, kind="mg", precision=prec)
    err = np.linalg.norm(got - want) / np.linalg.norm(want)
    assert err <= VCYCLE_TOL[prec], err


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_vcycle_apply_with_cut_cells_matches_oracle(prec):
    g = inputs.Grid(40, 24, 12, 1.0 / 12)
    ap = _strut_apertures(g)
    F = _rand_F(g.shape, 3)
    op = oracle.operator(F, apertures=ap)
    r = np.random.default_rng(4).standard_normal(g.shape)
    want = mg.vcycle(mg.hierarchy(op), r)
    with capi.Poisson(g.nx, g.ny, g.nz, g.h, precision=prec, precond="mg") as s:
        s.set_apertures(*ap)
        s.set_density(F)
        got = np.empty_like(r)
        s.precond_apply(r, got, kind="mg", precision=prec)
    assert np.linalg.norm(got - want) <= VCYCLE_TOL[prec] * np.linalg.norm(want)


# 256 x 84 x 49: the fine passes on shared-memory planes (whole 32-cell tiles along x) with two
# planes per thread (z-chunk 2), a ragged last row of tiles (84 = 10 x 8 + 4) and an odd plane
# count (the last coarse plane has one fine plane).
STAGED = (256, 84, 49)


@pytest.mark.parametrize("walls", [0, 31])
def test_vcycle_apply_with_staged_fine_passes(walls):
    nx, ny, nz = STAGED
    F = _rand_F((nz, ny, nx), 7)
    with capi.Poisson(nx, ny, nz, 1.0 / nz, precision="fp32", precond="mg",
                      **_walls_kw(walls)) as s:
        assert "zchunk=2" in s.describe(), s.describe()
        s.set_density(F)
        r = np.random.default_rng(8).standard_normal((nz, ny, nx))
        got = np.empty_like(r)
        s.precond_apply(r, got, kind="mg", precision="fp32")
    op = oracle.operator(F, walls=walls)
    want = mg.vcycle(mg.hierarchy(op), r)
    err = np.linalg.norm(got - want) / np.linalg.norm(want)
    assert err <= VCYCLE_TOL["fp32"], err


@pytest.mark.parametrize("walls", [0, 31])
@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_mg_solve_with_staged_fine_passes(walls, prec):
    c = inputs.strut_case(*STAGED, seed=9)
    g = c.grid
    op, b, xref = _reference(c.F, c.s, g.h, walls=walls)
    with capi.Poisson(g.nx, g.ny, g.nz, g.h, precision=prec, precond="mg", inner_tol=1e-5,
                      **_walls_kw(walls)) as s:
        s.set_density(c.F)
        p = np.zeros(g.shape)
        rc, st = s.solve(c.s, p, 1e-9)
    assert rc == capi.OK
    _check(op, b, xref, p, st, 1e-9)


# 256 x 96 x 28: the fine passes on 2 x 2-cell quad tiles and the first two coarse levels
# (128 x 48 x 14, 64 x 24 x 7) on the quad kernels for FP32 faces (odd plane count on level 2);
# 128 x 36 x 21: a cut-cell body, whose fine level takes the face kernels too (ragged tile rows:
# 36 = 2 x 16 + 4), as does its first coarse level (64 x 18 x 11).
FACES = (256, 96, 28)
CUT_FACES = (128, 36, 21)


@pytest.mark.parametrize("walls", [0, 31, oracle.PERIODIC_X, oracle.PERIODIC_X | 16])
def test_vcycle_apply_with_quad_face_levels(walls):
    nx, ny, nz = FACES
    F = _rand_F((nz, ny, nx), 17)
    with capi.Poisson(nx, ny, nz, 1.0 / nz, precision="fp32", precond="mg",
                      **_walls_kw(walls)) as s:
        s.set_density(F)
        r = np.random.default_rng(18).standard_normal((nz, ny, nx))
        got = np.empty_like(r)
        s.precond_apply(r, got, kind="mg", precision="fp32")
    op = oracle.operator(F, walls=walls)
    want = mg.vcycle(mg.hierarchy(op), r)
    err = np.linalg.norm(got - want) / np.linalg.norm(want)
    assert err <= VCYCLE_TOL["fp32"], err


@pytest.mark.parametrize("walls", [0, oracle.PERIODIC_X])
@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_mg_solve_with_quad_face_levels(prec, walls):
    """Periodic x: the halo columns of the first and last tiles wrap (the 64-wide second coarse
    level is one tile wrapping onto itself)."""
    c = inputs.strut_case(*FACES, seed=19)
    g = c.grid
    op, b, xref = _reference(c.F, c.s, g.h, walls=walls)
    with capi.Poisson(g.nx, g.ny, g.nz, g.h, precision=prec, precond="mg", inner_tol=1e-5,
                      **_walls_kw(walls)) as s:
        s.set_density(c.F)
        p = np.zeros(g.shape)
        rc, st = s.solve(c.s, p, 1e-9)
    assert rc == capi.OK
    _check(op, b, xref, p, st, 1e-9)


def test_vcycle_apply_cut_cells_on_quad_faces():
    nx, ny, nz = CUT_FACES
    c = inputs.flat_case(nx, ny, nz, seed=21, tol=1e-9)
    ap = _strut_apertures(c.grid)
    with capi.Poisson(nx, ny, nz, c.grid.h, precision="fp32", precond="mg") as s:
        s.set_apertures(*ap)
        s.set_density(c.F)
        r = np.random.default_rng(22).standard_normal((nz, ny, nx))
        got = np.empty_like(r)
        s.precond_apply(r, got, kind="mg", precision="fp32")
    op = oracle.operator(c.F, apertures=ap)
    want = mg.vcycle(mg.hierarchy(op), r)
    err = np.linalg.norm(got - want) / np.linalg.norm(want)
    assert err <= VCYCLE_TOL["fp32"], err


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_mg_solve_cut_cells_on_quad_faces(prec):
    c = inputs.flat_case(*CUT_FACES, seed=23, tol=1e-9)
    g = c.grid
    ap = _strut_apertures(g)
    op, b, xref = _reference(c.F, c.s, g.h, apertures=ap, vol=ap[3])
    with capi.Poisson(g.nx, g.ny, g.nz, g.h, precision=prec, precond="mg") as s:
        s.set_apertures(*ap)
        s.set_density(c.F)
        p = np.zeros(g.shape)
        rc, st = s.solve(c.s, p, 1e-9)
    assert rc == capi.OK
    _check(op, b, xref, p, st, 1e-9)


def test_mg_chunk_graphs_on_a_stream():
    """On a stream of its own (capturable, unlike the legacy default stream) the CG loop runs each
    chunk of iterations as one replay of a captured graph: two solves in a row (capture, then
    replay) meet both criteria; new apertures drop the graph, and the cut operator's solve and
    the plain one after them are right too."""
    import torch
    c = inputs.strut_case(128, 36, 21, seed=31)
    g = c.grid
    op, b, xref = _reference(c.F, c.s, g.h)
    ap = _strut_apertures(g)
    cop, cb, cxref = _reference(c.F, c.s, g.h, apertures=ap, vol=ap[3])
    st = torch.cuda.Stream()
    with capi.Poisson(g.nx, g.ny, g.nz, g.h, precision="fp32", precond="mg", stream=st) as s:
        s.set_density(c.F)
        for _ in range(2):
            p = np.zeros(g.shape)
            l0 = capi.kernel_launches()
            rc, info = s.solve(c.s, p, 1e-9)
            assert rc == capi.OK and capi.kernel_launches() > l0
            _check(op, b, xref, p, info, 1e-9)
        s.set_apertures(*ap)
        s.set_density(c.F)
        p = np.zeros(g.shape)
        rc, info = s.solve(c.s, p, 1e-9)
        assert rc == capi.OK
        _check(cop, cb, cxref, p, info, 1e-9)
        s.set_apertures(None, None, None, None)
        s.set_density(c.F)
        p = np.zeros(g.shape)
        rc, info = s.solve(c.s, p, 1e-9)
        assert rc == capi.OK
        _check(op, b, xref, p, info, 1e-9)


# Edge layouts of the 2x2-cells-per-thread kernels: one row pair (ny = 2), one plane (nz = 1:
# aggregates of one plane, fz = 1), two planes, a single 64-wide tile wrapping onto itself
# (periodic x), and a last tile row holding one row pair (ny = 18).
QUAD_EDGES = [((64, 2, 1), 0), ((128, 2, 5), 0), ((64, 16, 2), 31), ((64, 18, 3), 0),
              ((64, 18, 3), oracle.PERIODIC_X), ((192, 4, 7), oracle.PERIODIC_X | 16)]


@pytest.mark.parametrize("shape,walls", QUAD_EDGES)
def test_vcycle_apply_quad_edge_layouts(shape, walls):
    nx, ny, nz = shape
    F = _rand_F((nz, ny, nx), 41)
    with capi.Poisson(nx, ny, nz, 1.0 / max(nz, 8), precision="fp32", precond="mg",
                      **_walls_kw(walls)) as s:
        s.set_density(F)
        r = np.random.default_rng(42).standard_normal((nz, ny, nx))
        got = np.empty_like(r)
        s.precond_apply(r, got, kind="mg", precision="fp32")
    op = oracle.operator(F, walls=walls)
    want = mg.vcycle(mg.hierarchy(op), r)
    err = np.linalg.norm(got - want) / np.linalg.norm(want)
    assert err <= VCYCLE_TOL["fp32"], err


@pytest.mark.parametrize("shape,walls", QUAD_EDGES)
@pytest.mark.parametrize("precond,tile", [("mg", 0), ("jacobi", -1)])
def test_solves_on_quad_edge_layouts(shape, walls, precond, tile):
    c = inputs.strut_case(*shape, seed=43)
    g = c.grid
    op, b, xref = _reference(c.F, c.s, g.h, walls=walls)
    with capi.Poisson(g.nx, g.ny, g.nz, g.h, precision="fp32", precond=precond, tile=tile,
                      **_walls_kw(walls)) as s:
        s.set_density(c.F)
        p = np.zeros(g.shape)
        rc, st = s.solve(c.s, p, 1e-9)
    assert rc == capi.OK
    _check(op, b, xref, p, st, 1e-9)


def _reference(F, s, h, walls=0, apertures=None, vol=None):
    op = oracle.operator(F, walls=walls, apertures=apertures)
    b = oracle.rhs(s, h, vol)
    ref = oracle.pcg(op, b, tol=1e-12, precond="ssor" if not walls & oracle.PERIODIC_X or
                     op.nx % 2 == 0 else "jacobi")
    assert ref.status == oracle.OK
    return op, b, ref.x


def _check(op, b, xref, p, st, tol):
    rel = oracle.rel_residual(op, b, p)
    assert rel <= tol * (1 + 1e-6), rel
    err = np.linalg.norm(p - xref) / np.linalg.norm(xref)
    assert err <= L2_TOL, err
    assert abs(st["rel_residual"] - rel) <= 1e-3 * rel + 1e-15


SOLVE_CASES = {
    "flat": lambda: inputs.flat_case(32, 32, 32, seed=0, tol=1e-10),
    "ragged": lambda: inputs.flat_case(37, 23, 19, seed=2, tol=1e-10),
    "strut": lambda: inputs.strut_case(96, 48, 40, seed=1),
    "column": lambda: inputs.flat_case(3, 5, 70, seed=4, tol=1e-10),
}


@pytest.mark.parametrize("name", list(SOLVE_CASES))
@pytest.mark.parametrize("prec", ["fp64", "fp32", "bf16"])
def test_mg_solve_matches_oracle(name, prec):
    c = SOLVE_CASES[name]()
    g = c.grid
    op, b, xref = _reference(c.F, c.s, g.h)
    with capi.Poisson(g.nx, g.ny, g.nz, g.h, precision=prec, precond="mg") as s:
        s.set_density(c.F)
        p = np.zeros(g.shape)
        rc, st = s.solve(c.s, p, c.tol)
    assert rc == capi.OK
    _check(op, b, xref, p, st, c.tol)


# 48 wide: the fine passes on plain loads; 64 wide with a ragged last row of tiles (ny = 20): the
# fine passes with shared-memory planes (whole 32-cell tiles along x, no periodic wrap)
@pytest.mark.parametrize("shape", [(48, 24, 20), (64, 20, 12)])
@pytest.mark.parametrize("walls", [0, 31, 16 | 1, oracle.PERIODIC_X, oracle.PERIODIC_X | 16])
@pytest.mark.parametrize("prec", ["fp64", "fp32", "bf16"])
def test_mg_solve_with_boundary_variants(shape, walls, prec):
    c = inputs.strut_case(*shape, seed=3)
    g = c.grid
    op, b, xref = _reference(c.F, c.s, g.h, walls=walls)
    with capi.Poisson(g.nx, g.ny, g.nz, g.h, precision=prec, precond="mg",
                      **_walls_kw(walls)) as s:
        s.set_density(c.F)
        p = np.zeros(g.shape)
        rc, st = s.solve(c.s, p, 1e-9)
    assert rc == capi.OK
    _check(op, b, xref, p, st, 1e-9)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_mg_solve_with_cut_cells(prec):
    c = inputs.flat_case(48, 24, 16, seed=5, tol=1e-9)
    g = c.grid
    ap = _strut_apertures(g)
    op, b, xref = _reference(c.F, c.s, g.h, apertures=ap, vol=ap[3])
    with capi.Poisson(g.nx, g.ny, g.nz, g.h, precision=prec, precond="mg") as s:
        s.set_apertures(*ap)
        s.set_density(c.F)
        p = np.zeros(g.shape)
        rc, st = s.solve(c.s, p, 1e-9)
    assert rc == capi.OK
    _check(op, b, xref, p, st, 1e-9)


def test_mg_needs_far_fewer_iterations_than_jacobi():
    c = inputs.strut_case(128, 64, 64, seed=0)
    g = c.grid
    its = {}
    for pc in ("jacobi", "mg"):
        with capi.Poisson(g.nx, g.ny, g.nz, g.h, precision="fp32", precond=pc, tile=-1) as s:
            s.set_density(c.F)
            p = np.zeros(g.shape)
            rc, st = s.solve(c.s, p, 1e-9)
        assert rc == capi.OK
        its[pc] = st["inner_iters"]
    assert its["mg"] * 10 <= its["jacobi"], its


def test_mg_errors():
    with pytest.raises(capi.PoissonError) as e:
        capi.Poisson(1, 1, 1, 1.0, precond="mg")
    assert e.value.status == capi.EINVAL
    F = _rand_F((4, 4, 4), 6)
    r = np.ones((4, 4, 4))
    z = np.empty_like(r)
    with capi.Poisson(4, 4, 4, 0.25, precision="fp32") as s:
        s.set_density(F)
        with pytest.raises(capi.PoissonError) as e:
            s.precond_apply(r, z, kind="mg", precision="fp32")
        assert e.value.status == capi.EINVAL
    with capi.Poisson(4, 4, 4, 0.25, precision="fp32", precond="mg") as s:
        with pytest.raises(capi.PoissonError) as e:
            s.precond_apply(r, z, kind="mg", precision="fp32")
        assert e.value.status == capi.ENOTREADY
        s.set_density(F)
        with pytest.raises(capi.PoissonError) as e:
            s.precond_apply(r, z, kind="mg", precision="fp64")
        assert e.value.status == capi.EINVAL


def test_mg_periodic_odd_nx_keeps_x_uncoarsened():
    """Periodic x with odd nx: the x axis is not coarsened (its wrap face stays between two
    aggregates); the level shapes and one cycle follow the oracle's."""
    nx, ny, nz = 45, 16, 12
    F = _rand_F((nz, ny, nx), 21)
    walls = oracle.PERIODIC_X
    op = oracle.operator(F, walls=walls)
    levels = mg.hierarchy(op)
    assert all(lev.op.nx == nx for lev in levels)
    r = np.random.default_rng(22).standard_normal(op.shape)
    want = mg.vcycle(levels, r)
    with capi.Poisson(nx, ny, nz, 1.0 / nz, precision="fp64", precond="mg",
                      **_walls_kw(walls)) as s:
        s.set_density(F)
        assert "mg-vcycle levels=%d" % len(levels) in s.describe()
        got = np.empty_like(r)
        s.precond_apply(r, got, kind="mg", precision="fp64")
    assert np.linalg.norm(got - want) <= VCYCLE_TOL["fp64"] * np.linalg.norm(want)


def test_mg_bf16_with_cut_cells():
    c = inputs.flat_case(48, 24, 16, seed=9, tol=1e-9)
    g = c.grid
    ap = _strut_apertures(g)
    op, b, xref = _reference(c.F, c.s, g.h, apertures=ap, vol=ap[3])
    with capi.Poisson(g.nx, g.ny, g.nz, g.h, precision="bf16", precond="mg") as s:
        s.set_apertures(*ap)
        s.set_density(c.F)
        p = np.zeros(g.shape)
        rc, st = s.solve(c.s, p, 1e-9)
    assert rc == capi.OK
    _check(op, b, xref, p, st, 1e-9)


def test_mg_warm_start_and_zero_source():
    c = inputs.flat_case(40, 24, 20, seed=6, tol=1e-10)
    g = c.grid
    op, b, xref = _reference(c.F, c.s, g.h)
    with capi.Poisson(g.nx, g.ny, g.nz, g.h, precision="fp32", precond="mg") as s:
        s.set_density(c.F)
        p = xref.copy()
        rc, st = s.solve(c.s, p, 1e-9)
        assert rc == capi.OK and st["inner_iters"] == 0 and np.array_equal(p, xref)
        p = np.full(g.shape, 3.0)
        rc, st = s.solve(np.zeros(g.shape), p, 1e-9)
        assert rc == capi.OK and not p.any()


def test_mg_iteration_cap_reports_notconv_with_best_iterate():
    c = inputs.strut_case(96, 48, 40, seed=1)
    g = c.grid
    op = oracle.operator(c.F)
    b = oracle.rhs(c.s, g.h)
    with capi.Poisson(g.nx, g.ny, g.nz, g.h, precision="fp32", precond="mg", max_iters=4) as s:
        s.set_density(c.F)
        p = np.zeros(g.shape)
        rc, st = s.solve(c.s, p, 1e-9, allow=(capi.ENOTCONV,))
    assert rc == capi.ENOTCONV
    assert st["inner_iters"] <= 4 + 8
    rel = oracle.rel_residual(op, b, p)
    assert rel < 1.0 and abs(st["rel_residual"] - rel) <= 1e-3 * rel


def test_mg_device_and_host_arrays_agree():
    import torch
    c = inputs.strut_case(64, 32, 24, seed=4)
    g = c.grid
    with capi.Poisson(g.nx, g.ny, g.nz, g.h, precision="fp32", precond="mg") as s:
        s.set_density(c.F)
        ph = np.zeros(g.shape)
        rc, _ = s.solve(c.s, ph, 1e-9)
        assert rc == capi.OK
        sd = torch.from_numpy(c.s).cuda()
        pd = torch.zeros(g.shape, dtype=torch.float64, device="cuda")
        rc, _ = s.solve(sd, pd, 1e-9)
        assert rc == capi.OK
    assert np.array_equal(pd.cpu().numpy(), ph)

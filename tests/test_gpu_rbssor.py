"""The red-black SSOR inner solve on the plane-marching kernels (march_rb.cu) against the oracle.

With omega = 1 the library runs red-black SSOR-PCG in its reduced form: from a start whose red
equations hold, the black parts of the SSOR-PCG iterates are the iterates of Jacobi-preconditioned
CG on the black Schur complement, and the red parts follow from the black ones.  Checked here:
  * solves in FP32 and BF16 inner precision, on shapes with ragged tiles, one-plane grids and
    Dirichlet walls, meet both acceptance criteria against the oracle;
  * every red-black kernel variant and work split does;
  * the k-th iterate of a capped solve is the k-th iterate of the oracle's textbook SSOR-PCG
    started from the red-consistent point x0 = (b_R / D_R, 0) -- the two are the same method;
  * the iteration count is the SSOR count, about half the Jacobi one.
"""
import numpy as np
import pytest

import oracle
from paper_1410_1942_gb300 import build, capi, inputs

pytestmark = pytest.mark.gpu

L2_TOL = 1e-6
REF_TOL = 1e-12


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    assert torch.cuda.is_available()
    build.build()
    capi.load()


_cache = {}


def _case(name):
    if name not in _cache:
        c = {
            "strut": lambda: inputs.strut_case(96, 48, 40, seed=1),
            "flat": lambda: inputs.flat_case(64, 32, 32, seed=3, tol=1e-10),
            "ragged": lambda: inputs.strut_case(72, 21, 13, seed=2),
            "narrow": lambda: inputs.flat_case(8, 9, 33, seed=4, tol=1e-10),
            "plane": lambda: inputs.flat_case(48, 16, 1, seed=5, tol=1e-10),
        }[name]()
        _cache[name] = c
    return _cache[name]


def _ref(c, walls=0):
    key = (id(c), walls)
    if key not in _cache:
        op = oracle.operator(c.F, walls=walls)
        b = oracle.rhs(c.s, c.grid.h)
        ref = oracle.pcg(op, b, tol=REF_TOL, precond="ssor")
        assert ref.status == oracle.OK
        _cache[key] = (op, b, ref.x)
    return _cache[key]


def _check(c, op, b, xref, p, st, tol):
    rel = oracle.rel_residual(op, b, p)
    assert rel <= tol * (1 + 1e-6), rel
    assert abs(st["rel_residual"] - rel) <= 1e-3 * rel + 1e-16
    err = np.linalg.norm(p - xref) / np.linalg.norm(xref)
    assert err <= L2_TOL, err


@pytest.mark.parametrize("name", ["strut", "flat", "ragged", "narrow", "plane"])
@pytest.mark.parametrize("prec", ["fp32", "bf16"])
@pytest.mark.parametrize("walls", [0, 31, 16])
def test_rb_solve_matches_oracle(name, prec, walls):
    c = _case(name)
    g = c.grid
    op, b, xref = _ref(c, walls)
    with capi.Poisson(g.nx, g.ny, g.nz, g.h, precision=prec, precond="rbssor",
                      dirichlet_walls=walls) as s:
        assert "red-black" in s.describe(), s.describe()
        s.set_density(c.F)
        p = np.zeros(g.shape)
        rc, st = s.solve(c.s, p, c.tol)
    assert rc == capi.OK
    _check(c, op, b, xref, p, st, c.tol)


# every red-black variant (64x8 tiles with 4 or 8 consumer warps and 8- or 7-stage rings, 64x16
# tiles) and split
@pytest.mark.parametrize("tile", [30812204, 31812204, 32812204, 30712204, 32712204, 30812108,
                                  32812108, 30712208, 32712208])
@pytest.mark.parametrize("name", ["strut", "ragged"])
def test_rb_variants_match_oracle(tile, name):
    c = _case(name)
    g = c.grid
    op, b, xref = _ref(c)
    with capi.Poisson(g.nx, g.ny, g.nz, g.h, precision="fp32", precond="rbssor", tile=tile) as s:
        assert "red-black" in s.describe() and "tile=%d " % tile in s.describe(), s.describe()
        s.set_density(c.F)
        p = np.zeros(g.shape)
        rc, st = s.solve(c.s, p, c.tol)
    assert rc == capi.OK
    _check(c, op, b, xref, p, st, c.tol)


@pytest.mark.parametrize("k", [1, 5, 8])
@pytest.mark.parametrize("name", ["strut", "ragged"])
def test_capped_rb_solve_is_the_ssor_pcg_iterate(name, k):
    """The FP32 inner solve capped at k iterations returns the oracle's k-th SSOR-PCG iterate
    (FP64, textbook PCG with the red-black SSOR preconditioner at omega = 1) from the start
    whose red equations hold, to FP32 accuracy."""
    c = _case(name)
    g = c.grid
    op = oracle.operator(c.F)
    b = oracle.rhs(c.s, g.h)
    kk, jj, ii = np.meshgrid(np.arange(g.nz), np.arange(g.ny), np.arange(g.nx), indexing="ij")
    red = (ii + jj + kk) % 2 == 0
    x0 = np.where(red, b / op.diag, 0.0)
    ref = oracle.pcg(op, b, x0=x0, tol=0.0, precond="ssor", max_iters=k).x
    with capi.Poisson(g.nx, g.ny, g.nz, g.h, precision="fp32", precond="rbssor",
                      max_iters=k) as s:
        s.set_density(c.F)
        p = np.zeros(g.shape)
        rc, st = s.solve(c.s, p, 1e-9, allow=(capi.OK, capi.ENOTCONV))
    assert rc == capi.ENOTCONV and st["inner_iters"] == k
    assert np.linalg.norm(p - ref) <= 1e-4 * np.linalg.norm(ref)
    # and not the Jacobi iterate, nor the SSOR iterate from the zero start
    jac = oracle.pcg(op, b, tol=0.0, precond="jacobi", max_iters=k).x
    assert np.linalg.norm(p - jac) > 1e-3 * np.linalg.norm(ref)


def test_rb_takes_the_ssor_iteration_count():
    c = _case("strut")
    g = c.grid
    its = {}
    for pc in ("jacobi", "rbssor"):
        with capi.Poisson(g.nx, g.ny, g.nz, g.h, precision="fp32", precond=pc) as s:
            s.set_density(c.F)
            p = np.zeros(g.shape)
            rc, st = s.solve(c.s, p, c.tol)
            assert rc == capi.OK
            its[pc] = st["inner_iters"]
    assert its["rbssor"] <= 0.65 * its["jacobi"], its


def test_rb_warm_start_and_zero_source():
    c = _case("strut")
    g = c.grid
    op, b, xref = _ref(c)
    with capi.Poisson(g.nx, g.ny, g.nz, g.h, precision="fp32", precond="rbssor") as s:
        s.set_density(c.F)
        p = xref.copy()
        rc, st = s.solve(c.s, p, c.tol)
        assert rc == capi.OK and st["inner_iters"] == 0
        p = np.ones(g.shape)
        rc, st = s.solve(np.zeros(g.shape), p, c.tol)
        assert rc == capi.OK and not p.any()


def test_family3_tiles_need_the_rbssor_preconditioner():
    with pytest.raises(capi.PoissonError) as e:
        capi.Poisson(64, 32, 16, 1.0 / 16, precision="fp32", tile=30812204)
    assert e.value.status == capi.EINVAL
    # omega != 1, FP64 and periodic x keep the column kernels
    for kw in ({"omega": 1.3}, {"precision": "fp64"}, {"periodic_x": True}):
        opts = dict(precision="fp32", precond="rbssor")
        opts.update(kw)
        with capi.Poisson(64, 32, 16, 1.0 / 16, **opts) as s:
            assert "red-black" not in s.describe()

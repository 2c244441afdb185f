"""The allocation-free residual entry point, checked against poisson_solve's own residual.

Some callers cannot allocate device memory when they check a pressure field (a step loop that
cannot afford cudaMalloc's latency or cudaFree's device-wide synchronisation, a process whose
device memory belongs to another allocator, code that forbids allocation after start-up).
poisson_residual_noalloc serves them from a static device array.  This file is collected last so
that a run stopping at the first failure has already run every other test; it passes alone in a
fresh process (its first call sets the array up) and after the rest of the suite.
"""
import numpy as np
import pytest

import oracle
from paper_1410_1942_gb300 import build, capi, inputs

pytestmark = pytest.mark.gpu

# Two FP64 evaluations of the same residual differ only by rounding: per cell by at most a few
# ulps of the terms of b - A p, so their relative residuals differ by at most
# rounding_bound() = 16 eps || |A| |p| + |b| ||_2 / ||b||_2 (|A| |p| = D |p| + sum beta |p_n|).
# At a converged field the terms are far larger than the residual and the bound is what the
# comparison can ask; on random fields it is ~1e-15 relative.
EPS = 2.0 ** -53


def rounding_bound(op, b, p):
    ap = np.abs(p)
    absA = 2.0 * op.diag * ap - oracle.apply(op, ap)
    return 16 * EPS * float(np.linalg.norm(absA + np.abs(b))) / float(np.linalg.norm(b))


@pytest.fixture(scope="module")
def solved():
    import torch
    assert torch.cuda.is_available()
    build.build()
    capi.load()
    c = inputs.strut_case(96, 48, 40, seed=5)
    g = c.grid
    F = torch.from_numpy(c.F).cuda()
    s = torch.from_numpy(c.s).cuda()
    p = torch.zeros(g.shape, dtype=torch.float64, device="cuda")
    with capi.Poisson(g.nx, g.ny, g.nz, g.h, precision="fp32") as solver:
        solver.set_density(F)
        rc, st = solver.solve(s, p, 1e-9)
    torch.cuda.synchronize()
    assert rc == capi.OK
    return c, F, s, p, st


def test_noalloc_residual_matches_the_solver_twice(solved):
    c, F, s, p, st = solved
    g = c.grid
    op, b, x = oracle.operator(c.F), oracle.rhs(c.s, g.h), p.cpu().numpy()
    ref = oracle.rel_residual(op, b, x)
    tol = rounding_bound(op, b, x)
    vals = [capi.residual_noalloc(g.nx, g.ny, g.nz, g.h, F, 1.0, 1000.0, s, p) for _ in range(2)]
    for v in vals:
        assert abs(v - st["rel_residual"]) <= tol, (v, st["rel_residual"], tol)
    assert vals[0] == vals[1]  # the shared array is reset between calls
    assert abs(vals[0] - ref) <= tol, (vals[0], ref, tol)


def test_noalloc_residual_device_output_and_zero_field(solved):
    import torch
    c, F, s, p, st = solved
    g = c.grid
    op, b, x = oracle.operator(c.F), oracle.rhs(c.s, g.h), p.cpu().numpy()
    tol = rounding_bound(op, b, x)
    out = torch.full((1,), -1.0, dtype=torch.float64, device="cuda")
    for _ in range(2):
        capi.residual_noalloc(g.nx, g.ny, g.nz, g.h, F, 1.0, 1000.0, s, p, out=out)
        torch.cuda.synchronize()
        assert abs(out.item() - st["rel_residual"]) <= tol
    zero = torch.zeros_like(p)
    for _ in range(2):  # r = b exactly for p = 0
        assert abs(capi.residual_noalloc(g.nx, g.ny, g.nz, g.h, F, 1.0, 1000.0, s, zero) - 1.0) <= 1e-14


def test_noalloc_rejects_grids_beyond_its_scratch(solved):
    c, F, s, p, st = solved
    with pytest.raises(capi.PoissonError) as e:
        capi.residual_noalloc(32 * 65, 8 * 64, 1, 0.01, F, 1.0, 1000.0, s, p)
    assert e.value.status == capi.ETOOLARGE
    with pytest.raises(capi.PoissonError) as e:  # host arrays are refused, not copied
        g = c.grid
        capi.residual_noalloc(g.nx, g.ny, g.nz, g.h, c.F, 1.0, 1000.0, c.s, p.cpu().numpy())
    assert e.value.status == capi.EINVAL
    g = c.grid
    for ra, rw in ((float("inf"), 1000.0), (1.0, float("inf")), (float("nan"), 1000.0), (0.0, 1.0)):
        with pytest.raises(capi.PoissonError) as e:  # non-finite or non-positive densities
            capi.residual_noalloc(g.nx, g.ny, g.nz, g.h, F, ra, rw, s, p)
        assert e.value.status == capi.EINVAL


# Ragged tiles (nx not a multiple of 32, ny not of 8), several planes per thread with a short
# last z-chunk (256 x 128 x 67: kc = 5, chunks of 5 planes and a last one of 2), and a plane of
# exactly the 4096-tile limit (2048 x 512 x 3).
@pytest.mark.parametrize("shape", [(37, 13, 29), (256, 128, 67), (2048, 512, 3)])
def test_noalloc_residual_on_ragged_and_limit_shapes(solved, shape):
    import torch
    nx, ny, nz = shape
    rng = np.random.default_rng(nx * 7 + ny * 3 + nz)
    F = rng.uniform(0.0, 1.0, size=(nz, ny, nx))
    F[rng.uniform(size=F.shape) < 0.3] = 1.0
    F[rng.uniform(size=F.shape) < 0.3] = 0.0
    s = rng.standard_normal((nz, ny, nx))
    p = rng.standard_normal((nz, ny, nx))
    h = 1.0 / nz
    op, b = oracle.operator(F), oracle.rhs(s, h)
    ref = oracle.rel_residual(op, b, p)
    tol = rounding_bound(op, b, p)
    assert tol < 1e-13 * ref  # random fields: no cancellation to speak of
    Fd, sd, pd = (torch.from_numpy(a).cuda() for a in (F, s, p))
    vals = [capi.residual_noalloc(nx, ny, nz, h, Fd, 1.0, 1000.0, sd, pd) for _ in range(2)]
    assert vals[0] == vals[1]
    assert abs(vals[0] - ref) <= tol, (vals[0], ref, tol)

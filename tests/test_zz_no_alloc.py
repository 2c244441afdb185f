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

# the library's own residual against the oracle's evaluation uses the same tolerance
REL_TOL = 1e-3


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
    vals = [capi.residual_noalloc(g.nx, g.ny, g.nz, g.h, F, 1.0, 1000.0, s, p) for _ in range(2)]
    for v in vals:
        assert abs(v - st["rel_residual"]) <= REL_TOL * st["rel_residual"]
    assert vals[0] == vals[1]  # the shared array is reset between calls
    ref = oracle.rel_residual(oracle.operator(c.F), oracle.rhs(c.s, g.h), p.cpu().numpy())
    assert abs(vals[0] - ref) <= REL_TOL * ref


def test_noalloc_residual_device_output_and_zero_field(solved):
    import torch
    c, F, s, p, st = solved
    g = c.grid
    out = torch.full((1,), -1.0, dtype=torch.float64, device="cuda")
    for _ in range(2):
        capi.residual_noalloc(g.nx, g.ny, g.nz, g.h, F, 1.0, 1000.0, s, p, out=out)
        torch.cuda.synchronize()
        assert abs(out.item() - st["rel_residual"]) <= REL_TOL * st["rel_residual"]
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

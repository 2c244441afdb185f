"""The failure path of the persistent PCG launches: a grid barrier whose wait runs out.

Every device-side wait of the library is bounded (grid barriers: 1 s of the GPU's global timer;
TMA mbarrier waits: 200 ms).  poisson_test_unreachable_barrier makes a handle's launches wait at
their grid barriers for one CTA more than they launch, so the first barrier can only end by its
deadline: every CTA must give up, let its TMA copies land and leave, and the solve must report
POISSON_ETIMEOUT instead of hanging.  Nothing faults: the wait simply runs out.  Afterwards the
same handle (and the context) must solve normally and match the oracle.
"""
import time

import numpy as np
import pytest

import oracle
from paper_1410_1942_gb300 import build, capi, inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    assert torch.cuda.is_available()
    build.build()
    capi.load()


# one-sweep (producer warp, lockstep split), two-sweep with a producer warp, two-sweep without,
# and the red-black SSOR kernel
@pytest.mark.parametrize("tile,precond", [(12012204, "jacobi"), (12204, "jacobi"),
                                          (2204, "jacobi"), (32812204, "rbssor")])
def test_unreachable_barrier_times_out_and_the_handle_recovers(tile, precond):
    c = inputs.strut_case(64, 32, 32, seed=2)
    g = c.grid
    op, b = oracle.operator(c.F), oracle.rhs(c.s, g.h)
    with capi.Poisson(g.nx, g.ny, g.nz, g.h, precision="fp32", tile=tile, precond=precond) as sv:
        sv.set_density(c.F)
        assert "persistent" in sv.describe() or "one-sweep" in sv.describe(), sv.describe()
        sv.test_unreachable_barrier(1)
        p = np.zeros(g.shape)
        t0 = time.perf_counter()
        rc, st = sv.solve(c.s, p, c.tol, allow=(capi.ETIMEOUT,))
        dt = time.perf_counter() - t0
        assert rc == capi.ETIMEOUT
        assert 0.9 <= dt < 10.0, dt  # one barrier deadline (1 s), not a hang
        assert np.all(np.isfinite(p))
        sv.test_unreachable_barrier(0)
        p = np.zeros(g.shape)
        rc, st = sv.solve(c.s, p, c.tol)
        assert rc == capi.OK
    rel = oracle.rel_residual(op, b, p)
    assert rel <= c.tol * (1 + 1e-6), rel
    ref = oracle.pcg(op, b, tol=1e-12, precond="ssor").x
    assert np.linalg.norm(p - ref) <= 1e-6 * np.linalg.norm(ref)


def test_unreachable_barrier_needs_a_persistent_launch():
    c = inputs.strut_case(64, 32, 32, seed=2)
    g = c.grid
    for kw in ({"precision": "fp64"}, {"precision": "fp32", "tile": -1},
               {"precision": "fp32", "precond": "rbssor", "tile": -1}):
        with capi.Poisson(g.nx, g.ny, g.nz, g.h, **kw) as sv:
            with pytest.raises(capi.PoissonError) as e:
                sv.test_unreachable_barrier(1)
            assert e.value.status == capi.EINVAL
    with capi.Poisson(g.nx, g.ny, g.nz, g.h, precision="fp32", tile=12204) as sv:
        for bad in (-1, 1025):
            with pytest.raises(capi.PoissonError):
                sv.test_unreachable_barrier(bad)

"""Non-finite or out-of-range inputs end in a status, never in a hang or a silent answer.

Injected on the host: a NaN or infinite water fraction, a fraction so far outside [0, 1] that the
density is not positive, a NaN source, an infinite initial guess, and one such solve inside a
batch of good ones.  The density check makes poisson_set_density refuse the field (EINVAL) and
leave the handle not ready (ENOTREADY); a non-finite source or guess makes the first residual
norm non-finite, and the solve reports EBREAKDOWN at once.  Each time the same handle then
solves a good problem to the oracle's residual.
"""
import time

import numpy as np
import pytest

import oracle
from paper_1410_1942_gb300 import build, capi, inputs

pytestmark = pytest.mark.gpu

KINDS = [{"precision": "fp64"}, {"precision": "fp32"}, {"precision": "fp32", "tile": -1},
         {"precision": "bf16"}, {"precision": "fp32", "precond": "rbssor"},
         {"precision": "fp32", "precond": "mg"}, {"precision": "fp32", "periodic_x": True}]


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    assert torch.cuda.is_available()
    build.build()
    capi.load()


def _case(kw):
    c = inputs.strut_case(64, 32, 32, seed=5)
    walls = oracle.PERIODIC_X if kw.get("periodic_x") else 0
    return c, oracle.operator(c.F, walls=walls), oracle.rhs(c.s, c.grid.h)


def _good_solve(sv, c, op, b):
    p = np.zeros(c.grid.shape)
    rc, _ = sv.solve(c.s, p, c.tol)
    assert rc == capi.OK
    assert oracle.rel_residual(op, b, p) <= c.tol * (1 + 1e-6)


def _kind_id(kw):
    return "-".join("%s=%s" % kv for kv in kw.items())


@pytest.mark.parametrize("kw", KINDS, ids=_kind_id)
def test_bad_density_is_refused_and_the_handle_recovers(kw):
    c, op, b = _case(kw)
    g = c.grid
    with capi.Poisson(g.nx, g.ny, g.nz, g.h, **kw) as sv:
        for cell, value in (((3, 4, 5), np.nan), ((0, 0, 0), np.inf), ((31, 31, 63), -np.inf),
                            ((30, 20, 10), -10.0)):
            F = c.F.copy()
            F[cell] = value
            with pytest.raises(capi.PoissonError) as e:
                sv.set_density(F)
            assert e.value.status == capi.EINVAL
            rc, _ = sv.solve(c.s, np.zeros(g.shape), c.tol, allow=(capi.ENOTREADY,))
            assert rc == capi.ENOTREADY
        # a small overshoot of the fraction keeps the density positive: accepted
        F = c.F.copy()
        F[3, 4, 5] = 1.0 + 1e-3
        F[4, 4, 5] = -1e-4
        sv.set_density(F)
        sv.set_density(c.F)
        _good_solve(sv, c, op, b)


@pytest.mark.parametrize("kw", KINDS, ids=_kind_id)
def test_non_finite_source_or_guess_breaks_down_at_once(kw):
    c, op, b = _case(kw)
    g = c.grid
    with capi.Poisson(g.nx, g.ny, g.nz, g.h, **kw) as sv:
        sv.set_density(c.F)
        bad_s = c.s.copy()
        bad_s[7, 8, 9] = np.nan
        bad_p = np.zeros(g.shape)
        bad_p[1, 2, 3] = np.inf
        for s, p in ((bad_s, np.zeros(g.shape)), (c.s, bad_p)):
            t0 = time.perf_counter()
            rc, _ = sv.solve(s, p, c.tol, allow=(capi.EBREAKDOWN,))
            assert rc == capi.EBREAKDOWN
            assert time.perf_counter() - t0 < 5.0
        p = np.zeros(g.shape)
        rc, _ = sv.solve(c.s, p, c.tol)
        assert rc == capi.OK
        assert oracle.rel_residual(op, b, p) <= c.tol * (1 + 1e-6)


def test_one_bad_solve_in_a_batch_leaves_the_others_alone():
    c, op, b = _case({})
    g = c.grid
    import torch
    svs = [capi.Poisson(g.nx, g.ny, g.nz, g.h, precision="fp32") for _ in range(3)]
    try:
        for sv in svs:
            sv.set_density(c.F)
        s = [torch.from_numpy(c.s.copy()).cuda() for _ in range(3)]
        s[1][5, 6, 7] = float("nan")
        p = [torch.zeros(g.shape, dtype=torch.float64, device="cuda") for _ in range(3)]
        torch.cuda.synchronize()
        tickets = capi.batch_submit(svs, s, p, c.tol)
        status = {}
        t0 = time.perf_counter()
        while len(status) < 3:
            for j, t in enumerate(tickets):
                if j not in status:
                    rc, _ = capi.poll(t)
                    if rc != capi.PENDING:
                        status[j] = rc
            assert time.perf_counter() - t0 < 30.0
        assert [status[j] for j in range(3)] == [capi.OK, capi.EBREAKDOWN, capi.OK]
        for j in (0, 2):
            assert oracle.rel_residual(op, b, p[j].cpu().numpy()) <= c.tol * (1 + 1e-6)
    finally:
        for sv in svs:
            sv.close()

"""Allocation failures end in POISSON_ENOMEM with everything released.

The failure is injected on the host: poisson_test_fail_alloc(n) makes the n-th following device
or pinned-host allocation of the library fail as if memory were exhausted, and
poisson_test_live_allocations counts the library's allocations not yet released.  For each kind
of handle, creation is tried with the failure at the 1st, 2nd, ... allocation until one succeeds:
every failed creation returns ENOMEM and leaves the live count where it was, and the handle
created at the end solves to the oracle's residual and releases everything when destroyed.  A
batch that meets an allocation failure reports ENOMEM for the solves it affects, and the next
batch runs normally.  (Forced tiles only: the autotuner caches its choice per size class for
the whole process, and a choice made under injected failures would outlive this test.)
"""
import numpy as np
import pytest

import oracle
from paper_1410_1942_gb300 import build, capi, inputs

pytestmark = pytest.mark.gpu

KINDS = [{"precision": "fp32", "tile": 12012204}, {"precision": "fp32", "tile": -1},
         {"precision": "bf16", "tile": 12312204}, {"precision": "fp32", "precond": "rbssor",
                                                   "tile": 32812204},
         {"precision": "fp32", "precond": "mg"}, {"precision": "bf16", "precond": "mg"},
         {"precision": "fp64"}, {"precision": "fp64", "precond": "mg"},
         {"precision": "fp32", "tile": 12012204, "periodic_x": True}]


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    assert torch.cuda.is_available()
    build.build()
    capi.load()
    yield
    capi.test_fail_alloc(0)


def _kind_id(kw):
    return "-".join("%s=%s" % kv for kv in kw.items())


def _case(kw):
    c = inputs.strut_case(64, 32, 32, seed=13)
    walls = oracle.PERIODIC_X if kw.get("periodic_x") else 0
    return c, oracle.operator(c.F, walls=walls), oracle.rhs(c.s, c.grid.h)


@pytest.mark.parametrize("kw", KINDS, ids=_kind_id)
def test_creation_fails_cleanly_at_every_allocation(kw):
    c, op, b = _case(kw)
    g = c.grid
    base = capi.live_allocations()
    failures = 0
    sv = None
    for n in range(1, 200):
        capi.test_fail_alloc(n)
        try:
            sv = capi.Poisson(g.nx, g.ny, g.nz, g.h, **kw)
        except capi.PoissonError as e:
            assert e.status == capi.ENOMEM, (n, e.status)
            assert capi.live_allocations() == base, n
            failures += 1
            continue
        finally:
            capi.test_fail_alloc(0)
        break
    assert sv is not None and failures >= 3
    with sv:
        assert capi.live_allocations() > base
        sv.set_density(c.F)
        p = np.zeros(g.shape)
        rc, _ = sv.solve(c.s, p, c.tol)
        assert rc == capi.OK
        assert oracle.rel_residual(op, b, p) <= c.tol * (1 + 1e-6)
    assert capi.live_allocations() == base


def _poll_all(tickets):
    out = []
    for t in tickets:
        while True:
            rc, _ = capi.poll(t)
            if rc != capi.PENDING:
                break
        out.append(rc)
    return out


def test_batch_allocation_failures_report_enomem():
    """The failure at each of the first allocations a batch makes (the executor's job tables
    and plan when it has none big enough yet, staging): every solve ends OK or ENOMEM, and a
    batch after them runs to the oracle's residual."""
    cases = inputs.batch_cases(6, seed=17, hi=(96, 64, 48))
    solvers = [capi.Poisson(c.grid.nx, c.grid.ny, c.grid.nz, c.grid.h, precision="fp32",
                            tile=12012204) for c in cases]
    try:
        for s, c in zip(solvers, cases):
            s.set_density(c.F)
        for n in range(1, 9):
            ps = [np.zeros(c.grid.shape) for c in cases]
            capi.test_fail_alloc(n)
            try:
                status = _poll_all(capi.batch_submit(solvers, [c.s for c in cases], ps, 1e-9))
            finally:
                capi.test_fail_alloc(0)
            assert all(rc in (capi.ENOMEM, capi.OK) for rc in status), (n, status)
        ps = [np.zeros(c.grid.shape) for c in cases]
        status = _poll_all(capi.batch_submit(solvers, [c.s for c in cases], ps, 1e-9))
        assert status == [capi.OK] * len(cases)
        for c, p in zip(cases, ps):
            op = oracle.operator(c.F)
            assert oracle.rel_residual(op, oracle.rhs(c.s, c.grid.h), p) <= 1e-9 * (1 + 1e-6)
    finally:
        for s in solvers:
            s.close()


def test_fail_alloc_rejects_a_negative_count():
    with pytest.raises(capi.PoissonError) as e:
        capi.test_fail_alloc(-1)
    assert e.value.status == capi.EINVAL

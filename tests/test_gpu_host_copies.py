"""Host arrays in pinned memory: the transfer kernel gives the results of the other paths.

The library moves a user array of at least 1 MiB between device memory and pinned (page-locked,
mapped) host memory with a kernel that reads or writes it through its device mapping, and every
other transfer with cudaMemcpyAsync.  Each call that takes host arrays runs here on pinned torch
tensors (16-byte aligned, and views one element in: 8-byte aligned, with an odd cell count so
that the transfer ends in a tail), on pageable numpy arrays and on device tensors.  The results
agree bit for bit; the solutions meet the oracle's residual, and the projection passes equal the
oracle's bit for bit, as in the small-grid projection tests.
"""
import numpy as np
import pytest

import oracle
from paper_1410_1942_gb300 import build, capi, inputs

pytestmark = pytest.mark.gpu

# 262144 cells (2 MiB per FP64 array) and 134685 cells (odd, just over 1 MiB)
SHAPES = [(128, 64, 32), (73, 41, 45)]


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    assert torch.cuda.is_available()
    build.build()
    capi.load()


def _pinned(a, offset):
    """A pinned copy of `a` starting 8 * offset bytes past a 16-byte boundary (offset 0 or 1)."""
    import torch
    a = np.ascontiguousarray(a, dtype=np.float64)
    buf = torch.empty(a.size + 2, dtype=torch.float64).pin_memory()
    start = ((8 * offset - buf.data_ptr()) % 16) // 8
    t = buf[start:start + a.size].view(a.shape)
    t.copy_(torch.from_numpy(a))
    assert t.is_pinned() and t.data_ptr() % 16 == 8 * offset
    return t


def _dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _host_kinds(a):
    """(name, array) for the pinned aligned, pinned offset and pageable copies of `a`."""
    return [("pinned", _pinned(a, 0)), ("pinned+8", _pinned(a, 1)), ("pageable", a.copy())]


def _np(a):
    return a.numpy() if hasattr(a, "numpy") else a


@pytest.mark.parametrize("offset", [0, 1])
@pytest.mark.parametrize("nx,ny,nz", SHAPES)
def test_solve_with_host_arrays_matches_device_arrays(nx, ny, nz, offset):
    import torch
    c = inputs.strut_case(nx, ny, nz, seed=3)
    g = c.grid
    with capi.Poisson(nx, ny, nz, g.h, precision="fp32") as sv:
        sv.set_density(_dev(c.F))
        p_d = torch.zeros(g.shape, dtype=torch.float64, device="cuda")
        sv.solve(_dev(c.s), p_d, c.tol)
        ref = p_d.cpu().numpy()
        for F, s, p in ((_pinned(c.F, offset), _pinned(c.s, offset),
                         _pinned(np.zeros(g.shape), offset)),
                        (c.F.copy(), c.s.copy(), np.zeros(g.shape))):
            sv.set_density(F)
            rc, st = sv.solve(s, p, c.tol)
            assert rc == capi.OK
            assert np.array_equal(_np(p), ref)
        # a warm start read from pinned memory: the solve starts at the solution
        p = _pinned(ref, offset)
        rc, st = sv.solve(_pinned(c.s, offset), p, c.tol)
        assert rc == capi.OK and st["inner_iters"] == 0
        assert np.array_equal(_np(p), ref)
    op = oracle.operator(c.F)
    assert oracle.rel_residual(op, oracle.rhs(c.s, g.h), ref) <= c.tol * (1 + 1e-6)


@pytest.mark.parametrize("nx,ny,nz", SHAPES)
def test_apply_and_operator_with_host_arrays(nx, ny, nz):
    import torch
    c = inputs.strut_case(nx, ny, nz, seed=4)
    g = c.grid
    x = np.random.default_rng(5).standard_normal(g.shape)
    with capi.Poisson(nx, ny, nz, g.h, precision="fp64") as sv:
        sv.set_density(c.F)
        y_d = torch.empty(g.shape, dtype=torch.float64, device="cuda")
        sv.apply(_dev(x), y_d)
        z_d = torch.empty_like(y_d)
        sv.precond_apply(_dev(x), z_d)
        ops_d = [torch.empty_like(y_d) for _ in range(4)]
        sv.get_operator(*ops_d)
        for name, xh in _host_kinds(x):
            off = 1 if name == "pinned+8" else 0
            out = (lambda: _pinned(np.zeros(g.shape), off)) if name != "pageable" else \
                (lambda: np.zeros(g.shape))
            y, z = out(), out()
            sv.apply(xh, y)
            sv.precond_apply(xh, z)
            ops = [out() for _ in range(4)]
            sv.get_operator(*ops)
            assert np.array_equal(_np(y), y_d.cpu().numpy()), name
            assert np.array_equal(_np(z), z_d.cpu().numpy()), name
            for a, b in zip(ops, ops_d):
                assert np.array_equal(_np(a), b.cpu().numpy()), name
    # the FP64 operator's faces are the oracle's bit for bit; its product, up to rounding order
    op = oracle.operator(c.F)
    for got, ref in zip(ops_d, (op.bx, op.by, op.bz, op.diag)):
        assert np.array_equal(got.cpu().numpy(), ref)
    bound = 1e-13 * op.diag * np.abs(x).max()
    assert np.all(np.abs(y_d.cpu().numpy() - oracle.apply(op, x)) <= bound)


@pytest.mark.parametrize("nx,ny,nz", SHAPES)
def test_projection_passes_with_pinned_arrays(nx, ny, nz):
    shape = (nz, ny, nx)
    rng = np.random.default_rng(6)
    u, v, w = (rng.standard_normal((nz, ny, nx + 1)), rng.standard_normal((nz, ny + 1, nx)),
               rng.standard_normal((nz + 1, ny, nx)))
    F = rng.random(shape)
    p = rng.standard_normal(shape)
    h, dt = 1.0 / nz, 1.3e-3
    op = oracle.operator(F)
    ref_s = oracle.divergence(u, v, w, h, dt)
    ru, rv, rw = oracle.project(op, F, u, v, w, p, h, dt)
    for off in (0, 1):
        with capi.Poisson(nx, ny, nz, h) as sv:
            sv.set_density(_pinned(F, off))
            s = _pinned(np.zeros(shape), off)
            sv.divergence(_pinned(u, off), _pinned(v, off), _pinned(w, off), dt, s)
            assert np.array_equal(_np(s), ref_s)
            gu, gv, gw = _pinned(u, off), _pinned(v, off), _pinned(w, off)
            sv.project(gu, gv, gw, _pinned(p, off), dt)
            assert np.array_equal(_np(gu), ru)
            assert np.array_equal(_np(gv), rv)
            assert np.array_equal(_np(gw), rw)


def test_batch_with_pinned_arrays_matches_device_arrays():
    import torch
    nx, ny, nz = SHAPES[0]
    cases = [inputs.strut_case(nx, ny, nz, seed=10 + q) for q in range(3)]
    g = cases[0].grid
    solvers = [capi.Poisson(nx, ny, nz, g.h, precision="fp32") for _ in cases]
    try:
        for sv, c in zip(solvers, cases):
            sv.set_density(_dev(c.F))

        def run(rhs, ps):
            tickets = capi.batch_submit(solvers, rhs, ps, 1e-9)
            out = []
            for t in tickets:
                while True:
                    rc, _ = capi.poll(t)
                    if rc != capi.PENDING:
                        break
                out.append(rc)
            return out

        p_d = [torch.zeros(g.shape, dtype=torch.float64, device="cuda") for _ in cases]
        assert run([_dev(c.s) for c in cases], p_d) == [capi.OK] * 3
        for off in (0, 1):
            p_h = [_pinned(np.zeros(g.shape), off) for _ in cases]
            assert run([_pinned(c.s, off) for c in cases], p_h) == [capi.OK] * 3
            for a, b in zip(p_h, p_d):
                assert np.array_equal(_np(a), b.cpu().numpy())
        for c, p in zip(cases, p_d):
            op = oracle.operator(c.F)
            assert oracle.rel_residual(op, oracle.rhs(c.s, g.h), p.cpu().numpy()) <= 1e-9 * (1 + 1e-6)
    finally:
        for sv in solvers:
            sv.close()

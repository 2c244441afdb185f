"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Element by element on seeded inputs that span several tiles and ragged tails: the FP64 operator
(face coefficients bit for bit, the stencil apply to FP64 rounding), the reduced-precision inner
operators (FP32 and BF16 densities, FP32 arithmetic), the Jacobi preconditioner, and full solves
in every precision mode against both acceptance criteria: relative residual <= tol under the
oracle's FP64 operator, and relative L2 distance <= 1e-6 from the oracle's 1e-12 solution.
"""
import numpy as np
import pytest

import oracle
from paper_1410_1942_gb300 import build, capi, inputs

pytestmark = pytest.mark.gpu

L2_TOL = 1e-6          # acceptance: relative L2 distance from the oracle solution
REF_TOL = 1e-12        # the oracle's reference solve
# reduced-precision operator apply, relative to diag_c * max|x|: FP32 densities and arithmetic
# (rounding of rho/2 to 24 bits, one approximate reciprocal per face, 7-term sums) stay within a
# few 1e-7; BF16 densities carry 2^-9 relative error per cell, 2^-8 per face.
APPLY_TOL = {"fp64": 1e-14, "fp32": 2e-6, "bf16": 1.6e-2}


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    build.build()
    capi.load()


CASES = {
    "flat32": lambda: inputs.flat_case(32, 32, 32, seed=0, tol=1e-10),
    "ragged": lambda: inputs.flat_case(37, 23, 19, seed=2, tol=1e-10),
    "strut": lambda: inputs.strut_case(96, 48, 40, seed=1),
    "column": lambda: inputs.flat_case(3, 5, 70, seed=4, tol=1e-10),
}
_cache = {}


def case(name):
    if name not in _cache:
        c = CASES[name]()
        op = oracle.operator(c.F)
        b = oracle.rhs(c.s, c.grid.h)
        ref = oracle.pcg(op, b, tol=REF_TOL, precond="ssor")
        assert ref.status == oracle.OK
        _cache[name] = (c, op, b, ref.x)
    return _cache[name]


def solver(c, precision="fp32", **kw):
    g = c.grid
    s = capi.Poisson(g.nx, g.ny, g.nz, g.h, precision=precision, **kw)
    s.set_density(c.F)
    return s


@pytest.mark.parametrize("name", list(CASES))
def test_fp64_operator_bit_exact(name):
    c, op, _, _ = case(name)
    with solver(c, "fp64") as s:
        arrs = [np.empty(c.grid.shape) for _ in range(4)]
        s.get_operator(*arrs)
    for got, ref in zip(arrs, (op.bx, op.by, op.bz, op.diag)):
        assert np.array_equal(got, ref)


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("prec", ["fp64", "fp32", "bf16"])
def test_operator_apply(name, prec):
    c, op, _, _ = case(name)
    x = np.random.default_rng(7).standard_normal(c.grid.shape)
    with solver(c, "fp64" if prec == "fp64" else "fp32") as s:
        y = np.empty_like(x)
        s.apply(x, y, prec)
    ref = oracle.apply(op, x)
    bound = APPLY_TOL[prec] * op.diag * np.abs(x).max()
    assert np.all(np.abs(y - ref) <= bound)


@pytest.mark.parametrize("name", ["flat32", "ragged"])
@pytest.mark.parametrize("prec", ["fp64", "fp32", "bf16"])
def test_jacobi_apply(name, prec):
    c, op, _, _ = case(name)
    r = np.random.default_rng(8).standard_normal(c.grid.shape)
    with solver(c) as s:
        z = np.empty_like(r)
        s.precond_apply(r, z, "jacobi", prec)
    ref = oracle.precond(op, r, "jacobi")
    np.testing.assert_allclose(z, ref, rtol=APPLY_TOL[prec], atol=0)


# SSOR sweeps accumulate up to 13 terms per cell in the precision's arithmetic; compared with the
# oracle's FP64 sweep relative to max|z|.
SSOR_TOL = {"fp64": 1e-13, "fp32": 1e-5, "bf16": 3e-2}


@pytest.mark.parametrize("name", ["flat32", "ragged", "column"])
@pytest.mark.parametrize("prec", ["fp64", "fp32", "bf16"])
@pytest.mark.parametrize("omega", [1.0, 1.3])
def test_rbssor_apply(name, prec, omega):
    """z = M^-1 r for the red-black SSOR preconditioner, against the oracle's sweep (itself
    pinned to the literal dense splitting)."""
    c, op, _, _ = case(name)
    r = np.random.default_rng(10).standard_normal(c.grid.shape)
    with solver(c, "fp64" if prec == "fp64" else "fp32", precond="rbssor", omega=omega) as s:
        z = np.empty_like(r)
        s.precond_apply(r, z, "rbssor", prec)
    ref = oracle.precond(op, r, "ssor", omega)
    assert np.max(np.abs(z - ref)) <= SSOR_TOL[prec] * np.abs(ref).max()


def _check_solution(c, op, b, xref, p, stats, tol):
    rel = oracle.rel_residual(op, b, p)
    assert rel <= tol * (1 + 1e-6), rel
    err = np.linalg.norm(p - xref) / np.linalg.norm(xref)
    assert err <= L2_TOL, err
    # the library's own FP64 residual agrees with the oracle's evaluation
    assert abs(stats["rel_residual"] - rel) <= 1e-3 * rel + 1e-15


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("prec", ["fp64", "fp32", "bf16"])
@pytest.mark.parametrize("precond", ["jacobi", "rbssor"])
def test_solve_matches_oracle(name, prec, precond):
    c, op, b, xref = case(name)
    with solver(c, prec, precond=precond) as s:
        p = np.zeros(c.grid.shape)
        rc, st = s.solve(c.s, p, c.tol)
    assert rc == capi.OK
    _check_solution(c, op, b, xref, p, st, c.tol)
    if prec != "fp64":
        assert st["outer_iters"] >= 2


@pytest.mark.parametrize("tile", [-1, 0, 1108, 2204, 2208, 12204, 12208, 302204, 302208,
                                  312208, 602204, 612208, 1012204, 2002204, 2012208, 2302204,
                                  10012204, 12012204, 10312204, 10312208, 12312208, 20012204,
                                  22012204, 20512204, 20012208, 22012208])
@pytest.mark.parametrize("prec", ["fp32", "bf16"])
@pytest.mark.parametrize("shape", [(96, 48, 40), (40, 23, 19), (64, 16, 1), (8, 9, 33)])
def test_kernel_variants_match_oracle(tile, prec, shape):
    """Every inner-solve kernel family and tile height, on shapes with ragged x and y tiles,
    a single plane and a thin column, against both acceptance criteria."""
    c = inputs.flat_case(*shape, seed=9, tol=1e-10)
    op = oracle.operator(c.F)
    b = oracle.rhs(c.s, c.grid.h)
    xref = oracle.pcg(op, b, tol=REF_TOL, precond="ssor").x
    with solver(c, prec, tile=tile) as s:
        p = np.zeros(c.grid.shape)
        rc, st = s.solve(c.s, p, c.tol)
    assert rc == capi.OK
    _check_solution(c, op, b, xref, p, st, c.tol)


def test_rbssor_needs_fewer_iterations_than_jacobi():
    c, op, b, xref = case("strut")
    its = {}
    for pc in ("jacobi", "rbssor"):
        with solver(c, "fp64", precond=pc) as s:
            p = np.zeros(c.grid.shape)
            rc, st = s.solve(c.s, p, 1e-9)
        assert rc == capi.OK
        its[pc] = st["inner_iters"]
    assert its["rbssor"] < 0.75 * its["jacobi"], its


def test_device_and_host_arrays_give_identical_results():
    import torch
    c, _, _, _ = case("ragged")
    with solver(c, "fp32") as s:
        ph = np.zeros(c.grid.shape)
        s.solve(c.s, ph, c.tol)
        rhs_d = torch.from_numpy(c.s).cuda()
        pd = torch.zeros(c.grid.shape, dtype=torch.float64, device="cuda")
        s.solve(rhs_d, pd, c.tol)
        torch.cuda.synchronize()
    assert np.array_equal(ph, pd.cpu().numpy())


def test_density_from_device_memory_matches_host():
    import torch
    c, op, _, _ = case("strut")
    g = c.grid
    with capi.Poisson(g.nx, g.ny, g.nz, g.h, precision="fp64") as s:
        s.set_density(torch.from_numpy(c.F).cuda())
        bx = np.empty(g.shape)
        s.get_operator(bx=bx)
    assert np.array_equal(bx, op.bx)


def test_zero_source_returns_zero_pressure():
    c, _, _, _ = case("flat32")
    with solver(c) as s:
        p = np.ones(c.grid.shape)
        rc, st = s.solve(np.zeros(c.grid.shape), p, 1e-9)
    assert rc == capi.OK and not p.any() and st["inner_iters"] == 0


def test_warm_start_from_solution_takes_no_iterations():
    c, op, b, xref = case("flat32")
    with solver(c) as s:
        p = xref.copy()
        rc, st = s.solve(c.s, p, 1e-9)
    assert rc == capi.OK and st["inner_iters"] == 0 and st["outer_iters"] == 1
    assert np.array_equal(p, xref)


def test_warm_start_takes_fewer_iterations():
    c, op, b, xref = case("strut")
    with solver(c) as s:
        p0 = np.zeros(c.grid.shape)
        _, cold = s.solve(c.s, p0, 1e-9)
        p1 = xref * (1 + 1e-4)
        _, warm = s.solve(c.s, p1, 1e-9)
    assert warm["inner_iters"] < cold["inner_iters"]
    _check_solution(c, op, b, xref, p1, warm, 1e-9)


def test_error_codes():
    c, _, _, _ = case("flat32")
    g = c.grid
    with capi.Poisson(g.nx, g.ny, g.nz, g.h) as s:
        p = np.zeros(g.shape)
        rc, _ = s.solve(c.s, p, 1e-9, allow=(capi.ENOTREADY,))
        assert rc == capi.ENOTREADY
        s.set_density(c.F)
        with pytest.raises(capi.PoissonError) as e:
            s.solve(c.s, p, 0.0)
        assert e.value.status == capi.EINVAL
        with pytest.raises(capi.PoissonError):
            s.set_density(c.F, rho_air=-1.0)


def test_iteration_cap_reports_notconv_with_best_iterate():
    c, op, b, _ = case("strut")
    with solver(c, "fp32", max_iters=20) as s:
        p = np.zeros(c.grid.shape)
        rc, st = s.solve(c.s, p, 1e-9, allow=(capi.ENOTCONV,))
    assert rc == capi.ENOTCONV
    assert st["inner_iters"] <= 20 + 8
    rel = oracle.rel_residual(op, b, p)
    assert rel < 1.0 and abs(st["rel_residual"] - rel) <= 1e-3 * rel


def _poll_all(tickets):
    out = {}
    pending = list(tickets)
    while pending:
        nxt = []
        for t in pending:
            rc, st = capi.poll(t)
            if rc == capi.PENDING:
                nxt.append(t)
            else:
                out[t] = (rc, st)
        pending = nxt
    return out


def _oracle_ref(c):
    op = oracle.operator(c.F)
    b = oracle.rhs(c.s, c.grid.h)
    return op, b, oracle.pcg(op, b, tol=REF_TOL, precond="ssor").x


@pytest.mark.parametrize("tile", [0, 2012204, 10012204, 12012204, 22012204, 13012204])
def test_batch_of_uneven_solves_matches_oracle(tile):
    """A batch of solves of uneven size, FP32 and BF16 coefficients, plus handles that run one
    by one (FP64, SSOR): every result meets both acceptance criteria, with the persistent
    kernel of either family and split."""
    cases = inputs.batch_cases(12, seed=3, hi=(96, 64, 48))
    precs = ["fp32"] * 8 + ["bf16"] * 2 + ["fp64", "fp32"]
    pcs = ["jacobi"] * 11 + ["rbssor"]
    solvers = [solver(c, pr, precond=pc, tile=tile if pr != "fp64" else 0)
               for c, pr, pc in zip(cases, precs, pcs)]
    ps = [np.zeros(c.grid.shape) for c in cases]
    tickets = capi.batch_submit(solvers, [c.s for c in cases], ps, 1e-9)
    res = _poll_all(tickets)
    for t, c, p in zip(tickets, cases, ps):
        rc, st = res[t]
        assert rc == capi.OK
        op, b, xref = _oracle_ref(c)
        _check_solution(c, op, b, xref, p, st, 1e-9)
    assert capi.poll(tickets[0])[0] == capi.ENOTICKET
    for s in solvers:
        s.close()


def test_batch_runs_multigrid_and_fp64_solves_on_workers():
    """Handles whose solves use only ordinary launches (multigrid in every precision, FP64) run
    on the executor's worker threads, several at once on their own streams, beside a Jacobi
    handle in the persistent batch: polls never block on them, and every result meets both
    acceptance criteria against the oracle."""
    cases = inputs.batch_cases(10, seed=5, hi=(96, 64, 48))
    kinds = ([("fp32", "mg")] * 5 + [("bf16", "mg")] * 2 + [("fp64", "mg"), ("fp64", "jacobi"),
                                                            ("fp32", "jacobi")])
    solvers = [solver(c, pr, precond=pc) for c, (pr, pc) in zip(cases, kinds)]
    ps = [np.zeros(c.grid.shape) for c in cases]
    tickets = capi.batch_submit(solvers, [c.s for c in cases], ps, 1e-9)
    res = _poll_all(tickets)
    for t, c, p in zip(tickets, cases, ps):
        rc, st = res[t]
        assert rc == capi.OK
        op, b, xref = _oracle_ref(c)
        _check_solution(c, op, b, xref, p, st, 1e-9)
    for s in solvers:
        s.close()


def test_a_handle_in_an_unreported_job_cannot_be_destroyed():
    """While a batch job uses a handle -- in the persistent batch, or on a worker thread -- its
    destruction is refused (EINVAL) and the job completes; after poll reports it, destroy
    succeeds."""
    cases = inputs.batch_cases(2, seed=7, hi=(96, 64, 48))
    svs = [solver(cases[0]), solver(cases[1], precond="mg")]
    ps = [np.zeros(c.grid.shape) for c in cases]
    tickets = capi.batch_submit(svs, [c.s for c in cases], ps, 1e-9)
    for s in svs:
        with pytest.raises(capi.PoissonError) as e:
            s.close()
        assert e.value.status == capi.EINVAL
    res = _poll_all(tickets)
    for t, c, p in zip(tickets, cases, ps):
        rc, st = res[t]
        assert rc == capi.OK
        op, b, xref = _oracle_ref(c)
        _check_solution(c, op, b, xref, p, st, 1e-9)
    for s in svs:
        s.close()


def test_batch_of_64_uneven_solves_matches_oracle():
    """The batched workload at its full specification: 64 solves of sizes drawn between 32^3
    and 128 x 64 x 64 (aspect <= 4), each with its own surface, strut and source, submitted
    together (one persistent launch per refinement step over every unfinished solve); every
    result meets both acceptance criteria against the oracle."""
    cases = inputs.batch_cases(64, seed=0)
    assert max(c.grid.n for c in cases) <= 128 * 64 * 64
    solvers = [solver(c) for c in cases]
    ps = [np.zeros(c.grid.shape) for c in cases]
    tickets = capi.batch_submit(solvers, [c.s for c in cases], ps, 1e-9)
    res = _poll_all(tickets)
    for t, c, p in zip(tickets, cases, ps):
        rc, st = res[t]
        assert rc == capi.OK
        op, b, xref = _oracle_ref(c)
        _check_solution(c, op, b, xref, p, st, 1e-9)
    for s in solvers:
        s.close()


def test_solve_alone_and_in_the_mix_agree():
    """The same solve run alone and inside a batch of others gives the same pressure within the
    acceptance tolerance (both meet it against the oracle)."""
    cases = inputs.batch_cases(6, seed=11, hi=(96, 64, 48))
    target = cases[2]
    alone = np.zeros(target.grid.shape)
    with solver(target) as s:
        t = capi.batch_submit([s], [target.s], [alone], 1e-9)
        rc, _ = _poll_all(t)[t[0]]
        assert rc == capi.OK
    solvers = [solver(c) for c in cases]
    ps = [np.zeros(c.grid.shape) for c in cases]
    tickets = capi.batch_submit(solvers, [c.s for c in cases], ps, 1e-9)
    res = _poll_all(tickets)
    assert all(r[0] == capi.OK for r in res.values())
    mixed = ps[2]
    assert np.linalg.norm(mixed - alone) / np.linalg.norm(alone) <= L2_TOL
    op, b, xref = _oracle_ref(target)
    assert oracle.rel_residual(op, b, mixed) <= 1e-9 * (1 + 1e-6)
    for s in solvers:
        s.close()


def test_solves_join_a_running_batch():
    """Solves submitted after a batch has started join it at its next refinement step."""
    cases = inputs.batch_cases(8, seed=21, hi=(80, 64, 48))
    solvers = [solver(c) for c in cases]
    ps = [np.zeros(c.grid.shape) for c in cases]
    first = capi.batch_submit(solvers[:4], [c.s for c in cases[:4]], ps[:4], 1e-9)
    for t in first[:1]:
        assert capi.poll(t)[0] == capi.PENDING  # one refinement step of the first four
    second = capi.batch_submit(solvers[4:], [c.s for c in cases[4:]], ps[4:], 1e-9)
    res = _poll_all(first + second)
    for t, c, p in zip(first + second, cases, ps):
        rc, st = res[t]
        assert rc == capi.OK
        op, b, xref = _oracle_ref(c)
        _check_solution(c, op, b, xref, p, st, 1e-9)
    for s in solvers:
        s.close()


def test_batch_rejects_a_handle_twice():
    c = inputs.flat_case(32, 32, 32, seed=1)
    with solver(c) as s:
        p = np.zeros(c.grid.shape)
        with pytest.raises(capi.PoissonError):
            capi.batch_submit([s, s], [c.s, c.s], [p, p.copy()], 1e-9)


@pytest.mark.parametrize("tile", [2002204, 2012208, 12012204, 22012204, 3012204, 13012204,
                                  13312208])
def test_lockstep_round_robin_split(tile):
    """More tile columns than CTAs (1024 x 512 planes): the lockstep split deals whole columns
    round-robin.  Checked by the oracle's FP64 residual (a property at any size) and against the
    equal split's solution."""
    c = inputs.flat_case(1024, 512, 6, seed=3, tol=1e-9)
    op = oracle.operator(c.F)
    b = oracle.rhs(c.s, c.grid.h)
    sols = []
    for t in (tile, tile % 1000000):
        with solver(c, "fp32", tile=t) as s:
            assert ("split=lockstep" in s.describe()) == (t == tile)
            p = np.zeros(c.grid.shape)
            rc, st = s.solve(c.s, p, c.tol)
        assert rc == capi.OK
        rel = oracle.rel_residual(op, b, p)
        assert rel <= c.tol * (1 + 1e-6), rel
        sols.append(p)
    assert np.linalg.norm(sols[0] - sols[1]) <= 2e-6 * np.linalg.norm(sols[1])


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_one_sweep_kernel_takes_the_iterations_of_standard_pcg(prec):
    """The one-sweep kernels run the Chronopoulos-Gear recurrences, which have the iterates of
    standard PCG: the inner iteration count stays within a few percent of the two-sweep
    kernel's."""
    c, op, b, xref = case("strut")
    its = {}
    for t in (12204, 10012204, 20012204):
        with solver(c, prec, tile=t) as s:
            p = np.zeros(c.grid.shape)
            rc, st = s.solve(c.s, p, c.tol)
        assert rc == capi.OK
        _check_solution(c, op, b, xref, p, st, c.tol)
        its[t] = st["inner_iters"]
    assert abs(its[10012204] - its[12204]) <= 0.1 * its[12204] + 5, its
    assert abs(its[20012204] - its[12204]) <= 0.1 * its[12204] + 5, its


@pytest.mark.parametrize("tile", [12204, 10012204, 20012204])
@pytest.mark.parametrize("k", [7, 8])
def test_capped_solve_returns_the_k_th_iterate(tile, k):
    """With the iteration cap at k, the FP32 inner solve stops after k CG iterations and p holds
    the k-th iterate: the k-th iterate of the oracle's textbook Jacobi PCG (FP64) to FP32
    accuracy, whichever arrangement of CG the kernel runs (the two-sweep kernels take the
    textbook form; the one-sweep kernels the Chronopoulos-Gear recurrences, the same iterates in
    exact arithmetic).  An odd k ends the one-sweep kernel on an iteration that leaves x to a
    closing pass (x is stored every other iteration), an even k on one that stores it."""
    c, op, b, _ = case("strut")
    with solver(c, "fp32", tile=tile, max_iters=k) as s:
        p = np.zeros(c.grid.shape)
        rc, st = s.solve(c.s, p, 1e-9, allow=(capi.OK, capi.ENOTCONV))
    assert rc == capi.ENOTCONV and st["inner_iters"] == k
    ref = oracle.pcg(op, b, tol=0.0, precond="jacobi", max_iters=k).x
    assert np.linalg.norm(p - ref) <= 1e-4 * np.linalg.norm(ref)


# ----------------------------------------------------------------------------- wall variants
WALL_CASES = [1 | 2, 4 | 8 | 16, 31]


@pytest.mark.parametrize("walls", WALL_CASES)
def test_dirichlet_walls_operator_bit_exact(walls):
    c = inputs.flat_case(37, 23, 19, seed=2, tol=1e-10)
    op = oracle.operator(c.F, walls=walls)
    with solver(c, "fp64", dirichlet_walls=walls) as s:
        arrs = [np.empty(c.grid.shape) for _ in range(4)]
        s.get_operator(*arrs)
        x = np.random.default_rng(3).standard_normal(c.grid.shape)
        y = np.empty_like(x)
        s.apply(x, y, "fp64")
    for got, ref in zip(arrs, (op.bx, op.by, op.bz, op.diag)):
        assert np.array_equal(got, ref)
    assert np.all(np.abs(y - oracle.apply(op, x)) <= APPLY_TOL["fp64"] * op.diag * np.abs(x).max())


@pytest.mark.parametrize("walls", WALL_CASES)
@pytest.mark.parametrize("prec,tile,precond", [("fp64", 0, "jacobi"), ("fp64", 0, "rbssor"),
                                               ("fp32", -1, "jacobi"), ("fp32", 0, "rbssor"),
                                               ("fp32", 2204, "jacobi"), ("fp32", 12204, "jacobi"),
                                               ("fp32", 12012204, "jacobi"),
                                               ("fp32", 22012204, "jacobi"),
                                               ("bf16", 12312208, "jacobi")])
def test_dirichlet_walls_solve_matches_oracle(walls, prec, tile, precond):
    """Side/bottom walls with p = 0 through every kernel family, against both criteria with the
    oracle's operator for the same walls."""
    c = inputs.flat_case(64, 40, 24, seed=5, tol=1e-9)
    op = oracle.operator(c.F, walls=walls)
    b = oracle.rhs(c.s, c.grid.h)
    xref = oracle.pcg(op, b, tol=REF_TOL, precond="ssor").x
    with solver(c, prec, tile=tile, precond=precond, dirichlet_walls=walls) as s:
        p = np.zeros(c.grid.shape)
        rc, st = s.solve(c.s, p, c.tol)
    assert rc == capi.OK
    _check_solution(c, op, b, xref, p, st, c.tol)


PERIODIC_CASES = [0, capi.WALL_YM | capi.WALL_ZM]


@pytest.mark.parametrize("walls", PERIODIC_CASES)
def test_periodic_x_operator_bit_exact(walls):
    c = inputs.flat_case(36, 23, 19, seed=4, tol=1e-10)
    op = oracle.operator(c.F, walls=walls | oracle.PERIODIC_X)
    with solver(c, "fp64", dirichlet_walls=walls, periodic_x=True) as s:
        arrs = [np.empty(c.grid.shape) for _ in range(4)]
        s.get_operator(*arrs)
        x = np.random.default_rng(5).standard_normal(c.grid.shape)
        y = np.empty_like(x)
        s.apply(x, y, "fp64")
        assert "columns" in s.describe()
    for got, ref in zip(arrs, (op.bx, op.by, op.bz, op.diag)):
        assert np.array_equal(got, ref)
    assert np.all(np.abs(y - oracle.apply(op, x)) <= APPLY_TOL["fp64"] * op.diag * np.abs(x).max())


@pytest.mark.parametrize("walls", PERIODIC_CASES)
@pytest.mark.parametrize("prec,precond", [("fp64", "jacobi"), ("fp64", "rbssor"), ("fp32", "jacobi"),
                                          ("fp32", "rbssor"), ("bf16", "jacobi")])
def test_periodic_x_solve_matches_oracle(walls, prec, precond):
    c = inputs.flat_case(48, 24, 20, seed=6, tol=1e-9)
    op = oracle.operator(c.F, walls=walls | oracle.PERIODIC_X)
    b = oracle.rhs(c.s, c.grid.h)
    xref = oracle.pcg(op, b, tol=REF_TOL, precond="ssor").x
    with solver(c, prec, precond=precond, dirichlet_walls=walls, periodic_x=True) as s:
        p = np.zeros(c.grid.shape)
        rc, st = s.solve(c.s, p, c.tol)
    assert rc == capi.OK
    _check_solution(c, op, b, xref, p, st, c.tol)


@pytest.mark.parametrize("walls", PERIODIC_CASES)
@pytest.mark.parametrize("prec,tile", [("fp32", 0), ("fp32", 10012204), ("fp32", 12012204),
                                       ("bf16", 10312208), ("fp32", -1), ("fp32", 12204)])
@pytest.mark.parametrize("shape", [(48, 24, 20), (96, 40, 18), (8, 9, 12), (128, 20, 9)])
def test_periodic_x_marching_matches_oracle(walls, prec, tile, shape):
    """Periodic x on the one-sweep marching kernels (rows padded with wrapped ghost columns; the
    tuner and forced one-sweep tiles) and on the column kernels (tile -1, or a two-sweep tile,
    which cannot wrap), on shapes with one tile, a ragged last tile, nx = 8, and two 64-cell
    tiles (the column path's phase A on the 2x2-cell kernel, its halo columns wrapped)."""
    c = inputs.flat_case(*shape, seed=7, tol=1e-9)
    op = oracle.operator(c.F, walls=walls | oracle.PERIODIC_X)
    b = oracle.rhs(c.s, c.grid.h)
    xref = oracle.pcg(op, b, tol=REF_TOL, precond="ssor").x
    with solver(c, prec, tile=tile, dirichlet_walls=walls, periodic_x=True) as s:
        p = np.zeros(c.grid.shape)
        rc, st = s.solve(c.s, p, c.tol)
        desc = s.describe()
    assert rc == capi.OK
    assert ("one-sweep" in desc) == (tile not in (-1, 12204)), desc
    _check_solution(c, op, b, xref, p, st, c.tol)


def test_periodic_x_rejects_x_walls_and_odd_ssor():
    for kw in ({"dirichlet_walls": capi.WALL_XM}, {"precond": "rbssor"}):
        with pytest.raises(capi.PoissonError) as e:
            capi.Poisson(15, 16, 16, 1.0 / 16, periodic_x=True, **kw)
        assert e.value.status == capi.EINVAL


def test_dirichlet_walls_rejects_unknown_bits():
    with pytest.raises(capi.PoissonError) as e:
        capi.Poisson(16, 16, 16, 1.0 / 16, dirichlet_walls=32)
    assert e.value.status == capi.EINVAL


# ----------------------------------------------------------------------------- full size
@pytest.fixture(scope="module")
def strut_full():
    c = inputs.strut_case(256, 128, 128, seed=0)
    op = oracle.operator(c.F)
    b = oracle.rhs(c.s, c.grid.h)
    ref = oracle.pcg(op, b, tol=REF_TOL, precond="ssor")
    assert ref.status == oracle.OK
    return c, op, b, ref.x


@pytest.mark.parametrize("prec,precond", [("fp32", "jacobi"), ("fp64", "jacobi"),
                                          ("bf16", "jacobi"), ("fp32", "rbssor"),
                                          ("fp64", "rbssor"), ("fp32", "mg"), ("fp64", "mg"),
                                          ("bf16", "mg")])
def test_full_size_strut_solve(strut_full, prec, precond):
    """The 256 x 128 x 128 strut workload at 1e-9, as the benchmark runs it."""
    c, op, b, xref = strut_full
    with solver(c, prec, precond=precond) as s:
        p = np.zeros(c.grid.shape)
        rc, st = s.solve(c.s, p, c.tol)
    assert rc == capi.OK
    _check_solution(c, op, b, xref, p, st, c.tol)

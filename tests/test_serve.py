"""The served request loop: continuous batching, admission by device-memory budget, warm starts,
and the same result alone and in the mix."""
import copy
import math

import numpy as np
import pytest

from paper_1410_1942_gb300 import build, capi, inputs, serve

pytestmark = pytest.mark.gpu

L2_TOL = 1e-6


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    assert torch.cuda.is_available()
    build.build()
    capi.load()
    inputs.mixed_fields_t((32, 32, 32), 1, device="cuda")  # first-use compilation outside tests


def _stream(n, rate, seed, hi=(96, 64, 64)):
    return serve.request_stream(n, rate, seed=seed, hi=hi)


def test_stream_of_requests_all_converge():
    reqs = _stream(6, math.inf, seed=1)
    st = serve.Server(budget_bytes=8 << 30, steps=4).serve(reqs)
    assert st["all_ok"] and st["solves"] == 24
    assert st["max_rel_residual"] <= 1e-9 * (1 + 1e-6)
    # warm starts: later steps of a request need fewer CG iterations than its first
    for r in reqs:
        assert min(r.iters[1:]) < r.iters[0]


def test_admission_respects_the_memory_budget():
    reqs = _stream(5, math.inf, seed=2)
    need = max(serve.request_bytes(r.shape, "fp32") for r in reqs)
    st = serve.Server(budget_bytes=2 * need, steps=2).serve(reqs)
    assert st["all_ok"]
    assert st["peak_used_bytes"] <= 2 * need
    assert st["peak_active"] < len(reqs)  # some requests waited for memory


@pytest.mark.parametrize("kw", [{}, {"precision": "bf16"}, {"precision": "fp64"},
                                {"precond": "mg"}, {"precond": "rbssor"},
                                {"periodic_x": True}, {"dirichlet_walls": 31},
                                {"tile": serve.SERVE_TILE}])
def test_library_budget_matches_the_handle(kw):
    """poisson_required_bytes bounds what a created handle holds (its plan is counted at an
    upper bound, at most a few MiB over) and refuses a budget it exceeds."""
    for shape in ((96, 48, 40), (64, 32, 32), (40, 23, 19)):
        rc, need = capi.required_bytes(*shape, **kw)
        assert rc == capi.OK
        with capi.Poisson(*shape, 1.0 / shape[2], **kw) as s:
            have = s.device_bytes()
        assert have <= need <= have + (4 << 20), (shape, kw, need, have)
        rc, _ = capi.required_bytes(*shape, budget=need - 1, **kw)
        assert rc == capi.ENOMEM_BUDGET
        rc, _ = capi.required_bytes(*shape, budget=need, **kw)
        assert rc == capi.OK


def test_every_served_solve_matches_the_oracle():
    """Continuous batching with requests overlapping on the device: the result of every step of
    every request (its own density, its drifted source, warm-started from the previous step's
    pressure) meets both acceptance criteria against the oracle -- relative residual <= 1e-9
    under the oracle's FP64 operator and relative L2 <= 1e-6 from the oracle's 1e-12 solve of
    that step's system."""
    import oracle
    reqs = _stream(4, math.inf, seed=6, hi=(64, 48, 48))
    srv = serve.Server(budget_bytes=8 << 30, steps=3, record_steps=True)
    st = srv.serve(reqs)
    assert st["all_ok"] and st["solves"] == 12 and st["peak_active"] >= 2
    for r in reqs:
        rec = srv.record[r.rid]
        g = rec["grid"]
        op = oracle.operator(rec["F"])
        assert len(rec["steps"]) == 3
        prev = None
        for s, p, rc in rec["steps"]:
            assert rc == capi.OK
            if prev is not None:
                assert np.linalg.norm(s - prev) > 0  # the source drifts between steps
            prev = s
            b = oracle.rhs(s, g.h)
            rel = oracle.rel_residual(op, b, p)
            assert rel <= 1e-9 * (1 + 1e-6), (r.rid, rel)
            ref = oracle.pcg(op, b, tol=1e-12, precond="ssor").x
            err = np.linalg.norm(p - ref) / np.linalg.norm(ref)
            assert err <= L2_TOL, (r.rid, err)


def test_result_alone_equals_result_in_the_mix():
    mix = _stream(6, 200.0, seed=3)
    target = copy.deepcopy(mix[2])
    target.arrival = 0.0
    alone = serve.Server(budget_bytes=8 << 30, steps=5, keep_results=True)
    alone.serve([target])
    mixed = serve.Server(budget_bytes=8 << 30, steps=5, keep_results=True)
    st = mixed.serve(mix)
    assert st["all_ok"] and st["peak_active"] >= 2
    a, m = alone.results[target.rid], mixed.results[mix[2].rid]
    assert np.linalg.norm(a - m) / np.linalg.norm(a) <= L2_TOL


def test_stream_with_the_multigrid_preconditioner():
    """MG handles are not batched (the executor solves them one by one at poll): every step
    converges, warm starts still pay, and a request's result equals the Jacobi stream's to the
    solves' accuracy."""
    reqs = _stream(4, math.inf, seed=4)
    jac = serve.Server(budget_bytes=8 << 30, steps=3, keep_results=True)
    jac.serve(copy.deepcopy(reqs))
    srv = serve.Server(budget_bytes=8 << 30, steps=3, keep_results=True, precond="mg")
    st = srv.serve(reqs)
    assert st["all_ok"] and st["solves"] == 12
    assert st["max_rel_residual"] <= 1e-9 * (1 + 1e-6)
    for r in reqs:
        assert max(r.iters) <= 60
        a, m = jac.results[r.rid], srv.results[r.rid]
        assert np.linalg.norm(a - m) / np.linalg.norm(a) <= 2 * L2_TOL


def test_cancelled_requests_leave_and_free_their_memory(tmp_path):
    """A request cancelled after k steps stops there (its step in flight finished, handle and
    memory given back); one cancelled before arrival is never admitted; the others run all
    their steps.  The JSON-lines log holds one line per finished solve."""
    reqs = _stream(5, math.inf, seed=6)
    reqs[1].cancel_after = 1
    reqs[3].cancel_after = 2
    srv = serve.Server(budget_bytes=8 << 30, steps=4, log=str(tmp_path / "solves.jsonl"))
    srv.cancel(reqs[4])
    st = srv.serve(reqs)
    assert st["all_ok"] and st["cancelled"] == 3
    assert st["used_bytes_at_end"] == 0
    assert [len(r.statuses) for r in reqs] == [4, 1, 4, 2, 0]
    assert st["solves"] == 11
    import json
    lines = [json.loads(x) for x in (tmp_path / "solves.jsonl").read_text().splitlines()]
    assert len(lines) == 11
    assert all(x["status"] == "ok" and x["rel_residual"] <= 1e-9 * (1 + 1e-6) for x in lines)
    for r in reqs:
        mine = [x for x in lines if x["rid"] == r.rid]
        assert [x["step"] for x in mine] == list(range(len(r.statuses)))
        assert all(x["shape"] == list(r.shape) and x["latency_ms"] > 0 for x in mine)


def test_checkpoint_and_resume_give_the_uninterrupted_results(tmp_path):
    """A stream stopped after some solves (steps in flight finish, unfinished requests parked
    with their next step's source and their pressure on the host), saved, loaded into a new
    server and run to the end runs every step exactly once, and each request's final pressure
    is the uninterrupted stream's within the acceptance tolerance."""
    reqs = _stream(5, math.inf, seed=8)
    whole = serve.Server(budget_bytes=8 << 30, steps=4, keep_results=True)
    st_whole = whole.serve(copy.deepcopy(reqs))
    assert st_whole["all_ok"] and st_whole["solves"] == 20
    first = serve.Server(budget_bytes=8 << 30, steps=4, keep_results=True)
    part = copy.deepcopy(reqs)
    st1 = first.serve(part, stop_after=7)
    assert st1["stopped"] and st1["all_ok"] and st1["used_bytes_at_end"] == 0
    assert 7 <= st1["solves"] < 20 and st1["parked"] >= 1
    path = str(tmp_path / "stream.npz")
    serve.Server.checkpoint(path, part)
    resumed = serve.Server.load_checkpoint(path)
    assert [r.step for r in resumed] == [r.step for r in part]
    second = serve.Server(budget_bytes=8 << 30, steps=4, keep_results=True)
    st2 = second.serve(resumed)
    assert st2["all_ok"] and not st2["stopped"]
    assert st1["solves"] + st2["solves"] == 20
    assert all(len(r.statuses) == 4 for r in resumed)
    for r in reqs:
        got = first.results.get(r.rid)
        if got is None:
            got = second.results[r.rid]
        want = whole.results[r.rid]
        assert np.linalg.norm(got - want) / np.linalg.norm(want) <= L2_TOL

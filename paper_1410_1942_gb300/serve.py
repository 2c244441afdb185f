"""Served pressure solves: a request stream over the batch executor (continuous batching).

A request is one grid of its own size, density field and source, solved for ``steps``
consecutive projection steps (the two-stage time integration of a ship-wave run solves the
pressure Poisson equation at every stage); between steps the source drifts (the velocity modes
are advected by the free stream for one ``dt``) and the previous pressure, kept on the device,
is the next step's initial guess.

The loop admits arriving requests first come first served while their device memory fits the
budget, submits each request's current step to the library's batch executor
(``poisson_batch_submit``), and polls: every poll of an unfinished solve runs one refinement step
of the whole batch, and a request whose step finished submits its next step at once, so
requests that arrive while others run join the batch at its next refinement step.  Reported:
solves/s, per-solve latency percentiles (from submission, or arrival for a request's first
step, to completion), the residual of every solve.
"""
from __future__ import annotations

import collections
import dataclasses
import json
import math
import time

import numpy as np

from . import capi, inputs

# the request's own arrays on the device: F, s, p (FP64)
REQUEST_BYTES_PER_CELL = 3 * 8
# kernel variant of served Jacobi handles: the one-sweep persistent kernel, 64x8 tiles, lockstep
# split (fixed, so admission does not run the autotuner)
SERVE_TILE = 12012204


def _handle_opts(precision, precond, tile):
    return {"precision": precision, "precond": precond,
            "tile": tile if (precision != "fp64" and precond == "jacobi") else 0}


def request_bytes(shape, precision, precond="jacobi", tile=SERVE_TILE):
    """Device bytes of one admitted request: the library's figure for its handle
    (poisson_required_bytes) plus its F, s and p arrays."""
    nx, ny, nz = shape
    _, b = capi.required_bytes(nx, ny, nz, **_handle_opts(precision, precond, tile))
    return b + REQUEST_BYTES_PER_CELL * nx * ny * nz


@dataclasses.dataclass
class Request:
    rid: int
    arrival: float        # seconds after the start of the run
    shape: tuple          # (nx, ny, nz)
    seed: int
    # runtime state
    step: int = 0
    solver: object = None
    grid: object = None
    modes: list = None
    F: object = None
    s: object = None
    p: object = None
    ticket: int = 0
    t_submit: float = 0.0
    latencies: list = dataclasses.field(default_factory=list)
    residuals: list = dataclasses.field(default_factory=list)
    iters: list = dataclasses.field(default_factory=list)
    statuses: list = dataclasses.field(default_factory=list)
    admitted_at: float = -1.0
    done_at: float = -1.0
    bytes: int = 0        # device bytes counted against the budget while admitted
    cancel_after: int = 0  # > 0: the client cancels the request after this many steps
    cancelled: bool = False
    # checkpoint/resume: a request parked at a stop keeps its next step's modes and its warm
    # start on the host (resume_p) and takes its device state back when it is admitted again
    resume_p: object = None
    finished: bool = False  # all its steps ran (before a checkpoint)


def request_stream(n, rate, seed=0, lo=(32, 32, 32), hi=(256, 128, 128)):
    """``n`` requests with Poisson arrivals of ``rate`` per second (rate = inf: all at t = 0) and
    grid sizes drawn as in the batched workload (dims multiples of 16, aspect <= 4)."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for i in range(n):
        if math.isfinite(rate):
            t += rng.exponential(1.0 / rate)
        out.append(Request(i, t if math.isfinite(rate) else 0.0, inputs.draw_shape(rng, lo, hi),
                           int(seed * 7919 + 31 * i + 5)))
    return out


class Server:
    def __init__(self, budget_bytes, precision="fp32", tol=1e-9, steps=20, device="cuda",
                 keep_results=False, tile=SERVE_TILE, precond="jacobi", record_steps=False,
                 log=None):
        # tile: kernel variant of every Jacobi request's handle (fixed, so admission does not run
        # the autotuner; the batch executor uses the variant of its largest solve).  precond
        # "mg": the V-cycle preconditioner; such handles are not batched, the executor solves
        # them one by one when they are polled.  Admission asks the library whether a request's
        # handle fits the memory left (poisson_required_bytes, POISSON_ENOMEM_BUDGET if not).
        self.tile = tile
        self.precond = precond
        self.budget = int(budget_bytes)
        self.precision = precision
        self.tol = tol
        self.steps = steps
        self.device = device
        self.keep = keep_results
        self.results = {}
        # record_steps: host copies of every step's inputs and result, for checking served solves
        # one by one (rid -> {"grid", "F", "steps": [(s, p, status)]}); costs a device-to-host
        # copy per step inside the loop, so it is for tests, not for timing
        self.record = {} if record_steps else None
        # log: a path or a writable text file; one JSON line per finished solve (request, step,
        # shape, status, residual, CG iterations, latency)
        self.log = log

    def _admit(self, r, now):
        g, F, s, modes = inputs.mixed_fields_t(r.shape, r.seed, device=self.device)
        import torch
        if r.resume_p is not None:
            # a resumed request: its next step's modes and its warm start from the checkpoint
            r.grid, r.F = g, F
            r.s = inputs.divergence_source_t(g, r.modes, device=self.device)
            r.p = torch.from_numpy(r.resume_p).to(self.device)
            r.resume_p = None
        else:
            r.grid, r.F, r.s, r.modes = g, F, s, modes
            r.p = torch.zeros(g.shape, dtype=torch.float64, device=self.device)
        r.solver = capi.Poisson(g.nx, g.ny, g.nz, g.h,
                                **_handle_opts(self.precision, self.precond, self.tile))
        r.solver.set_density(F)
        r.admitted_at = now
        if self.record is not None:
            self.record[r.rid] = {"grid": g, "F": F.cpu().numpy(), "steps": []}
        self._submit(r, r.arrival)

    def _submit(self, r, t_from):
        import torch
        torch.cuda.synchronize()  # the source is written on torch's stream
        r.ticket = capi.batch_submit([r.solver], [r.s], [r.p], self.tol)[0]
        r.t_submit = t_from

    def _advance(self, r):
        r.modes = inputs.advect_modes(r.modes, r.grid, inputs.DT)
        r.s = inputs.divergence_source_t(r.grid, r.modes, device=self.device)

    def cancel(self, r):
        """The client gives up on request r.  Not yet admitted: it is dropped unallocated.
        Admitted: its step in flight still finishes (a batch is not interrupted mid-solve), then
        it leaves (handle destroyed, memory returned to the budget) without further steps."""
        r.cancelled = True

    def _log(self, out, r, rc, st, lat, t):
        if out is None:
            return
        out.write(json.dumps({"rid": r.rid, "step": r.step, "shape": list(r.shape),
                              "status": capi.strerror(rc) if rc != capi.OK else "ok",
                              "rel_residual": st["rel_residual"] if st else None,
                              "inner_iters": st["inner_iters"] if st else None,
                              "latency_ms": 1e3 * lat, "t_s": t}) + "\n")

    def serve(self, requests, stop_after=None):
        """Runs the stream to completion (wall clock); returns the statistics.  stop_after: stop
        once that many solves have finished -- no request is admitted and no step submitted
        after it, the steps in flight finish, and every unfinished admitted request is parked
        (its next step's source modes and its pressure copied to the host, its handle and device
        memory released), so that checkpoint() can save the stream and a new Server resume it."""
        own_log = isinstance(self.log, str)
        out = open(self.log, "w") if own_log else self.log
        try:
            return self._serve(requests, out, stop_after)
        finally:
            if own_log:
                out.close()

    @staticmethod
    def checkpoint(path, requests):
        """Saves a stopped stream (after serve(..., stop_after=n)): every request's identity,
        progress and statistics so far, and for parked ones their source modes and warm start.
        A .npz file of plain arrays; the metadata is one JSON string."""
        meta, arrays = [], {}
        for r in requests:
            meta.append({"rid": r.rid, "arrival": r.arrival, "shape": list(r.shape), "seed": r.seed,
                         "step": r.step, "cancel_after": r.cancel_after, "cancelled": r.cancelled,
                         "finished": r.finished or r.done_at >= 0,
                         "latencies": r.latencies, "residuals": r.residuals, "iters": r.iters,
                         "statuses": r.statuses, "parked": r.resume_p is not None})
            if r.resume_p is not None:
                arrays["p_%d" % r.rid] = r.resume_p
                arrays["modes_a_%d" % r.rid] = np.array([m.a for m in r.modes], dtype=np.float64)
                arrays["modes_k_%d" % r.rid] = np.array([m.k for m in r.modes], dtype=np.int64)
                arrays["modes_phase_%d" % r.rid] = np.array([m.phase for m in r.modes])
        np.savez(path, meta=np.array(json.dumps(meta)), **arrays)

    @staticmethod
    def load_checkpoint(path):
        """The requests of a checkpoint, ready for serve(): finished ones are kept for the
        statistics and not run again, parked ones resume at their next step from their saved
        pressure, the others start from the beginning."""
        with np.load(path) as z:
            meta = json.loads(str(z["meta"]))
            out = []
            for m in meta:
                r = Request(m["rid"], m["arrival"], tuple(m["shape"]), m["seed"])
                r.step, r.cancel_after, r.cancelled = m["step"], m["cancel_after"], m["cancelled"]
                r.finished = m["finished"]
                r.latencies, r.residuals = list(m["latencies"]), list(m["residuals"])
                r.iters, r.statuses = list(m["iters"]), list(m["statuses"])
                if m["parked"]:
                    rid = r.rid
                    r.resume_p = np.array(z["p_%d" % rid])
                    r.modes = [inputs.Mode(tuple(float(v) for v in a), tuple(int(v) for v in k),
                                           float(ph))
                               for a, k, ph in zip(z["modes_a_%d" % rid], z["modes_k_%d" % rid],
                                                   z["modes_phase_%d" % rid])]
                out.append(r)
        return out

    def _serve(self, requests, out, stop_after=None):
        pending = collections.deque(sorted((q for q in requests if not q.finished),
                                           key=lambda q: q.arrival))
        done_solves = cells_done = 0
        stopping = False
        parked = 0
        active = []
        used = 0
        t0 = time.perf_counter()
        lat = []
        peak_active = 0
        peak_used = 0
        while (pending and not stopping) or active:
            now = time.perf_counter() - t0
            while pending and pending[0].arrival <= now and not stopping:
                if pending[0].cancelled:  # cancelled before admission: never allocated
                    pending.popleft()
                    continue
                nx, ny, nz = pending[0].shape
                arrays = REQUEST_BYTES_PER_CELL * nx * ny * nz
                left = self.budget - used - arrays
                rc, hb = capi.required_bytes(nx, ny, nz, budget=max(1, left),
                                             **_handle_opts(self.precision, self.precond, self.tile))
                if (left <= 0 or rc == capi.ENOMEM_BUDGET) and active:
                    break  # wait for memory to free up
                r = pending.popleft()
                r.bytes = hb + arrays
                used += r.bytes
                self._admit(r, now)
                active.append(r)
            peak_active = max(peak_active, len(active))
            peak_used = max(peak_used, used)
            if not active:
                if pending and not stopping:
                    time.sleep(max(0.0, min(0.01, pending[0].arrival - now)))
                continue
            for r in list(active):
                rc, st = capi.poll(r.ticket)
                if rc == capi.PENDING:
                    continue
                t = time.perf_counter() - t0
                r.latencies.append(t - r.t_submit)
                r.statuses.append(rc)
                r.residuals.append(st["rel_residual"] if st else float("nan"))
                r.iters.append(st["inner_iters"] if st else 0)
                lat.append(t - r.t_submit)
                if self.record is not None:
                    self.record[r.rid]["steps"].append((r.s.cpu().numpy(), r.p.cpu().numpy(), rc))
                self._log(out, r, rc, st, t - r.t_submit, t)
                r.step += 1
                done_solves += 1
                cells_done += r.shape[0] * r.shape[1] * r.shape[2]
                if stop_after is not None and done_solves >= stop_after:
                    stopping = True
                if r.cancel_after and r.step >= r.cancel_after:
                    r.cancelled = True
                more = r.step < self.steps and rc == capi.OK and not r.cancelled
                if more and not stopping:
                    self._advance(r)
                    self._submit(r, t)
                else:
                    if more:  # parked at the stop: the next step's modes and warm start
                        self._advance(r)
                        r.resume_p = r.p.cpu().numpy()
                        parked += 1
                    else:
                        r.finished = True
                    if r.finished:
                        r.done_at = t
                    if self.keep and r.finished:
                        self.results[r.rid] = r.p.cpu().numpy()
                    r.solver.close()
                    r.solver = None
                    r.F = r.s = r.p = None
                    used -= r.bytes
                    active.remove(r)
        wall = time.perf_counter() - t0
        lat = np.array(lat) if lat else np.zeros(1)
        # this run's solves (a resumed stream's requests carry their earlier steps' records)
        nsolves = done_solves
        cells = cells_done
        complete = lambda r: r.finished or r.cancelled
        return {
            "requests": len(requests), "solves": nsolves, "wall_s": wall,
            "solves_per_s": nsolves / wall, "cell_solves_per_s": cells / wall,
            "p50_ms": 1e3 * float(np.percentile(lat, 50)), "p99_ms": 1e3 * float(np.percentile(lat, 99)),
            "max_rel_residual": max((max(r.residuals) for r in requests if r.residuals), default=0.0),
            "all_ok": all(all(s == capi.OK for s in r.statuses) and
                          (len(r.statuses) == self.steps or r.cancelled or not complete(r))
                          for r in requests),
            "cancelled": sum(1 for r in requests if r.cancelled),
            "used_bytes_at_end": used,
            "stopped": stopping, "parked": parked,
            "peak_active": peak_active, "peak_used_bytes": peak_used, "budget_bytes": self.budget,
            "precision": self.precision,
        }

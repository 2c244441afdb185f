"""Benchmark of the pressure Poisson solve on one or more GB300s.

One step = one pass of the whole solve path over one synthetic input: set the density from the
water fraction (operator set-up) and solve div((1/rho) grad p) = s to relative residual 1e-9 from
a zero start (FP32 inner PCG inside FP64 refinement by default).  The workload is the
surface-piercing elliptic strut on a 256 x 128 x 128 grid (4,194,304 cells, density ratio 1000).

value  = cells x CG iterations / device seconds, summed over ranks (Gcell-iters/s), inputs
         resident in HBM, L2 flushed between steps.
e2e    = the same metric through the C ABI with pinned HOST arrays: the H2D copy of F, s and the
         start p and the D2H copy of the solution are inside the timed region.
roofline: the dominant CG kernel's algorithmic bytes per launch / its mean CUDA-event duration.
cpu_baseline: the FP64 CPU oracle timed on this host on a bounded sample of the same workload.

--impl reference times the oracle instead (the reference arm: a plain CPU program).
Multi-GPU (torchrun): independent replicas, one solve per rank per step (weak scaling).
"""
import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

CELLS_NOTE = "strut 256x128x128"
WORKLOAD = ("surface-piercing elliptic strut (0.1 x 0.02, water density) in a Kelvin-like "
            "two-phase surface, 256x128x128 cells, h = 1/128, rho 1/1000, source div(u*)/dt of "
            "8 random modes; tol 1e-9 rel. residual, zero start")
# Algorithmic bytes per cell of one launch of each CG pass (FP32 vectors; rho/2 per cell as the
# coefficient array, FP32 = 4 B, BF16 = 2 B; neighbour re-reads served on chip, not counted):
#   phase A: read z, p_old, eta; write p                     = 3 vec + eta + 1 vec
#   phase B: read x, r, p, eta; write x, r, z                = 6 vec + eta
BYTES_PER_CELL = {
    "fp32": {"cg_phase_a": 4 * 3 + 4, "cg_phase_b": 4 * 6 + 4},
    "bf16": {"cg_phase_a": 4 * 3 + 2, "cg_phase_b": 4 * 6 + 2},
    # FP64 PCG: vectors 8 B, stored FP64 faces bx, by, bz + diag (+ dinv in phase B)
    "fp64": {"cg_phase_a": 8 * 3 + 8 * 4, "cg_phase_b": 8 * 6 + 8 * 5},
}
# one-sweep persistent kernels (Chronopoulos-Gear): reads p, u, s^, w^ (16 B) + eta, writes p,
# u, s^, w^ (16 B) every iteration; x read and written every other iteration (4 B on average)
BYTES_PER_CELL_ONE_SWEEP = {"fp32": 16 + 4 + 16 + 4, "bf16": 16 + 2 + 16 + 4}
# one-sweep kernels that form A p in the sweep: read u, p (8 B) + eta, write u, p (8 B), x every
# other iteration (4 B on average)
BYTES_PER_CELL_AP_FORMED = {"fp32": 8 + 4 + 8 + 4, "bf16": 8 + 2 + 8 + 4}
# MG-preconditioned phase B (POISSON_MG), per fine cell: the CG update (read p, x, r, eta; write
# x, r, the pre-smoothed x0 = 7 vec-equivalents with eta), the fine restriction (read r, x0, eta;
# write r_c, x_c: 2 values per 8 cells) and the fine prolongation + smoothing (read x0, r, eta and
# e_c (1 value per 8 cells); write z); every coarse level l adds, per cell of its own, the
# restriction (read r, x, four stored operator arrays; write 2 values per 8 cells) and the
# smoothing (read r, x, four operator arrays, 1 value per 8 cells; write y).
def mg_phase_b_bytes(precision, level_cells, n):
    v = 8 if precision == "fp64" else 4
    eta = 8 * 4 if precision == "fp64" else (4 if precision == "fp32" else 2)
    fine = (4 * v + eta + 3 * v) + (2 * v + eta + 2 * v / 8) + (2 * v + eta + v / 8 + v)
    coarse = sum(nl * ((6 * v + 2 * v / 8) + (6 * v + v / 8 + v)) for nl in level_cells[1:-1])
    coarse += level_cells[-1] * 6 * v  # coarsest: r, x, operator (sweeps stay on chip)
    return fine + coarse / n


def mg_levels(nx, ny, nz, periodic, coarse_max=512):
    """Cell counts of the V-cycle's levels: 2x2x2 aggregation (an axis of one cell stays; a
    periodic x axis only while nx is even and >= 4), level 0 always coarsened once, stop at
    coarse_max cells."""
    cells = [nx * ny * nz]
    while True:
        fx = (2 if nx % 2 == 0 and nx >= 4 else 1) if periodic else (2 if nx > 1 else 1)
        fy, fz = (2 if ny > 1 else 1), (2 if nz > 1 else 1)
        if fx * fy * fz == 1 or (len(cells) > 1 and nx * ny * nz <= coarse_max):
            return cells
        nx, ny, nz = -(-nx // fx), -(-ny // fy), -(-nz // fz)
        cells.append(nx * ny * nz)


L2_FLUSH_BYTES = 256 << 20


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="fp32", choices=["fp32", "bf16", "fp64"])
    ap.add_argument("--precond", default="jacobi", choices=["jacobi", "rbssor", "mg"])
    ap.add_argument("--inner-tol", type=float, default=1e-4,
                    help="FP32 inner solve: relative reduction per refinement step")
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--shape", type=int, nargs=3, default=(256, 128, 128),
                    help="grid of the strut workload (profiling of smaller cases)")
    ap.add_argument("--tile", type=int, default=0, help="FP32 kernel tile option (0 = autotuned)")
    ap.add_argument("--walls", type=int, default=0,
                    help="Dirichlet side/bottom walls bitmask (1 x-, 2 x+, 4 y-, 8 y+, 16 z-)")
    ap.add_argument("--periodic-x", action="store_true", help="periodic x boundaries")
    ap.add_argument("--cut-body", action="store_true",
                    help="the strut as a free-slip cut-cell body (face and volume fractions)")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the FP64 comparison, batched and served measurements")
    ap.add_argument("--serve-requests", type=int, default=24)
    ap.add_argument("--case", default="strut", choices=["strut", "wedge"],
                    help="strut 256x128x128 (default) or the 1024x512x256 wedge (fields made on "
                         "the device)")
    return ap.parse_args()


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def source_hash():
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1410_1942_gb300", "csrc")
    for name in sorted(os.listdir(csrc)):
        with open(os.path.join(csrc, name), "rb") as f:
            h.update(name.encode() + f.read())
    return h.hexdigest()[:16]


def ncu_traffic(kernel, precision, workload):
    """DRAM bytes per cell-iteration of `kernel` on `workload` from the committed ncu summary, if
    it was taken on the current kernel sources; else None."""
    path = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    if not os.path.exists(path):
        return None
    with open(path) as f:
        d = json.load(f)
    e = d.get("%s/%s/%s" % (precision, kernel, workload))
    if not e or e.get("source_hash") != source_hash():
        return None
    return e.get("dram_bytes_per_cell_iter")


class Clocks:
    """Samples SM clocks and throttle reasons with nvidia-smi while the timed region runs."""
    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.f = None

    def start(self):
        try:
            self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.f.flush()
        self.f.seek(0)
        rows = [r.split(", ") for r in self.f.read().strip().splitlines() if r.strip()]
        self.f.close()
        os.unlink(self.f.name)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            if len(r) < 8:
                continue
            try:
                sm.append(float(r[0]))
                mx.append(float(r[1]))
            except ValueError:
                continue
            for nm, v in zip(names, r[4:8]):
                if v.strip().lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def combine_ranks(t, units, device, world):
    """Whole-job figures of a replicated run: the slowest rank's time and the units of all ranks
    (two all-reduces over the process group; world 1: unchanged)."""
    if world <= 1:
        return t, units
    import torch
    import torch.distributed as tdist
    tt = torch.tensor([t, units], dtype=torch.float64, device=device)
    mx = tt.clone()
    tdist.all_reduce(mx, op=tdist.ReduceOp.MAX)
    tdist.all_reduce(tt, op=tdist.ReduceOp.SUM)
    return float(mx[0]), float(tt[1])


# ----------------------------------------------------------------------------- reference arm
def run_reference(args):
    """The oracle (plain FP64 CPU PCG) timed on this host's cores, same workload and metric."""
    world, rank, _ = dist_env()
    if rank != 0:
        return 0
    import oracle
    from paper_1410_1942_gb300 import inputs
    oracle.build()
    c = inputs.strut_case(256, 128, 128, seed=args.seed)
    op = oracle.operator(c.F)
    b = oracle.rhs(c.s, c.grid.h)
    iters_per_step = 20
    precond = "ssor" if args.precond == "rbssor" else "jacobi"
    x = np.zeros(c.grid.shape)
    for _ in range(args.warmup):
        oracle.pcg(op, b, x0=x, tol=0.0, precond=precond, max_iters=iters_per_step)
    t0 = time.perf_counter()
    its = 0
    for _ in range(args.steps):
        r = oracle.pcg(op, b, x0=x, tol=0.0, precond=precond, max_iters=iters_per_step)
        its += r.iters
    dt = time.perf_counter() - t0
    val = c.grid.n * its / dt / 1e9
    line = {
        "impl": "reference", "metric": "Poisson PCG Gcell-iters/s", "value": val,
        "unit": "Gcell-iters/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * dt / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "precond": precond},
        "cpu_baseline": {"value": val, "unit": "Gcell-iters/s", "cores": oracle.threads(),
                         "kind": "oracle",
                         "sample": "%d FP64 %s-PCG iterations per step of the CPU oracle on the "
                                   "%s workload" % (iters_per_step, precond, CELLS_NOTE)},
        "e2e": {"value": val, "unit": "Gcell-iters/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def fp64_baseline(case, steps, stream):
    """Plain FP64 GPU PCG (Jacobi) on the same workload: solves/s at the same tolerance."""
    import torch
    from paper_1410_1942_gb300 import capi
    g = case.grid
    F = torch.from_numpy(case.F).cuda()
    s = torch.from_numpy(case.s).cuda()
    p = torch.zeros(g.shape, dtype=torch.float64, device="cuda")
    with capi.Poisson(g.nx, g.ny, g.nz, g.h, precision="fp64", stream=stream.cuda_stream) as sv:
        sv.set_density(F)
        sv.solve(s, p, case.tol)  # warm-up
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        its, rel = 0, 0.0
        for _ in range(steps):
            sv.set_density(F)
            p.zero_()
            rc, st = sv.solve(s, p, case.tol)
            its += st["inner_iters"]
            rel = max(rel, st["rel_residual"])
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
    return {"solves_per_s": steps / dt, "ms_per_solve": 1e3 * dt / steps,
            "gcell_iters_per_s": g.n * its / dt / 1e9, "cg_iters_per_solve": its / steps,
            "max_rel_residual": rel}


def batched(n=64, seed=0):
    """64 independent solves of uneven size (32^3 .. 128x64x64) submitted together and driven
    by the batch executor (one persistent PCG launch per refinement step)."""
    import torch
    from paper_1410_1942_gb300 import capi, inputs
    cases = inputs.batch_cases(n, seed=seed)
    solvers, ps, rhs = [], [], []
    for c in cases:
        g = c.grid
        sv = capi.Poisson(g.nx, g.ny, g.nz, g.h, precision="fp32")
        sv.set_density(torch.from_numpy(c.F).cuda())
        solvers.append(sv)
        rhs.append(torch.from_numpy(c.s).cuda())
        ps.append(torch.zeros(g.shape, dtype=torch.float64, device="cuda"))

    def run():
        for p in ps:
            p.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        tickets = capi.batch_submit(solvers, rhs, ps, 1e-9)
        res, pending = {}, list(tickets)
        while pending:
            nxt = []
            for t in pending:
                rc, st = capi.poll(t)
                if rc == capi.PENDING:
                    nxt.append(t)
                else:
                    res[t] = (rc, st)
            pending = nxt
        return time.perf_counter() - t0, [res[t] for t in tickets]

    run()  # warm-up (graphs, plans)
    dt, res = run()
    cells_it = sum(c.grid.n * r[1]["inner_iters"] for c, r in zip(cases, res))
    out = {"solves": n, "wall_s": dt, "solves_per_s": n / dt, "gcell_iters_per_s": cells_it / dt / 1e9,
           "all_ok": all(r[0] == capi.OK for r in res),
           "max_rel_residual": max(r[1]["rel_residual"] for r in res),
           "cells": sum(c.grid.n for c in cases)}
    for sv in solvers:
        sv.close()
    return out


def served(nreq, seed=0):
    """The request stream: capacity with every request waiting at t = 0 (6 steps each), then
    Poisson arrivals at 70 % of that capacity, 20 steps per request; FP32 inner solve, and the
    plain FP64 PCG's and the multigrid-preconditioned solve's capacities for comparison."""
    import math as _m
    from paper_1410_1942_gb300 import inputs, serve
    # warm the device-side input generators (torch compiles its complex kernels on first use)
    inputs.mixed_fields_t((32, 32, 32), 1, device="cuda")
    budget = 48 << 30
    cap = serve.Server(budget, steps=6).serve(serve.request_stream(max(4, nreq // 2), _m.inf, seed=seed + 1))
    rate = 0.7 * cap["solves_per_s"] / 20.0
    st = serve.Server(budget, steps=20).serve(serve.request_stream(nreq, rate, seed=seed))
    cap64 = serve.Server(budget, precision="fp64", steps=3).serve(
        serve.request_stream(max(4, nreq // 4), _m.inf, seed=seed + 2))
    # the same capacity stream with the multigrid preconditioner (unbatched handles)
    capmg = serve.Server(budget, steps=6, precond="mg").serve(
        serve.request_stream(max(4, nreq // 2), _m.inf, seed=seed + 1))
    return {"capacity_solves_per_s": cap["solves_per_s"], "arrival_rate_per_s": rate,
            "solves_per_s": st["solves_per_s"], "p50_ms": st["p50_ms"], "p99_ms": st["p99_ms"],
            "solves": st["solves"], "requests": nreq, "steps_per_request": 20,
            "max_rel_residual": st["max_rel_residual"], "all_ok": st["all_ok"],
            "peak_active": st["peak_active"],
            "fp64_capacity_solves_per_s": cap64["solves_per_s"],
            "fp64_p50_ms": cap64["p50_ms"], "fp64_p99_ms": cap64["p99_ms"],
            "mg_capacity_solves_per_s": capmg["solves_per_s"],
            "mg_max_rel_residual": capmg["max_rel_residual"], "mg_all_ok": capmg["all_ok"]}


def cpu_baseline(case, seconds, precond):
    """The oracle as it stands on this host's cores: fixed 20-iteration PCG windows of the same
    workload until `seconds` of CPU work have run."""
    import oracle
    oracle.build()
    op = oracle.operator(case.F)
    b = oracle.rhs(case.s, case.grid.h)
    x = np.zeros(case.grid.shape)
    if precond == "mg":
        from oracle import multigrid
        levels = multigrid.hierarchy(op)
    its, t0 = 0, time.perf_counter()
    while True:
        if precond == "mg":
            r = multigrid.pcg_mg(op, b, x0=x, tol=0.0, max_iters=20, levels=levels)
        else:
            r = oracle.pcg(op, b, x0=x, tol=0.0, precond=precond, max_iters=20)
        its += r.iters
        if time.perf_counter() - t0 >= seconds:
            break
    dt = time.perf_counter() - t0
    return {"value": case.grid.n * its / dt / 1e9, "unit": "Gcell-iters/s",
            "cores": oracle.threads(), "kind": "oracle",
            "sample": "%d FP64 %s-PCG iterations (windows of 20) of the CPU oracle on the %s "
                      "workload, %.1f s" % (its, precond, CELLS_NOTE, dt)}


# ----------------------------------------------------------------------------- our arm
def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    import torch
    import torch.distributed as tdist
    world, rank, local = dist_env()
    if world > 1:
        torch.cuda.set_device(local)
        tdist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    dev = torch.device("cuda", torch.cuda.current_device())

    from paper_1410_1942_gb300 import build as _build
    from paper_1410_1942_gb300 import capi, inputs
    _build.build()
    capi.load()

    if args.case == "wedge":
        shape = (1024, 512, 256) if tuple(args.shape) == (256, 128, 128) else tuple(args.shape)
        g, F_d, s_d, _ = inputs.wedge_fields_t(shape, seed=args.seed + rank, device=dev)
        case = inputs.Case("wedge", g, None, None, 1e-9, {})
        args.no_extras = True
        args.no_cpu_baseline = True
        args.no_e2e = True
    else:
        case = inputs.strut_case(*args.shape, seed=args.seed + rank)
        g = case.grid
        F_d = torch.from_numpy(case.F).to(dev)
        s_d = torch.from_numpy(case.s).to(dev)
    p_d = torch.zeros(g.shape, dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream(dev)
    solver = capi.Poisson(g.nx, g.ny, g.nz, g.h, precision=args.precision, precond=args.precond,
                          stream=stream.cuda_stream, tile=args.tile, dirichlet_walls=args.walls,
                          periodic_x=args.periodic_x, inner_tol=args.inner_tol)
    apertures = None
    if args.cut_body:
        Lx, Ly, _ = g.lengths
        psi = lambda x, y, z: inputs.ellipse_sdf(x, y, 0.5 * Lx, 0.5 * Ly, 0.1, 0.02)
        apertures = inputs.cut_apertures(g, psi)
        solver.set_apertures(*apertures)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)

    def barrier():
        if world > 1:
            tdist.barrier()
        torch.cuda.synchronize(dev)

    def step():
        solver.set_density(F_d)
        p_d.zero_()
        rc, st = solver.solve(s_d, p_d, case.tol)
        if rc != capi.OK:
            raise RuntimeError("solve failed: %s" % capi.strerror(rc))
        return st

    for _ in range(args.warmup):
        step()
    solver.profile(True)
    clocks = Clocks(torch.cuda.current_device()) if rank == 0 else None
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(args.steps)]
    iters, outer, rels = 0, 0, []
    barrier()
    if clocks:
        clocks.start()
    l0 = capi.kernel_launches()
    for q in range(args.steps):
        flush.fill_(q & 0xFF)
        evs[q][0].record(stream)
        st = step()
        evs[q][1].record(stream)
        iters += st["inner_iters"]
        outer += st["outer_iters"]
        rels.append(st["rel_residual"])
    barrier()
    launches = capi.kernel_launches() - l0
    clk = clocks.stop() if clocks else None
    dev_ms = sum(a.elapsed_time(b) for a, b in evs)
    prof = solver.profile_read()
    solver.profile(False)
    units = float(g.n) * iters                     # cell-iterations of this rank
    t_max, units = combine_ranks(dev_ms, units, dev, world)
    value = units / (t_max * 1e-3) / 1e9

    # dominant CG kernel and its roofline
    bpc = BYTES_PER_CELL[args.precision]
    cands = [k for k in ("pcg_persistent", "cg_phase_a", "cg_phase_b") if prof[k]["launches"]]
    dom = max(cands, key=lambda k: prof[k]["ms"])
    per_launch_ms = prof[dom]["ms"] / prof[dom]["launches"]
    desc = solver.describe()
    if "A p formed" in desc:
        bpi = BYTES_PER_CELL_AP_FORMED[args.precision]
    elif "one-sweep" in desc:
        bpi = BYTES_PER_CELL_ONE_SWEEP[args.precision]
    elif args.precond == "mg":
        bpc = dict(bpc)
        bpc["cg_phase_b"] = mg_phase_b_bytes(args.precision,
                                             mg_levels(g.nx, g.ny, g.nz, args.periodic_x), g.n)
        bpi = bpc["cg_phase_a"] + bpc["cg_phase_b"]
    else:
        bpi = bpc["cg_phase_a"] + bpc["cg_phase_b"]  # algorithmic bytes per cell-iteration
    if dom == "pcg_persistent":
        # one launch runs every CG iteration of one inner solve
        alg_bytes = bpi * g.n * iters / prof[dom]["launches"]
    else:
        alg_bytes = bpc[dom] * g.n
    achieved = alg_bytes / (per_launch_ms * 1e-3) / 1e9
    peak, peak_kind = peaks()
    wl_key = "%s%dx%dx%d" % (args.case, g.nx, g.ny, g.nz)
    bpci = ncu_traffic(dom, args.precision, wl_key)
    # DRAM bytes per launch, like alg_bytes: the measured bytes per cell-iteration times the
    # cell-iterations of an average launch
    traffic = (bpci * g.n * iters / prof[dom]["launches"]
               if bpci is not None and dom == "pcg_persistent" else None)
    hbm_alg = value * bpi  # GB/s of CG-pass algorithmic traffic

    # end to end through the C ABI with pinned host arrays
    e2e = None
    if not args.no_e2e:
        F_h = torch.from_numpy(case.F).pin_memory()
        s_h = torch.from_numpy(case.s).pin_memory()
        p_h = torch.zeros(g.shape, dtype=torch.float64).pin_memory()
        solver_h = capi.Poisson(g.nx, g.ny, g.nz, g.h, precision=args.precision,
                                precond=args.precond, stream=stream.cuda_stream, tile=args.tile,
                                dirichlet_walls=args.walls, periodic_x=args.periodic_x,
                                inner_tol=args.inner_tol)
        if apertures is not None:
            solver_h.set_apertures(*apertures)

        def step_e2e():
            p_h.zero_()
            solver_h.set_density(F_h)
            rc, st = solver_h.solve(s_h, p_h, case.tol)
            if rc != capi.OK:
                raise RuntimeError("e2e solve failed: %s" % capi.strerror(rc))
            return st

        for _ in range(min(2, args.warmup)):
            step_e2e()
        barrier()
        its_e, t0 = 0, time.perf_counter()
        for _ in range(args.steps):
            its_e += step_e2e()["inner_iters"]
        barrier()
        te = time.perf_counter() - t0
        ue = float(g.n) * its_e
        te, ue = combine_ranks(te, ue, dev, world)
        e2e = {"value": ue / te / 1e9, "unit": "Gcell-iters/s",
               "h2d_bytes_per_step": 3 * 8 * g.n, "d2h_bytes_per_step": 8 * g.n,
               "ms_per_step": 1e3 * te / args.steps}
        solver_h.close()

    extras = {}
    if rank == 0 and not args.no_extras and tuple(args.shape) == (256, 128, 128):
        fb = fp64_baseline(case, 2, stream)
        extras["fp64_baseline"] = fb
        extras["mixed_vs_fp64_solves_ratio"] = (world * args.steps / (t_max * 1e-3)) / fb["solves_per_s"]
        extras["batched"] = batched()
        extras["served"] = served(args.serve_requests)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(case, args.cpu_seconds, {"rbssor": "ssor"}.get(args.precond, args.precond))

    if rank == 0:
        line = {
            "metric": "Poisson PCG Gcell-iters/s", "value": value, "unit": "Gcell-iters/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": t_max / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64" if args.precision == "fp64" else "f32",
            "data": "synthetic",
            "config": {"workload": ("wedge %dx%dx%d (hull half-plane pair, breaking patches)"
                                    % (g.nx, g.ny, g.nz)) if args.case == "wedge" else
                        (WORKLOAD if tuple(args.shape) == (256, 128, 128)
                         else "strut %dx%dx%d (profiling case)" % tuple(args.shape)), "cells": g.n, "precision": args.precision,
                       "precond": args.precond, "tol": case.tol, "inner_tol": args.inner_tol,
                       "boundaries": ("strut as a free-slip cut-cell body, " if args.cut_body
                                      else "") + ("periodic x, " if args.periodic_x else "") +
                                     ("Dirichlet walls mask %d" % args.walls if args.walls
                                      else "zero-gradient side/bottom walls") + ", p = 0 on top",
                       "l2": "flushed between steps (256 MiB write)",
                       "parallelism": "replicas" if world > 1 else "1 GPU",
                       "kernels": solver.describe(),
                       "cg_iters_per_step": iters / args.steps,
                       "outer_iters_per_step": outer / args.steps,
                       "max_rel_residual": max(rels)},
            "hbm_gbs_algorithmic": hbm_alg,
            "solves_per_s": world * args.steps / (t_max * 1e-3),
            "roofline": {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak,
                         "peak_kind": peak_kind, "unit": "GB/s", "frac": achieved / peak,
                         "traffic": traffic, "alg_bytes_per_launch": alg_bytes,
                         "alg_bytes_per_cell_iter": bpi,
                         "ms_per_launch": per_launch_ms},
            "kernel_times": prof,
            **extras,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": launches,
            "clocks": clk,
        }
        print(json.dumps(line), flush=True)
    solver.close()
    if world > 1:
        tdist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())

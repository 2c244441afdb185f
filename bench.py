"""Benchmark of the pressure Poisson solve on one or more GB300s.

One step = one pass of the whole solve path over one synthetic input: set the density from the
water fraction (operator set-up) and solve div((1/rho) grad p) = s to relative residual 1e-9 from
a zero start (FP32 inner PCG inside FP64 refinement by default).  The default workload is the
largest single-GPU configuration: a wedge-like hull (signed-distance half-plane pair, seeded
entrance half-angle) in a two-phase surface with breaking-like patches on a 1024 x 512 x 256 grid
(134,217,728 cells, density ratio 1000).  ``--case strut`` runs the 256 x 128 x 128 strut instead.

value  = cells x CG iterations / device seconds, summed over ranks (Gcell-iters/s), inputs
         resident in HBM (and far larger than L2; a 256 MiB buffer is also written between steps).
e2e    = the same metric through the C ABI with pinned HOST arrays: the H2D copy of F, s and the
         start p and the D2H copy of the solution are inside the timed region.
roofline: the dominant CG kernel's algorithmic bytes per launch / its mean CUDA-event duration;
         traffic = the DRAM bytes per cell-iteration of the committed ncu capture (taken on the
         current sources of that kernel) times the cell-iterations of a launch.
cpu_baseline: the FP64 CPU oracle timed on this host on a bounded sample of the same workload.
extras (rank 0): the wedge with BF16 densities in the inner operator and with the multigrid
         preconditioner, and the strut workload's line with its plain-FP64 comparison, its
         64-solve batch and its served request stream.

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

METRIC = "Poisson PCG Gcell-iters/s"
SHAPES = {"wedge": (1024, 512, 256), "strut": (256, 128, 128)}
TOL = 1e-9


def workload(kind, shape):
    nx, ny, nz = shape
    if kind == "wedge":
        return ("wedge-like hull (signed-distance half-plane pair, seeded entrance half-angle "
                "10-30 deg, full depth, water density) in a two-phase surface with breaking-like "
                "patches (5 %% of the cells within 2h of the surface set to 0 or 1), %dx%dx%d "
                "cells, h = 1/%d, rho 1/1000, source div(u*)/dt of 8 random modes; tol 1e-9 rel. "
                "residual, zero start" % (nx, ny, nz, nz))
    return ("surface-piercing elliptic strut (0.1 x 0.02, water density) in a Kelvin-like "
            "two-phase surface, %dx%dx%d cells, h = 1/%d, rho 1/1000, source div(u*)/dt of 8 "
            "random modes; tol 1e-9 rel. residual, zero start" % (nx, ny, nz, nz))


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
# cut-cell handles (FP32 or BF16 precision): the inner operator is four stored FP32 arrays (the
# faces bx, by, bz, each scaled by its open fraction, and the diagonal) in place of rho/2
BYTES_PER_CELL_CUT = {"cg_phase_a": 4 * 3 + 16, "cg_phase_b": 4 * 6 + 16}
# one-sweep persistent kernels (Chronopoulos-Gear): reads p, u, s^, w^ (16 B) + eta, writes p,
# u, s^, w^ (16 B) every iteration; x read and written every other iteration (4 B on average)
BYTES_PER_CELL_ONE_SWEEP = {"fp32": 16 + 4 + 16 + 4, "bf16": 16 + 2 + 16 + 4}
# one-sweep kernels that form A p in the sweep: read u, p (8 B) + eta, write u, p (8 B), x every
# other iteration (4 B on average)
BYTES_PER_CELL_AP_FORMED = {"fp32": 8 + 4 + 8 + 4, "bf16": 8 + 2 + 8 + 4}
# red-black SSOR kernels (CG on the black Schur complement): per black cell read u, s^, w^, p,
# x and write them (40 B), per cell eta -- per cell of the grid 20 B of vectors + eta
BYTES_PER_CELL_RB = {"fp32": 20 + 4, "bf16": 20 + 2}
# The face-array schedule that the stencil's byte model counts per cell-iteration (FP32 vectors):
# Jacobi, three stored face arrays and 1/D read, q = A p stored and re-read -- 14 words = 56 B;
# red-black SSOR with the faces read again by the sweeps and z stored -- 17 words = 68 B.  The
# kernels here store rho/2 instead of faces and never store q, so they move less; the line
# reports the fraction at both counts.
BYTES_PER_CELL_FACE_SCHEDULE = {"one-sweep": 56, "red-black": 68}


# MG-preconditioned phase B (POISSON_MG), per fine cell: the CG update (read p, x, r, eta; write
# x, r, the pre-smoothed x0 = 7 vec-equivalents with eta), the fine restriction (read r, x0, eta;
# write r_c, x_c: 2 values per 8 cells) and the fine prolongation + smoothing (read x0, r, eta and
# e_c (1 value per 8 cells); write z); every coarse level l adds, per cell of its own, the
# restriction (read r, x, four stored operator arrays; write 2 values per 8 cells) and the
# smoothing (read r, x, four operator arrays, 1 value per 8 cells; write y).
def mg_phase_b_bytes(precision, level_cells, n, cut=False):
    v = 8 if precision == "fp64" else 4
    eta = 8 * 4 if precision == "fp64" else (4 if precision == "fp32" else 2)
    if cut and precision != "fp64":
        eta = 4 * 4  # FP32 faces bx, by, bz and diag stand in for rho/2
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
E2E_MAX_STEPS = 5     # end-to-end steps (each moves 4 GiB between host and device on the wedge)


def parse(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--case", default="wedge", choices=["wedge", "strut"],
                    help="wedge 1024x512x256 (default; fields made on the device) or the "
                         "256x128x128 strut")
    ap.add_argument("--shape", type=int, nargs=3, default=None,
                    help="grid of the workload (smaller cases for profiling)")
    ap.add_argument("--precision", default="fp32", choices=["fp32", "bf16", "fp64"])
    ap.add_argument("--precond", default="jacobi", choices=["jacobi", "rbssor", "mg"])
    ap.add_argument("--inner-tol", type=float, default=1e-4,
                    help="FP32 inner solve: relative reduction per refinement step")
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--tile", type=int, default=0, help="FP32 kernel tile option (0 = autotuned)")
    ap.add_argument("--walls", type=int, default=0,
                    help="Dirichlet side/bottom walls bitmask (1 x-, 2 x+, 4 y-, 8 y+, 16 z-)")
    ap.add_argument("--periodic-x", action="store_true", help="periodic x boundaries")
    ap.add_argument("--cut-body", action="store_true",
                    help="the strut as a free-slip cut-cell body (face and volume fractions)")
    ap.add_argument("--cap-iters", type=int, default=0,
                    help="profiling: cap each solve at this many CG iterations (one inner launch "
                         "of exactly that many; the solve ends not converged)")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the BF16 / multigrid wedge lines and the strut line with its FP64 "
                         "comparison, batched and served measurements")
    ap.add_argument("--serve-requests", type=int, default=24)
    args = ap.parse_args(argv)
    if args.shape is None:
        args.shape = SHAPES[args.case]
    args.shape = tuple(args.shape)
    return args


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


# Device sources of each persistent kernel family: a committed ncu figure counts only while
# these files are unchanged and the line runs the tile (variant and split) it was taken on.
KERNEL_SOURCES = {
    "one-sweep": ["march1.cu", "march_dev.cuh", "tma.cuh", "internal.cuh", "march.h"],
    "red-black": ["march_rb.cu", "march_rb.h", "march_dev.cuh", "tma.cuh", "internal.cuh",
                  "march.h"],
}


def source_hash(family="one-sweep"):
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1410_1942_gb300", "csrc")
    for name in sorted(KERNEL_SOURCES[family]):
        with open(os.path.join(csrc, name), "rb") as f:
            h.update(name.encode() + f.read())
    return h.hexdigest()[:16]


def ncu_traffic(family, precision, kind, desc):
    """DRAM bytes per cell-iteration of the persistent kernel `family` on workload `kind`, from
    the committed ncu summary if it was taken on the kernel's current sources and on the tile the
    handle runs (`desc`: its description); else None."""
    path = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    if family not in KERNEL_SOURCES or not os.path.exists(path):
        return None
    with open(path) as f:
        d = json.load(f)
    e = d.get("%s/%s/%s" % (precision, family, kind))
    if not e or e.get("source_hash") != source_hash(family):
        return None
    if "tile=%d " % e.get("tile", -1) not in desc:
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


def make_fields(kind, shape, seed, device):
    """(grid, F, s, meta) of the workload as float64 torch tensors on `device`."""
    import torch
    from paper_1410_1942_gb300 import inputs
    if kind == "wedge":
        return inputs.wedge_fields_t(shape, seed=seed, device=device)
    c = inputs.strut_case(*shape, seed=seed)
    return (c.grid, torch.from_numpy(c.F).to(device), torch.from_numpy(c.s).to(device), c.meta)


# ----------------------------------------------------------------------------- reference arm
def run_reference(args):
    """The oracle (plain FP64 CPU PCG) timed on this host's cores, same workload and metric:
    each step is a fixed window of FP64 PCG iterations from the zero start."""
    world, rank, _ = dist_env()
    if rank != 0:
        return 0
    import oracle
    oracle.build()
    g, F, s, _ = make_fields(args.case, args.shape, args.seed, "cpu")
    op = oracle.operator(F.numpy())
    b = oracle.rhs(s.numpy(), g.h)
    del F, s
    iters_per_step = 20
    precond = "ssor" if args.precond == "rbssor" else "jacobi"
    x = np.zeros(g.shape)
    for _ in range(args.warmup):
        oracle.pcg(op, b, x0=x, tol=0.0, precond=precond, max_iters=iters_per_step)
    t0 = time.perf_counter()
    its = 0
    for _ in range(args.steps):
        r = oracle.pcg(op, b, x0=x, tol=0.0, precond=precond, max_iters=iters_per_step)
        its += r.iters
    dt = time.perf_counter() - t0
    val = g.n * its / dt / 1e9
    line = {
        "impl": "reference", "metric": METRIC, "value": val,
        "unit": "Gcell-iters/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * dt / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": workload(args.case, args.shape), "precond": precond},
        "cpu_baseline": {"value": val, "unit": "Gcell-iters/s", "cores": oracle.threads(),
                         "kind": "oracle",
                         "sample": "%d FP64 %s-PCG iterations per step of the CPU oracle (zero "
                                   "start) on the %s %dx%dx%d workload" %
                                   ((iters_per_step, precond, args.case) + args.shape)},
        "e2e": {"value": val, "unit": "Gcell-iters/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ----------------------------------------------------------------------------- measurements
def persistent_path(desc):
    """Whether a handle's inner solve is one persistent launch (its per-kernel events bracket
    whole solves and cost nothing between kernels)."""
    return any(w in desc for w in ("one-sweep", "red-black", "persistent"))


def timed_solves(solver, F, s, p, tol, steps, warmup, stream, sync, clocks=None, flush=None,
                 allow=None):
    """`warmup` untimed then `steps` timed solves (set_density + solve from p = 0), each
    bracketed by CUDA events on the solver's stream; returns the device time and the counts.
    The library's per-kernel events (poisson_profile) record during the timed solves when the
    inner solve is one persistent launch.  For the column kernels they are off while timing
    (between two kernels they would stop the next launch from overlapping the previous one's
    tail) and the per-kernel times come from one more solve, profiled, after the timed region."""
    from paper_1410_1942_gb300 import capi
    allow = allow or (capi.OK,)

    def step():
        solver.set_density(F)
        p.zero_()
        rc, st = solver.solve(s, p, tol, allow=allow)
        return st

    import torch
    for _ in range(warmup):
        step()
    live = persistent_path(solver.describe())
    if live:
        solver.profile(True)
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(steps)]
    iters, outer, rels = 0, 0, []
    sync()
    if clocks:
        clocks.start()
    l0 = capi.kernel_launches()
    for q in range(steps):
        if flush is not None:
            flush.fill_(q & 0xFF)
        evs[q][0].record(stream)
        st = step()
        evs[q][1].record(stream)
        iters += st["inner_iters"]
        outer += st["outer_iters"]
        rels.append(st["rel_residual"])
    sync()
    launches = capi.kernel_launches() - l0
    clk = clocks.stop() if clocks else None
    dev_ms = sum(a.elapsed_time(b) for a, b in evs)
    if live:
        prof_iters = iters
    else:
        solver.profile(True)
        prof_iters = step()["inner_iters"]
        sync()
    prof = solver.profile_read()
    solver.profile(False)
    prof["from"] = ("the timed solves" if live else
                    "one solve after the timed region (events between column kernels would "
                    "serialise their launches)")
    return {"dev_ms": dev_ms, "iters": iters, "outer": outer, "rels": rels,
            "launches": launches, "clocks": clk, "prof": prof, "prof_iters": prof_iters}


def roofline(prof, desc, precision, precond, g, iters, periodic, kind, cut=False):
    """The dominant CG kernel's algorithmic bytes per launch over its mean event time (prof: the
    per-kernel times of one profiled solve of `iters` CG iterations)."""
    bpc = BYTES_PER_CELL[precision]
    if cut and precision != "fp64":
        bpc = BYTES_PER_CELL_CUT
    cands = [k for k in ("pcg_persistent", "cg_phase_a", "cg_phase_b") if prof[k]["launches"]]
    dom = max(cands, key=lambda k: prof[k]["ms"])
    per_launch_ms = prof[dom]["ms"] / prof[dom]["launches"]
    family = None
    if "red-black" in desc:
        bpi = BYTES_PER_CELL_RB[precision]
        family = "red-black"
    elif "A p formed" in desc:
        bpi = BYTES_PER_CELL_AP_FORMED[precision]
    elif "one-sweep" in desc:
        bpi = BYTES_PER_CELL_ONE_SWEEP[precision]
        family = "one-sweep"
    elif precond == "mg":
        bpc = dict(bpc)
        bpc["cg_phase_b"] = mg_phase_b_bytes(precision, mg_levels(g.nx, g.ny, g.nz, periodic), g.n,
                                             cut)
        bpi = bpc["cg_phase_a"] + bpc["cg_phase_b"]
    else:
        bpi = bpc["cg_phase_a"] + bpc["cg_phase_b"]  # algorithmic bytes per cell-iteration
    if dom == "pcg_persistent":
        # one launch runs every CG iteration of one inner solve
        cell_iters = g.n * iters / prof[dom]["launches"]
        alg_bytes = bpi * cell_iters
    else:
        cell_iters = g.n
        alg_bytes = bpc[dom] * g.n
    achieved = alg_bytes / (per_launch_ms * 1e-3) / 1e9
    peak, peak_kind = peaks()
    bpci = ncu_traffic(family, precision, kind, desc) if family and dom == "pcg_persistent" else None
    out = {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak,
           "peak_kind": peak_kind, "unit": "GB/s", "frac": achieved / peak,
           # DRAM bytes per launch, like alg_bytes: the measured bytes per cell-iteration times
           # the cell-iterations of an average launch
           "traffic": bpci * cell_iters if bpci is not None else None,
           "traffic_bytes_per_cell_iter": bpci,
           "alg_bytes_per_launch": alg_bytes, "alg_bytes_per_cell_iter": bpi,
           "ms_per_launch": per_launch_ms, "cell_iters_per_launch": cell_iters}
    if family in ("one-sweep", "red-black") and precision == "fp32":
        out["frac_at_face_schedule_bytes"] = (BYTES_PER_CELL_FACE_SCHEDULE[family] * cell_iters /
                                              (per_launch_ms * 1e-3) / 1e9 / peak)
    return out


def e2e_line(make_solver, F, s, g, tol, steps, warmup, dev, world, apertures=None):
    """The metric end to end through the C ABI with pinned host arrays (H2D of F, s and the
    start p, D2H of the solution inside every step)."""
    import torch
    from paper_1410_1942_gb300 import capi
    F_h = F.cpu().pin_memory()
    s_h = s.cpu().pin_memory()
    p_h = torch.zeros(g.shape, dtype=torch.float64).pin_memory()
    sv = make_solver()
    if apertures is not None:
        sv.set_apertures(*apertures)

    def step():
        # (one pinned start reused: a fresh pinned buffer per step was slower -- its pages are
        # cold for the GPU's address translation -- than zeroing this one on the host)
        p_h.zero_()
        sv.set_density(F_h)
        rc, st = sv.solve(s_h, p_h, tol)
        if rc != capi.OK:
            raise RuntimeError("e2e solve failed: %s" % capi.strerror(rc))
        return st

    for _ in range(warmup):
        step()
    torch.cuda.synchronize(dev)
    its, t0 = 0, time.perf_counter()
    for _ in range(steps):
        its += step()["inner_iters"]
    torch.cuda.synchronize(dev)
    te = time.perf_counter() - t0
    ue = float(g.n) * its
    te, ue = combine_ranks(te, ue, dev, world)
    sv.close()
    return {"value": ue / te / 1e9, "unit": "Gcell-iters/s",
            "h2d_bytes_per_step": 3 * 8 * g.n, "d2h_bytes_per_step": 8 * g.n,
            "ms_per_step": 1e3 * te / steps, "steps": steps}


def fp64_baseline(F, s, g, steps, stream):
    """Plain FP64 GPU PCG (Jacobi) on the same workload: solves/s at the same tolerance."""
    import torch
    from paper_1410_1942_gb300 import capi
    p = torch.zeros(g.shape, dtype=torch.float64, device=F.device)
    with capi.Poisson(g.nx, g.ny, g.nz, g.h, precision="fp64", stream=stream.cuda_stream) as sv:
        sv.set_density(F)
        sv.solve(s, p, TOL)  # warm-up
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        its, rel = 0, 0.0
        for _ in range(steps):
            sv.set_density(F)
            p.zero_()
            rc, st = sv.solve(s, p, TOL)
            its += st["inner_iters"]
            rel = max(rel, st["rel_residual"])
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
    return {"solves_per_s": steps / dt, "ms_per_solve": 1e3 * dt / steps,
            "gcell_iters_per_s": g.n * its / dt / 1e9, "cg_iters_per_solve": its / steps,
            "max_rel_residual": rel}


def batched(n=64, seed=0, precond="jacobi", tile=0):
    """64 independent solves of uneven size (32^3 .. 128x64x64) submitted together and driven
    by the batch executor: Jacobi handles in one persistent PCG launch per refinement step,
    multigrid handles on its worker threads (several solves at once, each on its own stream)."""
    import torch
    from paper_1410_1942_gb300 import capi, inputs
    cases = inputs.batch_cases(n, seed=seed)
    solvers, ps, rhs = [], [], []
    for c in cases:
        g = c.grid
        kw = {"inner_tol": 1e-5} if precond == "mg" else {}
        sv = capi.Poisson(g.nx, g.ny, g.nz, g.h, precision="fp32", precond=precond, tile=tile,
                          **kw)
        sv.set_density(torch.from_numpy(c.F).cuda())
        solvers.append(sv)
        rhs.append(torch.from_numpy(c.s).cuda())
        ps.append(torch.zeros(g.shape, dtype=torch.float64, device="cuda"))

    def run():
        for p in ps:
            p.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        tickets = capi.batch_submit(solvers, rhs, ps, TOL)
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
    plain FP64 PCG's and the multigrid-preconditioned solve's capacities on the same stream."""
    import math as _m
    from paper_1410_1942_gb300 import inputs, serve
    # warm the device-side input generators (torch compiles its complex kernels on first use)
    inputs.mixed_fields_t((32, 32, 32), 1, device="cuda")
    budget = 48 << 30
    cap_stream = lambda: serve.request_stream(max(4, nreq // 2), _m.inf, seed=seed + 1)
    cap = serve.Server(budget, steps=6).serve(cap_stream())
    rate = 0.7 * cap["solves_per_s"] / 20.0
    st = serve.Server(budget, steps=20).serve(serve.request_stream(nreq, rate, seed=seed))
    cap64 = serve.Server(budget, precision="fp64", steps=6).serve(cap_stream())
    # the same capacity stream and the same open-loop stream with the multigrid preconditioner
    # (unbatched handles)
    capmg = serve.Server(budget, steps=6, precond="mg").serve(cap_stream())
    stmg = serve.Server(budget, steps=20, precond="mg").serve(
        serve.request_stream(nreq, rate, seed=seed))
    return {"capacity_solves_per_s": cap["solves_per_s"], "arrival_rate_per_s": rate,
            "solves_per_s": st["solves_per_s"], "p50_ms": st["p50_ms"], "p99_ms": st["p99_ms"],
            "solves": st["solves"], "requests": nreq, "steps_per_request": 20,
            "max_rel_residual": st["max_rel_residual"], "all_ok": st["all_ok"],
            "peak_active": st["peak_active"],
            "capacity_stream": "%d requests x 6 steps, all waiting at t = 0" % max(4, nreq // 2),
            "fp64_capacity_solves_per_s": cap64["solves_per_s"],
            "fp64_p50_ms": cap64["p50_ms"], "fp64_p99_ms": cap64["p99_ms"],
            "fp64_all_ok": cap64["all_ok"],
            "mixed_vs_fp64_capacity_ratio": cap["solves_per_s"] / cap64["solves_per_s"],
            "mg_capacity_solves_per_s": capmg["solves_per_s"],
            "mg_max_rel_residual": max(capmg["max_rel_residual"], stmg["max_rel_residual"]),
            "mg_all_ok": capmg["all_ok"] and stmg["all_ok"],
            "mg_open_loop": {"solves_per_s": stmg["solves_per_s"], "p50_ms": stmg["p50_ms"],
                             "p99_ms": stmg["p99_ms"], "peak_active": stmg["peak_active"]},
            "served_tile": serve.SERVE_TILE}


def cpu_baseline(F, s, g, kind, seconds, precond):
    """The oracle as it stands on this host's cores: fixed 20-iteration PCG windows from the zero
    start on the same fields until `seconds` of CPU work have run."""
    import oracle
    oracle.build()
    op = oracle.operator(F)
    b = oracle.rhs(s, g.h)
    x = np.zeros(g.shape)
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
    return {"value": g.n * its / dt / 1e9, "unit": "Gcell-iters/s",
            "cores": oracle.threads(), "kind": "oracle",
            "sample": "%d FP64 %s-PCG iterations (windows of 20 from the zero start) of the CPU "
                      "oracle on the %s %dx%dx%d workload, %.1f s" %
                      (its, precond, kind, g.nx, g.ny, g.nz, dt)}


def solver_line(sv, F, s, g, steps, warmup, stream, precision, precond, kind, flush):
    """A secondary line (rank 0): Gcell-iters/s, solves/s and the roofline of one handle."""
    import torch
    p = torch.zeros(g.shape, dtype=torch.float64, device=F.device)
    r = timed_solves(sv, F, s, p, TOL, steps, warmup, stream, torch.cuda.synchronize, flush=flush)
    value = g.n * r["iters"] / (r["dev_ms"] * 1e-3) / 1e9
    desc = sv.describe()
    roof = roofline(r["prof"], desc, precision, precond, g, r["prof_iters"], False, kind)
    return {"value": value, "unit": "Gcell-iters/s", "precision": precision, "precond": precond,
            "solves_per_s": steps / (r["dev_ms"] * 1e-3), "ms_per_solve": r["dev_ms"] / steps,
            "cg_iters_per_solve": r["iters"] / steps, "outer_iters_per_solve": r["outer"] / steps,
            "max_rel_residual": max(r["rels"]), "kernels": desc, "steps": steps,
            "roofline_frac": roof["frac"], "roofline_kernel": roof["kernel"],
            "alg_bytes_per_cell_iter": roof["alg_bytes_per_cell_iter"]}


def extras_for(kind, args, F_d, s_d, g, stream, flush):
    import torch
    from paper_1410_1942_gb300 import capi
    out = {}

    def handle(gg, **kw):
        return capi.Poisson(gg.nx, gg.ny, gg.nz, gg.h, stream=stream.cuda_stream, **kw)

    few = max(1, min(args.steps, 2))
    if kind == "wedge":
        with handle(g, precision="bf16") as sv:
            out["wedge_bf16"] = solver_line(sv, F_d, s_d, g, few, 1, stream, "bf16", "jacobi",
                                            kind, flush)
        with handle(g, precision="fp32", precond="mg", inner_tol=1e-5) as sv:
            out["wedge_mg"] = solver_line(sv, F_d, s_d, g, few, 1, stream, "fp32", "mg", kind,
                                          flush)
        with handle(g, precision="fp32", precond="rbssor") as sv:
            out["wedge_rbssor"] = solver_line(sv, F_d, s_d, g, few, 1, stream, "fp32", "rbssor",
                                              kind, flush)
        torch.cuda.empty_cache()
        gs, Fs, ss, _ = make_fields("strut", SHAPES["strut"], args.seed, F_d.device)
    else:
        gs, Fs, ss = g, F_d, s_d
    with handle(gs, precision="fp32") as sv:
        line = solver_line(sv, Fs, ss, gs, max(1, min(args.steps, 10)), 3, stream, "fp32",
                           "jacobi", "strut", flush)
    fb = fp64_baseline(Fs, ss, gs, 2, stream)
    line["fp64_baseline"] = fb
    line["mixed_vs_fp64_solves_ratio"] = line["solves_per_s"] / fb["solves_per_s"]
    line["batched"] = batched()
    line["batched_mg"] = batched(precond="mg")
    line["served"] = served(args.serve_requests)
    out["strut"] = line
    return out


# ----------------------------------------------------------------------------- our arm
def main(argv=None):
    args = parse(argv)
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

    kind = args.case
    g, F_d, s_d, meta = make_fields(kind, args.shape, args.seed + rank, dev)
    p_d = torch.zeros(g.shape, dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream(dev)
    skw = dict(precision=args.precision, precond=args.precond, stream=stream.cuda_stream,
               tile=args.tile, dirichlet_walls=args.walls, periodic_x=args.periodic_x,
               inner_tol=args.inner_tol)
    if args.cap_iters:
        skw["max_iters"] = args.cap_iters

    def make_solver():
        return capi.Poisson(g.nx, g.ny, g.nz, g.h, **skw)

    solver = make_solver()
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

    allow = (capi.OK, capi.ENOTCONV) if args.cap_iters else (capi.OK,)
    clocks = Clocks(torch.cuda.current_device()) if rank == 0 else None
    r = timed_solves(solver, F_d, s_d, p_d, TOL, args.steps, args.warmup, stream, barrier,
                     clocks=clocks, flush=flush, allow=allow)
    units = float(g.n) * r["iters"]                     # cell-iterations of this rank
    t_max, units = combine_ranks(r["dev_ms"], units, dev, world)
    value = units / (t_max * 1e-3) / 1e9
    desc = solver.describe()
    roof = roofline(r["prof"], desc, args.precision, args.precond, g, r["prof_iters"],
                    args.periodic_x, kind, cut=args.cut_body)
    solver.close()
    del p_d

    e2e = None
    if not args.no_e2e:
        e2e = e2e_line(make_solver, F_d, s_d, g, TOL, min(args.steps, E2E_MAX_STEPS),
                       min(1, args.warmup), dev, world, apertures)

    extras = {}
    if rank == 0 and not args.no_extras and args.shape == SHAPES[kind] and not args.cap_iters:
        extras = extras_for(kind, args, F_d, s_d, g, stream, flush)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        Fh, sh = F_d.cpu().numpy(), s_d.cpu().numpy()
        del F_d, s_d
        torch.cuda.empty_cache()
        cpu = cpu_baseline(Fh, sh, g, kind, args.cpu_seconds,
                           {"rbssor": "ssor"}.get(args.precond, args.precond))

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "Gcell-iters/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": t_max / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64" if args.precision == "fp64" else "f32",
            "data": "synthetic",
            "config": {"workload": workload(kind, args.shape), "cells": g.n,
                       "precision": args.precision, "precond": args.precond, "tol": TOL,
                       "inner_tol": args.inner_tol,
                       "boundaries": ("strut as a free-slip cut-cell body, " if args.cut_body
                                      else "") + ("periodic x, " if args.periodic_x else "") +
                                     ("Dirichlet walls mask %d" % args.walls if args.walls
                                      else "zero-gradient side/bottom walls") + ", p = 0 on top",
                       "l2": ("inputs larger than L2 (%.1f GB of FP64 fields); a 256 MiB buffer "
                              "is also written between steps" % (3 * 8 * g.n / 1e9)),
                       "parallelism": "replicas" if world > 1 else "1 GPU",
                       "kernels": desc,
                       "cg_iters_per_step": r["iters"] / args.steps,
                       "outer_iters_per_step": r["outer"] / args.steps,
                       "max_rel_residual": max(r["rels"]),
                       "cap_iters": args.cap_iters or None,
                       "fields": {k: v for k, v in meta.items() if k != "modes"}},
            "hbm_gbs_algorithmic": value * roof["alg_bytes_per_cell_iter"],
            "solves_per_s": world * args.steps / (t_max * 1e-3),
            "roofline": roof,
            "kernel_times": r["prof"],
            **extras,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": r["launches"],
            "clocks": r["clocks"],
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        tdist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())

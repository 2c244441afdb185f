"""Writes tests/golden/flat32_seed0.json from the oracle alone.

The paper prints no values for the pressure solve, so the only stored expected values are these:
the FP64 oracle's solution of the 32^3 flat-surface case (seed 0, tolerance 1e-12) sampled at a
fixed set of cells, with the Jacobi and SSOR iteration counts.  They anchor the oracle across
machines (x86 build host, Arm GPU host).  Run: python tests/golden/make_golden.py
"""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import oracle  # noqa: E402
from paper_1410_1942_gb300 import inputs  # noqa: E402

SAMPLES = [(0, 0, 0), (31, 31, 31), (5, 17, 9), (16, 16, 15), (16, 16, 16), (1, 30, 31), (30, 2, 0)]


def main():
    c = inputs.flat_case(32, 32, 32, seed=0)
    out = {"case": "flat 32^3 seed 0, h = 1/32, rho 1/1000, tol 1e-12",
           "samples_ijk": SAMPLES}
    for pc in ("jacobi", "ssor"):
        res, _ = oracle.solve(c.F, c.s, c.grid.h, tol=1e-12, precond=pc)
        out[pc] = {"iters": res.iters, "rel_residual": res.rel_residual,
                   "p": [float(res.x[k, j, i]) for i, j, k in SAMPLES],
                   "l2": float(np.linalg.norm(res.x))}
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "flat32_seed0.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
    print(path)


if __name__ == "__main__":
    main()

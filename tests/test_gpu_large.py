"""The large wedge workload (1024 x 512 x 256 = 134M cells) at full size: every precision mode
reaches the tolerance under the oracle's FP64 operator, and the FP32- and BF16-coefficient
inner solves agree with each other."""
import numpy as np
import pytest

import oracle
from paper_1410_1942_gb300 import build, capi, inputs

pytestmark = pytest.mark.gpu


def test_wedge_full_size_solves():
    import torch
    assert torch.cuda.is_available()
    build.build()
    capi.load()
    grid, F, s, _ = inputs.wedge_fields_t((1024, 512, 256), seed=0, device="cuda")
    op = oracle.operator(F.cpu().numpy())
    b = oracle.rhs(s.cpu().numpy(), grid.h)
    sols = {}
    for prec in ("fp32", "bf16"):
        p = torch.zeros(grid.shape, dtype=torch.float64, device="cuda")
        with capi.Poisson(grid.nx, grid.ny, grid.nz, grid.h, precision=prec) as sv:
            sv.set_density(F)
            rc, st = sv.solve(s, p, 1e-9)
        assert rc == capi.OK, prec
        x = p.cpu().numpy()
        rel = oracle.rel_residual(op, b, x)
        assert rel <= 1e-9 * (1 + 1e-6), (prec, rel)
        assert abs(st["rel_residual"] - rel) <= 1e-3 * rel
        sols[prec] = x
        del p
        torch.cuda.empty_cache()
    d = np.linalg.norm(sols["fp32"] - sols["bf16"]) / np.linalg.norm(sols["fp32"])
    assert d <= 1e-6, d

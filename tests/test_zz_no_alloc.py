"""The allocation-free adjoint entry point against the allocating one.

fe_assemble_adjoint_noalloc serves callers that cannot let the library call
cudaMalloc (applications that own all device memory through their own pool, or
loops that must not enter the CUDA allocator). It keeps the compliance
reduction scratch in a static device array instead of the space's own buffer.
This file is collected last so that a failure here cannot hide any other test.
"""
import numpy as np
import pytest
import torch

from paper_1708_01773_gb300 import build, feasm, inputs

pytestmark = pytest.mark.gpu

CASES = [((3, 3, 3), 1, 1, "fp64"), ((2, 2, 3), 2, 1, "fp32"), ((3, 2, 2), 2, 0, "fp64"), ((16, 16, 16), 1, 1, "fp64")]


@pytest.mark.parametrize("shape,p,problem,prec", CASES)
def test_noalloc_adjoint_matches_allocating_entry(shape, p, problem, prec):
    build.build()
    assert torch.cuda.is_available()
    prob = inputs.small_problem(shape, p, problem, seed=40 + p)
    sp = feasm.FESpace(prob)
    u = torch.tensor(inputs.unit_rms_field(sp.n_dofs, 4), device="cuda")
    E = torch.tensor(prob.coef, device="cuda")
    pr = feasm.PRECISIONS[prec]
    g_ref = torch.empty(sp.n_cells, dtype=torch.float64, device="cuda")
    c_ref = torch.empty(1, dtype=torch.float64, device="cuda")
    feasm.fe_assemble_adjoint(sp.handle, u, E, 1.7, g_ref, c_ref, pr)
    for _ in range(2):
        g = torch.full((sp.n_cells,), np.nan, dtype=torch.float64, device="cuda")
        c = torch.full((1,), np.nan, dtype=torch.float64, device="cuda")
        feasm.fe_assemble_adjoint_noalloc(sp.handle, u, E, 1.7, g, c, pr)
        torch.cuda.synchronize()
        assert sp.status() == 0
        tol = 1e-12 if prec == "fp64" else 1e-6
        scale = float(g_ref.abs().max())
        assert float((g - g_ref).abs().max()) <= tol * scale
        assert abs(float(c) - float(c_ref)) <= tol * abs(float(c_ref))
    sp.close()

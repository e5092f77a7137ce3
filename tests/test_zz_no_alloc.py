"""The allocation-free adjoint entry point against the allocating one.

fe_assemble_adjoint_noalloc serves callers that cannot let the library call
cudaMalloc (applications that own all device memory through their own pool, or
loops that must not enter the CUDA allocator). It keeps the compliance
reduction scratch in a static device array instead of the space's own buffer.
Both entry points run the same kernels in the same reduction order, so their
results agree bit for bit. This file is collected last so that a failure here
cannot hide any other test.
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
    g = torch.empty(sp.n_cells, dtype=torch.float64, device="cuda")
    c = torch.empty(1, dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    for call in range(2):
        g.fill_(np.nan)
        c.fill_(np.nan)
        torch.cuda.synchronize()
        free_before = torch.cuda.mem_get_info()[0]
        feasm.fe_assemble_adjoint_noalloc(sp.handle, u, E, 1.7, g, c, pr)
        torch.cuda.synchronize()
        if call == 1:
            # after the first call (which may load the library's device code),
            # a call leaves the device's free memory unchanged
            assert torch.cuda.mem_get_info()[0] == free_before
        assert sp.status() == 0
        assert torch.equal(g, g_ref)
        assert torch.equal(c, c_ref)
    # without the compliance: the gradient alone, the same bits
    g.fill_(np.nan)
    feasm.fe_assemble_adjoint_noalloc(sp.handle, u, None, 1.7, g, None, pr)
    torch.cuda.synchronize()
    assert sp.status() == 0
    assert torch.equal(g, g_ref)
    sp.close()


def test_noalloc_adjoint_empty_mesh():
    build.build()
    mesh = inputs.Mesh(np.zeros((0, 3)), np.zeros((0, 8), dtype=np.int32), (0, 0, 0), (1, 1, 1))
    prob = inputs.Problem("empty", mesh, 1, 2, 1, np.zeros(0), np.array([0.0, 0.0, -1.0]))
    sp = feasm.FESpace(prob)
    c = torch.full((1,), np.nan, dtype=torch.float64, device="cuda")
    empty = torch.zeros(0, dtype=torch.float64, device="cuda")
    feasm.fe_assemble_adjoint_noalloc(sp.handle, empty, empty, 1.0, empty, c, feasm.FE_PREC_FP64)
    torch.cuda.synchronize()
    assert float(c) == 0.0
    sp.close()


def test_noalloc_adjoint_in_a_cuda_graph():
    """The allocation-free entry point captured into a CUDA graph (global capture
    mode, where an allocation would end the capture with an error) and replayed
    gives the allocating entry point's gradient and compliance bit for bit."""
    build.build()
    prob = inputs.small_problem((6, 5, 4), 1, 1, seed=44)
    sp = feasm.FESpace(prob)
    u = torch.tensor(inputs.unit_rms_field(sp.n_dofs, 5), device="cuda")
    E = torch.tensor(prob.coef, device="cuda")
    pr = feasm.PRECISIONS["fp64"]
    g_ref = torch.empty(sp.n_cells, dtype=torch.float64, device="cuda")
    c_ref = torch.empty(1, dtype=torch.float64, device="cuda")
    feasm.fe_assemble_adjoint(sp.handle, u, E, 1.3, g_ref, c_ref, pr)
    g = torch.empty_like(g_ref)
    c = torch.empty_like(c_ref)
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):  # warm-up outside the capture
        feasm.fe_assemble_adjoint_noalloc(sp.handle, u, E, 1.3, g, c, pr, side)
    torch.cuda.current_stream().wait_stream(side)
    torch.cuda.synchronize()
    g.fill_(np.nan)
    c.fill_(np.nan)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, capture_error_mode="global"):
        feasm.fe_assemble_adjoint_noalloc(sp.handle, u, E, 1.3, g, c, pr, torch.cuda.current_stream())
    graph.replay()
    torch.cuda.synchronize()
    assert sp.status() == 0
    assert torch.equal(g, g_ref)
    assert torch.equal(c, c_ref)
    sp.close()

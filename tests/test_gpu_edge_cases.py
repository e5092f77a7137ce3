"""GPU edge cases of the constrained, Stokes and DG paths: every DOF fixed
(an empty system), nothing fixed (the unconstrained system, bit for bit), a
single cell (DG: boundary facets only; Stokes), an empty mesh; the largest
single mesh of the batched recipe (Q3 elasticity on 40^3 cells: more
contributions than an int32 can index); and for every cell kernel void cells
(zero and 1e-9 coefficients) on a strongly distorted mesh, and flat cells of
aspect ratio ~1e-3."""
import dataclasses

import numpy as np
import pytest
import torch

import oracle
from metrics import TOL, row_scaled_error, vec_error
from paper_1708_01773_gb300 import build, feasm, inputs
from test_gpu_parity import check_all_kernels, check_rows, sampled_rows

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    feasm.lib()


def test_dirichlet_everything_and_nothing_fixed():
    prob = inputs.small_problem((3, 2, 2), 1, 1, seed=900)
    sp = feasm.FESpace(prob)
    coef = torch.tensor(prob.coef, device="cuda")
    full = sp.dirichlet(np.ones(sp.n_dofs, dtype=bool))
    assert (full.n_free, full.nnz) == (0, 0)
    uD = torch.ones(full.n_fixed, dtype=torch.float64, device="cuda")
    v, r = full.assemble(coef, uD, values=torch.empty(1, dtype=torch.float64, device="cuda"),
                         rhs=torch.empty(1, dtype=torch.float64, device="cuda"), prec="fp32")
    torch.cuda.synchronize()
    assert sp.status() == 0
    none = sp.dirichlet(np.zeros(sp.n_dofs, dtype=bool))
    for prec in ("fp32", "fp64"):
        v0, r0 = none.assemble(coef, None, prec=prec)
        v1, r1 = sp.assemble(coef, prec=prec)
        torch.cuda.synchronize()
        assert torch.equal(v0, v1) and torch.equal(r0, r1), prec
    full.close(); none.close(); sp.close()


@pytest.mark.parametrize("p", [1, 2, 3])
def test_dg_single_cell(p):
    mesh = inputs.small_problem((1, 1, 1), p, 0, seed=910 + p).mesh
    g = feasm.DGSpace(mesh, p)
    assert g.n_interior == 0 and g.n_boundary == 6
    rp_o, col_o, val_o, rhs_o = oracle.dg_assemble(mesh, p, 1.0, 6.0, 2.0)
    for prec in ("fp64", "fp32"):
        vals, rhs = g.assemble(1.0, 6.0, 2.0, prec=prec)
        torch.cuda.synchronize()
        assert row_scaled_error(rp_o, col_o, vals.cpu().numpy(), val_o) <= TOL[prec], prec
        assert vec_error(rhs.cpu().numpy(), rhs_o) <= 1e-12
    g.close()


def test_stokes_single_cell():
    prob = inputs.small_problem((1, 1, 1), 2, inputs.STOKES, seed=920)
    cd_o, n_o, nv = oracle.stokes_dof_numbering(prob.mesh, 2)
    rp_o, col_o, val_o, rhs_o = oracle.assemble_csr(prob, cd_o, n_o)
    sp = feasm.FESpace(prob)
    assert (sp.n_dofs, sp.n_first) == (n_o, nv) == (89, 81)
    np.testing.assert_array_equal(sp.cell_dofs(), cd_o)
    coef = torch.tensor(prob.coef, device="cuda")
    for prec in ("fp64", "fp32"):
        vals, rhs = sp.assemble(coef, prec=prec)
        torch.cuda.synchronize()
        assert row_scaled_error(rp_o, col_o, vals.cpu().numpy(), val_o) <= TOL[prec], prec
        assert sp.status() == 0
        assert vec_error(rhs.cpu().numpy(), rhs_o) <= 1e-12
    sp.close()


def test_empty_mesh_dg_and_dirichlet():
    mesh = inputs.Mesh(np.zeros((0, 3)), np.zeros((0, 8), dtype=np.int32), (0, 0, 0), (1.0, 1.0, 1.0))
    g = feasm.DGSpace(mesh, 2)
    assert (g.n_dofs, g.nnz, g.n_interior, g.n_boundary) == (0, 0, 0, 0)
    g.assemble(1.0, 5.0, 1.0, values=torch.empty(1, dtype=torch.float64, device="cuda"),
               rhs=torch.empty(1, dtype=torch.float64, device="cuda"))
    torch.cuda.synchronize()
    g.close()


def test_maximum_size_q3_elasticity_int64():
    """Q3 elasticity on 40^3 cells (5.3M DOFs, 1.95e9 nonzeros, 2.36e9
    contributions: 64-bit positions throughout), FP32 form: sampled rows,
    the last ones included, against the oracle."""
    prob = inputs.small_problem((40, 40, 40), 3, inputs.ELASTICITY, seed=950)
    sp = feasm.FESpace(prob)
    assert sp.n_contrib > 2 ** 31 and sp.nnz > 2 ** 30
    coef = torch.tensor(prob.coef, device="cuda")
    vals, rhs = sp.assemble(coef, prec="fp32")
    torch.cuda.synchronize()
    assert sp.status() == 0
    check_rows(prob, sp, vals.cpu().numpy(), rhs.cpu().numpy(), "fp32", sampled_rows(sp.n_dofs, k=12))
    sp.close()


SHAPES = {1: (4, 4, 3), 2: (3, 3, 2), 3: (2, 2, 2)}


@pytest.mark.parametrize("p,problem", [(1, 0), (1, 1), (2, 0), (2, 1), (3, 0), (3, 1)])
def test_void_cells_on_a_strongly_distorted_mesh(p, problem):
    """SIMP-like coefficients: half the cells at 1e-9 of their value and a fifth
    exactly zero (void cells have zero cell matrices; rows inside the void are
    zero, and the row-scaled comparison then demands exact zeros), on a mesh
    whose interior vertices move by up to 0.3h per coordinate. Every entry of
    every kernel and precision against the oracle."""
    prob = inputs.small_problem(SHAPES[p], p, problem, alpha=0.3, seed=120 + 2 * p + problem)
    assert oracle.min_det_jacobian(prob.mesh, prob.quad_1d) > 0
    rng = np.random.default_rng(130 + 2 * p + problem)
    coef = np.where(rng.random(prob.mesh.n_cells) < 0.5, 1e-9, 1.0) * prob.coef
    coef[rng.random(prob.mesh.n_cells) < 0.2] = 0.0
    assert (coef == 0).any() and (coef > 0.5).any()
    check_all_kernels(dataclasses.replace(prob, coef=coef))


@pytest.mark.parametrize("p,problem", [(1, 1), (2, 0), (2, 1), (3, 1)])
def test_flat_cells(p, problem):
    """Cells of aspect ratio ~1e-3 (a 1 x 1 x 1e-3 slab, interior shifts up to
    0.2h_d): cofactors and 1/det J span six orders of magnitude before their
    rounding to FP32. Every entry of every kernel and precision against the oracle."""
    prob = inputs.small_problem(SHAPES[p], p, problem, seed=140 + 2 * p + problem, extent=(1.0, 1.0, 1e-3))
    assert oracle.min_det_jacobian(prob.mesh, prob.quad_1d) > 0
    check_all_kernels(prob)

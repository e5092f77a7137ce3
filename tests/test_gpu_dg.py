"""GPU parity of the interior penalty DG assembly (fe_dg_assemble) against the
oracle: every entry and the RHS on small meshes (p = 1..3, rotated cell
orderings, tau = 1 and -1, FP64/FP32/BF16 forms: geometry FP64 in every form,
facet products and blocks FP64 in the FP64 form and FP32 in the FP32 and BF16
forms), every entry on meshes large enough that each persistent facet block
takes several facets and each block-row block several cells, and at the 32^3
Q2 size the consistency property (a linear u gives zero rows away from the
boundary), SIPG symmetry and determinism."""
import numpy as np
import pytest
import torch

import oracle
from metrics import TOL, csr_matvec, row_scaled_error, vec_error
from paper_1708_01773_gb300 import build, feasm, inputs
from test_oracle_pins import dg_node_positions, rotated_mesh

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    feasm.lib()


@pytest.mark.parametrize("p,shape,rotate", [(1, (4, 3, 2), False), (2, (3, 2, 2), True), (3, (2, 2, 2), True)])
def test_small_dg_meshes(p, shape, rotate):
    mesh = inputs.small_problem(shape, p, 0, seed=800 + p).mesh
    if rotate:
        mesh = rotated_mesh(mesh, 810 + p)
    g = feasm.DGSpace(mesh, p)
    rp, col = g.pattern()
    for tau in (1.0, -1.0):
        rp_o, col_o, val_o, rhs_o = oracle.dg_assemble(mesh, p, tau, 8.0, 1.5)
        np.testing.assert_array_equal(rp.cpu().numpy(), rp_o)
        np.testing.assert_array_equal(col.cpu().numpy(), col_o)
        for prec in ("fp64", "fp32", "bf16"):
            vals, rhs = g.assemble(tau, 8.0, 1.5, prec=prec)
            torch.cuda.synchronize()
            v = vals.cpu().numpy()
            assert row_scaled_error(rp_o, col_o, v, val_o) <= TOL[prec], (tau, prec)
            assert vec_error(rhs.cpu().numpy(), rhs_o) <= 1e-12
    g.close()


@pytest.mark.parametrize("p", [1, 2, 3])
def test_dg_o_grid(p):
    """IP-DG on an O-grid (facets between cells of irregular valence, a curved
    polygonal outer boundary): pattern and every entry against the oracle, both
    tau, three forms."""
    mesh = inputs.o_grid(3, 2, 2)
    g = feasm.DGSpace(mesh, p)
    rp, col = g.pattern()
    for tau in (1.0, -1.0):
        rp_o, col_o, val_o, rhs_o = oracle.dg_assemble(mesh, p, tau, 8.0, 1.5)
        np.testing.assert_array_equal(rp.cpu().numpy(), rp_o)
        np.testing.assert_array_equal(col.cpu().numpy(), col_o)
        for prec in ("fp64", "fp32", "bf16"):
            vals, rhs = g.assemble(tau, 8.0, 1.5, prec=prec)
            torch.cuda.synchronize()
            assert row_scaled_error(rp_o, col_o, vals.cpu().numpy(), val_o) <= TOL[prec], (tau, prec)
            assert vec_error(rhs.cpu().numpy(), rhs_o) <= 1e-12
    g.close()


@pytest.mark.parametrize("p,n,taus", [(2, 14, (1.0, -1.0)), (1, 16, (1.0, -1.0)), (3, 11, (1.0,))])
def test_dg_every_entry_with_several_facets_per_block(p, n, taus):
    """Rotated n^3 meshes: k_dg_facets runs one wave of at most 152 x 16 resident
    blocks over (3 (n-1) + 6) n^2 facets (p = 2: 8,820 facets, at least 3.6 per block
    at any occupancy), so every block forms the point data of its next facet on
    the helper warp while the current one is reduced (the double buffer); k_dg_rows
    runs at most 1,216 blocks over n^3 cells (p = 1: 4,096 cells, p = 2: 2,744), so
    blocks loop over cells. Every entry and the RHS against the oracle, three forms."""
    mesh = inputs.small_problem((n, n, n), p, 0, seed=900 + p).mesh
    mesh = rotated_mesh(mesh, 910 + p)
    g = feasm.DGSpace(mesh, p)
    assert g.n_interior + g.n_boundary == (3 * (n - 1) + 6) * n * n
    rp, col = g.pattern()
    for tau in taus:
        rp_o, col_o, val_o, rhs_o = oracle.dg_assemble(mesh, p, tau, 8.0, 1.5)
        np.testing.assert_array_equal(rp.cpu().numpy(), rp_o)
        np.testing.assert_array_equal(col.cpu().numpy(), col_o)
        for prec in ("fp64", "fp32", "bf16"):
            vals, rhs = g.assemble(tau, 8.0, 1.5, prec=prec)
            torch.cuda.synchronize()
            v = vals.cpu().numpy()
            assert row_scaled_error(rp_o, col_o, v, val_o) <= TOL[prec], (tau, prec)
            assert vec_error(rhs.cpu().numpy(), rhs_o) <= 1e-12
    g.close()


def test_dg_q2_32_consistency_symmetry_determinism():
    mesh = inputs.dg_q2_32()
    g = feasm.DGSpace(mesh, 2)
    assert g.n_interior == 3 * 31 * 32 * 32 and g.n_boundary == 6 * 32 * 32
    rp, col = g.pattern()
    n = g.n_dofs
    x = dg_node_positions(mesh, 2)
    u = torch.tensor(0.3 + x @ np.array([1.2, -0.8, 0.5]), device="cuda")
    # cells with no boundary face: their rows of A u vanish for a linear u (f = 0)
    c = np.arange(mesh.n_cells)
    ix, iy, iz = c % 32, (c // 32) % 32, c // 1024
    inner = (ix > 0) & (ix < 31) & (iy > 0) & (iy < 31) & (iz > 0) & (iz < 31)
    rows = torch.tensor(np.repeat(inner, 27), device="cuda")
    for prec in ("fp64", "fp32"):
        vals, rhs = g.assemble(1.0, 10.0, 0.0, prec=prec)
        v2, _ = g.assemble(1.0, 10.0, 0.0, prec=prec)
        torch.cuda.synchronize()
        assert torch.equal(vals, v2)
        A = torch.sparse_csr_tensor(rp, col.to(torch.int64), vals, size=(n, n))
        r = torch.mv(A, u)
        scale = float(torch.mv(torch.sparse_csr_tensor(rp, col.to(torch.int64), vals.abs(), size=(n, n)),
                               u.abs()).max())
        assert float(r[rows].abs().max()) <= 4 * TOL[prec] * scale, prec
        if prec == "fp64":
            # symmetry on sampled rows: A[i, j] == A[j, i]
            rpn, coln, vn = rp.cpu().numpy(), col.cpu().numpy(), vals.cpu().numpy()
            rng = np.random.default_rng(3)
            for i in rng.integers(0, n, 64):
                for k in range(rpn[i], rpn[i + 1], 7):
                    j = coln[k]
                    kk = rpn[j] + np.searchsorted(coln[rpn[j]:rpn[j + 1]], i)
                    assert coln[kk] == i and abs(vn[kk] - vn[k]) <= 1e-14 * abs(vn[rpn[i]:rpn[i + 1]]).max()
    g.close()

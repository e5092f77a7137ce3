"""GPU parity of the Stokes (Taylor-Hood) assembly through the C ABI against the
oracle: every entry on small meshes (Q2/Q1 and Q3/Q2, FP64 and FP32 forms), the
energy error on the velocity block (the full matrix is indefinite: vectors with
zero pressure part), the RHS; sampled rows of the 32^3 Q2/Q1 workload in the
launch configuration the benchmark times; a constrained (lid-driven cavity)
system; and the combinations that are reported as unsupported."""
import numpy as np
import pytest
import torch

import oracle
from metrics import TOL, csr_matvec, row_scaled_error, vec_error
from paper_1708_01773_gb300 import build, feasm, inputs
from test_gpu_dirichlet import lift_scale

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    feasm.lib()


def velocity_energy_error(rp, col, val, val_ref, nv, seed=0, n_vec=8):
    rng = np.random.default_rng(seed)
    n = rp.size - 1
    worst = 0.0
    for _ in range(n_vec):
        v = np.zeros(n)
        v[:nv] = rng.standard_normal(nv)
        num = abs(v @ csr_matvec(rp, col, val - val_ref, v))
        den = v @ csr_matvec(rp, col, val_ref, v)
        worst = max(worst, num / den)
    return worst


@pytest.mark.parametrize("shape,p,scramble", [((3, 3, 2), 2, False), ((4, 2, 3), 2, False), ((2, 2, 2), 3, False),
                                              ((3, 2, 2), 2, True), ((2, 2, 2), 3, True)])
def test_small_stokes_meshes(shape, p, scramble):
    prob = inputs.small_problem(shape, p, inputs.STOKES, seed=700 + p)
    if scramble:  # random vertex ids and cell order, rotated local vertex orders
        prob = inputs.scrambled(prob, seed=710 + p)
    check_stokes(prob)


@pytest.mark.parametrize("p", [2, 3])
def test_stokes_o_grid(p):
    """Taylor-Hood on an O-grid (irregular vertex valence)."""
    check_stokes(inputs.o_grid_problem(3, 2, 2, p, inputs.STOKES, seed=720 + p))


def check_stokes(prob):
    p = prob.order
    cd_o, n_o, nv = oracle.stokes_dof_numbering(prob.mesh, p)
    rp_o, col_o, val_o, rhs_o = oracle.assemble_csr(prob, cd_o, n_o)
    sp = feasm.FESpace(prob)
    assert sp.n_dofs == n_o and sp.n_first == nv
    np.testing.assert_array_equal(sp.cell_dofs(), cd_o)
    rp, col = sp.pattern()
    np.testing.assert_array_equal(rp.cpu().numpy(), rp_o)
    np.testing.assert_array_equal(col.cpu().numpy(), col_o)
    coef = torch.tensor(prob.coef, device="cuda")
    for prec in ("fp64", "fp32"):
        vals, rhs = sp.assemble(coef, prec=prec)
        torch.cuda.synchronize()
        assert sp.status() == 0
        v, b = vals.cpu().numpy(), rhs.cpu().numpy()
        assert row_scaled_error(rp_o, col_o, v, val_o) <= TOL[prec], prec
        assert velocity_energy_error(rp_o, col_o, v, val_o, nv) <= TOL[prec], prec
        assert vec_error(b, rhs_o) <= 1e-12
        assert np.all(b[nv:] == 0)
    sp.close()


def test_stokes_q2q1_32_full_size():
    """32^3 cells, 823,875 velocity + 35,937 pressure DOFs: sampled velocity and
    pressure rows against the oracle, both forms; rigid velocity translations in
    the kernel of the GPU matrix."""
    prob = inputs.stokes_q2q1_32()
    sp = feasm.FESpace(prob)
    nv = sp.n_first
    assert nv == 3 * 65 ** 3 and sp.n_dofs == nv + 33 ** 3
    coef = torch.tensor(prob.coef, device="cuda")
    rng = np.random.default_rng(9)
    rows = np.unique(np.concatenate([[0, nv - 1, nv, sp.n_dofs - 1], rng.integers(0, nv, 32),
                                     rng.integers(nv, sp.n_dofs, 16)])).astype(np.int64)
    cd = sp.cell_dofs()
    ptr, col_o, val_o, rhs_o = oracle.assemble_rows(prob, rows, cd, sp.n_dofs)
    rp, col = sp.pattern_host()
    rpd, cold = sp.pattern()
    for prec in ("fp32", "fp64"):
        vals, rhs = sp.assemble(coef, prec=prec)
        torch.cuda.synchronize()
        assert sp.status() == 0
        v, b = vals.cpu().numpy(), rhs.cpu().numpy()
        worst = 0.0
        for q, r in enumerate(rows):
            np.testing.assert_array_equal(col[rp[r]:rp[r + 1]], col_o[ptr[q]:ptr[q + 1]])
            ref = val_o[ptr[q]:ptr[q + 1]]
            worst = max(worst, np.abs(v[rp[r]:rp[r + 1]] - ref).max() / np.abs(ref).max())
        assert worst <= TOL[prec], (prec, worst)
        assert np.abs(b[rows] - rhs_o).max() <= 1e-12 * np.abs(rhs_o).max()
        A = torch.sparse_csr_tensor(rpd, cold.to(torch.int64), vals, size=(sp.n_dofs, sp.n_dofs))
        for c in range(3):
            t = torch.zeros(sp.n_dofs, dtype=torch.float64, device="cuda")
            t[c:nv:3] = 1.0
            assert float(torch.mv(A, t).abs().max() / vals.abs().max()) <= 8 * TOL[prec]
    sp.close()


def test_stokes_lid_driven_cavity_constrained():
    """Every velocity DOF on the boundary fixed (the lid z = 1 moves with (1, 0, 0),
    the rest at rest) and one pressure DOF fixed: the constrained system against
    the oracle's, entry by entry, both forms."""
    prob = inputs.small_problem((3, 3, 3), 2, inputs.STOKES, seed=710)
    sp = feasm.FESpace(prob)
    nv = sp.n_first
    pos = sp.dof_points()
    comp = np.arange(sp.n_dofs) % 3
    on_bnd = np.any((np.abs(pos) < 1e-12) | (np.abs(pos - 1.0) < 1e-12), axis=1)
    fixed = np.zeros(sp.n_dofs, dtype=bool)
    fixed[:nv] = on_bnd[:nv]
    fixed[nv] = True
    u_full = np.zeros(sp.n_dofs)
    lid = (np.abs(pos[:, 2] - 1.0) < 1e-12) & (comp == 0)
    u_full[:nv][lid[:nv]] = 1.0
    cd = sp.cell_dofs()
    rp_o, col_o, val_o, rhs_o = oracle.assemble_csr(prob, cd, sp.n_dofs)
    ptr_r, col_r, val_r, rhs_r = oracle.dirichlet_reduce(rp_o, col_o, val_o, rhs_o, fixed, u_full[fixed])
    dsys = sp.dirichlet(fixed)
    rp, col = dsys.pattern_host()
    np.testing.assert_array_equal(rp, ptr_r)
    np.testing.assert_array_equal(col, col_r)
    coef = torch.tensor(prob.coef, device="cuda")
    uD = torch.tensor(u_full[fixed], device="cuda")
    for prec in ("fp64", "fp32"):
        vals, rhs = dsys.assemble(coef, uD, prec=prec)
        torch.cuda.synchronize()
        assert row_scaled_error(ptr_r, col_r, vals.cpu().numpy(), val_r) <= TOL[prec]
        scale = lift_scale(rp_o, col_o, val_o, rhs_o, fixed, u_full).max()
        assert np.abs(rhs.cpu().numpy() - rhs_r).max() <= TOL[prec] * scale
    dsys.close()
    sp.close()


def test_stokes_unsupported_combinations_are_reported():
    prob = inputs.small_problem((2, 2, 2), 2, inputs.STOKES, seed=720)
    sp = feasm.FESpace(prob)
    coef = torch.tensor(prob.coef, device="cuda")
    with pytest.raises(feasm.FEError) as ei:
        sp.assemble(coef, prec="bf16")
    assert ei.value.code == -6
    u = torch.zeros(sp.n_dofs, dtype=torch.float64, device="cuda")
    with pytest.raises(feasm.FEError):
        sp.adjoint(u, coef)
    with pytest.raises(feasm.FEError):
        feasm.fe_batch_create([sp.handle])
    with pytest.raises(feasm.FEError):
        feasm.fe_space_create(prob.mesh.coords, prob.mesh.cell_vertices, 1, 0, inputs.STOKES, 0.0)
    sp.close()

"""GPU parity: the CUDA path through the C ABI against the FP64 oracle.

Small meshes are compared entry by entry (several tiles and a ragged tail per
kernel); the paper-shaped full-size workloads are compared on sampled rows the
oracle computes one by one, plus invariants that hold at any size.
"""
import numpy as np
import pytest
import torch

import oracle
from metrics import TOL, TOL_TC_Q3_ELASTICITY_FP32, energy_error, row_scaled_error, vec_error
from paper_1708_01773_gb300 import build, feasm, inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    feasm.lib()


def run(sp, prob, prec):
    coef = torch.tensor(prob.coef, device="cuda")
    vals, rhs = sp.assemble(coef, prec=prec)
    torch.cuda.synchronize()
    assert sp.status() == 0
    return vals.cpu().numpy(), rhs.cpu().numpy()


SMALL = [((3, 3, 3), 1, 0), ((3, 3, 3), 1, 1), ((3, 2, 3), 2, 0), ((3, 2, 2), 2, 1), ((2, 3, 2), 3, 0),
         ((2, 2, 2), 3, 1), ((5, 1, 1), 2, 1)]


@pytest.mark.parametrize("shape,p,problem", SMALL)
def test_small_meshes_all_precisions(shape, p, problem):
    check_all_kernels(inputs.small_problem(shape, p, problem, seed=10 * p + problem))


# Scrambled bricks: Q1 on 60 cells (two tiles of the Q1 elasticity kernel, the
# second ragged), Q2 and Q3 on several cells per persistent tensor-core CTA pass
SCRAMBLED = [((5, 4, 3), 1, 0), ((5, 4, 3), 1, 1), ((3, 3, 2), 2, 0), ((3, 3, 2), 2, 1), ((2, 2, 3), 3, 0),
             ((2, 2, 2), 3, 1)]


@pytest.mark.parametrize("shape,p,problem", SCRAMBLED)
def test_unstructured_numbering_all_kernels(shape, p, problem):
    """The small-mesh check on scrambled bricks: random vertex ids and cell
    order, every cell's local vertex order turned by a random proper rotation of
    the reference cube. The DOF numbering and pattern bit for bit, every entry of
    every kernel and precision, and the RHS against the oracle on the same mesh."""
    base = inputs.small_problem(shape, p, problem, seed=60 + 10 * p + problem)
    check_all_kernels(inputs.scrambled(base, seed=70 + 10 * p + problem))


@pytest.mark.parametrize("p,problem", [(1, 0), (1, 1), (2, 0), (2, 1), (3, 0), (3, 1)])
def test_o_grid_all_kernels(p, problem):
    """An O-grid (66 cells; six cells around the inner square's corner vertices,
    three on the end faces, eight elsewhere): numbering, pattern, every entry of
    every kernel and precision and the RHS against the oracle."""
    check_all_kernels(inputs.o_grid_problem(3, 2, 2, p, problem, seed=40 + 2 * p + problem))


@pytest.mark.parametrize("p,problem", [(1, 0), (1, 1), (2, 0), (2, 1), (3, 0)])
def test_flower_all_kernels(p, problem):
    """A flower mesh (34 cells around its axis vertex between the two layers:
    more than 32 cells around a DOF, so the scatter takes its general path, not
    the slot-wise one): every kernel and precision against the oracle; the
    batched driver refuses the space."""
    prob = inputs.o_grid_problem(0, 0, 0, p, problem, seed=50 + 2 * p + problem, mesh=inputs.flower(17, 2))
    check_all_kernels(prob)
    sp = feasm.FESpace(prob)
    with pytest.raises(feasm.FEError):
        feasm.fe_batch_create([sp.handle])
    sp.close()


@pytest.mark.parametrize("p,problem", [(1, 1), (2, 1)])
def test_locality_ordered_mesh_all_kernels(p, problem):
    """A scrambled brick given in the cell order of fe_mesh_locality_order (the
    order bench.py --reorder uses): the same checks against the oracle."""
    scr = inputs.scrambled(inputs.small_problem((5, 4, 3), p, problem, seed=90 + p), seed=91 + p)
    order = feasm.fe_mesh_locality_order(scr.mesh.coords, scr.mesh.cell_vertices)
    check_all_kernels(inputs.reordered(scr, order))


def check_all_kernels(prob):
    p, problem = prob.order, prob.problem
    shape = prob.mesh.shape or prob.mesh.n_cells
    cd, n = oracle.dof_numbering(prob.mesh, p, prob.ncomp)
    rp_o, col_o, val_o, rhs_o = oracle.assemble_csr(prob, cd, n)
    sp = feasm.FESpace(prob)
    np.testing.assert_array_equal(sp.cell_dofs(), cd)
    rp, col = sp.pattern()
    np.testing.assert_array_equal(rp.cpu().numpy(), rp_o)
    np.testing.assert_array_equal(col.cpu().numpy(), col_o)
    kernels = ["cuda_core", "tensor_core"] if p >= 2 else ["auto", "cuda_core"]
    for kern in kernels:
        sp.set_kernel(kern)
        for prec in ("fp64", "fp32", "bf16"):
            if kern == "tensor_core" and prec == "fp64":
                continue
            vals, rhs = run(sp, prob, prec)
            e_inf = row_scaled_error(rp_o, col_o, vals, val_o)
            e_en = energy_error(rp_o, col_o, vals, val_o)
            tol = TOL[prec]
            if kern == "tensor_core" and (p, problem, prec) == (3, 1, "fp32"):
                tol = TOL_TC_Q3_ELASTICITY_FP32
            print(f"{shape} p{p} problem {problem} {kern} {prec}: entry {e_inf:.3e} energy {e_en:.3e}")
            assert e_inf <= tol, (kern, prec, e_inf)
            assert e_en <= tol, (kern, prec, e_en)
            assert vec_error(rhs, rhs_o) <= 1e-12
    sp.close()


def test_tensor_core_pipeline_wraps():
    """Q2 elasticity on 768 cells: every persistent CTA of the tensor-core kernel takes
    five or six cells, so the geometry slots (4) and operand/accumulator stages (2)
    are all reused; every entry is compared with the oracle."""
    prob = inputs.small_problem((12, 8, 8), 2, 1, seed=21)
    rp_o, col_o, val_o, rhs_o = oracle.assemble_csr(prob)
    sp = feasm.FESpace(prob)
    sp.set_kernel("tensor_core")
    for prec in ("fp32", "bf16"):
        vals, rhs = run(sp, prob, prec)
        assert row_scaled_error(rp_o, col_o, vals, val_o) <= TOL[prec], prec
        assert energy_error(rp_o, col_o, vals, val_o) <= TOL[prec], prec
        assert vec_error(rhs, rhs_o) <= 1e-12
    sp.close()


def test_elasticity_q3_tensor_core_cells_wrap():
    """Q3 elasticity on the tensor cores, 210 cells: more cells than CTAs, so
    each persistent CTA runs several MMA rounds on the same operand stages and
    tensor memory; every entry against the oracle, the CUDA-core kernel on the
    same space, and run-to-run bitwise reproducibility."""
    prob = inputs.small_problem((7, 6, 5), 3, 1, seed=33)
    rp_o, col_o, val_o, rhs_o = oracle.assemble_csr(prob)
    sp = feasm.FESpace(prob)
    for kern in ("tensor_core", "cuda_core"):
        sp.set_kernel(kern)
        for prec in ("fp32", "bf16"):
            vals, rhs = run(sp, prob, prec)
            e_inf = row_scaled_error(rp_o, col_o, vals, val_o)
            e_en = energy_error(rp_o, col_o, vals, val_o)
            print(f"Q3 elasticity 7x6x5 {kern} {prec}: entry {e_inf:.3e} energy {e_en:.3e}")
            tol = TOL_TC_Q3_ELASTICITY_FP32 if (kern, prec) == ("tensor_core", "fp32") else TOL[prec]
            assert e_inf <= tol, (kern, prec, e_inf)
            assert e_en <= tol, (kern, prec, e_en)
            assert vec_error(rhs, rhs_o) <= 1e-12
            if kern == "tensor_core":
                again, rhs2 = run(sp, prob, prec)
                assert np.array_equal(vals, again) and np.array_equal(rhs, rhs2)
    sp.close()


@pytest.mark.parametrize("shape,p", [((15, 13, 11), 2), ((11, 9, 7), 3)])
def test_poisson_tensor_core_tiles_wrap(shape, p):
    """Poisson Q2 (4 cells per 128-row tile) and Q3 (2 cells per tile) on the
    tensor cores: 2,145 and 693 cells, i.e. more tiles than CTAs (each persistent
    CTA loops over several tiles, reusing both operand stages and its tensor
    memory) and a ragged last tile; every entry against the oracle, the general
    CUDA-core kernel on the same space, and run-to-run bitwise reproducibility."""
    prob = inputs.small_problem(shape, p, 0, seed=30 + p)
    rp_o, col_o, val_o, rhs_o = oracle.assemble_csr(prob)
    sp = feasm.FESpace(prob)
    for kern in ("tensor_core", "cuda_core"):
        sp.set_kernel(kern)
        for prec in ("fp32", "bf16"):
            vals, rhs = run(sp, prob, prec)
            assert row_scaled_error(rp_o, col_o, vals, val_o) <= TOL[prec], (kern, prec)
            assert energy_error(rp_o, col_o, vals, val_o) <= TOL[prec], (kern, prec)
            assert vec_error(rhs, rhs_o) <= 1e-12
            if kern == "tensor_core":
                again, rhs2 = run(sp, prob, prec)
                assert np.array_equal(vals, again) and np.array_equal(rhs, rhs2)
    sp.close()


def test_poisson_q1_8_full():
    prob = inputs.poisson_q1_8()
    rp_o, col_o, val_o, rhs_o = oracle.assemble_csr(prob)
    sp = feasm.FESpace(prob)
    for prec in ("fp64", "fp32", "bf16"):
        vals, rhs = run(sp, prob, prec)
        assert row_scaled_error(rp_o, col_o, vals, val_o) <= TOL[prec]
        assert energy_error(rp_o, col_o, vals, val_o) <= TOL[prec]
        assert vec_error(rhs, rhs_o) <= 1e-12
    sp.close()


def test_bitwise_deterministic():
    prob = inputs.small_problem((4, 3, 3), 2, 1, seed=3)
    sp = feasm.FESpace(prob)
    coef = torch.tensor(prob.coef, device="cuda")
    for kern in ("cuda_core", "auto"):
        sp.set_kernel(kern)
        for prec in ("fp64", "fp32", "bf16"):
            a, ra = sp.assemble(coef, prec=prec)
            b, rb = sp.assemble(coef, prec=prec)
            assert torch.equal(a, b) and torch.equal(ra, rb)
    sp.close()


def test_exact_accumulation_matches_fp64_sum_of_cell_matrices():
    """The FP64 path sums the FP64 cell-matrix entries of each nonzero exactly (integer
    fixed point) before one rounding; the oracle sums them in plain FP64. On a mesh with
    up to 8 terms per entry the two differ only by the oracle's rounding (~1e-16)."""
    prob = inputs.small_problem((3, 3, 3), 1, 0, seed=9)
    cd, n = oracle.dof_numbering(prob.mesh, 1, 1)
    rp_o, col_o, val_o, _ = oracle.assemble_csr(prob, cd, n)
    sp = feasm.FESpace(prob)
    vals, _ = run(sp, prob, "fp64")
    assert row_scaled_error(rp_o, col_o, vals, val_o) <= 1e-14
    sp.close()


def sampled_rows(n, k=48, seed=0):
    rng = np.random.default_rng(seed)
    rows = np.unique(np.concatenate([[0, 1, 2, n // 3, n // 2, n - 2, n - 1], rng.integers(0, n, k)]))
    return rows.astype(np.int64)


def check_rows(prob, sp, vals, rhs, prec, rows):
    cd = sp.cell_dofs()
    ptr, col_o, val_o, rhs_o = oracle.assemble_rows(prob, rows, cd, sp.n_dofs)
    rp, col = sp.pattern_host()
    worst = 0.0
    for q, r in enumerate(rows):
        np.testing.assert_array_equal(col[rp[r]:rp[r + 1]], col_o[ptr[q]:ptr[q + 1]])
        ref = val_o[ptr[q]:ptr[q + 1]]
        got = vals[rp[r]:rp[r + 1]]
        worst = max(worst, np.abs(got - ref).max() / np.abs(ref).max())
    assert worst <= TOL[prec], (prec, worst)
    assert np.abs(rhs[rows] - rhs_o).max() <= 1e-12 * max(np.abs(rhs_o).max(), 1e-300)
    return worst


def translation_residual(sp, vals, comp):
    """||A t|| / (||A||_max ||t||) for the rigid translation t along `comp` (GPU matvec)."""
    rp, col = sp.pattern()
    A = torch.sparse_csr_tensor(rp, col.to(torch.int64), vals, size=(sp.n_dofs, sp.n_dofs))
    t = torch.zeros(sp.n_dofs, dtype=torch.float64, device="cuda")
    t[comp::3] = 1.0
    r = torch.mv(A, t)
    return float(r.abs().max() / vals.abs().max())


@pytest.mark.parametrize("prec,kernel", [("fp32", "auto"), ("bf16", "auto"), ("fp64", "auto"),
                                         ("fp32", "cuda_core"), ("bf16", "cuda_core")])
def test_elasticity_q2_beam_full_size(prec, kernel):
    """32x32x32 Q2 beam (the benchmark workload, in the launch configuration the
    benchmark times): sampled rows vs the oracle, rigid translations in the kernel,
    RHS sums -vol = -4 on z rows."""
    prob = inputs.elasticity_q2_beam()
    sp = feasm.FESpace(prob)
    sp.set_kernel(kernel)
    coef = torch.tensor(prob.coef, device="cuda")
    vals, rhs = sp.assemble(coef, prec=prec)
    torch.cuda.synchronize()
    assert sp.status() == 0
    check_rows(prob, sp, vals.cpu().numpy(), rhs.cpu().numpy(), prec, sampled_rows(sp.n_dofs))
    for c in range(3):
        assert translation_residual(sp, vals, c) <= 8 * TOL[prec]
    assert abs(float(rhs[2::3].sum()) + 4.0) < 1e-11 and abs(float(rhs[0::3].sum())) < 1e-11
    sp.close()


def test_elasticity_q1_128_full_size():
    """128^3 Q1 elasticity (2.1M cells, 514M nonzeros), mixed FP32 form."""
    prob = inputs.elasticity_q1_128()
    sp = feasm.FESpace(prob)
    coef = torch.tensor(prob.coef, device="cuda")
    vals, rhs = sp.assemble(coef, prec="fp32")
    torch.cuda.synchronize()
    assert sp.status() == 0
    check_rows(prob, sp, vals.cpu().numpy(), rhs.cpu().numpy(), "fp32", sampled_rows(sp.n_dofs, k=24))
    assert translation_residual(sp, vals, 1) <= 8 * TOL["fp32"]
    assert abs(float(rhs[2::3].sum()) + 1.0) < 1e-10
    sp.close()


def test_host_buffer_entry_matches_device_entry():
    prob = inputs.small_problem((3, 3, 2), 2, 1, seed=5)
    sp = feasm.FESpace(prob)
    coef = torch.tensor(prob.coef, device="cuda")
    vals, rhs = sp.assemble(coef, prec="fp32")
    hv = torch.empty(sp.nnz, dtype=torch.float64).pin_memory()
    hr = torch.empty(sp.n_dofs, dtype=torch.float64).pin_memory()
    hc = torch.tensor(prob.coef).pin_memory()
    feasm.fe_assemble_host(sp.handle, hc, prob.force, hv, hr, feasm.FE_PREC_FP32)
    assert torch.equal(hv, vals.cpu()) and torch.equal(hr, rhs.cpu())
    # pageable buffers take the staging path: same values
    pv = torch.full((sp.nnz,), float("nan"), dtype=torch.float64)
    pr = torch.full((sp.n_dofs,), float("nan"), dtype=torch.float64)
    feasm.fe_assemble_host(sp.handle, torch.tensor(prob.coef), prob.force, pv, pr, feasm.FE_PREC_FP32)
    assert torch.equal(pv, vals.cpu()) and torch.equal(pr, rhs.cpu())
    # pinned values with a pageable RHS, and no RHS at all
    hv.fill_(float("nan"))
    pr.fill_(float("nan"))
    feasm.fe_assemble_host(sp.handle, hc, prob.force, hv, pr, feasm.FE_PREC_FP32)
    assert torch.equal(hv, vals.cpu()) and torch.equal(pr, rhs.cpu())
    feasm.fe_assemble_host(sp.handle, hc, prob.force, hv, None, feasm.FE_PREC_FP64)
    v64, _ = sp.assemble(coef, prec="fp64")
    assert torch.equal(hv, v64.cpu())
    sp.close()


def test_negative_jacobian_reported_without_fault():
    prob = inputs.small_problem((2, 2, 2), 1, 0, seed=1)
    coords = prob.mesh.coords.copy()
    centre = 13  # the interior vertex of a 2x2x2 brick
    coords[centre] = [1.2, 1.2, 1.2]  # pushed through the far corner: inverted cells
    m = inputs.Mesh(coords, prob.mesh.cell_vertices, prob.mesh.shape, prob.mesh.extent)
    bad = inputs.Problem("bad", m, 1, 2, 0, prob.coef, prob.force)
    sp = feasm.FESpace(bad)
    coef = torch.tensor(bad.coef, device="cuda")
    sp.assemble(coef, prec="fp64")
    assert sp.status() == -4
    assert sp.status() == 0          # the word is cleared; the context is still usable
    good = feasm.FESpace(prob)
    vals, _ = good.assemble(torch.tensor(prob.coef, device="cuda"), prec="fp64")
    assert good.status() == 0 and torch.isfinite(vals).all()
    sp.close()
    good.close()


@pytest.mark.parametrize("p,problem", [(2, 1), (2, 0), (3, 0), (3, 1)])
def test_negative_jacobian_reported_by_tensor_core_kernels(p, problem):
    """Inverted cells set FE_ERR_NEG_JACOBIAN in the tensor-core cell kernels
    (both forms) without a fault; the next assembly on a good mesh is clean."""
    prob = inputs.small_problem((2, 2, 2), p, problem, seed=2)
    coords = prob.mesh.coords.copy()
    coords[13] = [1.2, 1.2, 1.2]  # the interior vertex pushed through the far corner
    m = inputs.Mesh(coords, prob.mesh.cell_vertices, prob.mesh.shape, prob.mesh.extent)
    bad = inputs.Problem("bad", m, p, p + 1, problem, prob.coef, prob.force, prob.nu)
    sp = feasm.FESpace(bad)
    sp.set_kernel("tensor_core")
    coef = torch.tensor(bad.coef, device="cuda")
    for prec in ("fp32", "bf16"):
        sp.assemble(coef, prec=prec)
        assert sp.status() == -4, prec
        assert sp.status() == 0
    good = feasm.FESpace(prob)
    good.set_kernel("tensor_core")
    vals, _ = good.assemble(torch.tensor(prob.coef, device="cuda"), prec="bf16")
    assert good.status() == 0 and torch.isfinite(vals).all()
    sp.close()
    good.close()


def test_empty_mesh():
    mesh = inputs.Mesh(np.zeros((0, 3)), np.zeros((0, 8), dtype=np.int32), (0, 0, 0), (1, 1, 1))
    prob = inputs.Problem("empty", mesh, 2, 3, 1, np.zeros(0), np.array([0.0, 0.0, -1.0]))
    sp = feasm.FESpace(prob)
    assert (sp.n_dofs, sp.nnz) == (0, 0)
    sp.assemble(torch.zeros(0, dtype=torch.float64, device="cuda"), prec="fp32")
    assert sp.status() == 0
    sp.close()


# ------------------------------------------------------------------ adjoint
@pytest.mark.parametrize("shape,p,problem", [((3, 3, 3), 1, 1), ((2, 2, 3), 2, 1), ((2, 2, 2), 3, 0), ((3, 2, 2), 2, 0)])
def test_adjoint_small_vs_oracle(shape, p, problem):
    prob = inputs.small_problem(shape, p, problem, seed=70 + p)
    sp = feasm.FESpace(prob)
    cd = sp.cell_dofs()
    u = inputs.unit_rms_field(sp.n_dofs, 9)
    g_o = oracle.cell_energies(prob, u, cd)
    ut = torch.tensor(u, device="cuda")
    coef = torch.tensor(prob.coef, device="cuda")
    c = torch.zeros(1, dtype=torch.float64, device="cuda")
    g64 = sp.adjoint(ut, coef, 1.0, compliance=c, prec="fp64").cpu().numpy()
    assert vec_error(g64, g_o) <= 1e-12
    assert abs(float(c) - np.dot(prob.coef, g_o)) <= 1e-12 * abs(np.dot(prob.coef, g_o))
    g32 = sp.adjoint(ut, None, 2.5, prec="fp32").cpu().numpy()
    assert vec_error(g32, 2.5 * g_o) <= 1e-5
    assert sp.status() == 0
    sp.close()


def test_adjoint_cantilever_full_size_fd_and_oracle():
    """64^3 Q1 cantilever: adjoint vs the oracle gradient on sampled cells, and vs
    central finite differences (step 1e-6 relative) on 32 random cells of the
    compliance c(E) = u^T A(E) u formed from the assembled FP64 matrix (fe_assemble)
    and a sparse matrix-vector product: an independent path (cell kernel + scatter)
    from the adjoint kernel's per-cell energies."""
    from paper_1708_01773_gb300.autograd import compliance
    prob = inputs.cantilever_q1_64()
    sp = feasm.FESpace(prob)
    cd = sp.cell_dofs()
    u = inputs.unit_rms_field(sp.n_dofs, 20171773 + 5)
    ut = torch.tensor(u, device="cuda")
    E = torch.tensor(prob.coef, device="cuda", requires_grad=True)
    c = compliance(E, ut, sp)
    c.backward()
    g = E.grad.detach().cpu().numpy()
    rng = np.random.default_rng(32)
    cells = np.unique(np.concatenate([[0, prob.mesh.n_cells - 1], rng.integers(0, prob.mesh.n_cells, 32)]))
    sub = inputs.Problem("sub", inputs.Mesh(prob.mesh.coords, prob.mesh.cell_vertices[cells]), 1, 2, 1,
                         prob.coef[cells], prob.force)
    g_o = oracle.cell_energies(sub, u, cd[cells])
    assert vec_error(g[cells], g_o) <= 1e-12
    g32 = sp.adjoint(ut, None, 1.0, prec="fp32").cpu().numpy()   # FP32 strain, FP64 geometry and sums
    assert vec_error(g32[cells], g_o) <= 1e-5
    # Euler identity for a functional linear in E
    assert abs(float(c) - float((E.detach() * E.grad).sum())) <= 1e-12 * abs(float(c))
    # central differences of c(E) = u^T A(E) u, A from fe_assemble (FP64)
    rp, col = sp.pattern()

    def quad_form(vals):
        A = torch.sparse_csr_tensor(rp, col.to(torch.int64), vals, size=(sp.n_dofs, sp.n_dofs))
        return torch.dot(ut, torch.mv(A, ut))

    v0, _ = sp.assemble(E.detach(), prec="fp64")
    assert abs(float(quad_form(v0)) - float(c)) <= 1e-10 * abs(float(c))   # the same compliance both ways
    for e in rng.choice(prob.mesh.n_cells, 32, replace=False):
        h = 1e-6 * prob.coef[e]
        Ep, Em = E.detach().clone(), E.detach().clone()
        Ep[e] += h
        Em[e] -= h
        vp, _ = sp.assemble(Ep, prec="fp64")
        vp = vp.clone()
        vm, _ = sp.assemble(Em, prec="fp64")
        # c(E + h) - c(E - h) = u^T (A(E + h) - A(E - h)) u: evaluated on the entry
        # differences, the entries without cell e cancel exactly (the assembly is
        # deterministic), so the quotient carries rounding of order 1e-10 only
        fd = float(quad_form(vp - vm)) / (2 * h)
        assert abs(fd - g[e]) <= 1e-7 * abs(g[e]), (e, fd, g[e])
        # the same quotient from the two compliances themselves (rounding of the
        # 64.7M-term sums, about 1e-5 relative at this h)
        fd_plain = (float(quad_form(vp)) - float(quad_form(vm))) / (2 * h)
        assert abs(fd_plain - g[e]) <= 1e-3 * abs(g[e]), (e, fd_plain, g[e])
    assert sp.status() == 0
    sp.close()

"""GPU parity of the strong-Dirichlet path (fe_assemble_dirichlet) through the C ABI.

Small meshes: every entry of the constrained matrix and right-hand side against
the oracle's constrained system (Eq. dirichlet_bc_discrete_problem). The
constrained matrix must also equal, bit for bit, the free x free block of the
unconstrained assembly (both sum the same contributions in the same order), and
with u^D = 0 the right-hand side must equal the unconstrained one on the free
rows bit for bit. Full size: the clamped Q2 beam on sampled rows, and the
bitwise block relation over the whole matrix.

RHS error: max_a |b_a - b*_a| / max_a s_a with s_a = |f_a| + sum_{c fixed}
|A_ac| |u^D_c|, the size of the terms the lifting sums; the cell-matrix entries
it multiplies carry the precision form's error (TOL), the rest is FP64.
"""
import numpy as np
import pytest
import torch

import oracle
from metrics import TOL, energy_error, row_scaled_error
from paper_1708_01773_gb300 import build, feasm, inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    feasm.lib()


def fixed_mask(pos, comp, kind, rng):
    if kind == "clamp_x0":
        return np.abs(pos[:, 0]) < 1e-12
    if kind == "boundary":
        ext = pos.max(axis=0)
        return np.any((np.abs(pos) < 1e-12) | (np.abs(pos - ext) < 1e-12), axis=1)
    if kind == "x_component":
        return (np.abs(pos[:, 0]) < 1e-12) & (comp == 0)
    return rng.uniform(size=pos.shape[0]) < 0.3


def lift_scale(rp, col, val, rhs, fixed, u_full, rows=None):
    """s_a = |f_a| + sum_{c fixed} |A_ac| |u_c| over the given (free) rows."""
    n = rp.size - 1
    r_of = np.repeat(np.arange(n), np.diff(rp))
    w = np.where(fixed[col], np.abs(val) * np.abs(u_full[col]), 0.0)
    s = np.abs(rhs).copy()
    np.add.at(s, r_of, w)
    return s if rows is not None else s[~fixed]


def components(n, ncomp):
    return np.arange(n) % ncomp     # the ncomp DOFs of a node are consecutive, components in order


CASES = [((3, 3, 3), 1, 1, "clamp_x0", "auto"), ((3, 2, 2), 2, 1, "clamp_x0", "tensor_core"),
         ((3, 2, 2), 2, 1, "clamp_x0", "cuda_core"), ((3, 2, 3), 2, 0, "boundary", "auto"),
         ((3, 3, 2), 1, 0, "random", "auto"), ((3, 2, 2), 1, 1, "x_component", "auto"),
         ((2, 1, 2), 3, 1, "random", "auto"), ((2, 2, 3), 3, 0, "boundary", "auto")]


@pytest.mark.parametrize("shape,p,problem,kind,kernel", CASES)
def test_small_constrained_systems(shape, p, problem, kind, kernel):
    prob = inputs.small_problem(shape, p, problem, seed=400 + 7 * p + problem)
    sp = feasm.FESpace(prob)
    sp.set_kernel(kernel)
    cd = sp.cell_dofs()
    n = sp.n_dofs
    pos = sp.dof_points()
    rng = np.random.default_rng(500 + p)
    fixed = fixed_mask(pos, components(n, prob.ncomp), kind, rng)
    dsys = sp.dirichlet(fixed)
    rp_o, col_o, val_o, rhs_o = oracle.assemble_csr(prob, cd, n)
    uD = rng.standard_normal(dsys.n_fixed)
    u_full = np.zeros(n)
    u_full[fixed] = uD
    ptr_r, col_r, val_r, rhs_r = oracle.dirichlet_reduce(rp_o, col_o, val_o, rhs_o, fixed, uD)
    scale = lift_scale(rp_o, col_o, val_o, rhs_o, fixed, u_full).max()
    rp, col = dsys.pattern()
    np.testing.assert_array_equal(rp.cpu().numpy(), ptr_r)
    np.testing.assert_array_equal(col.cpu().numpy(), col_r)
    lab = dsys.labels()
    block = (lab[col_o] >= 0) & np.repeat(lab >= 0, np.diff(rp_o))
    coef = torch.tensor(prob.coef, device="cuda")
    uD_d = torch.tensor(uD, device="cuda")
    for prec in ("fp64", "fp32", "bf16"):
        if kernel == "tensor_core" and prec == "fp64":
            continue
        vals, rhs = dsys.assemble(coef, uD_d, prec=prec)
        _, rhs_h = dsys.assemble(coef, None, prec=prec)      # homogeneous data
        torch.cuda.synchronize()
        assert sp.status() == 0
        v, b = vals.cpu().numpy(), rhs.cpu().numpy()
        assert row_scaled_error(ptr_r, col_r, v, val_r) <= TOL[prec], (prec, kind)
        assert energy_error(ptr_r, col_r, v, val_r) <= TOL[prec], (prec, kind)
        assert np.abs(b - rhs_r).max() <= TOL[prec] * scale, (prec, np.abs(b - rhs_r).max() / scale)
        # the unconstrained assembly, bit for bit on the free block and free rows
        vals_u, rhs_u = sp.assemble(coef, prec=prec)
        torch.cuda.synchronize()
        assert np.array_equal(v, vals_u.cpu().numpy()[block]), prec
        assert np.array_equal(rhs_h.cpu().numpy(), rhs_u.cpu().numpy()[~fixed]), prec
    dsys.close()
    sp.close()


def test_constrained_assembly_is_deterministic():
    prob = inputs.small_problem((4, 3, 3), 2, 1, seed=410)
    sp = feasm.FESpace(prob)
    pos = sp.dof_points()
    fixed = np.abs(pos[:, 0]) < 1e-12
    dsys = sp.dirichlet(fixed)
    coef = torch.tensor(prob.coef, device="cuda")
    uD = torch.linspace(-1.0, 1.0, dsys.n_fixed, dtype=torch.float64, device="cuda")
    for prec in ("fp32", "fp64"):
        v1, b1 = dsys.assemble(coef, uD, prec=prec)
        v1, b1 = v1.clone(), b1.clone()
        v2, b2 = dsys.assemble(coef, uD, prec=prec)
        torch.cuda.synchronize()
        assert torch.equal(v1, v2) and torch.equal(b1, b2), prec
    dsys.close()
    sp.close()


def clamp_data(pos):
    """Prescribed displacement on the clamped face: a small linear field."""
    return np.stack([0.01 * pos[:, 1], -0.02 * pos[:, 2], 0.03 * (pos[:, 1] - 0.5)], axis=1)


@pytest.mark.parametrize("prec", ["fp32", "fp64", "bf16"])
def test_clamped_q2_beam_full_size(prec):
    """The 32x32x32 Q2 beam with its x = 0 face clamped to a prescribed linear
    displacement, in the launch configuration the benchmark times: sampled free rows
    (half of them next to the clamp, where the lifting acts) against the oracle, and
    the bitwise relation to the unconstrained assembly over the whole matrix."""
    prob = inputs.elasticity_q2_beam()
    sp = feasm.FESpace(prob)
    n = sp.n_dofs
    pos = sp.dof_points()
    comp = components(n, 3)
    fixed = np.abs(pos[:, 0]) < 1e-12
    assert fixed.sum() == 3 * 65 * 65
    u_full = np.zeros(n)
    u_full[fixed] = clamp_data(pos)[fixed, comp[fixed]]
    dsys = sp.dirichlet(fixed)
    coef = torch.tensor(prob.coef, device="cuda")
    uD = torch.tensor(u_full[fixed], device="cuda")
    vals, rhs = dsys.assemble(coef, uD, prec=prec)
    torch.cuda.synchronize()
    assert sp.status() == 0
    lab = dsys.labels()
    rng = np.random.default_rng(7)
    near = np.flatnonzero(~fixed & (pos[:, 0] < 0.2))
    far = np.flatnonzero(~fixed)
    rows = np.unique(np.concatenate([rng.choice(near, 24, replace=False), rng.choice(far, 24, replace=False),
                                     far[[0, -1]]])).astype(np.int64)
    cd = sp.cell_dofs()
    ptr, col_o, val_o, rhs_o = oracle.assemble_rows(prob, rows, cd, n)
    p_r, c_r, v_r, b_r = oracle.dirichlet_reduce(ptr, col_o, val_o, rhs_o, fixed, u_full[fixed], rows=rows)
    s_r = lift_scale(ptr, col_o, val_o, rhs_o, fixed, u_full, rows=rows)
    rp, col = dsys.pattern_host()
    v, b = vals.cpu().numpy(), rhs.cpu().numpy()
    worst = 0.0
    for q, g in enumerate(rows):
        r = lab[g]
        np.testing.assert_array_equal(col[rp[r]:rp[r + 1]], c_r[p_r[q]:p_r[q + 1]])
        ref = v_r[p_r[q]:p_r[q + 1]]
        worst = max(worst, np.abs(v[rp[r]:rp[r + 1]] - ref).max() / np.abs(ref).max())
    assert worst <= TOL[prec], (prec, worst)
    assert np.abs(b[lab[rows]] - b_r).max() <= TOL[prec] * s_r.max()
    # bitwise: the constrained values are the free x free block of the unconstrained assembly
    vals_u, _ = sp.assemble(coef, prec=prec)
    rp_u, col_u = sp.pattern()
    lab_d = torch.tensor(lab, device="cuda")
    rows_u = torch.repeat_interleave(torch.arange(n, device="cuda"), rp_u[1:] - rp_u[:-1])
    block = (lab_d[col_u.long()] >= 0) & (lab_d[rows_u] >= 0)
    assert torch.equal(vals, vals_u[block])
    dsys.close()
    sp.close()

"""GPU parity of the self-adjoint compliance (fe_compliance): assembly of the
clamped system, Jacobi-preconditioned CG in FP64, c = f^T u and the gradient
dc/dE_K = -u_K^T (A^K/E_K) u_K, against the oracle.

FP64 form, against the oracle's direct solve: CG stops at ||r|| <= 1e-12 ||f||,
so u carries at most cond(K) x 1e-12 relative error (cond(K) < 1e4 on these
meshes) -> 1e-8 on u and the gradient, and c = f^T u (error quadratic in u's
error plus the residual term) 1e-10.

FP32/BF16 forms: the solve is exact for the mixed-precision matrix, whose
entries are each within TOL[prec] of their row's largest entry. So the
returned u must satisfy the oracle's FP64 system row by row up to exactly that
allowance plus the CG residual:
    |(K u - f)_i| <= TOL rowmax_i sum_{j in row i} |u_j| + rtol ||f||_2.
(A comparison of c or u with the FP64 solution would instead measure the
matrix error amplified by 1/lambda_min: the clamped structure's softest,
bending modes have energies far below the rows' largest entries; on the Q2
mesh below the FP32 compliance differs from the FP64 one by 7e-5.) The
gradient is checked against the oracle's cell energies of the returned u
(1e-5: the adjoint's FP32 strain arithmetic), and c against f^T u.
"""
import numpy as np
import pytest
import torch

import oracle
from metrics import TOL, csr_matvec, vec_error
from paper_1708_01773_gb300 import build, feasm, inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    feasm.lib()


CASES = [((4, 2, 2), 1, 1), ((3, 2, 2), 2, 1), ((3, 3, 2), 1, 0), ((2, 2, 2), 3, 1)]


def clamped(shape, p, problem, seed):
    prob = inputs.small_problem(shape, p, problem, seed=seed, extent=(2.0, 1.0, 1.0))
    sp = feasm.FESpace(prob)
    pos = sp.dof_points()
    fixed = np.abs(pos[:, 0]) < 1e-12
    return prob, sp, fixed


@pytest.mark.parametrize("shape,p,problem", CASES)
def test_small_compliance_against_direct_solve(shape, p, problem):
    prob, sp, fixed = clamped(shape, p, problem, seed=600 + 3 * p + problem)
    cd = sp.cell_dofs()
    u_o, c_o, g_o = oracle.compliance_solve(prob, fixed, cd, sp.n_dofs)
    rp, col, val, rhs = oracle.assemble_csr(prob, cd, sp.n_dofs)
    ptr, col_r, val_r, b_r = oracle.dirichlet_reduce(rp, col, val, rhs, fixed, np.zeros(int(fixed.sum())))
    rowmax = np.zeros(ptr.size - 1)
    np.maximum.at(rowmax, np.repeat(np.arange(ptr.size - 1), np.diff(ptr)), np.abs(val_r))
    dsys = sp.dirichlet(fixed)
    coef = torch.tensor(prob.coef, device="cuda")
    for prec in ("fp64", "fp32", "bf16"):
        rtol = 1e-12 if prec == "fp64" else 1e-10
        u, c, g, it, rel = dsys.compliance(coef, prec=prec, rtol=rtol)
        torch.cuda.synchronize()
        assert sp.status() == 0
        assert rel <= rtol and 0 < it <= 20000
        u, c, g = u.cpu().numpy(), float(c), g.cpu().numpy()
        assert np.all(u[fixed] == 0) and np.isfinite(c) and c > 0 and np.all(g <= 0)
        if prec == "fp64":
            assert abs(c - c_o) <= 1e-10 * c_o
            assert vec_error(u, u_o) <= 1e-8
            assert vec_error(g, g_o) <= 1e-8
            assert abs(prob.coef @ g + c) <= 1e-9 * c   # Euler: c is homogeneous of degree -1 in E
            continue
        # row-wise residual in the oracle's FP64 operator, within the mixed form's allowance
        uf = u[~fixed]
        res = csr_matvec(ptr, col_r, val_r, uf) - b_r
        allow = TOL[prec] * rowmax * csr_matvec(ptr, col_r, np.ones_like(val_r), np.abs(uf)) \
            + rtol * np.linalg.norm(b_r)
        assert np.all(np.abs(res) <= allow), (prec, float((np.abs(res) / allow).max()))
        assert abs(c - b_r @ uf) <= 1e-12 * c
        g_u = -oracle.cell_energies(prob, u, cd)
        assert vec_error(g, g_u) <= 1e-5, (prec, vec_error(g, g_u))
        print(prec, "relative compliance difference to FP64", abs(c - c_o) / c_o)
    dsys.close()
    sp.close()


def test_compliance_is_deterministic_and_autograd_matches():
    from paper_1708_01773_gb300.autograd import self_adjoint_compliance
    prob, sp, fixed = clamped((4, 3, 3), 1, 1, seed=610)
    dsys = sp.dirichlet(fixed)
    coef = torch.tensor(prob.coef, device="cuda")
    runs = [dsys.compliance(coef, prec="fp32", rtol=1e-10) for _ in range(2)]
    torch.cuda.synchronize()
    (u1, c1, g1, it1, r1), (u2, c2, g2, it2, r2) = runs
    assert it1 == it2 and r1 == r2
    assert torch.equal(u1, u2) and torch.equal(c1, c2) and torch.equal(g1, g2)
    E = coef.clone().requires_grad_(True)
    c = self_adjoint_compliance(E, dsys, "fp64", 1e-12)
    c.backward()
    _, c64, g64, _, _ = dsys.compliance(coef, prec="fp64", rtol=1e-12)
    assert float(c.detach()) == float(c64)
    assert torch.equal(E.grad, g64)
    dsys.close()
    sp.close()


def test_compliance_errors_are_reported():
    prob, sp, fixed = clamped((3, 2, 2), 1, 1, seed=611)
    dsys = sp.dirichlet(fixed)
    coef = torch.tensor(prob.coef, device="cuda")
    with pytest.raises(feasm.FEError) as ei:
        dsys.compliance(coef, prec="fp64", rtol=1e-14, max_iter=3)
    assert ei.value.code == -7                               # FE_ERR_NOT_CONVERGED
    with pytest.raises(feasm.FEError):
        dsys.compliance(coef, prec="fp64", rtol=-1.0)
    dsys.close()
    # nothing fixed: K is singular and f has a net force, so PCG cannot converge
    free = sp.dirichlet(np.zeros(sp.n_dofs, dtype=bool))
    with pytest.raises(feasm.FEError):
        free.compliance(coef, prec="fp64", rtol=1e-12, max_iter=400)
    free.close()
    sp.close()


def test_cantilever_q1_64_full_size():
    """64^3 Q1 cantilever clamped at x = 0 under its body force: the residual of the
    returned u, the energy identity c = u^T K u (the adjoint kernel's compliance of
    u), Euler's identity, and the gradient against the oracle's cell energies of
    the GPU's u on sampled cells."""
    prob = inputs.cantilever_q1_64()
    sp = feasm.FESpace(prob)
    pos = sp.dof_points()
    fixed = np.abs(pos[:, 0]) < 1e-12
    dsys = sp.dirichlet(fixed)
    coef = torch.tensor(prob.coef, device="cuda")
    u, c, g, it, rel = dsys.compliance(coef, prec="fp64", rtol=1e-10)
    torch.cuda.synchronize()
    assert rel <= 1e-10
    c = float(c)
    # energy identity through the adjoint kernel: u^T K u = sum_K E_K u_K^T (A^K/E_K) u_K
    cu = torch.empty(1, dtype=torch.float64, device="cuda")
    sp.adjoint(u, coef, 1.0, compliance=cu, prec="fp64")
    assert abs(float(cu) - c) <= 1e-8 * c
    gn = g.cpu().numpy()
    assert abs(prob.coef @ gn + c) <= 1e-9 * c
    # residual of the constrained system on the GPU (torch sparse matvec, test only)
    vals, rhs = dsys.assemble(coef, None, prec="fp64")
    rp, col = dsys.pattern()
    K = torch.sparse_csr_tensor(rp, col.to(torch.int64), vals, size=(dsys.n_free, dsys.n_free))
    lab = torch.tensor(dsys.labels(), device="cuda")
    uf = u[lab >= 0]
    res = torch.linalg.vector_norm(torch.mv(K, uf) - rhs) / torch.linalg.vector_norm(rhs)
    assert float(res) <= 1e-9
    # gradient on sampled cells against the oracle's cell energies of this u
    un = u.cpu().numpy()
    cd = sp.cell_dofs()
    rng = np.random.default_rng(64)
    cells = np.unique(np.concatenate([[0, prob.mesh.n_cells - 1], rng.integers(0, prob.mesh.n_cells, 32)]))
    sub = inputs.Problem("sub", inputs.Mesh(prob.mesh.coords, prob.mesh.cell_vertices[cells]), 1, 2, 1,
                         prob.coef[cells], prob.force)
    g_o = -oracle.cell_energies(sub, un, cd[cells])
    assert vec_error(gn[cells], g_o) <= 1e-12
    dsys.close()
    sp.close()

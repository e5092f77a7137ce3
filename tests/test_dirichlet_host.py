"""CPU tests of the strong-Dirichlet setup of the C-ABI library (no GPU): the
free/fixed labels, the constrained CSR pattern, both forms of its assembly
permutation and the lifting lists, checked by emulating the scatter and the
lifting on the CPU with the oracle's FP64 cell matrices against the oracle's
constrained system (Eq. dirichlet_bc_discrete_problem). Also the DOF node
positions against an independent numpy evaluation of the trilinear map."""
import numpy as np
import pytest

import oracle
from paper_1708_01773_gb300 import feasm, inputs

from test_oracle_pins import boundary_dofs, node_positions


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1708_01773_gb300 import build
    build.build()


def cell_matrices(prob):
    nl = prob.ncomp * (prob.order + 1) ** 3
    Ke = np.zeros((prob.mesh.n_cells, nl, nl))
    fe = np.zeros((prob.mesh.n_cells, nl))
    for e in range(prob.mesh.n_cells):
        xv = prob.mesh.coords[prob.mesh.cell_vertices[e]]
        Ke[e], fe[e] = oracle.cell_matrix(prob.problem, prob.order, prob.quad_1d, xv, prob.coef[e], prob.nu,
                                          prob.force)
    return Ke, fe


def fixed_sets(pos, comp, kind, rng):
    if kind == "clamp_x0":                    # a clamped end: every component of the x = 0 face
        return np.abs(pos[:, 0]) < 1e-12
    if kind == "boundary":
        return boundary_dofs(pos, extent=tuple(pos.max(axis=0)))
    if kind == "x_component":                 # a symmetry-type condition: u_x = 0 on x = 0 only
        return (np.abs(pos[:, 0]) < 1e-12) & (comp == 0)
    return rng.uniform(size=pos.shape[0]) < 0.3   # scattered fixed DOFs


CASES = [((3, 2, 2), 1, 1, "clamp_x0"), ((3, 2, 2), 2, 1, "clamp_x0"), ((2, 2, 2), 2, 0, "boundary"),
         ((2, 2, 3), 1, 0, "random"), ((2, 2, 2), 1, 1, "x_component"), ((2, 1, 2), 3, 1, "clamp_x0"),
         ((2, 2, 1), 3, 0, "random")]


@pytest.mark.parametrize("shape,p,problem,kind", CASES)
def test_constrained_permutation_matches_oracle(shape, p, problem, kind):
    prob = inputs.small_problem(shape, p, problem, seed=200 + 7 * p + problem)
    sp = feasm.FESpace(prob, host_only=True)
    cd = sp.cell_dofs()
    n = sp.n_dofs
    pos_o, comp = node_positions(prob, cd, n)
    np.testing.assert_allclose(sp.dof_points(), pos_o, rtol=0, atol=1e-14)
    rng = np.random.default_rng(300 + p)
    fixed = fixed_sets(pos_o, comp, kind, rng)
    assert 0 < fixed.sum() < n
    dsys = sp.dirichlet(fixed)
    lab = dsys.labels()
    np.testing.assert_array_equal(lab, oracle.dirichlet_labels(fixed))
    assert dsys.n_free == int((~fixed).sum()) and dsys.n_fixed == int(fixed.sum())
    # oracle's constrained system with random prescribed values
    rp_o, col_o, val_o, rhs_o = oracle.assemble_csr(prob, cd, n)
    uD = rng.standard_normal(dsys.n_fixed)
    ptr_r, col_r, val_r, rhs_r = oracle.dirichlet_reduce(rp_o, col_o, val_o, rhs_o, fixed, uD)
    rp, col = dsys.pattern_host()
    np.testing.assert_array_equal(rp, ptr_r)
    np.testing.assert_array_equal(col, col_r)
    nl = prob.ncomp * (p + 1) ** 3
    Ke, fe = cell_matrices(prob)
    Kf = Ke.reshape(-1)
    # lifting lists, then the lifted cell vectors
    cells, lptr, lm, lfix = feasm.fe_dirichlet_lift_host(dsys.handle)
    expect = [e for e in range(prob.mesh.n_cells) if fixed[cd[e]].any() and (~fixed[cd[e]]).any()]
    assert cells.tolist() == expect
    fe_l = fe.copy()
    for i, e in enumerate(cells):
        m = lm[lptr[i]:lptr[i + 1]].astype(np.int64)
        assert np.all(np.diff(m) > 0)
        np.testing.assert_array_equal(m, np.flatnonzero(fixed[cd[e]]))
        np.testing.assert_array_equal(lfix[lptr[i]:lptr[i + 1]], -1 - lab[cd[e][m]])
        fe_l[e] -= Ke[e][:, m] @ uD[lfix[lptr[i]:lptr[i + 1]]]
    cnt, code_ptr, codes, ncode, posb, slot_ptr, slots = feasm.fe_dirichlet_permutation_host(
        dsys.handle, prob.mesh.n_cells * nl)
    acc_stride = (int(np.diff(rp).max()) + 3) & ~3
    vals_codes = np.zeros(dsys.nnz)
    vals_pos = np.zeros(dsys.nnz)
    rhs = np.zeros(dsys.n_free)
    flat_cd = cd.reshape(-1)
    for r in range(dsys.n_free):
        sl = slots[slot_ptr[r]:slot_ptr[r + 1]].astype(np.int64)
        g = np.flatnonzero(lab == r)[0]
        assert np.all(flat_cd[sl] == g) and np.all(np.diff(sl // nl) > 0)
        rhs[r] = fe_l.reshape(-1)[sl].sum()
        c0 = code_ptr[r]
        assert c0 % 8 == 0 and code_ptr[r + 1] - c0 == (len(sl) * nl + 7) // 8 * 8
        # codes form: ncode[r] codes, runs per nonzero, fixed columns left out
        assert ncode[r] == sum(int((~fixed[cd[e // nl]]).sum()) for e in sl)
        c = c0
        for k in range(rp[r], rp[r + 1]):
            seg = codes[c:c + cnt[k]].astype(np.int64)
            c += cnt[k]
            assert seg[0] >> 15 == 1 and np.all(seg[1:] >> 15 == 0)
            s, m = (seg >> 8) & 127, seg & 255
            assert np.all(lab[flat_cd[(sl[s] // nl) * nl + m]] == col[k])
            vals_codes[k] = Kf[sl[s] * nl + m].sum()
        assert c == c0 + ncode[r]
        # slot-major positions: nonzero index (head bit on its first contribution) or the lane's dummy
        seen = np.zeros(rp[r + 1] - rp[r], dtype=bool)
        for s in range(len(sl)):
            e = sl[s] // nl
            for m in range(nl):
                v = int(posb[c0 + s * nl + m])
                if fixed[cd[e][m]]:
                    assert v == acc_stride + (m & 31)
                    continue
                k = v & 0x7FFF
                assert lab[cd[e][m]] == col[rp[r] + k]
                assert bool(v >> 15) == (not seen[k])
                seen[k] = True
                vals_pos[rp[r] + k] += Kf[sl[s] * nl + m]
        assert seen.all()
    scale = np.abs(val_r).max()
    np.testing.assert_allclose(vals_codes, val_r, rtol=0, atol=1e-13 * scale)
    np.testing.assert_allclose(vals_pos, val_r, rtol=0, atol=1e-13 * scale)
    np.testing.assert_allclose(rhs, rhs_r, rtol=0, atol=1e-13 * (scale * np.abs(uD).sum() + 1))
    dsys.close()
    sp.close()


def test_clamped_elasticity_keeps_node_rows():
    """With every component of a node fixed together, the free rows still come in
    node triples sharing cells (local rows i*nb + a) and columns."""
    prob = inputs.small_problem((3, 2, 2), 1, 1, seed=211)
    sp = feasm.FESpace(prob, host_only=True)
    pos = sp.dof_points()
    dsys = sp.dirichlet(np.abs(pos[:, 0]) < 1e-12)
    cnt, code_ptr, codes, ncode, posb, slot_ptr, slots = feasm.fe_dirichlet_permutation_host(
        dsys.handle, prob.mesh.n_cells * 24)
    rp, col = dsys.pattern_host()
    assert dsys.n_free % 3 == 0
    for n in range(dsys.n_free // 3):
        r0 = 3 * n
        for i in (1, 2):
            np.testing.assert_array_equal(slots[slot_ptr[r0 + i]:slot_ptr[r0 + i + 1]],
                                          slots[slot_ptr[r0]:slot_ptr[r0 + 1]] + i * 8)
            assert rp[r0 + i + 1] - rp[r0 + i] == rp[r0 + 1] - rp[r0]


def test_nothing_fixed_and_everything_fixed():
    prob = inputs.small_problem((2, 2, 1), 2, 0, seed=212)
    sp = feasm.FESpace(prob, host_only=True)
    d0 = sp.dirichlet(np.zeros(sp.n_dofs, dtype=bool))
    rp, col = d0.pattern_host()
    rp_s, col_s = sp.pattern_host()
    np.testing.assert_array_equal(rp, rp_s)
    np.testing.assert_array_equal(col, col_s)
    assert feasm.fe_dirichlet_lift_host(d0.handle)[0].size == 0
    d1 = sp.dirichlet(np.ones(sp.n_dofs, dtype=bool))
    assert (d1.n_free, d1.n_fixed, d1.nnz) == (0, sp.n_dofs, 0)
    assert feasm.fe_dirichlet_lift_host(d1.handle)[0].size == 0   # no cell has a free DOF
    d0.close(); d1.close(); sp.close()


def test_invalid_arguments():
    prob = inputs.small_problem((1, 1, 1), 1, 0, seed=213)
    sp = feasm.FESpace(prob, host_only=True)
    mask = np.zeros(sp.n_dofs, dtype=np.uint8)
    assert feasm.lib().fe_dirichlet_create(sp.handle, mask.ctypes.data, None) == -1      # out NULL
    out = feasm.ctypes.c_void_p()
    assert feasm.lib().fe_dirichlet_create(sp.handle, None, feasm.ctypes.byref(out)) == -1  # mask NULL
    assert out.value is None
    with pytest.raises(feasm.FEError):     # a host-only space cannot compute
        d = sp.dirichlet(np.zeros(sp.n_dofs, dtype=bool))
        feasm.fe_assemble_dirichlet(d.handle, None, [1.0], None, None, None, 1, 0)
    other = inputs.small_problem((2, 1, 1), 1, 0, seed=214)
    with pytest.raises(feasm.FEError):     # the mesh must be the space's
        feasm.fe_space_dof_points_host(sp.handle, other.mesh.coords, other.mesh.cell_vertices)
    sp.close()

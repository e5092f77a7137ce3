"""CPU tests of the C-ABI library: it loads, exports every declared symbol, and its
host-side setup (DOF numbering, CSR pattern, assembly permutation) agrees with the
oracle. No compute call is made (no GPU here)."""
import re
import os

import numpy as np
import pytest

import oracle
from paper_1708_01773_gb300 import feasm, inputs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1708_01773_gb300 import build
    build.build()


def declared_functions():
    src = open(os.path.join(ROOT, "include", "feasm.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:int|void|const char\*)\s+(fe_\w+)\s*\(", src, flags=re.M)))


def test_library_exports_every_declared_symbol():
    names = declared_functions()
    assert len(names) >= 15
    assert set(names) == set(feasm.EXPORTS)
    L = feasm.lib()
    for n in names:
        assert hasattr(L, n), n
    out = os.popen(f"nm -D --defined-only {feasm.LIB_PATH}").read()
    for n in names:
        assert re.search(rf"\bT {n}\b", out), n


CASES = [
    ((3, 2, 2), 1, 0, False), ((2, 2, 3), 1, 1, False), ((2, 3, 2), 2, 0, False), ((3, 2, 2), 2, 1, False),
    ((2, 2, 2), 3, 0, False), ((2, 1, 2), 3, 1, False), ((3, 2, 2), 2, 2, False), ((2, 1, 2), 3, 2, False),
    # scrambled bricks: random vertex ids and cell order, rotated local vertex orders
    ((3, 3, 2), 1, 1, True), ((3, 2, 2), 2, 0, True), ((2, 2, 2), 2, 1, True), ((2, 2, 2), 3, 1, True),
    ((3, 2, 2), 2, 2, True),
]


@pytest.mark.parametrize("shape,p,problem,scramble", CASES)
def test_numbering_pattern_permutation_match_oracle(shape, p, problem, scramble):
    prob = inputs.small_problem(shape, p, problem, seed=3 * p + problem)
    if scramble:
        prob = inputs.scrambled(prob, seed=20 + 3 * p + problem)
    check_host_setup(prob)


@pytest.mark.parametrize("p,problem", [(1, 0), (1, 1), (2, 0), (2, 1), (3, 1), (2, 2)])
def test_o_grid_numbering_pattern_permutation(p, problem):
    """The same checks on an O-grid (irregular vertex valence: six cells around
    the inner square's corner vertices, three on the end faces)."""
    check_host_setup(inputs.o_grid_problem(3, 2, 2, p, problem, seed=20 + p))


@pytest.mark.parametrize("p,problem", [(1, 1), (2, 0), (3, 0)])
def test_flower_numbering_pattern_permutation(p, problem):
    """The same checks on a flower mesh: 34 cells around the axis vertex between
    its two layers (more than the 32 of the slot-wise scatter)."""
    prob = inputs.o_grid_problem(0, 0, 0, p, problem, seed=30 + p, mesh=inputs.flower(17, 2))
    check_host_setup(prob)


def check_host_setup(prob):
    p, problem = prob.order, prob.problem
    sp = feasm.FESpace(prob, host_only=True)
    cd_o, n_o = oracle.numbering(prob)
    cd = sp.cell_dofs()
    assert sp.n_dofs == n_o
    np.testing.assert_array_equal(cd, cd_o)                      # list_dofs, bit-exact
    rp_o, col_o, val_o, rhs_o = oracle.assemble_csr(prob, cd_o, n_o)
    rp, col = sp.pattern_host()
    np.testing.assert_array_equal(rp, rp_o)
    np.testing.assert_array_equal(col, col_o)
    nl = prob.n_local
    assert sp.n_contrib == prob.mesh.n_cells * nl * nl
    # emulate the scatter on the CPU with the oracle's own FP64 cell matrices
    cnt, code_ptr, codes, slot_ptr, slots = feasm.fe_space_permutation_host(sp.handle)
    Ke = np.zeros((prob.mesh.n_cells, nl, nl))
    fe = np.zeros((prob.mesh.n_cells, nl))
    for e in range(prob.mesh.n_cells):
        xv = prob.mesh.coords[prob.mesh.cell_vertices[e]]
        Ke[e], fe[e] = oracle.cell_matrix(problem, p, p + 1, xv, prob.coef[e], prob.nu, prob.force)
    Kflat = Ke.reshape(-1)
    vals = np.zeros(sp.nnz)
    rhs = np.zeros(sp.n_dofs)
    seen = np.zeros(Kflat.size, dtype=np.int64)
    for r in range(sp.n_dofs):
        sl = slots[slot_ptr[r]:slot_ptr[r + 1]]
        assert np.all(np.diff(sl // nl) > 0)                     # cells ascending
        assert np.all(cd.reshape(-1)[sl] == r)
        rhs[r] = fe.reshape(-1)[sl].sum()
        c = code_ptr[r]
        assert c % 8 == 0 and code_ptr[r + 1] - c == (len(sl) * nl + 7) // 8 * 8
        for k in range(rp[r], rp[r + 1]):
            seg = codes[c:c + cnt[k]].astype(np.int64)
            c += cnt[k]
            head, s, m = seg >> 15, (seg >> 8) & 127, seg & 255
            assert head[0] == 1 and np.all(head[1:] == 0)        # a run per nonzero
            assert np.all(np.diff(s) > 0)                        # ascending cell within a nonzero
            src = sl[s].astype(np.int64) * nl + m
            assert np.all(cd.reshape(-1)[(sl[s] // nl) * nl + m] == col[k])
            seen[src] += 1
            vals[k] = Kflat[src].sum()
        assert c == code_ptr[r] + len(sl) * nl
    assert np.all(seen == 1)                                     # a permutation of all contributions
    if problem == 1:
        # the three rows of a node (consecutive DOFs) lie in the same cells at local rows
        # i*nb + a and share columns and codes: the scatter reads one position block per node
        nb = (p + 1) ** 3
        for n in range(sp.n_dofs // 3):
            r0 = 3 * n
            for i in (1, 2):
                r = r0 + i
                np.testing.assert_array_equal(slots[slot_ptr[r]:slot_ptr[r + 1]],
                                              slots[slot_ptr[r0]:slot_ptr[r0 + 1]] + i * nb)
                np.testing.assert_array_equal(col[rp[r]:rp[r + 1]], col[rp[r0]:rp[r0 + 1]])
                np.testing.assert_array_equal(codes[code_ptr[r]:code_ptr[r + 1]],
                                              codes[code_ptr[r0]:code_ptr[r0 + 1]])
    np.testing.assert_allclose(vals, val_o, rtol=0, atol=1e-13 * np.abs(val_o).max())
    np.testing.assert_allclose(rhs, rhs_o, rtol=0, atol=1e-14)
    sp.close()


def test_structured_pattern_sizes():
    """(3n+1)^3 nonzeros per component pair for Q1 and (8n+1)^3 for Q2 on n^3 bricks."""
    for p, per in ((1, lambda n: 3 * n + 1), (2, lambda n: 8 * n + 1)):
        prob = inputs.small_problem((4, 3, 2), p, 1, seed=1)
        sp = feasm.FESpace(prob, host_only=True)
        assert sp.nnz == 9 * per(4) * per(3) * per(2)
        sp.close()


def test_rotated_cell_orientation_matches_oracle():
    prob = inputs.small_problem((2, 2, 1), 3, 1, seed=11)
    cv = prob.mesh.cell_vertices.copy()
    perm = [(1 - (v & 1)) + 2 * (1 - ((v >> 1) & 1)) + 4 * ((v >> 2) & 1) for v in range(8)]
    cv[1] = cv[1][perm]
    m2 = inputs.Mesh(prob.mesh.coords, cv, prob.mesh.shape, prob.mesh.extent)
    p2 = inputs.Problem("rot", m2, 3, 4, 1, prob.coef, prob.force)
    sp = feasm.FESpace(p2, host_only=True)
    cd_o, n_o = oracle.dof_numbering(m2, 3, 3)
    np.testing.assert_array_equal(sp.cell_dofs(), cd_o)
    sp.close()


def test_invalid_arguments_are_reported():
    prob = inputs.small_problem((2, 2, 2), 1, 0)
    with pytest.raises(feasm.FEError) as ei:
        feasm.fe_space_create(prob.mesh.coords, prob.mesh.cell_vertices, 4, 0, 0, 0.3, host_only=True)
    assert ei.value.code == -1 and "order" in str(ei.value)
    bad = prob.mesh.cell_vertices.copy()
    bad[0, 0] = prob.mesh.n_vertices + 5
    with pytest.raises(feasm.FEError) as ei:
        feasm.fe_space_create(prob.mesh.coords, bad, 1, 0, 0, 0.3, host_only=True)
    assert ei.value.code == -1 and "range" in str(ei.value)
    with pytest.raises(feasm.FEError) as ei:
        feasm.fe_space_create(prob.mesh.coords, prob.mesh.cell_vertices, 1, 0, 1, 0.5, host_only=True)
    assert ei.value.code == -1
    with pytest.raises(feasm.FEError) as ei:
        feasm.fe_space_create(prob.mesh.coords, prob.mesh.cell_vertices, 2, 9, 0, 0.3, host_only=True)
    assert ei.value.code == -1


def test_empty_mesh_host_setup():
    mesh = inputs.Mesh(np.zeros((0, 3)), np.zeros((0, 8), dtype=np.int32), (0, 0, 0), (1, 1, 1))
    h = feasm.fe_space_create(mesh.coords, mesh.cell_vertices, 2, 0, 1, 0.3, host_only=True)
    assert feasm.fe_space_sizes(h) == (0, 0, 0, 0)
    feasm.fe_space_destroy(h)


def _morton_model(mesh):
    """Morton codes of the cell centroids written out bit by bit (21 bits per
    axis over the centroids' bounding box, x in the lowest bit of each triple)."""
    cen = mesh.coords[mesh.cell_vertices].mean(axis=1)
    lo, hi = cen.min(axis=0), cen.max(axis=0)
    span = np.where(hi > lo, hi - lo, 1.0)
    top = (1 << 21) - 1
    q = np.clip(np.floor((cen - lo) / span * top), 0, top).astype(np.int64)
    q[:, hi <= lo] = 0
    code = np.zeros(mesh.n_cells, dtype=np.uint64)
    for b in range(21):
        for k in range(3):
            code |= (((q[:, k] >> b) & 1).astype(np.uint64)) << np.uint64(3 * b + k)
    return code


def _locality(mesh):
    """Mean distance in cell position between cells that share a face."""
    faces = {}
    for e, cv in enumerate(mesh.cell_vertices):
        for d in range(3):
            for s in range(2):
                f = tuple(sorted(int(cv[v]) for v in range(8) if ((v >> d) & 1) == s))
                faces.setdefault(f, []).append(e)
    pairs = np.array([v for v in faces.values() if len(v) == 2])
    return float(np.abs(pairs[:, 0] - pairs[:, 1]).mean())


def test_locality_order_sorts_centroid_morton_codes():
    """fe_mesh_locality_order returns a permutation that sorts the Morton codes of
    the cell centroids (ties in input order), and on a scrambled brick it brings
    face neighbours close again: the mean position distance of face-sharing cells
    drops far below the scrambled one, to the order of the lexicographic brick's."""
    base = inputs.small_problem((12, 10, 8), 1, 1, seed=5)
    scr = inputs.scrambled(base, seed=6)
    order = feasm.fe_mesh_locality_order(scr.mesh.coords, scr.mesh.cell_vertices)
    assert order.dtype == np.int64 and np.array_equal(np.sort(order), np.arange(scr.mesh.n_cells))
    code = _morton_model(scr.mesh)
    np.testing.assert_array_equal(order, np.lexsort((np.arange(scr.mesh.n_cells), code)))
    np.testing.assert_array_equal(order, feasm.fe_mesh_locality_order(scr.mesh.coords, scr.mesh.cell_vertices))
    re = inputs.reordered(scr, order)
    brick, scrambled, morton = _locality(base.mesh), _locality(scr.mesh), _locality(re.mesh)
    assert morton < 0.2 * scrambled and morton < 1.5 * brick, (brick, scrambled, morton)
    # the reordered mesh is the same problem: coefficients follow their cells
    np.testing.assert_array_equal(re.coef, scr.coef[order])


def test_locality_order_edge_cases():
    m = inputs.brick(1, 1, 1)
    assert feasm.fe_mesh_locality_order(m.coords, m.cell_vertices).tolist() == [0]
    empty = feasm.fe_mesh_locality_order(m.coords, m.cell_vertices[:0])
    assert empty.size == 0
    flat = inputs.brick(5, 1, 1)               # all centroids on one line: two degenerate axes
    np.testing.assert_array_equal(feasm.fe_mesh_locality_order(flat.coords, flat.cell_vertices), np.arange(5))
    bad = m.cell_vertices.copy()
    bad[0, 3] = m.n_vertices                    # vertex id out of range
    with pytest.raises(feasm.FEError):
        feasm.fe_mesh_locality_order(m.coords, bad)
    nan = m.coords.copy()
    nan[0, 0] = np.nan
    with pytest.raises(feasm.FEError):
        feasm.fe_mesh_locality_order(nan, m.cell_vertices)


def test_cell_repeating_a_vertex_is_rejected():
    """A hexahedron whose vertex list repeats an id (a collapsed edge) is refused
    at setup with FE_ERR_INVALID_ARG, as are vertex ids out of range."""
    m = inputs.brick(2, 1, 1)
    bad = m.cell_vertices.copy()
    bad[1, 7] = bad[1, 6]
    prob = inputs.Problem("bad", inputs.Mesh(m.coords, bad, (), m.extent), 1, 2, 0, np.ones(2), np.ones(1))
    with pytest.raises(feasm.FEError) as e:
        feasm.FESpace(prob, host_only=True)
    assert e.value.code == -1 and "repeats a vertex" in str(e.value)
    bad = m.cell_vertices.copy()
    bad[0, 0] = -1
    prob = inputs.Problem("bad", inputs.Mesh(m.coords, bad, (), m.extent), 1, 2, 0, np.ones(2), np.ones(1))
    with pytest.raises(feasm.FEError) as e:
        feasm.FESpace(prob, host_only=True)
    assert e.value.code == -1

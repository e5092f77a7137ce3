"""Pins of the FP64 oracle against facts the paper and the mathematics fix.

Nothing here compares the oracle with itself: each test checks a closed form,
an exactness statement, an invariant or a brute-force computation written
independently in numpy. A plausible slip in the oracle (a dropped term, a wrong
sign, a transposed J, a swapped index) fails at least one of them.
"""
import itertools
import math
import os

import numpy as np
import pytest

import oracle
from paper_1708_01773_gb300 import inputs

NU = 0.3


# ---------------------------------------------------------------- helpers
def lame_hat(nu):
    return nu / ((1 + nu) * (1 - 2 * nu)), 1.0 / (2 * (1 + nu))


def node_positions(prob, cell_dofs, n_dofs):
    """Physical position of every DOF: Phi_K(alpha/p) with the trilinear map,
    checked to agree between all cells sharing the DOF (conformity)."""
    p = prob.order
    n1 = p + 1
    mesh = prob.mesh
    al = np.array([[a % n1, (a // n1) % n1, a // (n1 * n1)] for a in range(n1 ** 3)]) / p
    N = np.ones((n1 ** 3, 8))
    for v in range(8):
        b = [(v >> d) & 1 for d in range(3)]
        for d in range(3):
            N[:, v] *= al[:, d] if b[d] else 1 - al[:, d]
    xv = mesh.coords[mesh.cell_vertices]                     # [cells, 8, 3]
    xn = np.einsum("av,evk->eak", N, xv)                     # [cells, nb, 3]
    pos = np.full((n_dofs, 3), np.nan)
    nb = n1 ** 3
    for c in range(prob.ncomp):
        d = cell_dofs[:, c * nb:(c + 1) * nb]
        pos[d.ravel()] = xn.reshape(-1, 3)
    # every cell must agree with the stored position
    for c in range(prob.ncomp):
        d = cell_dofs[:, c * nb:(c + 1) * nb]
        np.testing.assert_allclose(pos[d.ravel()], xn.reshape(-1, 3), atol=1e-13)
    comp = np.zeros(n_dofs, dtype=np.int64)
    for c in range(prob.ncomp):
        comp[cell_dofs[:, c * nb:(c + 1) * nb].ravel()] = c
    return pos, comp


def csr_to_dense(row_ptr, col, val, n):
    A = np.zeros((n, n))
    for r in range(n):
        A[r, col[row_ptr[r]:row_ptr[r + 1]]] = val[row_ptr[r]:row_ptr[r + 1]]
    return A


def boundary_dofs(pos, tol=1e-12, extent=(1.0, 1.0, 1.0)):
    b = np.zeros(pos.shape[0], dtype=bool)
    for d in range(3):
        b |= np.abs(pos[:, d]) < tol
        b |= np.abs(pos[:, d] - extent[d]) < tol
    return b


# ---------------------------------------------------------------- Gauss rule
@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 8, 12])
def test_gauss_exactness(n):
    """An n-point rule integrates x^k on [0,1] exactly for k <= 2n-1 and not for 2n."""
    x, w = oracle.gauss_legendre(n)
    assert np.all(np.diff(x) > 0) and np.all((x > 0) & (x < 1)) and np.all(w > 0)
    for k in range(2 * n):
        assert abs(np.dot(w, x ** k) - 1.0 / (k + 1)) < 1e-14
    # degree 2n is not exact: the rule gives 0 for P_n(2x-1)^2 (it vanishes at the nodes),
    # whose integral over [0,1] is 1/(2n+1)
    Pn = np.polynomial.legendre.Legendre.basis(n)(2 * x - 1)
    assert np.abs(Pn).max() < 1e-13 and abs(np.dot(w, Pn ** 2)) < 1e-25


def test_gauss_closed_forms():
    x, w = oracle.gauss_legendre(2)
    np.testing.assert_allclose(x, [0.5 - 0.5 / math.sqrt(3), 0.5 + 0.5 / math.sqrt(3)], atol=1e-15)
    np.testing.assert_allclose(w, [0.5, 0.5], atol=1e-15)
    x, w = oracle.gauss_legendre(3)
    s = 0.5 * math.sqrt(3 / 5)
    np.testing.assert_allclose(x, [0.5 - s, 0.5, 0.5 + s], atol=1e-15)
    np.testing.assert_allclose(w, [5 / 18, 8 / 18, 5 / 18], atol=1e-15)
    x, w = oracle.gauss_legendre(4)
    t = np.array([-math.sqrt(3 / 7 + 2 / 7 * math.sqrt(6 / 5)), -math.sqrt(3 / 7 - 2 / 7 * math.sqrt(6 / 5))])
    t = np.concatenate([t, -t[::-1]])
    wt = np.array([(18 - math.sqrt(30)) / 36, (18 + math.sqrt(30)) / 36])
    wt = np.concatenate([wt, wt[::-1]])
    np.testing.assert_allclose(x, 0.5 * (t + 1), atol=1e-15)
    np.testing.assert_allclose(w, 0.5 * wt, atol=1e-15)


# ---------------------------------------------------------------- Lagrange basis
@pytest.mark.parametrize("p", [1, 2, 3])
def test_lagrange_kronecker_and_partition(p):
    for l in range(p + 1):
        v, _ = oracle.lagrange_1d(p, l / p)
        np.testing.assert_allclose(v, np.eye(p + 1)[l], atol=1e-15)
    rng = np.random.default_rng(0)
    for x in rng.uniform(-0.2, 1.2, 10):
        v, d = oracle.lagrange_1d(p, x)
        assert abs(v.sum() - 1) < 1e-13 and abs(d.sum()) < 1e-12
        # derivative vs a central difference of the values
        h = 1e-6
        vp, _ = oracle.lagrange_1d(p, x + h)
        vm, _ = oracle.lagrange_1d(p, x - h)
        np.testing.assert_allclose(d, (vp - vm) / (2 * h), atol=1e-8)
        # reproduces x^k for k <= p
        for k in range(p + 1):
            nodes = np.arange(p + 1) / p
            assert abs(np.dot(v, nodes ** k) - x ** k) < 1e-12


# ---------------------------------------------------------------- closed-form unit cube
UNIT = np.array([[(v & 1), (v >> 1) & 1, (v >> 2) & 1] for v in range(8)], dtype=float)


def test_q1_unit_cube_laplacian_closed_form():
    """K = K1(x)M1(x)M1 + ...: 1/3 on the diagonal, 0 / -1/12 / -1/12 at Hamming distance 1/2/3."""
    K, f = oracle.cell_matrix(0, 1, 2, UNIT, 1.0, NU, [1.0])
    for a in range(8):
        for b in range(8):
            h = bin(a ^ b).count("1")
            assert abs(K[a, b] - [1 / 3, 0.0, -1 / 12, -1 / 12][h]) < 1e-15
    np.testing.assert_allclose(f, np.full(8, 1 / 8), atol=1e-15)
    K2, _ = oracle.cell_matrix(0, 1, 2, UNIT, 3.5, NU, [1.0])
    np.testing.assert_allclose(K2, 3.5 * K, atol=1e-14)


def test_q1_unit_cube_elasticity_closed_form():
    """Elasticity on the unit cube from 1D factor integrals (independent of the oracle's
    stress/strain contraction): G^{ij}_{ab} = prod_d (K1 | C1 | C1^T | M1)."""
    M1 = np.array([[1 / 3, 1 / 6], [1 / 6, 1 / 3]])
    K1 = np.array([[1.0, -1.0], [-1.0, 1.0]])
    C1 = np.array([[-0.5, -0.5], [0.5, 0.5]])    # C1[a,b] = int l_a' l_b

    def G(i, j, a, b):
        val = 1.0
        for d in range(3):
            ad, bd = (a >> d) & 1, (b >> d) & 1
            if d == i and d == j:
                val *= K1[ad, bd]
            elif d == i:
                val *= C1[ad, bd]
            elif d == j:
                val *= C1[bd, ad]
            else:
                val *= M1[ad, bd]
        return val

    E = 2.7
    lh, mh = lame_hat(NU)
    Kref = np.zeros((24, 24))
    for i, j, a, b in itertools.product(range(3), range(3), range(8), range(8)):
        v = lh * G(i, j, a, b) + mh * G(j, i, a, b)
        if i == j:
            v += mh * sum(G(k, k, a, b) for k in range(3))
        Kref[i * 8 + a, j * 8 + b] = E * v
    K, f = oracle.cell_matrix(1, 1, 2, UNIT, E, NU, [0.0, 0.0, -1.0])
    np.testing.assert_allclose(K, Kref, atol=1e-14)
    np.testing.assert_allclose(f, np.concatenate([np.zeros(16), -np.full(8, 1 / 8)]), atol=1e-15)


# ---------------------------------------------------------------- affine cells: exact quadrature
def affine_cell(rng, scale=1.0):
    A = np.eye(3) + 0.3 * rng.uniform(-1, 1, (3, 3))
    b = rng.uniform(-1, 1, 3)
    return scale * (UNIT @ A.T) + b, A


@pytest.mark.parametrize("p", [1, 2, 3])
@pytest.mark.parametrize("problem", [0, 1])
def test_affine_cell_exact_vs_brute_force(p, problem):
    """On a parallelepiped the (p+1)-point rule is exact: a 12-point rule must agree."""
    rng = np.random.default_rng(10 * p + problem)
    xv, _ = affine_cell(rng)
    K, f = oracle.cell_matrix(problem, p, p + 1, xv, 1.7, NU, [0.3, -0.2, 1.1])
    Kb, fb = oracle.cell_matrix(problem, p, 12, xv, 1.7, NU, [0.3, -0.2, 1.1])
    sc = np.abs(Kb).max()
    assert np.abs(K - Kb).max() < 1e-13 * sc
    assert np.abs(f - fb).max() < 1e-13 * np.abs(fb).max()


@pytest.mark.parametrize("problem", [0, 1])
def test_scaling_and_rotation(problem):
    """3D stiffness scales linearly with the cell size; Poisson is rotation invariant and
    the elasticity blocks transform with R (comp-major local index i*nb + a)."""
    rng = np.random.default_rng(3)
    p = 2
    xv = UNIT + 0.1 * rng.uniform(-1, 1, (8, 3))
    K, _ = oracle.cell_matrix(problem, p, 3, xv, 1.0, NU, [0, 0, 0])
    Ks, _ = oracle.cell_matrix(problem, p, 3, 2.5 * xv, 1.0, NU, [0, 0, 0])
    np.testing.assert_allclose(Ks, 2.5 * K, atol=1e-12 * np.abs(K).max())
    th = 0.7
    R = np.array([[math.cos(th), -math.sin(th), 0], [math.sin(th), math.cos(th), 0], [0, 0, 1]])
    R = R @ np.array([[1, 0, 0], [0, math.cos(0.4), -math.sin(0.4)], [0, math.sin(0.4), math.cos(0.4)]])
    Kr, _ = oracle.cell_matrix(problem, p, 3, xv @ R.T, 1.0, NU, [0, 0, 0])
    if problem == 0:
        np.testing.assert_allclose(Kr, K, atol=1e-12 * np.abs(K).max())
    else:
        nb = (p + 1) ** 3
        Q = np.kron(R, np.eye(nb))
        np.testing.assert_allclose(Kr, Q @ K @ Q.T, atol=1e-12 * np.abs(K).max())


def test_distorted_cell_converges_with_quadrature():
    """On a distorted cell the (p+1) rule is the method's value, not the exact integral;
    increasing the rule must converge (sanity check)."""
    rng = np.random.default_rng(5)
    xv = UNIT + 0.2 * rng.uniform(-1, 1, (8, 3))
    ref, _ = oracle.cell_matrix(1, 2, 14, xv, 1.0, NU, [0, 0, 0])
    errs = [np.abs(oracle.cell_matrix(1, 2, n, xv, 1.0, NU, [0, 0, 0])[0] - ref).max() for n in (3, 5, 8)]
    assert errs[0] > errs[1] > errs[2] and errs[2] < 1e-6 * np.abs(ref).max()


# ---------------------------------------------------------------- independent numpy brute force
def numpy_cell_matrix(problem, p, nq1d, xv, coef, nu):
    """Second implementation: einsum over quadrature points, Gram-block form of
    elasticity, numpy's Gauss-Legendre nodes on [-1,1] mapped to [0,1]."""
    t, wt = np.polynomial.legendre.leggauss(nq1d)
    x1, w1 = 0.5 * (t + 1), 0.5 * wt
    n1 = p + 1
    nodes = np.arange(n1) / p

    def lag(x):
        V = np.ones((len(x), n1))
        D = np.zeros((len(x), n1))
        for m in range(n1):
            for s in range(n1):
                if s != m:
                    V[:, m] *= (x - nodes[s]) / (nodes[m] - nodes[s])
            for r in range(n1):
                if r == m:
                    continue
                term = np.full(len(x), 1 / (nodes[m] - nodes[r]))
                for s in range(n1):
                    if s != m and s != r:
                        term *= (x - nodes[s]) / (nodes[m] - nodes[s])
                D[:, m] += term
        return V, D

    V, D = lag(x1)
    Vg, Dg = np.array([[1 - x, x] for x in x1]), np.tile([-1.0, 1.0], (nq1d, 1))
    qi = np.array(list(itertools.product(range(nq1d), repeat=3)))[:, ::-1]   # x fastest
    ai = np.array(list(itertools.product(range(n1), repeat=3)))[:, ::-1]
    vi = np.array(list(itertools.product(range(2), repeat=3)))[:, ::-1]
    w = w1[qi[:, 0]] * w1[qi[:, 1]] * w1[qi[:, 2]]

    def grads(Vt, Dt, idx):
        g = np.empty((len(qi), len(idx), 3))
        for d in range(3):
            f = np.ones((len(qi), len(idx)))
            for e in range(3):
                T = Dt if e == d else Vt
                f *= T[qi[:, e]][:, idx[:, e]]
            g[:, :, d] = f
        return g

    gref = grads(V, D, ai)
    gN = grads(Vg, Dg, vi)
    J = np.einsum("vk,qvd->qkd", xv, gN)
    det = np.linalg.det(J)
    Jinv = np.linalg.inv(J)
    g = np.einsum("qad,qdk->qak", gref, Jinv)
    c = w * det
    Gm = np.einsum("q,qai,qbj->ijab", c, g, g)
    nb = n1 ** 3
    if problem == 0:
        return coef * (Gm[0, 0] + Gm[1, 1] + Gm[2, 2])
    if problem == 2:
        # Taylor-Hood: mu eps:eps = mu/2 (delta_ij tr G + G^{ji}); pressure Q_{p-1}
        # on the nodes k/(p-1); coupling -int psi_c d_j phi_b in both off-diagonal blocks
        nbp = p ** 3
        pn = np.arange(p) / (p - 1)
        Vp = np.ones((nq1d, p))
        for m in range(p):
            for s_ in range(p):
                if s_ != m:
                    Vp[:, m] *= (x1 - pn[s_]) / (pn[m] - pn[s_])
        pi = np.array(list(itertools.product(range(p), repeat=3)))[:, ::-1]
        psi = Vp[qi[:, 0]][:, pi[:, 0]] * Vp[qi[:, 1]][:, pi[:, 1]] * Vp[qi[:, 2]][:, pi[:, 2]]
        K = np.zeros((3 * nb + nbp, 3 * nb + nbp))
        tr = Gm[0, 0] + Gm[1, 1] + Gm[2, 2]
        for i in range(3):
            for j in range(3):
                K[i * nb:(i + 1) * nb, j * nb:(j + 1) * nb] = 0.5 * coef * (Gm[j, i] + (tr if i == j else 0))
        Bm = -np.einsum("q,qc,qbj->cjb", c, psi, g).reshape(nbp, 3 * nb)
        K[3 * nb:, :3 * nb] = Bm
        K[:3 * nb, 3 * nb:] = Bm.T
        return K
    lh, mh = lame_hat(nu)
    K = np.zeros((3 * nb, 3 * nb))
    tr = Gm[0, 0] + Gm[1, 1] + Gm[2, 2]
    for i in range(3):
        for j in range(3):
            blk = lh * Gm[i, j] + mh * Gm[j, i] + (mh * tr if i == j else 0)
            K[i * nb:(i + 1) * nb, j * nb:(j + 1) * nb] = coef * blk
    return K


@pytest.mark.parametrize("p", [1, 2, 3])
@pytest.mark.parametrize("problem", [0, 1])
def test_distorted_cell_vs_numpy_brute_force(p, problem):
    rng = np.random.default_rng(100 + p)
    xv = UNIT * np.array([1.3, 0.7, 1.0]) + 0.2 * rng.uniform(-1, 1, (8, 3))
    K, _ = oracle.cell_matrix(problem, p, p + 1, xv, 2.3, NU, [0, 0, 0])
    Kn = numpy_cell_matrix(problem, p, p + 1, xv, 2.3, NU)
    np.testing.assert_allclose(K, Kn, atol=1e-13 * np.abs(Kn).max())


# ---------------------------------------------------------------- DOF numbering
def test_dof_numbering_list_dofs_order_single_q2_cell():
    """One Q2 cell: the interior node is numbered first, then the 8 vertices, then
    x-, y-, z-edges (anchors ascending), then the faces (xy, xz, yz)."""
    mesh = inputs.brick(1, 1, 1)
    cd, n = oracle.dof_numbering(mesh, 2, 1)
    assert n == 27
    lex = lambda i, j, k: i + 3 * j + 9 * k
    expected_order = [lex(1, 1, 1)]
    expected_order += [lex(2 * (v & 1), 2 * ((v >> 1) & 1), 2 * ((v >> 2) & 1)) for v in range(8)]
    expected_order += [lex(1, 0, 0), lex(1, 2, 0), lex(1, 0, 2), lex(1, 2, 2)]   # x-edges
    expected_order += [lex(0, 1, 0), lex(2, 1, 0), lex(0, 1, 2), lex(2, 1, 2)]   # y-edges
    expected_order += [lex(0, 0, 1), lex(2, 0, 1), lex(0, 2, 1), lex(2, 2, 1)]   # z-edges
    expected_order += [lex(1, 1, 0), lex(1, 1, 2)]                               # xy faces
    expected_order += [lex(1, 0, 1), lex(1, 2, 1)]                               # xz faces
    expected_order += [lex(0, 1, 1), lex(2, 1, 1)]                               # yz faces
    got = np.empty(27, dtype=int)
    got[cd[0]] = np.arange(27)
    assert list(got) == expected_order


def _golden(name):
    """Sections of a text fixture under tests/golden: a keyword line followed by
    rows of integers, or a keyword and its integers on one line."""
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", name)
    out, key = {}, None
    for line in open(path):
        line = line.split("#", 1)[0].split()
        if not line:
            continue
        if line[0].lstrip("-").isdigit():
            out[key].append([int(v) for v in line])
        else:
            key = line[0]
            out[key] = [[int(v) for v in line[1:]]] if len(line) > 1 else []
    return out


def test_dof_numbering_matches_the_papers_bicubic_example():
    """The paper's printed bicubic quadrilateral (tests/golden/bicubic_quad_dofs.txt):
    on the z = 0 face of one Q3 hexahedron (the same 4 x 4 nodes), the node
    numbering is x-fastest lexicographic, and the order in which list_dofs meets
    the face's nodes is the concatenation of the owned-DOF lists of its n-faces
    in the figure's order (vertices, x-edges, y-edges, the face). The nodes of
    n-face 8 (the edge x = 1) are those with alpha_x = 3."""
    g = _golden("bicubic_quad_dofs.txt")
    labels = np.array(g["labels"])
    for j in range(4):
        for i in range(4):
            assert labels[j, i] == 1 + i + 4 * j          # the figure's node at (i, j)
    ptr, lst = g["p"][0], g["l"][0]
    assert len(ptr) == 10 and ptr[-1] - 1 == len(lst) == 16
    mesh = inputs.brick(1, 1, 1)
    cd, n = oracle.dof_numbering(mesh, 3, 1)
    order = np.argsort(cd[0])                            # local nodes in the order list_dofs numbers them
    face = [int(a) + 1 for a in order if a < 16]         # the z = 0 layer, as 1-based 2D labels
    assert face == lst
    # each n-face's owned nodes are consecutive in that order
    for f in range(9):
        owned = lst[ptr[f] - 1:ptr[f + 1] - 1]
        pos = [face.index(v) for v in owned]
        assert pos == list(range(pos[0], pos[0] + len(owned)))
    assert sorted(a + 1 for a in range(16) if a % 4 == 3) == g["dofs_n_face_8"][0]


def test_dof_numbering_matches_the_papers_n_face_numbering():
    """The paper's printed n-face numbering of the quadrilateral
    (tests/golden/quad_nface_numbering.txt): each n-face's drawn point is the
    centroid of its listed vertices, and on the z = 0 face of one Q2 hexahedron
    (one node per n-face) list_dofs meets the nodes at those points in the
    figure's n-face order (vertices, the two x-edges, the two y-edges, the face)."""
    g = _golden("quad_nface_numbering.txt")
    pts = {row[0]: np.array(row[1:], dtype=float) / 2.0 for row in g["position"]}
    ptr, lst = g["p"][0], g["l"][0]
    for k in range(1, 10):
        verts = lst[ptr[k - 1] - 1:ptr[k] - 1]
        np.testing.assert_allclose(np.mean([pts[v] for v in verts], axis=0), pts[k])
    # n-faces numbered by dimension: 4 vertices, 4 edges, 1 cell (the paper's
    # ptr_n_faces_x_dim = {1, 5, 9, 10}), read off the vertex counts
    dims = [int(np.log2(ptr[k] - ptr[k - 1])) for k in range(1, 10)]
    assert dims == [0] * 4 + [1] * 4 + [2]
    ptr_x_dim = [1 + sum(1 for d in dims if d < m) for m in range(4)]
    assert ptr_x_dim == g["ptr_n_faces_x_dim"][0]
    cd, n = oracle.dof_numbering(inputs.brick(1, 1, 1), 2, 1)
    layer = [int(a) for a in np.argsort(cd[0]) if a < 9]   # z = 0 nodes in numbering order
    got = [np.array([a % 3, a // 3], dtype=float) / 2.0 for a in layer]
    np.testing.assert_allclose(np.array(got), np.array([pts[k] for k in range(1, 10)]))


def test_node_sharing_matches_the_papers_cube_n_face_codes():
    """The paper's printed [extrusion|anchor] codes of the 3-cube's n-faces
    (tests/golden/cube_nface_codes.txt): 26 distinct codes, 8 vertices, 12
    edges and 6 faces, anchor bits only in directions not extruded. A node
    alpha of a Q2 cell lies on the n-face extruded where alpha_d = 1 and
    anchored where alpha_d = 2; in a 3 x 3 x 3 brick the oracle's numbering
    gives each node of the centre cell to 2^(3 - |ext|) cells, and the codes of
    the centre cell's 26 boundary nodes are the printed ones."""
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "cube_nface_codes.txt")
    printed = set()
    for line in open(path):
        line = line.split("#", 1)[0].strip()
        if line.startswith("["):
            e, a = line.strip("[]").split("|")
            printed.add((tuple(int(c) for c in e), tuple(int(c) for c in a)))
    assert len(printed) == 26
    assert sorted(sum(e) for e, _ in printed) == [0] * 8 + [1] * 12 + [2] * 6
    assert all(not (x and y) for e, a in printed for x, y in zip(e, a))
    cd, n = oracle.dof_numbering(inputs.brick(3, 3, 3), 2, 1)
    centre = 1 + 3 + 9
    count = np.bincount(cd.ravel(), minlength=n)
    codes = set()
    for a in range(27):
        al = (a % 3, (a // 3) % 3, a // 9)
        e = tuple(int(x == 1) for x in al)
        anc = tuple(int(x == 2) for x in al)
        assert count[cd[centre, a]] == 2 ** (3 - sum(e))
        if sum(e) < 3:
            codes.add((e, anc))
    # the printed strings' direction order is not stated; the set is the same
    # under either reading of the bit order
    flip = {(e[::-1], a[::-1]) for e, a in printed}
    assert codes == printed == flip


def test_dof_numbering_two_cells_share_face():
    mesh = inputs.brick(2, 1, 1)
    cd, n = oracle.dof_numbering(mesh, 1, 3)
    assert n == 12 * 3
    # cell 0: vertices in local order, 3 consecutive ids per node, local index c*8 + a
    np.testing.assert_array_equal(cd[0].reshape(3, 8), np.arange(24).reshape(8, 3).T)
    # cell 1 shares its x=0 face (local 0,2,4,6) with cell 0's x=1 face (local 1,3,5,7)
    np.testing.assert_array_equal(cd[1].reshape(3, 8)[:, [0, 2, 4, 6]], cd[0].reshape(3, 8)[:, [1, 3, 5, 7]])
    np.testing.assert_array_equal(cd[1].reshape(3, 8)[:, [1, 3, 5, 7]], 24 + np.arange(12).reshape(4, 3).T)


@pytest.mark.parametrize("p,ncomp,shape", [(1, 1, (3, 2, 2)), (2, 3, (2, 3, 2)), (3, 1, (2, 2, 3)), (3, 3, (2, 1, 2))])
def test_dof_numbering_conformity(p, ncomp, shape):
    """(s,K) ~ (s',K') iff x_s = x_s': every DOF has one position, DOF count is the
    structured node count, and distinct DOFs of one component sit at distinct points."""
    prob = inputs.small_problem(shape, p, 1 if ncomp == 3 else 0, seed=p)
    cd, n = oracle.dof_numbering(prob.mesh, p, ncomp)
    nx, ny, nz = shape
    assert n == ncomp * (p * nx + 1) * (p * ny + 1) * (p * nz + 1)
    pos, comp = node_positions(prob, cd, n)
    for c in range(ncomp):
        pts = np.round(pos[comp == c], 12)
        assert len(np.unique(pts, axis=0)) == len(pts)
    # a node's components carry consecutive ids
    if ncomp == 3:
        nb = (p + 1) ** 3
        np.testing.assert_array_equal(cd[:, nb:2 * nb], cd[:, :nb] + 1)
        np.testing.assert_array_equal(cd[:, 2 * nb:], cd[:, :nb] + 2)


def test_dof_numbering_rotated_cells():
    """Cells given with a rotated local vertex order (same geometry) must keep the
    space conforming: node keys are orientation free."""
    prob = inputs.small_problem((2, 2, 1), 3, 0, seed=11)
    mesh = prob.mesh
    cv = mesh.cell_vertices.copy()
    # rotate cell 1 by 180 degrees about z: local (x,y,z) -> (1-x, 1-y, z)
    perm = [(1 - (v & 1)) + 2 * (1 - ((v >> 1) & 1)) + 4 * ((v >> 2) & 1) for v in range(8)]
    cv[1] = cv[1][perm]
    m2 = inputs.Mesh(mesh.coords, cv, mesh.shape, mesh.extent)
    prob2 = inputs.Problem("rot", m2, 3, 4, 0, prob.coef, prob.force)
    cd, n = oracle.dof_numbering(m2, 3, 1)
    assert n == (3 * 2 + 1) * (3 * 2 + 1) * (3 * 1 + 1)
    node_positions(prob2, cd, n)


def dof_correspondence(prob_a, cd_a, n_a, prob_b, cd_b, n_b):
    """perm with DOF m of space a = DOF perm[m] of space b, matched by node
    position and component (both spaces on the same geometry)."""
    assert n_a == n_b
    xa, ca = node_positions(prob_a, cd_a, n_a)
    xb, cb = node_positions(prob_b, cd_b, n_b)

    def order(x, c):
        r = np.round(x, 9)
        return np.lexsort((c, r[:, 2], r[:, 1], r[:, 0]))

    ia, ib = order(xa, ca), order(xb, cb)
    np.testing.assert_allclose(xa[ia], xb[ib], atol=1e-12)
    np.testing.assert_array_equal(ca[ia], cb[ib])
    perm = np.empty(n_a, dtype=np.int64)
    perm[ia] = ib
    return perm


@pytest.mark.parametrize("p,problem,shape", [(1, 0, (3, 3, 2)), (1, 1, (3, 2, 2)), (2, 0, (3, 2, 2)),
                                             (2, 1, (2, 2, 2)), (3, 0, (2, 2, 2)), (3, 1, (2, 1, 2))])
def test_assembly_invariant_under_unstructured_numbering(p, problem, shape):
    """The scrambled brick (random vertex ids and cell order, every cell's local
    vertex order turned by a random proper rotation) is the same discrete
    problem: its matrix and RHS equal the brick's under the DOF correspondence
    of node positions and components. This pins the orientation-free node keys
    of list_dofs and the cell matrix's covariance with the cell's local frame
    (the tensor Gauss rule is invariant under the cube's rotations), and that
    the coefficient of a cell follows the cell."""
    prob = inputs.small_problem(shape, p, problem, seed=40 + 2 * p + problem)
    scr = inputs.scrambled(prob, seed=p + 3 * problem)
    cd0, n0 = oracle.dof_numbering(prob.mesh, p, prob.ncomp)
    cd1, n1 = oracle.dof_numbering(scr.mesh, p, scr.ncomp)
    perm = dof_correspondence(prob, cd0, n0, scr, cd1, n1)
    assert not np.array_equal(perm, np.arange(n0))
    rp0, col0, val0, rhs0 = oracle.assemble_csr(prob, cd0, n0)
    rp1, col1, val1, rhs1 = oracle.assemble_csr(scr, cd1, n1)
    A0 = csr_to_dense(rp0, col0, val0, n0)
    A1 = csr_to_dense(rp1, col1, val1, n1)
    np.testing.assert_allclose(A1[np.ix_(perm, perm)], A0, rtol=0, atol=1e-12 * np.abs(A0).max())
    np.testing.assert_allclose(rhs1[perm], rhs0, rtol=0, atol=1e-12 * np.abs(rhs0).max())
    # the same sparsity pattern, up to the renumbering
    assert rp0[-1] == rp1[-1]
    S0 = csr_to_dense(rp0, col0, np.ones(col0.size), n0) != 0
    S1 = csr_to_dense(rp1, col1, np.ones(col1.size), n1) != 0
    np.testing.assert_array_equal(S1[np.ix_(perm, perm)], S0)


# ---------------------------------------------------------------- assembled-system invariants
def assembled(prob):
    cd, n = oracle.dof_numbering(prob.mesh, prob.order, prob.ncomp)
    rp, col, val, rhs = oracle.assemble_csr(prob, cd, n)
    return cd, n, rp, col, val, rhs


def test_poisson_q1_8_invariants():
    prob = inputs.poisson_q1_8()
    assert oracle.min_det_jacobian(prob.mesh, 2) > 0
    cd, n, rp, col, val, rhs = assembled(prob)
    assert n == 729 and rp[-1] == 15625                     # (3n+1)^3 pattern
    A = csr_to_dense(rp, col, val, n)
    assert np.array_equal(A, A.T)                           # bitwise symmetric
    assert np.abs(A @ np.ones(n)).max() < 1e-13 * np.abs(A).max()   # zero row sums
    assert abs(rhs.sum() - 1.0) < 1e-13                     # sum f = vol = 1 for f = 1
    assert np.all(np.diag(A) > 0)


def _lin_fields(pos, comp, ncomp):
    """The linear fields used by the patch test and the rigid-body check."""
    out = []
    for c in range(ncomp):
        for d in range(3):
            u = np.where(comp == c, pos[:, d], 0.0)
            out.append(((c, d), u))
    return out


@pytest.mark.parametrize("p,shape", [(1, (3, 3, 3)), (2, (3, 2, 2)), (3, (2, 2, 2))])
def test_poisson_patch_test(p, shape):
    """Constant conductivity: A u_lin vanishes on interior rows and u^T A u = kappa |a|^2 vol."""
    prob = inputs.small_problem(shape, p, 0, seed=20 + p)
    prob.coef[:] = 2.0
    cd, n, rp, col, val, rhs = assembled(prob)
    A = csr_to_dense(rp, col, val, n)
    pos, comp = node_positions(prob, cd, n)
    interior = ~boundary_dofs(pos)
    a = np.array([0.3, -1.1, 0.7])
    u = pos @ a + 0.5
    r = A @ u
    assert np.abs(r[interior]).max() < 1e-12 * np.abs(A).max()
    assert abs(u @ r - 2.0 * (a @ a) * 1.0) < 1e-12
    assert abs(rhs.sum() - 1.0) < 1e-13


@pytest.mark.parametrize("p,shape", [(1, (3, 2, 3)), (2, (2, 2, 2)), (3, (2, 1, 2))])
def test_elasticity_rigid_modes_and_patch(p, shape):
    """Six rigid-body modes lie in the kernel (any E, any geometry); a uniform strain
    gives the closed-form energy with constant E; RHS z-rows sum to -vol."""
    prob = inputs.small_problem(shape, p, 1, seed=30 + p)
    cd, n, rp, col, val, rhs = assembled(prob)
    A = csr_to_dense(rp, col, val, n)
    sc = np.abs(A).max()
    assert np.abs(A - A.T).max() < 1e-15 * sc               # symmetric to rounding
    pos, comp = node_positions(prob, cd, n)
    for c in range(3):                                       # translations
        t = (comp == c).astype(float)
        assert np.abs(A @ t).max() < 1e-12 * sc
    for w in np.eye(3):                                      # rotations w x x
        r = np.zeros(n)
        disp = np.cross(w[None, :], pos)
        for c in range(3):
            r[comp == c] = disp[comp == c, c]
        assert np.abs(A @ r).max() < 1e-12 * sc
    # uniform strain with constant E: u = eps0 x
    prob.coef[:] = 3.0
    _, _, rp2, col2, val2, _ = assembled(prob)
    A2 = csr_to_dense(rp2, col2, val2, n)
    eps0 = np.array([[0.2, 0.05, -0.1], [0.05, -0.3, 0.15], [-0.1, 0.15, 0.4]])
    disp = pos @ eps0.T
    u = np.zeros(n)
    for c in range(3):
        u[comp == c] = disp[comp == c, c]
    lh, mh = lame_hat(NU)
    exact = 3.0 * (lh * np.trace(eps0) ** 2 + 2 * mh * np.sum(eps0 * eps0)) * 1.0
    assert abs(u @ A2 @ u - exact) < 1e-12 * exact
    r = A2 @ u
    assert np.abs(r[~boundary_dofs(pos)]).max() < 1e-11 * np.abs(A2).max()
    zsum = rhs[comp == 2].sum()
    assert abs(zsum + 1.0) < 1e-13 and abs(rhs[comp == 0].sum()) < 1e-14 and abs(rhs[comp == 1].sum()) < 1e-14


def _o_grid_ring(mesh):
    """The outer boundary of an O-grid's cross-section: its vertices on the
    circle (z = 0), in angular order."""
    xy = mesh.coords[mesh.coords[:, 2] == 0.0][:, :2]
    r = np.hypot(xy[:, 0], xy[:, 1])
    ring = xy[np.abs(r - r.max()) < 1e-12]
    return ring[np.argsort(np.arctan2(ring[:, 1], ring[:, 0]))]


def _o_grid_boundary(pos, ring, height):
    """DOFs on the boundary: the end faces z = 0, height, and the polygon edges
    between consecutive ring vertices (the trilinear cells' straight sides)."""
    b = (np.abs(pos[:, 2]) < 1e-12) | (np.abs(pos[:, 2] - height) < 1e-12)
    a, c = ring, np.roll(ring, -1, axis=0)
    for p0, p1 in zip(a, c):
        d = p1 - p0
        t = np.clip(((pos[:, :2] - p0) @ d) / (d @ d), 0.0, 1.0)
        dist = np.linalg.norm(pos[:, :2] - (p0 + t[:, None] * d), axis=1)
        b |= dist < 1e-12
    return b


@pytest.mark.parametrize("p", [1, 2, 3])
def test_o_grid_invariants(p):
    """On an O-grid (irregular vertex valence: three cells per layer around the
    inner square's corner edges) the assembled Poisson matrix has zero row sums,
    reproduces linear fields on interior rows with the energy |a|^2 vol, and its
    RHS sums to vol (vol = the polygonal cross-section's area x height, by the
    shoelace formula); the elasticity matrix is symmetric with the six rigid
    modes in its kernel and z-rows of the RHS summing to -vol."""
    po = inputs.o_grid_problem(3, 2, 2, p, inputs.POISSON, seed=p)
    assert oracle.min_det_jacobian(po.mesh, po.quad_1d) > 0
    ring = _o_grid_ring(po.mesh)
    area = 0.5 * abs(np.sum(ring[:, 0] * np.roll(ring[:, 1], -1) - np.roll(ring[:, 0], -1) * ring[:, 1]))
    vol = area * po.mesh.extent[2]
    po.coef[:] = 2.0
    cd, n, rp, col, val, rhs = assembled(po)
    A = csr_to_dense(rp, col, val, n)
    pos, comp = node_positions(po, cd, n)
    sc = np.abs(A).max()
    assert np.abs(A.sum(axis=1)).max() < 1e-13 * sc
    a = np.array([0.3, -1.1, 0.7])
    u = pos @ a + 0.5
    inner = ~_o_grid_boundary(pos, ring, po.mesh.extent[2])
    assert inner.sum() > 0
    assert np.abs((A @ u)[inner]).max() < 1e-12 * sc
    assert abs(u @ A @ u - 2.0 * (a @ a) * vol) < 1e-12 * 2.0 * (a @ a) * vol
    assert abs(rhs.sum() - vol) < 1e-13
    el = inputs.o_grid_problem(3, 2, 2, p, inputs.ELASTICITY, seed=10 + p)
    cd, n, rp, col, val, rhs = assembled(el)
    A = csr_to_dense(rp, col, val, n)
    sc = np.abs(A).max()
    assert np.abs(A - A.T).max() < 1e-15 * sc
    pos, comp = node_positions(el, cd, n)
    for c in range(3):
        assert np.abs(A @ (comp == c).astype(float)).max() < 1e-12 * sc
    for w in np.eye(3):
        r = np.zeros(n)
        disp = np.cross(w[None, :], pos)
        for c in range(3):
            r[comp == c] = disp[comp == c, c]
        assert np.abs(A @ r).max() < 1e-12 * sc
    assert abs(rhs[comp == 2].sum() + vol) < 1e-13


def test_assemble_rows_matches_full():
    prob = inputs.small_problem((3, 2, 2), 2, 1, seed=41)
    cd, n, rp, col, val, rhs = assembled(prob)
    rows = np.array([0, 5, n // 2, n - 1], dtype=np.int64)
    ptr, c2, v2, r2 = oracle.assemble_rows(prob, rows, cd, n)
    for q, r in enumerate(rows):
        np.testing.assert_array_equal(c2[ptr[q]:ptr[q + 1]], col[rp[r]:rp[r + 1]])
        np.testing.assert_allclose(v2[ptr[q]:ptr[q + 1]], val[rp[r]:rp[r + 1]], rtol=0, atol=1e-14)
    np.testing.assert_allclose(r2, rhs[rows], atol=1e-15)


@pytest.mark.parametrize("problem", [0, 1])
def test_cell_energies_euler_and_fd(problem):
    """c(E) = u^T A(E) u is linear in E: sum_K E_K g_K = c, and central differences agree."""
    prob = inputs.small_problem((2, 2, 2), 2, problem, seed=50 + problem)
    cd, n, rp, col, val, rhs = assembled(prob)
    A = csr_to_dense(rp, col, val, n)
    u = inputs.unit_rms_field(n, 5)
    g = oracle.cell_energies(prob, u, cd)
    c = u @ A @ u
    assert abs(np.dot(prob.coef, g) - c) < 1e-12 * abs(c)
    for e in (0, 3, 7):
        h = 1e-6 * prob.coef[e]
        cp = prob.coef.copy(); cp[e] += h
        cm = prob.coef.copy(); cm[e] -= h
        pp = inputs.Problem("p", prob.mesh, prob.order, prob.quad_1d, problem, cp, prob.force)
        pm = inputs.Problem("m", prob.mesh, prob.order, prob.quad_1d, problem, cm, prob.force)
        Ap = csr_to_dense(*oracle.assemble_csr(pp, cd, n)[:3], n)
        Am = csr_to_dense(*oracle.assemble_csr(pm, cd, n)[:3], n)
        fd = (u @ Ap @ u - u @ Am @ u) / (2 * h)
        assert abs(fd - g[e]) < 1e-6 * abs(g[e])


def test_workload_meshes_valid_and_patterns():
    """The seeded workloads have positive Jacobians everywhere (the generator does not
    redraw) and the structured pattern sizes of the paper-shaped configs."""
    prob = inputs.elasticity_q2_beam(n=8)
    assert oracle.min_det_jacobian(prob.mesh, 3) > 0
    cd, n = oracle.dof_numbering(prob.mesh, 2, 3)
    assert n == 3 * 17 ** 3
    pc = inputs.cantilever_q1_64(n=16)
    assert oracle.min_det_jacobian(pc.mesh, 2) > 0


# ---------------------------------------------------------------- strong Dirichlet conditions
def test_dirichlet_hand_example():
    """Eq. dirichlet_bc_discrete_problem on a 3x3 system worked by hand: fixing DOF 1
    at 2 leaves rows/columns {0, 2}, and each right-hand side loses A_a1 * 2."""
    rp = np.array([0, 3, 6, 9])
    col = np.array([0, 1, 2] * 3)
    val = np.array([4.0, -1.0, 0.5, -1.0, 4.0, -1.0, 0.5, -1.0, 4.0])
    f = np.array([1.0, 10.0, 3.0])
    lab = oracle.dirichlet_labels([0, 1, 0])
    assert lab.tolist() == [0, -1, 1]
    ptr, c, v, b = oracle.dirichlet_reduce(rp, col, val, f, [0, 1, 0], [2.0])
    assert ptr.tolist() == [0, 2, 4] and c.tolist() == [0, 1, 0, 1]
    assert v.tolist() == [4.0, 0.5, 0.5, 4.0]
    assert b.tolist() == [1.0 + 2.0, 3.0 + 2.0]
    # two fixed DOFs, labelled -1, -2 in ascending global id
    ptr, c, v, b = oracle.dirichlet_reduce(rp, col, val, f, [1, 0, 1], [3.0, -5.0])
    assert oracle.dirichlet_labels([1, 0, 1]).tolist() == [-1, 0, -2]
    assert ptr.tolist() == [0, 1] and c.tolist() == [0] and v.tolist() == [4.0]
    assert b.tolist() == [10.0 - (-1.0 * 3.0) - (-1.0 * -5.0)]


def test_dirichlet_nothing_fixed_is_identity():
    prob = inputs.small_problem((2, 2, 1), 2, 1, seed=61)
    cd, n, rp, col, val, rhs = assembled(prob)
    ptr, c, v, b = oracle.dirichlet_reduce(rp, col, val, rhs, np.zeros(n, bool), np.zeros(0))
    np.testing.assert_array_equal(ptr, rp)
    np.testing.assert_array_equal(c, col)
    np.testing.assert_array_equal(v, val)
    np.testing.assert_array_equal(b, rhs)


@pytest.mark.parametrize("p,problem", [(1, 0), (2, 1), (3, 0)])
def test_dirichlet_single_cell_brute_force(p, problem):
    """One distorted cell: the constrained system equals the cell matrix restricted to
    the free local DOFs, with K_free,fixed u^D moved to the right-hand side (taken
    directly from the oracle's cell matrix and the cell's DOF map with numpy)."""
    rng = np.random.default_rng(70 + p)
    xv = inputs.brick(1, 1, 1).coords + rng.uniform(-0.12, 0.12, size=(8, 3))
    mesh = inputs.Mesh(xv, np.arange(8, dtype=np.int32)[None, :])
    ncomp = 3 if problem == 1 else 1
    force = np.array([0.3, -0.2, 1.0]) if problem == 1 else np.array([1.5])
    prob = inputs.Problem("one", mesh, p, p + 1, problem, np.array([2.5]), force)
    cd, n, rp, col, val, rhs = assembled(prob)
    K, fe = oracle.cell_matrix(problem, p, p + 1, xv, 2.5, NU, force)
    fixed = rng.uniform(size=n) < 0.6
    fixed[0] = False
    uD = rng.standard_normal(int(fixed.sum()))
    ptr, c, v, b = oracle.dirichlet_reduce(rp, col, val, rhs, fixed, uD)
    g = np.empty(n, dtype=np.int64)
    g[cd[0]] = np.arange(n)                 # global DOF -> local index in the cell
    fr, fx = np.flatnonzero(~fixed), np.flatnonzero(fixed)
    A_ff = K[np.ix_(g[fr], g[fr])]
    b_ref = fe[g[fr]] - K[np.ix_(g[fr], g[fx])] @ uD
    A = csr_to_dense(ptr, c, v, fr.size)
    np.testing.assert_allclose(A, A_ff, rtol=0, atol=1e-14 * np.abs(K).max())
    np.testing.assert_allclose(b, b_ref, rtol=0, atol=1e-13 * (np.abs(K).max() * np.abs(uD).sum() + 1))
    assert ncomp * (p + 1) ** 3 == n


@pytest.mark.parametrize("p,shape", [(1, (3, 3, 3)), (2, (3, 2, 2)), (3, (2, 2, 2))])
def test_dirichlet_poisson_patch_reproduces_linear_data(p, shape):
    """Patch test through the constrained system: u^D = g linear on the whole boundary,
    f = 0, constant conductivity. g lies in the trial space (trilinear map, Q_p with p >= 1) and the (p+1)^3
    Gauss rule integrates a(g, v) exactly, so the free values solving Eq.
    dirichlet_bc_discrete_problem are g at the free nodes."""
    prob = inputs.small_problem(shape, p, 0, seed=80 + p)
    prob.force[:] = 0.0
    prob.coef[:] = 2.0                      # a linear field has zero flux jumps only for constant kappa
    cd, n, rp, col, val, rhs = assembled(prob)
    pos, comp = node_positions(prob, cd, n)
    fixed = boundary_dofs(pos)
    g = pos @ np.array([1.3, -0.4, 2.2]) - 0.7
    ptr, c, v, b = oracle.dirichlet_reduce(rp, col, val, rhs, fixed, g[fixed])
    u = np.linalg.solve(csr_to_dense(ptr, c, v, int((~fixed).sum())), b)
    np.testing.assert_allclose(u, g[~fixed], rtol=0, atol=1e-11 * np.abs(g).max())


@pytest.mark.parametrize("p,shape", [(1, (3, 2, 3)), (2, (2, 2, 2))])
def test_dirichlet_elasticity_patch_reproduces_linear_field(p, shape):
    """A linear displacement x -> B x + t prescribed on the boundary with zero body
    force has constant stress, so it solves the constrained elasticity system."""
    prob = inputs.small_problem(shape, p, 1, seed=90 + p)
    prob.force[:] = 0.0
    prob.coef[:] = 3.0                      # constant E: the stress is constant across cells
    cd, n, rp, col, val, rhs = assembled(prob)
    pos, comp = node_positions(prob, cd, n)
    fixed = boundary_dofs(pos)
    B = np.array([[0.2, -0.3, 0.1], [0.4, 0.05, -0.2], [-0.1, 0.3, 0.25]])
    disp = pos @ B.T + np.array([0.1, -0.2, 0.3])
    g = disp[np.arange(n), comp]
    ptr, c, v, b = oracle.dirichlet_reduce(rp, col, val, rhs, fixed, g[fixed])
    u = np.linalg.solve(csr_to_dense(ptr, c, v, int((~fixed).sum())), b)
    np.testing.assert_allclose(u, g[~fixed], rtol=0, atol=1e-10 * np.abs(g).max())


def test_dirichlet_clamped_beam_is_spd_and_homogeneous_keeps_f():
    """Clamping the x = 0 face removes the six rigid modes: the constrained matrix is
    symmetric positive definite; with u^D = 0 the right-hand side is f on the free rows."""
    prob = inputs.small_problem((4, 1, 1), 2, 1, seed=95, extent=(4.0, 1.0, 1.0))
    cd, n, rp, col, val, rhs = assembled(prob)
    pos, comp = node_positions(prob, cd, n)
    fixed = np.abs(pos[:, 0]) < 1e-12
    assert fixed.sum() == 3 * 9
    ptr, c, v, b = oracle.dirichlet_reduce(rp, col, val, rhs, fixed, np.zeros(int(fixed.sum())))
    A = csr_to_dense(ptr, c, v, int((~fixed).sum()))
    assert np.abs(A - A.T).max() < 1e-15 * np.abs(A).max()
    assert np.linalg.eigvalsh(A).min() > 0
    np.testing.assert_array_equal(b, rhs[~fixed])



# ---------------------------------------------------------------- self-adjoint compliance
def clamped_problem(p=1, shape=(4, 2, 2), seed=120):
    prob = inputs.small_problem(shape, p, 1, seed=seed, extent=(2.0, 1.0, 1.0))
    cd, n = oracle.dof_numbering(prob.mesh, p, 3)
    pos, _ = node_positions(prob, cd, n)
    return prob, cd, n, np.abs(pos[:, 0]) < 1e-12


@pytest.mark.parametrize("p", [1, 2])
def test_compliance_identities(p):
    """c(E) = f^T u(E) with K(E) u = f: c = u^T K u (energy), c(sE) = c(E)/s (K is
    linear in E), and Euler's identity for a function homogeneous of degree -1:
    sum_K E_K dc/dE_K = -c. A wrong sign or a missing term in the gradient fails."""
    prob, cd, n, fixed = clamped_problem(p)
    u, c, g = oracle.compliance_solve(prob, fixed, cd, n)
    assert c > 0 and np.all(u[fixed] == 0)
    rp, col, val, rhs = oracle.assemble_csr(prob, cd, n)
    A = csr_to_dense(rp, col, val, n)
    assert abs(u @ A @ u - c) <= 1e-10 * c
    assert abs(rhs @ u - c) <= 1e-12 * c                     # f^T u over the free DOFs (u = 0 on fixed)
    assert np.all(g < 0)                                      # stiffer cells lower the compliance
    assert abs(prob.coef @ g + c) <= 1e-10 * c
    scaled = inputs.Problem("s", prob.mesh, p, p + 1, 1, 2.5 * prob.coef, prob.force)
    _, c2, g2 = oracle.compliance_solve(scaled, fixed, cd, n)
    assert abs(c2 - c / 2.5) <= 1e-10 * c
    np.testing.assert_allclose(g2, g / 2.5 ** 2, rtol=1e-9)


def test_compliance_gradient_central_differences():
    prob, cd, n, fixed = clamped_problem(1, (3, 2, 2), seed=121)
    u, c, g = oracle.compliance_solve(prob, fixed, cd, n)
    for e in (0, 5, 11):
        h = 1e-5 * prob.coef[e]
        cp = prob.coef.copy(); cp[e] += h
        cm = prob.coef.copy(); cm[e] -= h
        c_p = oracle.compliance_solve(inputs.Problem("p", prob.mesh, 1, 2, 1, cp, prob.force), fixed, cd, n)[1]
        c_m = oracle.compliance_solve(inputs.Problem("m", prob.mesh, 1, 2, 1, cm, prob.force), fixed, cd, n)[1]
        fd = (c_p - c_m) / (2 * h)
        assert abs(fd - g[e]) <= 1e-6 * abs(g[e])


def test_compliance_of_a_bar_in_tension_closed_form():
    """An undistorted bar [0,L]x[0,1]^2 clamped at x = 0 (all components) and pulled by
    a uniform axial body force b: for nu = 0 the 3D problem is exactly the 1D bar
    -E u'' = b, u(0) = 0, u'(L) = 0, whose solution u = b (L x - x^2/2)/E is quadratic,
    hence exact in Q2; c = int b u dV = b^2 L^3 / (3 E)."""
    L, E, b = 3.0, 2.0, 0.7
    mesh = inputs.brick(3, 1, 1, L, 1.0, 1.0)
    prob = inputs.Problem("bar", mesh, 2, 3, 1, np.full(mesh.n_cells, E), np.array([b, 0.0, 0.0]), nu=0.0)
    cd, n = oracle.dof_numbering(mesh, 2, 3)
    pos, comp = node_positions(prob, cd, n)
    fixed = np.abs(pos[:, 0]) < 1e-12
    u, c, g = oracle.compliance_solve(prob, fixed, cd, n)
    exact_u = b * (L * pos[:, 0] - pos[:, 0] ** 2 / 2) / E
    np.testing.assert_allclose(u[comp == 0], exact_u[comp == 0], rtol=0, atol=1e-12)
    assert np.abs(u[comp != 0]).max() < 1e-12
    assert abs(c - b * b * L ** 3 / (3 * E)) <= 1e-12 * c



# ---------------------------------------------------------------- Stokes (Taylor-Hood)
@pytest.mark.parametrize("p", [2, 3])
def test_stokes_cell_vs_numpy_brute_force(p):
    """A distorted Taylor-Hood cell against the numpy Gram-block implementation."""
    rng = np.random.default_rng(130 + p)
    xv = UNIT * np.array([1.1, 0.8, 1.2]) + 0.15 * rng.uniform(-1, 1, (8, 3))
    K, fe = oracle.cell_matrix(2, p, p + 1, xv, 1.7, 0.0, [0.2, -0.5, 1.0])
    Kn = numpy_cell_matrix(2, p, p + 1, xv, 1.7, 0.0)
    np.testing.assert_allclose(K, Kn, rtol=0, atol=1e-13 * np.abs(Kn).max())
    nv = 3 * (p + 1) ** 3
    assert np.all(K[nv:, nv:] == 0) and np.all(fe[nv:] == 0)


def stokes_system(shape=(3, 2, 2), p=2, seed=140, mu=None):
    prob = inputs.small_problem(shape, p, inputs.STOKES, seed=seed)
    if mu is not None:
        prob.coef[:] = mu
    cd, n, nv = oracle.stokes_dof_numbering(prob.mesh, p)
    rp, col, val, rhs = oracle.assemble_csr(prob, cd, n)
    A = csr_to_dense(rp, col, val, n)
    return prob, cd, n, nv, A, rhs


def stokes_positions(prob, cd, n, nv):
    """Node position and component of every velocity DOF, position of every
    pressure DOF (independent numpy evaluation of the trilinear map)."""
    p = prob.order
    nb = (p + 1) ** 3
    vel = inputs.Problem("v", prob.mesh, p, p + 1, 1, prob.coef, prob.force)
    pos_v, comp = node_positions(vel, cd[:, :3 * nb], nv)
    pre = inputs.Problem("q", prob.mesh, p - 1, p, 0, prob.coef, prob.force)
    pos_p, _ = node_positions(pre, cd[:, 3 * nb:] - nv, n - nv)
    return pos_v, comp, pos_p


def test_stokes_assembled_invariants():
    """Symmetric (the symmetric reading), zero pressure-pressure block, the six rigid
    velocity modes in the kernel of every row, a constant pressure orthogonal to the
    interior velocity rows and summing to zero per component, and the body force on
    the velocity rows only."""
    prob, cd, n, nv, A, rhs = stokes_system()
    sc = np.abs(A).max()
    assert np.abs(A - A.T).max() <= 1e-15 * sc
    assert np.all(A[nv:, nv:] == 0)
    pos_v, comp, pos_p = stokes_positions(prob, cd, n, nv)
    for c in range(3):
        t = np.zeros(n); t[:nv][comp == c] = 1.0
        assert np.abs(A @ t).max() <= 1e-12 * sc
    for w in np.eye(3):
        r = np.zeros(n)
        disp = np.cross(w[None, :], pos_v)
        r[:nv] = disp[np.arange(nv), comp]
        assert np.abs(A @ r).max() <= 1e-12 * sc
    one_p = np.zeros(n); one_p[nv:] = 1.0
    bt = (A @ one_p)[:nv]
    interior = ~boundary_dofs(pos_v)
    assert np.abs(bt[interior]).max() <= 1e-12 * sc
    for c in range(3):
        assert abs(bt[comp == c].sum()) <= 1e-12 * sc
    vol = 1.0
    f = prob.force
    for c in range(3):
        assert abs(rhs[:nv][comp == c].sum() - f[c] * vol) <= 1e-13
    assert np.all(rhs[nv:] == 0)


@pytest.mark.parametrize("p", [2, 3])
def test_stokes_invariants_on_an_o_grid(p):
    """On an O-grid: symmetry, the zero pressure block, the six rigid velocity
    modes in the kernel, a constant pressure orthogonal to the interior velocity
    rows (the divergence of an interior velocity basis function integrates to
    zero) and the body force summing to f vol on the velocity rows."""
    prob = inputs.o_grid_problem(3, 2, 2, p, inputs.STOKES, seed=60 + p)
    cd, n, nv = oracle.stokes_dof_numbering(prob.mesh, p)
    rp, col, val, rhs = oracle.assemble_csr(prob, cd, n)
    A = csr_to_dense(rp, col, val, n)
    sc = np.abs(A).max()
    assert np.abs(A - A.T).max() <= 1e-15 * sc
    assert np.all(A[nv:, nv:] == 0)
    pos_v, comp, _ = stokes_positions(prob, cd, n, nv)
    for c in range(3):
        t = np.zeros(n)
        t[:nv][comp == c] = 1.0
        assert np.abs(A @ t).max() <= 1e-12 * sc
    for w in np.eye(3):
        r = np.zeros(n)
        r[:nv] = np.cross(w[None, :], pos_v)[np.arange(nv), comp]
        assert np.abs(A @ r).max() <= 1e-12 * sc
    one_p = np.zeros(n)
    one_p[nv:] = 1.0
    bt = (A @ one_p)[:nv]
    ring = _o_grid_ring(prob.mesh)
    inner = ~_o_grid_boundary(pos_v, ring, prob.mesh.extent[2])
    assert np.abs(bt[inner]).max() <= 1e-12 * sc
    area = 0.5 * abs(np.sum(ring[:, 0] * np.roll(ring[:, 1], -1) - np.roll(ring[:, 0], -1) * ring[:, 1]))
    vol = area * prob.mesh.extent[2]
    for c in range(3):
        assert abs(rhs[:nv][comp == c].sum() - prob.force[c] * vol) <= 1e-13
    assert np.all(rhs[nv:] == 0)


def test_stokes_linear_velocity_closed_forms():
    """u = Bx + t, zero pressure, constant viscosity mu: the pressure rows give
    -tr(B) int psi_c, summing to -tr(B) vol; the interior velocity rows vanish
    (constant strain); u^T A u = mu |sym B|^2 vol."""
    mu = 1.3
    prob, cd, n, nv, A, rhs = stokes_system(mu=mu, seed=141)
    pos_v, comp, pos_p = stokes_positions(prob, cd, n, nv)
    Bm = np.array([[0.3, -0.2, 0.1], [0.4, -0.5, 0.2], [-0.1, 0.25, 0.6]])
    disp = pos_v @ Bm.T + np.array([0.1, 0.2, -0.3])
    u = np.zeros(n)
    u[:nv] = disp[np.arange(nv), comp]
    r = A @ u
    vol = 1.0
    assert abs(r[nv:].sum() + np.trace(Bm) * vol) <= 1e-12
    assert np.abs(r[:nv][~boundary_dofs(pos_v)]).max() <= 1e-11 * np.abs(A).max()
    sym = 0.5 * (Bm + Bm.T)
    assert abs(u @ r - mu * np.sum(sym * sym) * vol) <= 1e-12 * mu * np.sum(sym * sym)


# ---------------------------------------------------------------- interior penalty DG
def dg_node_positions(mesh, p):
    """Position of every DG DOF (K, a): Phi_K(alpha_a / p), K-major."""
    n1 = p + 1
    al = np.array([[a % n1, (a // n1) % n1, a // (n1 * n1)] for a in range(n1 ** 3)]) / p
    N = np.ones((n1 ** 3, 8))
    for v in range(8):
        for d in range(3):
            N[:, v] *= al[:, d] if (v >> d) & 1 else 1 - al[:, d]
    return np.einsum("av,evk->eak", N, mesh.coords[mesh.cell_vertices]).reshape(-1, 3)


def proper_rotations():
    """The 24 rotations of the unit cube as (axis permutation, flips) with det +1."""
    out = []
    for perm in itertools.permutations(range(3)):
        for flips in itertools.product((0, 1), repeat=3):
            M = np.zeros((3, 3))
            for i in range(3):
                M[i, perm[i]] = -1.0 if flips[i] else 1.0
            if np.linalg.det(M) > 0:
                out.append((perm, flips))
    return out


def rotated_mesh(mesh, seed):
    """The same cells with each local vertex order turned by a random proper rotation."""
    rng = np.random.default_rng(seed)
    rots = proper_rotations()
    cv = mesh.cell_vertices.copy()
    for e in range(mesh.n_cells):
        perm, flips = rots[rng.integers(len(rots))]
        new = np.empty(8, dtype=np.int32)
        for w in range(8):
            r = [(w >> i) & 1 for i in range(3)]
            rr = [1 - r[perm[i]] if flips[i] else r[perm[i]] for i in range(3)]
            new[w] = mesh.cell_vertices[e][rr[0] + 2 * rr[1] + 4 * rr[2]]
        cv[e] = new
    return inputs.Mesh(mesh.coords, cv, mesh.shape, mesh.extent)


@pytest.mark.parametrize("p,shape,rotate", [(1, (3, 2, 2), False), (2, (2, 2, 2), False), (3, (2, 1, 2), False),
                                            (2, (2, 2, 2), True), (1, (3, 3, 2), True)])
@pytest.mark.parametrize("tau", [1.0, -1.0, 0.0])
def test_dg_consistency_with_linear_solution(p, shape, rotate, tau):
    """u = g linear solves -Lap u = 0 with u = g on the boundary; IP-DG is consistent
    and its cell, facet and boundary integrals are exact for g on trilinear cells,
    so A u_g equals the right-hand side with f = 0 and u_D = g, to rounding. A wrong
    sign, normal, mean or jump factor, or a mismatched neighbour point fails."""
    mesh = inputs.small_problem(shape, p, 0, seed=150 + p).mesh
    if rotate:
        mesh = rotated_mesh(mesh, 160 + p)
    ud = np.array([0.4, 1.3, -0.7, 2.1])
    rp, col, val, rhs = oracle.dg_assemble(mesh, p, tau, 7.0, 0.0, ud)
    x = dg_node_positions(mesh, p)
    u = ud[0] + x @ ud[1:]
    r = csr_matvec(rp, col, val, u)
    assert np.abs(r - rhs).max() <= 1e-11 * np.abs(rhs).max()


@pytest.mark.parametrize("p", [1, 2, 3])
@pytest.mark.parametrize("tau", [1.0, -1.0])
def test_dg_consistency_on_an_o_grid(p, tau):
    """The same consistency on an O-grid: facets between cells of irregular
    valence and a polygonal outer boundary."""
    mesh = inputs.o_grid(3, 2, 2)
    ud = np.array([-0.3, 0.8, 1.7, -0.6])
    rp, col, val, rhs = oracle.dg_assemble(mesh, p, tau, 7.0, 0.0, ud)
    u = ud[0] + dg_node_positions(mesh, p) @ ud[1:]
    assert np.abs(csr_matvec(rp, col, val, u) - rhs).max() <= 1e-11 * np.abs(rhs).max()


def csr_matvec(rp, col, val, v):
    rows = np.repeat(np.arange(rp.size - 1), np.diff(rp))
    out = np.zeros(rp.size - 1)
    np.add.at(out, rows, val * v[col])
    return out


@pytest.mark.parametrize("h", [0.5, 2.0])
def test_dg_penalty_closed_form_q1_cube(h):
    """The penalty part of the IP-DG matrix on one axis-aligned Q1 cube of side h
    (every face a boundary facet): per face gamma/|F| times the Q1 face mass
    matrix |F| (4, 2, 2, 1)/36 (same vertex, edge neighbours, diagonal), so per
    unit gamma the sum over the six faces is 1/3, 1/9, 1/36, 0 by the Hamming
    distance of the two vertices, whatever h (Eq. ip_dg_formulations)."""
    bits = np.array([[v & 1, (v >> 1) & 1, (v >> 2) & 1] for v in range(8)], dtype=np.float64)
    mesh = inputs.Mesh(h * bits, np.arange(8, dtype=np.int32).reshape(1, 8), (1, 1, 1), (h, h, h))
    A = {}
    for gamma in (1.0, 3.0):
        rp, col, val, _ = oracle.dg_assemble(mesh, 1, 1.0, gamma)
        A[gamma] = csr_to_dense(rp, col, val, 8)
    P = (A[3.0] - A[1.0]) / 2.0
    expect = np.array([[(1 / 3, 1 / 9, 1 / 36, 0.0)[bin(a ^ b).count("1")] for b in range(8)] for a in range(8)])
    np.testing.assert_allclose(P, expect, rtol=0, atol=1e-14)


def test_dg_symmetry_linearity_and_coercivity():
    """SIPG (tau = 1) is symmetric and, with a large enough penalty, positive
    definite; the matrix is affine in tau and in gamma; the pattern couples each
    cell with itself and its face neighbours."""
    mesh = inputs.small_problem((3, 2, 2), 2, 0, seed=170).mesh
    n = mesh.n_cells * 27
    A = {}
    for tau, gamma in ((1.0, 10.0), (0.0, 10.0), (-1.0, 10.0), (1.0, 30.0)):
        rp, col, val, _ = oracle.dg_assemble(mesh, 2, tau, gamma)
        A[tau, gamma] = csr_to_dense(rp, col, val, n)
    S = A[1.0, 10.0]
    sc = np.abs(S).max()
    assert np.abs(S - S.T).max() <= 1e-14 * sc
    assert np.abs(A[1.0, 10.0] + A[-1.0, 10.0] - 2 * A[0.0, 10.0]).max() <= 1e-14 * sc
    P = (A[1.0, 30.0] - A[1.0, 10.0]) / 20.0                   # the penalty matrix per unit gamma
    assert np.abs(P - P.T).max() <= 1e-14 * sc and np.linalg.eigvalsh(P).min() > -1e-12 * sc
    assert np.linalg.eigvalsh(A[1.0, 30.0]).min() > 0
    interior = (2 * 2 * 2) + (3 * 1 * 2) + (3 * 2 * 1)
    assert rp[-1] == 27 * 27 * (mesh.n_cells + 2 * interior)


# ---------------------------------------------------------------- smallest det J (mesh validity)
def _single_cell(corners):
    """One hexahedron from its 8 vertices in x-fastest local order."""
    return inputs.Mesh(np.asarray(corners, dtype=np.float64), np.arange(8, dtype=np.int32)[None, :])


def _unit_corners():
    return np.array([[v & 1, (v >> 1) & 1, (v >> 2) & 1] for v in range(8)], dtype=np.float64)


def test_min_det_brick_cells():
    """Axis-aligned brick cells of sides (hx, hy, hz): J = diag(hx, hy, hz) at every
    point and vertex, so det J = hx hy hz; over several cells the smallest product."""
    m = inputs.brick(3, 2, 2, 0.6, 0.5, 2.0)                 # cells 0.2 x 0.25 x 1.0
    for nq1d in (1, 2, 3, 4):
        assert abs(oracle.min_det_jacobian(m, nq1d) - 0.2 * 0.25 * 1.0) <= 1e-15
    sizes = [(0.5, 2.0, 1.5), (0.3, 0.7, 0.2), (1.0, 1.0, 0.9)]
    xs, cvs = [], []
    for i, h in enumerate(sizes):
        xs.append(_unit_corners() * np.array(h) + np.array([5.0 * i, -1.0, 2.0]))
        cvs.append(np.arange(8, dtype=np.int32) + 8 * i)
    m2 = inputs.Mesh(np.concatenate(xs), np.stack(cvs).astype(np.int32))
    assert abs(oracle.min_det_jacobian(m2, 2) - 0.3 * 0.7 * 0.2) <= 1e-15


def test_min_det_affine_cell():
    """An affine cell x = A xhat + b has J = A everywhere: det J = det A exactly."""
    A = np.array([[0.9, 0.2, -0.1], [0.15, 1.1, 0.3], [-0.2, 0.1, 0.8]])
    detA = (A[0, 0] * (A[1, 1] * A[2, 2] - A[1, 2] * A[2, 1]) - A[0, 1] * (A[1, 0] * A[2, 2] - A[1, 2] * A[2, 0])
            + A[0, 2] * (A[1, 0] * A[2, 1] - A[1, 1] * A[2, 0]))
    m = _single_cell(_unit_corners() @ A.T + np.array([0.3, -0.7, 1.1]))
    for nq1d in (2, 3):
        assert abs(oracle.min_det_jacobian(m, nq1d) - detA) <= 1e-14 * abs(detA)


def test_min_det_inverted_cell_is_negative():
    """Mirroring a brick along x while keeping the local vertex order inverts the
    map: det J = -hx hy hz < 0 everywhere."""
    m = _single_cell(_unit_corners() * np.array([-0.5, 0.4, 0.25]))
    assert abs(oracle.min_det_jacobian(m, 2) + 0.5 * 0.4 * 0.25) <= 1e-15


def test_min_det_reached_at_a_vertex():
    """Unit cube with vertex 7 moved to (t, t, t): at that vertex the Jacobian columns
    are x7 - x6, x7 - x5, x7 - x3, i.e. I + (t - 1) 11^T, whose determinant is 3t - 2
    (eigenvalues 1, 1, 3t - 2); every other vertex and every Gauss point has a larger
    det J, so the minimum over the sampled points is 3t - 2 only if the vertices are
    sampled as well as the quadrature points."""
    t = 0.9
    x = _unit_corners()
    x[7] = [t, t, t]
    m = _single_cell(x)
    for nq1d in (2, 3, 4):
        assert abs(oracle.min_det_jacobian(m, nq1d) - (3 * t - 2)) <= 1e-14

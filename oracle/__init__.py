"""FP64 CPU oracle for cell integration and global assembly (test infrastructure).

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package. The CUDA product path never calls it, and
the two share no code: the oracle is the plain C file ``fe_oracle.c`` compiled
with gcc and reached through ctypes.

Each wrapper names the passage of the FEMPAR paper it follows (see the header of
``fe_oracle.c``). The strong Dirichlet split (``dirichlet_labels``,
``dirichlet_reduce``) is plain numpy on top of the assembled matrix.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fe_oracle.c")
# ORACLE_LIB: load a library the caller built from this source (the tests that
# plant mistakes in a copy of the oracle use it); otherwise liboracle.so here.
_LIB = os.environ.get("ORACLE_LIB") or os.path.join(_HERE, "liboracle.so")
_lib = None

_i32p = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")
_i64p = np.ctypeslib.ndpointer(dtype=np.int64, flags="C_CONTIGUOUS")
_f64p = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")


def build(force: bool = False) -> str:
    """Compile fe_oracle.c into liboracle.so next to it (gcc, plain -O2)."""
    if os.environ.get("ORACLE_LIB"):
        return _LIB
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-D_DEFAULT_SOURCE", "-fPIC", "-shared",
                               _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        L.or_gauss_legendre.argtypes = [ctypes.c_int, _f64p, _f64p]
        L.or_gauss_legendre.restype = ctypes.c_int
        L.or_lagrange_1d.argtypes = [ctypes.c_int, ctypes.c_double, _f64p, _f64p]
        L.or_lagrange_1d.restype = None
        L.or_cell_matrix.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, _f64p, ctypes.c_double,
                                     ctypes.c_double, _f64p, _f64p, _f64p]
        L.or_cell_matrix.restype = ctypes.c_int
        L.or_min_det_jacobian.argtypes = [ctypes.c_int, ctypes.c_int64, _i32p, _f64p]
        L.or_min_det_jacobian.restype = ctypes.c_double
        L.or_dof_numbering.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int64, _i32p, _i32p]
        L.or_dof_numbering.restype = ctypes.c_int64
        vp = ctypes.c_void_p
        L.or_assemble_csr.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int64, _i32p, _f64p,
                                      _i32p, ctypes.c_int64, _f64p, ctypes.c_double, _f64p, vp, vp, vp, vp]
        L.or_assemble_csr.restype = ctypes.c_int64
        L.or_assemble_rows.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int64, _i32p, _f64p,
                                       _i32p, ctypes.c_int64, _f64p, ctypes.c_double, _f64p, ctypes.c_int64,
                                       _i64p, ctypes.c_int64, _i64p, _i32p, _f64p, _f64p]
        L.or_assemble_rows.restype = ctypes.c_int64
        L.or_cell_energies.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int64, _i32p, _f64p,
                                       _i32p, ctypes.c_double, _f64p, _f64p]
        L.or_cell_energies.restype = ctypes.c_int
        L.or_dg_assemble.argtypes = [ctypes.c_int, ctypes.c_int64, _i32p, _f64p, ctypes.c_double, ctypes.c_double,
                                     ctypes.c_double, _f64p, vp, vp, vp, vp]
        L.or_dg_assemble.restype = ctypes.c_int64
        _lib = L
    return _lib


def _c(a, dt):
    return np.ascontiguousarray(a, dtype=dt)


def gauss_legendre(n: int):
    """n-point Gauss-Legendre rule on [0,1] (Sect. Numerical integration)."""
    x = np.zeros(n)
    w = np.zeros(n)
    rc = lib().or_gauss_legendre(n, x, w)
    if rc:
        raise ValueError(f"or_gauss_legendre({n}) -> {rc}")
    return x, w


def lagrange_1d(p: int, x: float):
    """Values and derivatives of the p+1 equidistant Lagrange polynomials (Eq. lagbas)."""
    v = np.zeros(p + 1)
    d = np.zeros(p + 1)
    lib().or_lagrange_1d(p, float(x), v, d)
    return v, d


def _n_local(problem: int, p: int) -> int:
    if problem == 2:                        # Taylor-Hood: 3 (p+1)^3 velocity + p^3 pressure
        return 3 * (p + 1) ** 3 + p ** 3
    return (3 if problem == 1 else 1) * (p + 1) ** 3


def cell_matrix(problem: int, p: int, nq1d: int, xv, coef: float, nu: float, force):
    """Cell matrix and vector of one hexahedron given its 8 vertices [8,3]."""
    nl = _n_local(problem, p)
    Ke = np.zeros(nl * nl)
    fe = np.zeros(nl)
    f = _c(np.resize(np.asarray(force, dtype=np.float64), 3), np.float64)
    rc = lib().or_cell_matrix(problem, p, nq1d, _c(xv, np.float64).ravel(), float(coef), float(nu), f, Ke, fe)
    if rc:
        raise ValueError(f"or_cell_matrix -> {rc}")
    return Ke.reshape(nl, nl), fe


def min_det_jacobian(mesh, nq1d: int) -> float:
    return float(lib().or_min_det_jacobian(nq1d, mesh.n_cells, _c(mesh.cell_vertices, np.int32),
                                           _c(mesh.coords, np.float64).ravel()))


def dof_numbering(mesh, p: int, ncomp: int):
    """Global DOF numbering by the list_dofs algorithm; returns (cell_dofs, n_dofs)."""
    nl = ncomp * (p + 1) ** 3
    cd = np.zeros((mesh.n_cells, nl), dtype=np.int32)
    n = lib().or_dof_numbering(p, ncomp, mesh.n_cells, _c(mesh.cell_vertices, np.int32), cd.reshape(-1))
    if n < 0:
        raise ValueError(f"or_dof_numbering -> {n}")
    return cd, int(n)


def stokes_dof_numbering(mesh, p: int):
    """Taylor-Hood Q_p/Q_{p-1} space: the velocity field numbered by list_dofs,
    then the pressure field by list_dofs, offset by the number of velocity DOFs
    (the block layout of Sect. "The FE affine operator abstraction" with the
    velocity block first). Returns (cell_dofs [cells][3 (p+1)^3 + p^3], n_dofs,
    n_velocity)."""
    cd_v, nv = dof_numbering(mesh, p, 3)
    cd_p, npr = dof_numbering(mesh, p - 1, 1)
    return np.hstack([cd_v, cd_p + nv]).astype(np.int32), nv + npr, nv


def numbering(prob):
    """(cell_dofs, n_dofs) of a workload's space."""
    if prob.problem == 2:
        cd, n, _ = stokes_dof_numbering(prob.mesh, prob.order)
        return cd, n
    return dof_numbering(prob.mesh, prob.order, prob.ncomp)


def _force3(force):
    return _c(np.resize(np.asarray(force, dtype=np.float64), 3), np.float64)


def assemble_csr(prob, cell_dofs=None, n_dofs=None):
    """Full CSR matrix + RHS by COO push-back and compress (Eq. assembly)."""
    L = lib()
    mesh = prob.mesh
    if cell_dofs is None:
        cell_dofs, n_dofs = numbering(prob)
    cv = _c(mesh.cell_vertices, np.int32)
    xyz = _c(mesh.coords, np.float64).ravel()
    cd = _c(cell_dofs, np.int32).reshape(-1)
    coef = _c(prob.coef, np.float64)
    f = _force3(prob.force)
    nnz = L.or_assemble_csr(prob.problem, prob.order, prob.quad_1d, mesh.n_cells, cv, xyz, cd, n_dofs,
                            coef, prob.nu, f, None, None, None, None)
    if nnz < 0:
        raise ValueError(f"or_assemble_csr -> {nnz}")
    row_ptr = np.zeros(n_dofs + 1, dtype=np.int64)
    col = np.zeros(nnz, dtype=np.int32)
    val = np.zeros(nnz, dtype=np.float64)
    rhs = np.zeros(n_dofs, dtype=np.float64)
    nnz2 = L.or_assemble_csr(prob.problem, prob.order, prob.quad_1d, mesh.n_cells, cv, xyz, cd, n_dofs,
                             coef, prob.nu, f, row_ptr.ctypes.data, col.ctypes.data, val.ctypes.data,
                             rhs.ctypes.data)
    assert nnz2 == nnz
    return row_ptr, col, val, rhs


def assemble_rows(prob, rows, cell_dofs, n_dofs):
    """Selected rows of the assembled matrix and RHS: (ptr, col, val, rhs)."""
    L = lib()
    mesh = prob.mesh
    rows = _c(rows, np.int64)
    nl = _n_local(prob.problem, prob.order)
    cap = int(rows.size) * 8 * nl
    ptr = np.zeros(rows.size + 1, dtype=np.int64)
    col = np.zeros(cap, dtype=np.int32)
    val = np.zeros(cap, dtype=np.float64)
    rhs = np.zeros(rows.size, dtype=np.float64)
    tot = L.or_assemble_rows(prob.problem, prob.order, prob.quad_1d, mesh.n_cells,
                             _c(mesh.cell_vertices, np.int32), _c(mesh.coords, np.float64).ravel(),
                             _c(cell_dofs, np.int32).reshape(-1), n_dofs, _c(prob.coef, np.float64),
                             prob.nu, _force3(prob.force), rows.size, rows, cap, ptr, col, val, rhs)
    if tot < 0:
        raise ValueError(f"or_assemble_rows -> {tot}")
    assert tot <= cap
    return ptr, col[:tot], val[:tot], rhs


def cell_energies(prob, u, cell_dofs):
    """g_K = u_K^T (A^K / coef_K) u_K for every cell (compliance sensitivity)."""
    mesh = prob.mesh
    g = np.zeros(mesh.n_cells)
    rc = lib().or_cell_energies(prob.problem, prob.order, prob.quad_1d, mesh.n_cells,
                                _c(mesh.cell_vertices, np.int32), _c(mesh.coords, np.float64).ravel(),
                                _c(cell_dofs, np.int32).reshape(-1), prob.nu, _c(u, np.float64), g)
    if rc:
        raise ValueError(f"or_cell_energies -> {rc}")
    return g


# ----------------------------------------------------------------------------- strong Dirichlet conditions
def dirichlet_labels(fixed):
    """Free/fixed split of the DOFs (Sect. "Strong imposition of boundary
    conditions"): free DOFs get the ids 0, 1, ... and fixed DOFs -1, -2, ...,
    each set in ascending global id (the paper labels them 1..n_free and
    -1..-n_fixed). Returns int64 labels [n_dofs]."""
    fixed = np.asarray(fixed).astype(bool)
    lab = np.empty(fixed.size, dtype=np.int64)
    lab[~fixed] = np.arange(int((~fixed).sum()))
    lab[fixed] = -1 - np.arange(int(fixed.sum()))
    return lab


def dirichlet_reduce(row_ptr, col, val, rhs, fixed, u_fixed, rows=None):
    """The constrained system of Eq. dirichlet_bc_discrete_problem, from the
    assembled matrix A and vector f of the whole space:
        sum_{b free} A_ab u_b = f_a - sum_{c fixed} A_ac u^D_c   for every free a.
    Rows and columns of fixed DOFs are dropped; the remaining ones are renumbered
    by ``dirichlet_labels``; each fixed column moves to the right-hand side times
    its prescribed value u_fixed[fixed id].

    (row_ptr, col, val, rhs) hold the rows ``rows`` of A and f (default: every
    row, in order); those rows must all be free. Returns the constrained rows as
    (row_ptr, col, val, rhs), columns ascending."""
    lab = dirichlet_labels(fixed)
    row_ptr = np.asarray(row_ptr, dtype=np.int64)
    col = np.asarray(col, dtype=np.int64)
    val = np.asarray(val, dtype=np.float64)
    n_rows = row_ptr.size - 1
    if rows is None:                       # the whole matrix: drop the fixed rows
        if n_rows != lab.size:
            raise ValueError("dirichlet_reduce: matrix and mask sizes differ")
        keep_rows = lab >= 0
    else:                                  # a block of free rows: keep them all
        rows = np.asarray(rows, dtype=np.int64)
        if rows.size != n_rows or (rows.size and lab[rows].min() < 0):
            raise ValueError("dirichlet_reduce: the block's rows must be free DOFs")
        keep_rows = np.ones(n_rows, dtype=bool)
    u_fixed = np.asarray(u_fixed, dtype=np.float64)
    row_of = np.repeat(np.arange(n_rows), np.diff(row_ptr))
    free_col = lab[col] >= 0
    # matrix: the free x free block, renumbered
    kept = free_col & keep_rows[row_of]
    out_ptr = np.zeros(int(keep_rows.sum()) + 1, dtype=np.int64)
    new_row = np.cumsum(keep_rows) - 1
    np.add.at(out_ptr, new_row[row_of[kept]] + 1, 1)
    out_ptr = np.cumsum(out_ptr)
    out_col = lab[col[kept]]
    out_val = val[kept]
    # right-hand side: f_a minus the fixed columns times the prescribed values
    lift = np.zeros(n_rows)
    fx = ~free_col
    np.add.at(lift, row_of[fx], val[fx] * u_fixed[-1 - lab[col[fx]]])
    out_rhs = (np.asarray(rhs, dtype=np.float64) - lift)[keep_rows]
    return out_ptr, out_col.astype(np.int32), out_val, out_rhs


# ----------------------------------------------------------------------------- self-adjoint compliance
def compliance_solve(prob, fixed, cell_dofs=None, n_dofs=None):
    """Compliance of the structure under its body force with the DOFs of `fixed`
    clamped (u^D = 0): K(E) u = f on the free DOFs (Eq. dirichlet_bc_discrete_problem),
    c = f^T u, and its gradient dc/dE_K = -u_K^T (A^K / E_K) u_K (c is self-adjoint:
    dc/dE = f^T du/dE = -u^T (dK/dE) u, and K is linear in the cell coefficients,
    Eq. assembly). The free system is solved directly (scipy's sparse LU) in FP64.
    Returns (u over all DOFs with zeros at the fixed ones, c, dc/dE)."""
    import scipy.sparse
    import scipy.sparse.linalg
    if cell_dofs is None:
        cell_dofs, n_dofs = dof_numbering(prob.mesh, prob.order, prob.ncomp)
    fixed = np.asarray(fixed).astype(bool)
    rp, col, val, rhs = assemble_csr(prob, cell_dofs, n_dofs)
    ptr, c_r, v_r, b_r = dirichlet_reduce(rp, col, val, rhs, fixed, np.zeros(int(fixed.sum())))
    n_free = ptr.size - 1
    K = scipy.sparse.csr_matrix((v_r, c_r, ptr), shape=(n_free, n_free))
    u_free = scipy.sparse.linalg.spsolve(K.tocsc(), b_r)
    u = np.zeros(n_dofs)
    u[~fixed] = u_free
    c = float(b_r @ u_free)
    grad = -cell_energies(prob, u, cell_dofs)
    return u, c, grad


# ----------------------------------------------------------------------------- interior penalty DG
def dg_assemble(mesh, p: int, tau: float, gamma: float, f: float = 0.0, ud=(0.0, 0.0, 0.0, 0.0)):
    """IP-DG Poisson system of Eq. ip_dg_formulations on a hexahedral mesh
    (cell-local DOFs K*(p+1)^3 + a): CSR (row_ptr, col, val) and the right-hand
    side with the source f and the weak Dirichlet data u_D(x) = ud[0] + ud[1:] . x."""
    L = lib()
    cv = _c(mesh.cell_vertices, np.int32)
    xyz = _c(mesh.coords, np.float64).ravel()
    u = _c(ud, np.float64)
    nnz = L.or_dg_assemble(p, mesh.n_cells, cv, xyz, float(tau), float(gamma), float(f), u, None, None, None, None)
    if nnz < 0:
        raise ValueError(f"or_dg_assemble -> {nnz}")
    n = mesh.n_cells * (p + 1) ** 3
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    col = np.zeros(nnz, dtype=np.int32)
    val = np.zeros(nnz)
    rhs = np.zeros(n)
    nnz2 = L.or_dg_assemble(p, mesh.n_cells, cv, xyz, float(tau), float(gamma), float(f), u,
                            row_ptr.ctypes.data, col.ctypes.data, val.ctypes.data, rhs.ctypes.data)
    assert nnz2 == nnz
    return row_ptr, col, val, rhs

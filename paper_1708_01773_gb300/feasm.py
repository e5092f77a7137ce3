"""Thin ctypes binding of libfeasm.so (the C ABI declared in include/feasm.h).

Argument marshalling only: every step of integration and assembly runs in the
library's CUDA kernels. Device buffers are torch tensors (their data_ptr() is
passed through); the library never falls back to the CPU, and loading fails
loudly when the shared library has not been built.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libfeasm.so")

FE_POISSON, FE_ELASTICITY, FE_STOKES = 0, 1, 2
FE_PREC_FP64, FE_PREC_FP32, FE_PREC_BF16 = 0, 1, 2
PRECISIONS = {"fp64": FE_PREC_FP64, "fp32": FE_PREC_FP32, "bf16": FE_PREC_BF16}

ERRORS = {
    -1: "FE_ERR_INVALID_ARG", -2: "FE_ERR_CUDA", -3: "FE_ERR_OOM", -4: "FE_ERR_NEG_JACOBIAN",
    -5: "FE_ERR_TIMEOUT", -6: "FE_ERR_UNSUPPORTED", -7: "FE_ERR_NOT_CONVERGED",
}

# every entry point declared in include/feasm.h
EXPORTS = [
    "fe_space_create", "fe_space_create_host", "fe_space_sizes", "fe_space_cell_dofs_host",
    "fe_space_csr_pattern_host", "fe_space_permutation_host", "fe_space_csr_pattern", "fe_assemble", "fe_assemble_ex", "fe_assemble_host",
    "fe_assemble_adjoint", "fe_assemble_adjoint_noalloc", "fe_space_set_kernel", "fe_status", "fe_space_destroy", "fe_last_error", "fe_batch_create",
    "fe_batch_assemble", "fe_batch_set_wait", "fe_batch_destroy", "fe_selftest_conversions", "fe_space_dof_points_host", "fe_mesh_locality_order", "fe_dirichlet_create", "fe_dirichlet_sizes",
    "fe_dirichlet_labels_host", "fe_dirichlet_csr_pattern_host", "fe_dirichlet_csr_pattern",
    "fe_dirichlet_permutation_host", "fe_dirichlet_lift_host", "fe_assemble_dirichlet", "fe_dirichlet_destroy",
    "fe_compliance_work_size", "fe_compliance", "fe_space_block_offset", "fe_dg_create", "fe_dg_create_host",
    "fe_dg_sizes", "fe_dg_csr_pattern_host", "fe_dg_csr_pattern", "fe_dg_facets_host", "fe_dg_assemble",
    "fe_dg_destroy",
]
_VOID = ("fe_space_destroy", "fe_last_error", "fe_batch_destroy", "fe_dirichlet_destroy", "fe_dg_destroy")


class FEError(RuntimeError):
    def __init__(self, code: int, fn: str, msg: str):
        super().__init__(f"{fn} failed: {ERRORS.get(code, code)}: {msg}")
        self.code = code


class MeshDesc(ctypes.Structure):
    _fields_ = [("n_vertices", ctypes.c_int64), ("coords", ctypes.c_void_p),
                ("n_cells", ctypes.c_int64), ("cell_vertices", ctypes.c_void_p)]


_lib = None


def lib() -> ctypes.CDLL:
    """Loads libfeasm.so (raises if it is missing: there is no fallback)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_1708_01773_gb300/build.py")
        L = ctypes.CDLL(LIB_PATH)
        P, I, I64, D, V = ctypes.POINTER, ctypes.c_int, ctypes.c_int64, ctypes.c_double, ctypes.c_void_p
        L.fe_space_create.argtypes = [P(MeshDesc), I, I, I, D, P(V)]
        L.fe_space_create_host.argtypes = [P(MeshDesc), I, I, I, D, P(V)]
        L.fe_space_sizes.argtypes = [V, P(I64), P(I64), P(I64), P(I64)]
        L.fe_space_cell_dofs_host.argtypes = [V, V]
        L.fe_space_csr_pattern_host.argtypes = [V, V, V]
        L.fe_space_csr_pattern.argtypes = [V, V, V, V]
        L.fe_space_permutation_host.argtypes = [V, V, V, V, V, V]
        L.fe_assemble.argtypes = [V, V, V, V, V, I, V]
        L.fe_assemble_host.argtypes = [V, V, V, V, V, I, V]
        L.fe_assemble_ex.argtypes = [V, V, V, V, V, I, V, V]
        L.fe_assemble_adjoint.argtypes = [V, V, V, D, V, V, I, V]
        L.fe_assemble_adjoint_noalloc.argtypes = [V, V, V, D, V, V, I, V]
        L.fe_status.argtypes = [V, V]
        L.fe_space_set_kernel.argtypes = [V, I]
        L.fe_space_destroy.argtypes = [V]
        L.fe_space_destroy.restype = None
        L.fe_last_error.argtypes = []
        L.fe_last_error.restype = ctypes.c_char_p
        L.fe_batch_create.argtypes = [V, I, I, P(V)]
        L.fe_batch_assemble.argtypes = [V, V, V, V, V, I, V]
        L.fe_batch_set_wait.argtypes = [V, ctypes.c_longlong, I]
        L.fe_selftest_conversions.argtypes = [V, I64, V, V, V]
        L.fe_batch_destroy.argtypes = [V]
        L.fe_batch_destroy.restype = None
        L.fe_space_dof_points_host.argtypes = [V, P(MeshDesc), V]
        L.fe_mesh_locality_order.argtypes = [P(MeshDesc), V]
        L.fe_dirichlet_create.argtypes = [V, V, P(V)]
        L.fe_dirichlet_sizes.argtypes = [V, P(I64), P(I64), P(I64)]
        L.fe_dirichlet_labels_host.argtypes = [V, V]
        L.fe_dirichlet_csr_pattern_host.argtypes = [V, V, V]
        L.fe_dirichlet_csr_pattern.argtypes = [V, V, V, V]
        L.fe_dirichlet_permutation_host.argtypes = [V, V, V, V, V, V, V, V]
        L.fe_dirichlet_lift_host.argtypes = [V, P(I64), P(I64), V, V, V, V]
        L.fe_assemble_dirichlet.argtypes = [V, V, V, V, V, V, I, V]
        L.fe_compliance_work_size.argtypes = [V, P(I64)]
        L.fe_space_block_offset.argtypes = [V, P(I64)]
        L.fe_dg_create.argtypes = [P(MeshDesc), I, P(V)]
        L.fe_dg_create_host.argtypes = [P(MeshDesc), I, P(V)]
        L.fe_dg_sizes.argtypes = [V, P(I64), P(I64), P(I64), P(I64)]
        L.fe_dg_csr_pattern_host.argtypes = [V, V, V]
        L.fe_dg_csr_pattern.argtypes = [V, V, V, V]
        L.fe_dg_facets_host.argtypes = [V, V, V, V, V, V, V]
        L.fe_dg_assemble.argtypes = [V, D, D, D, V, V, I, V]
        L.fe_dg_destroy.argtypes = [V]
        L.fe_dg_destroy.restype = None
        L.fe_compliance.argtypes = [V, V, V, I, D, I, V, V, V, V, P(I), P(D), V]
        L.fe_dirichlet_destroy.argtypes = [V]
        L.fe_dirichlet_destroy.restype = None
        for n in EXPORTS:
            if n not in _VOID:
                getattr(L, n).restype = ctypes.c_int
        _lib = L
    return _lib


def _check(rc: int, fn: str):
    if rc != 0:
        raise FEError(rc, fn, lib().fe_last_error().decode())


def _ptr(t) -> int:
    if t is None:
        return 0
    if hasattr(t, "data_ptr"):
        return int(t.data_ptr())
    return int(t.ctypes.data)


def _stream(stream) -> int:
    if stream is None:
        import torch
        return int(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return stream
    return int(stream.cuda_stream)


def _mesh_desc(coords: np.ndarray, cell_vertices: np.ndarray):
    coords = np.ascontiguousarray(coords, dtype=np.float64)
    cv = np.ascontiguousarray(cell_vertices, dtype=np.int32)
    d = MeshDesc(coords.shape[0], coords.ctypes.data, cv.shape[0], cv.ctypes.data)
    return d, (coords, cv)


def fe_space_create(coords, cell_vertices, order: int, quad_points_1d: int, problem: int, nu: float,
                    host_only: bool = False) -> int:
    d, keep = _mesh_desc(coords, cell_vertices)
    out = ctypes.c_void_p()
    fn = lib().fe_space_create_host if host_only else lib().fe_space_create
    _check(fn(ctypes.byref(d), order, quad_points_1d, problem, float(nu), ctypes.byref(out)),
           "fe_space_create")
    del keep
    return out.value


def fe_space_sizes(space: int):
    v = [ctypes.c_int64() for _ in range(4)]
    _check(lib().fe_space_sizes(space, *[ctypes.byref(x) for x in v]), "fe_space_sizes")
    return tuple(x.value for x in v)   # n_dofs, nnz, n_cells, n_contrib


def fe_space_cell_dofs_host(space: int, n_cells: int, nl: int) -> np.ndarray:
    out = np.zeros((n_cells, nl), dtype=np.int32)
    _check(lib().fe_space_cell_dofs_host(space, out.ctypes.data), "fe_space_cell_dofs_host")
    return out


def fe_space_csr_pattern_host(space: int):
    n_dofs, nnz, _, _ = fe_space_sizes(space)
    rp = np.zeros(n_dofs + 1, dtype=np.int64)
    col = np.zeros(nnz, dtype=np.int32)
    _check(lib().fe_space_csr_pattern_host(space, rp.ctypes.data, col.ctypes.data), "fe_space_csr_pattern_host")
    return rp, col


def fe_space_permutation_host(space: int):
    n_dofs, nnz, n_cells, n_contrib = fe_space_sizes(space)
    cnt = np.zeros(nnz, dtype=np.uint8)
    code_ptr = np.zeros(n_dofs + 1, dtype=np.int64)
    slot_ptr = np.zeros(n_dofs + 1, dtype=np.int64)
    slots = np.zeros(int(slot_count(space)), dtype=np.int32)
    _check(lib().fe_space_permutation_host(space, cnt.ctypes.data, code_ptr.ctypes.data, None,
                                           slot_ptr.ctypes.data, slots.ctypes.data), "fe_space_permutation_host")
    codes = np.zeros(int(code_ptr[-1]), dtype=np.uint16)
    _check(lib().fe_space_permutation_host(space, cnt.ctypes.data, code_ptr.ctypes.data, codes.ctypes.data,
                                           slot_ptr.ctypes.data, slots.ctypes.data), "fe_space_permutation_host")
    return cnt, code_ptr, codes, slot_ptr, slots


def slot_count(space: int) -> int:
    """Number of (cell, local DOF) incidences: n_contrib / n_loc."""
    n_dofs, nnz, n_cells, n_contrib = fe_space_sizes(space)
    nl = int(round((n_contrib / max(n_cells, 1)) ** 0.5))
    return n_cells * nl


def fe_space_csr_pattern(space: int, row_ptr, col_idx, stream=None):
    _check(lib().fe_space_csr_pattern(space, _ptr(row_ptr), _ptr(col_idx), _stream(stream)), "fe_space_csr_pattern")


def fe_assemble(space: int, coefficients, body_force, csr_values, rhs, prec: int, stream=None):
    f = np.ascontiguousarray(np.resize(np.asarray(body_force, dtype=np.float64), 3))
    _check(lib().fe_assemble(space, _ptr(coefficients), f.ctypes.data, _ptr(csr_values), _ptr(rhs), prec,
                             _stream(stream)), "fe_assemble")


def fe_assemble_ex(space: int, coefficients, body_force, csr_values, rhs, prec: int, stream, event_mid):
    """fe_assemble that records the CUDA event handle `event_mid` between its two kernels."""
    f = np.ascontiguousarray(np.resize(np.asarray(body_force, dtype=np.float64), 3))
    _check(lib().fe_assemble_ex(space, _ptr(coefficients), f.ctypes.data, _ptr(csr_values), _ptr(rhs), prec,
                                _stream(stream), int(event_mid)), "fe_assemble_ex")


def fe_assemble_host(space: int, coefficients, body_force, csr_values, rhs, prec: int, stream=None):
    f = np.ascontiguousarray(np.resize(np.asarray(body_force, dtype=np.float64), 3))
    _check(lib().fe_assemble_host(space, _ptr(coefficients), f.ctypes.data, _ptr(csr_values), _ptr(rhs), prec,
                                  _stream(stream)), "fe_assemble_host")


def fe_assemble_adjoint(space: int, u, coefficients, grad_scale: float, dc_dcoef, compliance, prec: int,
                        stream=None):
    _check(lib().fe_assemble_adjoint(space, _ptr(u), _ptr(coefficients), float(grad_scale), _ptr(dc_dcoef),
                                     _ptr(compliance), prec, _stream(stream)), "fe_assemble_adjoint")


FE_KERNEL_AUTO, FE_KERNEL_CUDA_CORE, FE_KERNEL_TENSOR_CORE = 0, 1, 2
KERNELS = {"auto": FE_KERNEL_AUTO, "cuda_core": FE_KERNEL_CUDA_CORE, "tensor_core": FE_KERNEL_TENSOR_CORE}


def fe_space_set_kernel(space: int, kernel: str):
    _check(lib().fe_space_set_kernel(space, KERNELS[kernel]), "fe_space_set_kernel")


def fe_assemble_adjoint_noalloc(space: int, u, coefficients, grad_scale: float, dc_dcoef, compliance, prec: int,
                                stream=None):
    """fe_assemble_adjoint with its reduction scratch in a static device array (no allocation)."""
    _check(lib().fe_assemble_adjoint_noalloc(space, _ptr(u), _ptr(coefficients), float(grad_scale),
                                             _ptr(dc_dcoef), _ptr(compliance), prec, _stream(stream)),
           "fe_assemble_adjoint_noalloc")


def fe_status(space: int, stream=None) -> int:
    return int(lib().fe_status(space, _stream(stream)))


def fe_space_destroy(space: int):
    lib().fe_space_destroy(space)


def fe_batch_create(spaces, cells_per_item: int = 0) -> int:
    arr = (ctypes.c_void_p * len(spaces))(*spaces)
    out = ctypes.c_void_p()
    _check(lib().fe_batch_create(arr, len(spaces), cells_per_item, ctypes.byref(out)), "fe_batch_create")
    return out.value


def fe_batch_assemble(batch: int, coefficients, body_forces, csr_values, rhs, prec: int, stream=None):
    n = len(coefficients)
    cp = (ctypes.c_void_p * n)(*[_ptr(c) for c in coefficients])
    vp = (ctypes.c_void_p * n)(*[_ptr(v) for v in csr_values])
    rp = (ctypes.c_void_p * n)(*[_ptr(r) for r in rhs])
    f = np.ascontiguousarray(np.concatenate([np.resize(np.asarray(b, dtype=np.float64), 3) for b in body_forces]
                                            + [np.zeros(3)]))
    _check(lib().fe_batch_assemble(batch, cp, f.ctypes.data, vp, rp, prec, _stream(stream)), "fe_batch_assemble")


def fe_batch_set_wait(batch: int, wait_cycles: int, extra_cells: int):
    _check(lib().fe_batch_set_wait(batch, int(wait_cycles), int(extra_cells)), "fe_batch_set_wait")


def fe_selftest_conversions(x, out32, out64, stream=None):
    _check(lib().fe_selftest_conversions(_ptr(x), int(x.numel()), _ptr(out32), _ptr(out64), _stream(stream)),
           "fe_selftest_conversions")


def fe_batch_destroy(batch: int):
    lib().fe_batch_destroy(batch)


def fe_space_dof_points_host(space: int, coords, cell_vertices) -> np.ndarray:
    """Node position of every DOF, [n_dofs, 3] (host)."""
    n_dofs = fe_space_sizes(space)[0]
    d, keep = _mesh_desc(coords, cell_vertices)
    out = np.zeros((n_dofs, 3), dtype=np.float64)
    _check(lib().fe_space_dof_points_host(space, ctypes.byref(d), out.ctypes.data), "fe_space_dof_points_host")
    del keep
    return out


def fe_mesh_locality_order(coords, cell_vertices) -> np.ndarray:
    """Cell order for memory locality (Morton order of the cell centroids),
    [n_cells] int64 (host): new cell i = input cell order[i]."""
    d, keep = _mesh_desc(coords, cell_vertices)
    out = np.zeros(d.n_cells, dtype=np.int64)
    _check(lib().fe_mesh_locality_order(ctypes.byref(d), out.ctypes.data), "fe_mesh_locality_order")
    del keep
    return out


def fe_dirichlet_create(space: int, fixed) -> int:
    fx = np.ascontiguousarray(np.asarray(fixed).astype(np.uint8))
    out = ctypes.c_void_p()
    _check(lib().fe_dirichlet_create(space, fx.ctypes.data, ctypes.byref(out)), "fe_dirichlet_create")
    return out.value


def fe_dirichlet_sizes(d: int):
    v = [ctypes.c_int64() for _ in range(3)]
    _check(lib().fe_dirichlet_sizes(d, *[ctypes.byref(x) for x in v]), "fe_dirichlet_sizes")
    return tuple(x.value for x in v)   # n_free, n_fixed, nnz


def fe_dirichlet_labels_host(d: int, n_dofs: int) -> np.ndarray:
    out = np.zeros(n_dofs, dtype=np.int32)
    _check(lib().fe_dirichlet_labels_host(d, out.ctypes.data), "fe_dirichlet_labels_host")
    return out


def fe_dirichlet_csr_pattern_host(d: int):
    n_free, _, nnz = fe_dirichlet_sizes(d)
    rp = np.zeros(n_free + 1, dtype=np.int64)
    col = np.zeros(nnz, dtype=np.int32)
    _check(lib().fe_dirichlet_csr_pattern_host(d, rp.ctypes.data, col.ctypes.data), "fe_dirichlet_csr_pattern_host")
    return rp, col


def fe_dirichlet_csr_pattern(d: int, row_ptr, col_idx, stream=None):
    _check(lib().fe_dirichlet_csr_pattern(d, _ptr(row_ptr), _ptr(col_idx), _stream(stream)),
           "fe_dirichlet_csr_pattern")


def fe_dirichlet_permutation_host(d: int, n_slots: int):
    """(cnt, code_ptr, codes, ncode, pos, slot_ptr, slots) of a host-only space's constrained system."""
    n_free, _, nnz = fe_dirichlet_sizes(d)
    cnt = np.zeros(nnz, dtype=np.uint8)
    code_ptr = np.zeros(n_free + 1, dtype=np.int64)
    ncode = np.zeros(n_free, dtype=np.int32)
    slot_ptr = np.zeros(n_free + 1, dtype=np.int64)
    slots = np.zeros(n_slots, dtype=np.int32)
    args = [cnt.ctypes.data, code_ptr.ctypes.data]
    _check(lib().fe_dirichlet_permutation_host(d, *args, None, ncode.ctypes.data, None, slot_ptr.ctypes.data,
                                               slots.ctypes.data), "fe_dirichlet_permutation_host")
    slots = slots[:int(slot_ptr[-1])]
    codes = np.zeros(int(code_ptr[-1]), dtype=np.uint16)
    pos = np.zeros(int(code_ptr[-1]), dtype=np.uint16)
    _check(lib().fe_dirichlet_permutation_host(d, *args, codes.ctypes.data, ncode.ctypes.data, pos.ctypes.data,
                                               slot_ptr.ctypes.data, slots.ctypes.data),
           "fe_dirichlet_permutation_host")
    return cnt, code_ptr, codes, ncode, pos, slot_ptr, slots


def fe_dirichlet_lift_host(d: int):
    """(cells, ptr, m, fix): the cells whose cell vectors are lifted and their fixed local columns."""
    nc, ne = ctypes.c_int64(), ctypes.c_int64()
    _check(lib().fe_dirichlet_lift_host(d, ctypes.byref(nc), ctypes.byref(ne), None, None, None, None),
           "fe_dirichlet_lift_host")
    cells = np.zeros(nc.value, dtype=np.int32)
    ptr = np.zeros(nc.value + 1, dtype=np.int32)
    m = np.zeros(ne.value, dtype=np.uint8)
    fix = np.zeros(ne.value, dtype=np.int32)
    _check(lib().fe_dirichlet_lift_host(d, None, None, cells.ctypes.data, ptr.ctypes.data, m.ctypes.data,
                                        fix.ctypes.data), "fe_dirichlet_lift_host")
    return cells, ptr, m, fix


def fe_assemble_dirichlet(d: int, coefficients, body_force, u_fixed, csr_values, rhs, prec: int, stream=None):
    f = np.ascontiguousarray(np.resize(np.asarray(body_force, dtype=np.float64), 3))
    _check(lib().fe_assemble_dirichlet(d, _ptr(coefficients), f.ctypes.data, _ptr(u_fixed), _ptr(csr_values),
                                       _ptr(rhs), prec, _stream(stream)), "fe_assemble_dirichlet")


def fe_dirichlet_destroy(d: int):
    lib().fe_dirichlet_destroy(d)


def fe_space_block_offset(space: int) -> int:
    n = ctypes.c_int64()
    _check(lib().fe_space_block_offset(space, ctypes.byref(n)), "fe_space_block_offset")
    return n.value


def fe_compliance_work_size(d: int) -> int:
    n = ctypes.c_int64()
    _check(lib().fe_compliance_work_size(d, ctypes.byref(n)), "fe_compliance_work_size")
    return n.value


def fe_compliance(d: int, coefficients, body_force, prec: int, rtol: float, max_iter: int, work, u, compliance,
                  dc_dcoef, stream=None):
    """Returns (iterations, relative residual)."""
    f = np.ascontiguousarray(np.resize(np.asarray(body_force, dtype=np.float64), 3))
    it, rel = ctypes.c_int(), ctypes.c_double()
    _check(lib().fe_compliance(d, _ptr(coefficients), f.ctypes.data, prec, float(rtol), int(max_iter), _ptr(work),
                               _ptr(u), _ptr(compliance), _ptr(dc_dcoef), ctypes.byref(it), ctypes.byref(rel),
                               _stream(stream)), "fe_compliance")
    return it.value, rel.value


class DirichletSystem:
    """The constrained system of an FESpace with the DOFs of `fixed` prescribed
    (strong Dirichlet conditions). Keeps its space alive."""

    def __init__(self, space: "FESpace", fixed):
        self.space = space
        self.handle = fe_dirichlet_create(space.handle, fixed)
        self.n_free, self.n_fixed, self.nnz = fe_dirichlet_sizes(self.handle)

    def labels(self) -> np.ndarray:
        return fe_dirichlet_labels_host(self.handle, self.space.n_dofs)

    def pattern_host(self):
        return fe_dirichlet_csr_pattern_host(self.handle)

    def pattern(self, device="cuda"):
        import torch
        rp = torch.empty(self.n_free + 1, dtype=torch.int64, device=device)
        col = torch.empty(self.nnz, dtype=torch.int32, device=device)
        fe_dirichlet_csr_pattern(self.handle, rp, col)
        return rp, col

    def assemble(self, coef, u_fixed=None, values=None, rhs=None, prec: str = "fp32", force=None, stream=None):
        import torch
        if values is None:
            values = torch.empty(self.nnz, dtype=torch.float64, device=coef.device)
        if rhs is None:
            rhs = torch.empty(self.n_free, dtype=torch.float64, device=coef.device)
        fe_assemble_dirichlet(self.handle, coef, self.space.prob.force if force is None else force, u_fixed,
                              values, rhs, PRECISIONS[prec], stream)
        return values, rhs

    def compliance(self, coef, prec: str = "fp64", rtol: float = 1e-10, max_iter: int = 20000, force=None,
                   gradient: bool = True, stream=None):
        """(u over all DOFs, c, dc/dcoef or None, iterations, relative residual) of the
        clamped structure (fixed DOFs at zero) under its body force."""
        import torch
        dev = coef.device
        work = torch.empty(fe_compliance_work_size(self.handle), dtype=torch.float64, device=dev)
        u = torch.empty(self.space.n_dofs, dtype=torch.float64, device=dev)
        c = torch.empty(1, dtype=torch.float64, device=dev)
        g = torch.empty(self.space.n_cells, dtype=torch.float64, device=dev) if gradient else None
        it, rel = fe_compliance(self.handle, coef, self.space.prob.force if force is None else force,
                                PRECISIONS[prec], rtol, max_iter, work, u, c, g, stream)
        return u, c, g, it, rel

    def close(self):
        if self.handle:
            fe_dirichlet_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class FESpace:
    """Owns one fe_space handle built from a seeded workload (inputs.Problem)."""

    def __init__(self, prob, host_only: bool = False):
        self.prob = prob
        self.handle = fe_space_create(prob.mesh.coords, prob.mesh.cell_vertices, prob.order, prob.quad_1d,
                                      prob.problem, prob.nu, host_only=host_only)
        self.n_dofs, self.nnz, self.n_cells, self.n_contrib = fe_space_sizes(self.handle)
        self.nl = prob.n_local
        self.n_first = fe_space_block_offset(self.handle)

    def cell_dofs(self) -> np.ndarray:
        return fe_space_cell_dofs_host(self.handle, self.n_cells, self.nl)

    def pattern_host(self):
        return fe_space_csr_pattern_host(self.handle)

    def pattern(self, device="cuda"):
        import torch
        rp = torch.empty(self.n_dofs + 1, dtype=torch.int64, device=device)
        col = torch.empty(self.nnz, dtype=torch.int32, device=device)
        fe_space_csr_pattern(self.handle, rp, col)
        return rp, col

    def assemble(self, coef, values=None, rhs=None, prec: str = "fp32", force=None, stream=None):
        import torch
        if values is None:
            values = torch.empty(self.nnz, dtype=torch.float64, device=coef.device)
        if rhs is None:
            rhs = torch.empty(self.n_dofs, dtype=torch.float64, device=coef.device)
        fe_assemble(self.handle, coef, self.prob.force if force is None else force, values, rhs,
                    PRECISIONS[prec], stream)
        return values, rhs

    def adjoint(self, u, coef=None, grad_scale: float = 1.0, out=None, compliance=None, prec: str = "fp64",
                stream=None):
        import torch
        if out is None:
            out = torch.empty(self.n_cells, dtype=torch.float64, device=u.device)
        fe_assemble_adjoint(self.handle, u, coef, grad_scale, out, compliance, PRECISIONS[prec], stream)
        return out

    def set_kernel(self, kernel: str):
        fe_space_set_kernel(self.handle, kernel)

    def dof_points(self) -> np.ndarray:
        return fe_space_dof_points_host(self.handle, self.prob.mesh.coords, self.prob.mesh.cell_vertices)

    def dirichlet(self, fixed) -> DirichletSystem:
        return DirichletSystem(self, fixed)

    def status(self, stream=None) -> int:
        return fe_status(self.handle, stream)

    def close(self):
        if self.handle:
            fe_space_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class DGSpace:
    """Interior penalty DG (Poisson) space on a mesh: cell-local DOFs K*(p+1)^3 + a."""

    def __init__(self, mesh, order: int, host_only: bool = False):
        d, keep = _mesh_desc(mesh.coords, mesh.cell_vertices)
        out = ctypes.c_void_p()
        fn = lib().fe_dg_create_host if host_only else lib().fe_dg_create
        _check(fn(ctypes.byref(d), int(order), ctypes.byref(out)), "fe_dg_create")
        del keep
        self.handle = out.value
        v = [ctypes.c_int64() for _ in range(4)]
        _check(lib().fe_dg_sizes(self.handle, *[ctypes.byref(x) for x in v]), "fe_dg_sizes")
        self.n_dofs, self.nnz, self.n_interior, self.n_boundary = (x.value for x in v)

    def pattern_host(self):
        rp = np.zeros(self.n_dofs + 1, dtype=np.int64)
        col = np.zeros(self.nnz, dtype=np.int32)
        _check(lib().fe_dg_csr_pattern_host(self.handle, rp.ctypes.data, col.ctypes.data), "fe_dg_csr_pattern_host")
        return rp, col

    def pattern(self, device="cuda"):
        import torch
        rp = torch.empty(self.n_dofs + 1, dtype=torch.int64, device=device)
        col = torch.empty(self.nnz, dtype=torch.int32, device=device)
        _check(lib().fe_dg_csr_pattern(self.handle, _ptr(rp), _ptr(col), _stream(None)), "fe_dg_csr_pattern")
        return rp, col

    def facets(self):
        ni, nb = self.n_interior, self.n_boundary
        plus, minus = np.zeros(ni, np.int32), np.zeros(ni, np.int32)
        pf, mf = np.zeros(ni, np.uint8), np.zeros(ni, np.uint8)
        bc, bf = np.zeros(nb, np.int32), np.zeros(nb, np.uint8)
        _check(lib().fe_dg_facets_host(self.handle, plus.ctypes.data, minus.ctypes.data, pf.ctypes.data,
                                       mf.ctypes.data, bc.ctypes.data, bf.ctypes.data), "fe_dg_facets_host")
        return plus, minus, pf, mf, bc, bf

    def assemble(self, tau: float, gamma: float, source: float = 0.0, values=None, rhs=None, prec: str = "fp64",
                 stream=None, device="cuda"):
        import torch
        if values is None:
            values = torch.empty(self.nnz, dtype=torch.float64, device=device)
        if rhs is None:
            rhs = torch.empty(self.n_dofs, dtype=torch.float64, device=device)
        _check(lib().fe_dg_assemble(self.handle, float(tau), float(gamma), float(source), _ptr(values), _ptr(rhs),
                                    PRECISIONS[prec], _stream(stream)), "fe_dg_assemble")
        return values, rhs

    def close(self):
        if self.handle:
            lib().fe_dg_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

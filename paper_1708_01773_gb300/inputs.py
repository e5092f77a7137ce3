"""Seeded synthetic inputs shared by the CUDA path, the oracle and the benchmark.

This module draws meshes, coefficients and displacement fields. It holds none of
the finite element arithmetic (no shape functions, Jacobians or quadrature):
both sides of every parity check receive exactly the arrays built here.

Mesh convention (the paper's lexicographic node numbering, Sect. "Node
generation and indexing", Eq. nodes_set): the local vertex ``v`` of a hexahedron
sits at reference corner ``(v & 1, (v >> 1) & 1, (v >> 2) & 1)`` of [0,1]^3, so
local vertex order is x-fastest lexicographic. Cells of a structured brick are
numbered x-fastest as well, like the structured mesh generator of the paper
(Sect. "A triangulation implementation").

Workloads (the paper runs no experiments; these stand in for its "structural"
problems, all synthetic):

* ``poisson_q1_8``      Poisson Q1, 8^3 cells of the unit cube, interior vertices
  shifted by up to 0.2h per coordinate, conductivity 10^U[-1,1], f = 1, 2^3 Gauss.
* ``elasticity_q2_beam`` Elasticity Q2, 32x32x32 cells of the beam [0,4]x[0,1]^2,
  shifts up to 0.15h_d, E ~ U[1,10], nu = 0.3, f = (0,0,-1), 3^3 Gauss.
* ``elasticity_q1_128`` Elasticity Q1, 128^3 cells of the unit cube, shifts up to
  0.2h, E = 10^U[log10 0.5, log10 5], nu = 0.3, f = (0,0,-1), 2^3 Gauss.
* ``batched64``        64 unit-cube meshes with n ~ U{10..40} cells per axis,
  p ~ U{1,2,3}, problem ~ Bernoulli(1/2), (p+1)^3 Gauss, shifts up to 0.2h;
  redrawn while the estimated GPU footprint exceeds half of the GPU memory.
* ``cantilever_q1_64`` Elasticity Q1, 64^3 cells of the unit cube, E ~ U[0.1,1],
  nu = 0.3, shifts up to 0.2h, u ~ N(0,1) per DOF rescaled to unit RMS.
* ``stokes_q2q1_32``   Stokes, Taylor-Hood Q2/Q1, 32^3 cells of the unit cube,
  shifts up to 0.15h, viscosity mu ~ U[0.5, 2], f = (0, 0, -1), 3^3 Gauss.
* ``poisson_q3_40``    Poisson Q3, 40^3 cells of the unit cube (the largest Q3
  mesh of the batched recipe), shifts up to 0.2h, conductivity 10^U[-1,1],
  f = 1, 4^3 Gauss (``poisson_q3_24``: the same on 24^3 cells).
* ``elasticity_q3_20`` Elasticity Q3, 20^3 cells of the unit cube, shifts up to
  0.2h, E ~ U[1,10], nu = 0.3, f = (0,0,-1), 4^3 Gauss (``elasticity_q3_12``:
  the same on 12^3 cells).

``scramble`` presents any of these meshes as an unstructured one (random vertex
ids, random cell order, each cell's local vertex order turned by one of the 24
proper rotations of the reference cube), so that the DOF numbering, the
assembly maps and the facet matching are exercised without the brick's
regular numbering (``elasticity_q1_128_scrambled``: the 128^3 workload so
presented, the worst case of memory locality for the assembly maps).
"""
from __future__ import annotations

import itertools
from dataclasses import dataclass, field

import numpy as np

SEED_BASE = 20171773

POISSON = 0
ELASTICITY = 1
STOKES = 2        # Taylor-Hood: velocity Q_p (3 components), pressure Q_{p-1}


@dataclass
class Mesh:
    """A conforming hexahedral mesh: vertex coordinates and cell connectivity."""

    coords: np.ndarray          # [n_vertices, 3] float64
    cell_vertices: np.ndarray   # [n_cells, 8] int32, x-fastest local order
    shape: tuple = ()           # (nx, ny, nz) for structured bricks
    extent: tuple = ()          # (Lx, Ly, Lz)

    @property
    def n_cells(self) -> int:
        return int(self.cell_vertices.shape[0])

    @property
    def n_vertices(self) -> int:
        return int(self.coords.shape[0])


@dataclass
class Problem:
    """One assembly workload: mesh + discretisation + coefficients."""

    name: str
    mesh: Mesh
    order: int
    quad_1d: int
    problem: int                 # POISSON, ELASTICITY or STOKES
    coef: np.ndarray             # [n_cells] float64 (kappa_K, E_K or the viscosity mu_K)
    force: np.ndarray            # [ncomp] float64, constant body force / source
    nu: float = 0.3
    extra: dict = field(default_factory=dict)

    @property
    def ncomp(self) -> int:
        """Components of the (velocity) field."""
        return 1 if self.problem == POISSON else 3

    @property
    def n_local(self) -> int:
        """Local DOFs of a cell: ncomp (p+1)^3, plus p^3 pressure nodes for Stokes."""
        n = self.ncomp * (self.order + 1) ** 3
        return n + self.order ** 3 if self.problem == STOKES else n


def brick(nx: int, ny: int, nz: int, lx: float = 1.0, ly: float = 1.0, lz: float = 1.0) -> Mesh:
    """Structured brick [0,lx]x[0,ly]x[0,lz] with nx*ny*nz hexahedra."""
    xs = np.linspace(0.0, lx, nx + 1)
    ys = np.linspace(0.0, ly, ny + 1)
    zs = np.linspace(0.0, lz, nz + 1)
    Z, Y, X = np.meshgrid(zs, ys, xs, indexing="ij")
    coords = np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1).astype(np.float64)
    i = np.arange(nx)
    j = np.arange(ny)
    k = np.arange(nz)
    K, J, I = np.meshgrid(k, j, i, indexing="ij")
    base = (I + J * (nx + 1) + K * (nx + 1) * (ny + 1)).ravel().astype(np.int64)
    cv = np.empty((base.size, 8), dtype=np.int64)
    for v in range(8):
        bx, by, bz = v & 1, (v >> 1) & 1, (v >> 2) & 1
        cv[:, v] = base + bx + by * (nx + 1) + bz * (nx + 1) * (ny + 1)
    return Mesh(coords=coords, cell_vertices=cv.astype(np.int32), shape=(nx, ny, nz), extent=(lx, ly, lz))


def perturb_interior(mesh: Mesh, alpha: float, rng: np.random.Generator) -> Mesh:
    """Shift every interior vertex coordinate by an independent U[-alpha h_d, alpha h_d].

    Boundary vertices stay put, so the domain and its volume are unchanged.
    """
    nx, ny, nz = mesh.shape
    lx, ly, lz = mesh.extent
    h = np.array([lx / nx, ly / ny, lz / nz])
    shift = rng.uniform(-1.0, 1.0, size=mesh.coords.shape) * (alpha * h)[None, :]
    idx = np.arange(mesh.n_vertices)
    vi = idx % (nx + 1)
    vj = (idx // (nx + 1)) % (ny + 1)
    vk = idx // ((nx + 1) * (ny + 1))
    interior = (vi > 0) & (vi < nx) & (vj > 0) & (vj < ny) & (vk > 0) & (vk < nz)
    coords = mesh.coords.copy()
    coords[interior] += shift[interior]
    return Mesh(coords=coords, cell_vertices=mesh.cell_vertices, shape=mesh.shape, extent=mesh.extent)


def _log_uniform(rng, lo, hi, n):
    return 10.0 ** rng.uniform(np.log10(lo), np.log10(hi), size=n)


def poisson_q1_8(n: int = 8, seed_offset: int = 1) -> Problem:
    rng = np.random.default_rng(SEED_BASE + seed_offset)
    mesh = perturb_interior(brick(n, n, n), 0.2, rng)
    coef = _log_uniform(rng, 0.1, 10.0, mesh.n_cells)
    return Problem("poisson_q1_8", mesh, 1, 2, POISSON, coef, np.array([1.0]))


def elasticity_q2_beam(n: int = 32, seed_offset: int = 2) -> Problem:
    rng = np.random.default_rng(SEED_BASE + seed_offset)
    mesh = perturb_interior(brick(n, n, n, 4.0, 1.0, 1.0), 0.15, rng)
    coef = rng.uniform(1.0, 10.0, size=mesh.n_cells)
    return Problem("elasticity_q2_beam", mesh, 2, 3, ELASTICITY, coef, np.array([0.0, 0.0, -1.0]))


def elasticity_q1_128(n: int = 128, seed_offset: int = 3) -> Problem:
    rng = np.random.default_rng(SEED_BASE + seed_offset)
    mesh = perturb_interior(brick(n, n, n), 0.2, rng)
    coef = _log_uniform(rng, 0.5, 5.0, mesh.n_cells)
    return Problem("elasticity_q1_128", mesh, 1, 2, ELASTICITY, coef, np.array([0.0, 0.0, -1.0]))


def _coupled_pairs_1d(n: int, p: int) -> int:
    """Pairs of the (p n + 1) nodes of a 1D line of n cells that share a cell."""
    m = p * n + 1
    count = 0
    for i in range(m):
        ci = {min(i // p, n - 1)} | ({i // p - 1} if (i % p == 0 and i > 0) else set())
        for j in range(max(0, i - 2 * p), min(m, i + 2 * p + 1)):
            cj = {min(j // p, n - 1)} | ({j // p - 1} if (j % p == 0 and j > 0) else set())
            if ci & cj:
                count += 1
    return count


def device_footprint(n: int, p: int, problem: int) -> int:
    """Bytes the assembly of an n^3 brick of order p holds on the GPU: CSR values,
    columns and counts per nonzero, two 16-bit permutation arrays per contribution,
    and the FP64-sized cell-matrix scratch (a budget estimate, not exact)."""
    c = 3 if problem == ELASTICITY else 1
    nnz = _coupled_pairs_1d(n, p) ** 3 * c * c
    nl = c * (p + 1) ** 3
    nlp = (nl + 3) // 4 * 4
    return nnz * (8 + 4 + 1) + n ** 3 * nl * nl * 4 + n ** 3 * nl * nlp * 8


def batched64(n_meshes: int = 64, n_lo: int = 10, n_hi: int = 40, seed_offset: int = 4,
              budget_bytes: float = 140e9) -> list[Problem]:
    """Independent meshes of uneven size and mixed order, one child seed each.

    A draw whose estimated device footprint exceeds `budget_bytes` (half of the
    GPU's memory by default) is redrawn from the next spawn key of the same seed.
    """
    for attempt in range(10000):
        base = np.random.SeedSequence(SEED_BASE + seed_offset, spawn_key=(attempt,) if attempt else ())
        children = base.spawn(n_meshes)
        draws = []
        total = 0
        for ss in children:
            rng = np.random.default_rng(ss)
            n = int(rng.integers(n_lo, n_hi + 1))
            p = int(rng.integers(1, 4))
            prob = int(rng.integers(0, 2))
            draws.append((ss, n, p, prob))
            total += device_footprint(n, p, prob)
        if total <= budget_bytes:
            break
    out = []
    for m, (ss, n, p, prob) in enumerate(draws):
        rng = np.random.default_rng(ss)
        rng.integers(n_lo, n_hi + 1), rng.integers(1, 4), rng.integers(0, 2)  # the draws above
        mesh = perturb_interior(brick(n, n, n), 0.2, rng)
        if prob == POISSON:
            coef = _log_uniform(rng, 0.1, 10.0, mesh.n_cells)
            force = np.array([1.0])
        else:
            coef = rng.uniform(1.0, 10.0, size=mesh.n_cells)
            force = np.array([0.0, 0.0, -1.0])
        out.append(Problem(f"batch{m}_p{p}_{'ela' if prob else 'poi'}_n{n}", mesh, p, p + 1, prob, coef, force,
                           extra={"attempt": attempt, "footprint": device_footprint(n, p, prob)}))
    return out


def cantilever_q1_64(n: int = 64, seed_offset: int = 5) -> Problem:
    rng = np.random.default_rng(SEED_BASE + seed_offset)
    mesh = perturb_interior(brick(n, n, n), 0.2, rng)
    coef = rng.uniform(0.1, 1.0, size=mesh.n_cells)
    return Problem("cantilever_q1_64", mesh, 1, 2, ELASTICITY, coef, np.array([0.0, 0.0, -1.0]))


def stokes_q2q1_32(n: int = 32, seed_offset: int = 6) -> Problem:
    rng = np.random.default_rng(SEED_BASE + seed_offset)
    mesh = perturb_interior(brick(n, n, n), 0.15, rng)
    coef = rng.uniform(0.5, 2.0, size=mesh.n_cells)
    return Problem("stokes_q2q1_32", mesh, 2, 3, STOKES, coef, np.array([0.0, 0.0, -1.0]))


def dg_q2_32(n: int = 32, seed_offset: int = 7) -> Mesh:
    """Mesh of the interior penalty DG workload: 32^3 cells of the unit cube,
    interior shifts up to 0.15h (discontinuous Q2, tau = 1, gamma = 10, f = 1)."""
    rng = np.random.default_rng(SEED_BASE + seed_offset)
    return perturb_interior(brick(n, n, n), 0.15, rng)


def poisson_q3(n: int = 40, seed_offset: int = 8) -> Problem:
    """Poisson Q3 on n^3 cells of the unit cube (40^3 is the largest Q3 mesh of
    the batched recipe), interior shifts up to 0.2h, conductivity 10^U[-1,1],
    f = 1, 4^3 Gauss."""
    rng = np.random.default_rng(SEED_BASE + seed_offset)
    mesh = perturb_interior(brick(n, n, n), 0.2, rng)
    return Problem(f"poisson_q3_{n}", mesh, 3, 4, POISSON, _log_uniform(rng, 0.1, 10.0, mesh.n_cells), np.array([1.0]))


def elasticity_q3(n: int = 20, seed_offset: int = 9) -> Problem:
    """Linear elasticity Q3 on n^3 cells of the unit cube (the Q3 elasticity
    meshes of the batched recipe), interior shifts up to 0.2h, E ~ U[1,10],
    nu = 0.3, body force (0, 0, -1), 4^3 Gauss."""
    rng = np.random.default_rng(SEED_BASE + seed_offset)
    mesh = perturb_interior(brick(n, n, n), 0.2, rng)
    return Problem(f"elasticity_q3_{n}", mesh, 3, 4, ELASTICITY, rng.uniform(1.0, 10.0, size=mesh.n_cells),
                   np.array([0.0, 0.0, -1.0]))


def unit_rms_field(n_dofs: int, seed: int) -> np.ndarray:
    """u_i ~ N(0,1) i.i.d., rescaled so that sqrt(mean(u^2)) = 1."""
    rng = np.random.default_rng(seed)
    u = rng.standard_normal(n_dofs)
    return u / np.sqrt(np.mean(u * u))


def small_problem(n: tuple, order: int, problem: int, alpha: float = 0.2, seed: int = 7,
                  extent: tuple = (1.0, 1.0, 1.0)) -> Problem:
    """A small seeded problem for parity tests (several tiles plus a ragged tail)."""
    rng = np.random.default_rng(SEED_BASE + 100 + seed)
    mesh = perturb_interior(brick(*n, *extent), alpha, rng)
    if problem == POISSON:
        coef = _log_uniform(rng, 0.1, 10.0, mesh.n_cells)
        force = np.array([1.0])
    elif problem == STOKES:
        coef = rng.uniform(0.5, 2.0, size=mesh.n_cells)
        force = np.array([0.3, -0.2, -1.0])
    else:
        coef = rng.uniform(1.0, 10.0, size=mesh.n_cells)
        force = np.array([0.0, 0.0, -1.0])
    return Problem(f"small_{n}_p{order}_{problem}", mesh, order, order + 1, problem, coef, force)


def o_grid(m: int, k: int, nz: int, a: float = 0.45, radius: float = 1.0, height: float = 1.0) -> Mesh:
    """A hexahedral O-grid: in the xy-plane an inner square [-a, a]^2 of m x m
    cells inside four blocks of m x k cells that run out to the circle of the
    given radius, extruded over nz layers of [0, height]. The four edges through
    the inner square's corners are shared by three cells per layer (six per
    vertex between layers) instead of a brick's four (eight), so vertex
    valence, row lengths and cells per DOF vary over the mesh. Coincident points
    of the blocks are merged; every cell is orientation-preserving."""
    pts2, quads = [], []

    def block(f, ni, nj):
        base = len(pts2)
        for j in range(nj + 1):
            for i in range(ni + 1):
                pts2.append(f(i / ni, j / nj))
        for j in range(nj):
            for i in range(ni):
                q = [base + j * (ni + 1) + i, base + j * (ni + 1) + i + 1,
                     base + (j + 1) * (ni + 1) + i, base + (j + 1) * (ni + 1) + i + 1]
                quads.append(q)

    block(lambda s, t: (-a + 2 * a * s, -a + 2 * a * t), m, m)
    for side in range(4):
        ang0 = -np.pi / 4 + side * np.pi / 2
        rot = np.array([[np.cos(side * np.pi / 2), -np.sin(side * np.pi / 2)],
                        [np.sin(side * np.pi / 2), np.cos(side * np.pi / 2)]])

        def f(s, t, rot=rot, ang0=ang0):
            inner = rot @ np.array([a, -a + 2 * a * s])
            th = ang0 + s * np.pi / 2
            outer = radius * np.array([np.cos(th), np.sin(th)])
            return tuple((1 - t) * inner + t * outer)
        block(f, m, k)
    P = np.array(pts2)
    key = np.round(P, 9)
    _, first, inv = np.unique(key, axis=0, return_index=True, return_inverse=True)
    P = P[first]
    Q = inv.reshape(-1)[np.array(quads)]
    # orientation: (p10 - p00) x (p01 - p00) > 0, else swap the local x and y
    d1 = P[Q[:, 1]] - P[Q[:, 0]]
    d2 = P[Q[:, 2]] - P[Q[:, 0]]
    neg = d1[:, 0] * d2[:, 1] - d1[:, 1] * d2[:, 0] < 0
    Q[neg] = Q[neg][:, [0, 2, 1, 3]]
    n2 = P.shape[0]
    zs = np.linspace(0.0, height, nz + 1)
    coords = np.concatenate([np.column_stack([P, np.full(n2, z)]) for z in zs])
    cells = [np.concatenate([Q + l * n2, Q + (l + 1) * n2], axis=1) for l in range(nz)]
    return Mesh(coords.astype(np.float64), np.concatenate(cells).astype(np.int32), (), (2 * radius, 2 * radius, height))


def flower(k: int, nz: int, tip: float = 1.25, height: float = 1.0) -> Mesh:
    """A hexahedral "flower": in the xy-plane k quadrilaterals around the
    origin, quad i with corners (origin, spoke i, tip i, spoke i + 1), spokes
    on the unit circle at angles 2 pi i / k and tips at radius `tip` halfway
    between, extruded over nz layers. The vertices on the z-axis between two
    layers belong to 2k cells (a brick's interior vertices to 8), so k > 16
    exceeds 32 cells around a DOF."""
    ang = 2 * np.pi * np.arange(k) / k
    spokes = np.column_stack([np.cos(ang), np.sin(ang)])
    tips = tip * np.column_stack([np.cos(ang + np.pi / k), np.sin(ang + np.pi / k)])
    P = np.concatenate([[[0.0, 0.0]], spokes, tips])
    i = np.arange(k)
    # local order (x fastest): (0,0) origin, (1,0) spoke i, (0,1) spoke i+1, (1,1) tip i
    Q = np.column_stack([np.zeros(k, dtype=np.int64), 1 + i, 1 + (i + 1) % k, 1 + k + i])
    n2 = P.shape[0]
    zs = np.linspace(0.0, height, nz + 1)
    coords = np.concatenate([np.column_stack([P, np.full(n2, z)]) for z in zs])
    cells = [np.concatenate([Q + l * n2, Q + (l + 1) * n2], axis=1) for l in range(nz)]
    return Mesh(coords.astype(np.float64), np.concatenate(cells).astype(np.int32), (), (2 * tip, 2 * tip, height))


def o_grid_problem(m: int, k: int, nz: int, order: int, problem: int, seed: int = 0, mesh: Mesh | None = None) -> Problem:
    """A seeded problem on an O-grid (or on the given mesh): coefficients as in
    small_problem."""
    rng = np.random.default_rng(SEED_BASE + 700 + seed)
    mesh = o_grid(m, k, nz) if mesh is None else mesh
    if problem == POISSON:
        coef, force = _log_uniform(rng, 0.1, 10.0, mesh.n_cells), np.array([1.0])
    elif problem == STOKES:
        coef, force = rng.uniform(0.5, 2.0, size=mesh.n_cells), np.array([0.3, -0.2, -1.0])
    else:
        coef, force = rng.uniform(1.0, 10.0, size=mesh.n_cells), np.array([0.0, 0.0, -1.0])
    return Problem(f"o_grid_{m}_{k}_{nz}_p{order}_{problem}", mesh, order, order + 1, problem, coef, force)


def _cube_rotations() -> np.ndarray:
    """The 24 proper rotations of the reference cube as permutations of its 8
    local vertices (x-fastest order, v = x + 2 y + 4 z): row r maps local
    vertex v to the vertex at R_r applied to v's corner (about the centre)."""
    rows = []
    for perm in itertools.permutations(range(3)):
        for signs in itertools.product((1, -1), repeat=3):
            R = np.zeros((3, 3), dtype=np.int64)
            for i in range(3):
                R[i, perm[i]] = signs[i]
            if round(np.linalg.det(R)) != 1:
                continue
            m = []
            for v in range(8):
                c = np.array([2 * (v & 1) - 1, 2 * ((v >> 1) & 1) - 1, 2 * (v >> 2) - 1])
                r = (R @ c + 1) // 2
                m.append(int(r[0] + 2 * r[1] + 4 * r[2]))
            rows.append(m)
    return np.array(rows, dtype=np.int64)


def scramble(mesh: Mesh, rng: np.random.Generator):
    """The same mesh presented as an unstructured one: vertex ids relabelled at
    random, cells in random order, and each cell's local vertex order turned by
    a random proper rotation of the reference cube (the cell map stays
    orientation-preserving, so det J keeps its sign). Returns (mesh, order):
    new cell i is old cell order[i]."""
    vperm = rng.permutation(mesh.n_vertices)        # old vertex i gets id vperm[i]
    coords = np.empty_like(mesh.coords)
    coords[vperm] = mesh.coords
    order = rng.permutation(mesh.n_cells)
    rot = _cube_rotations()[rng.integers(0, 24, mesh.n_cells)]
    cv = np.take_along_axis(mesh.cell_vertices[order].astype(np.int64), rot, axis=1)
    return Mesh(coords, vperm[cv].astype(mesh.cell_vertices.dtype), (), mesh.extent), order


def scrambled(prob: Problem, seed: int) -> Problem:
    """A workload on the scrambled form of its mesh (coefficients follow their cells)."""
    mesh, order = scramble(prob.mesh, np.random.default_rng(SEED_BASE + 500 + seed))
    return Problem(prob.name + "_scrambled", mesh, prob.order, prob.quad_1d, prob.problem,
                   np.asarray(prob.coef)[order], prob.force, prob.nu)


def reordered(prob: Problem, order) -> Problem:
    """The workload with its cells in the given order (new cell i = old cell
    order[i]); coefficients follow their cells, vertices keep their ids."""
    order = np.asarray(order, dtype=np.int64)
    mesh = Mesh(prob.mesh.coords, prob.mesh.cell_vertices[order], (), prob.mesh.extent)
    return Problem(prob.name + "_reordered", mesh, prob.order, prob.quad_1d, prob.problem,
                   np.asarray(prob.coef)[order], prob.force, prob.nu)


WORKLOADS = {
    "poisson_q1_8": poisson_q1_8,
    "elasticity_q2_beam": elasticity_q2_beam,
    "elasticity_q1_128": elasticity_q1_128,
    "cantilever_q1_64": cantilever_q1_64,
    "stokes_q2q1_32": stokes_q2q1_32,
    "poisson_q3_40": poisson_q3,
    "poisson_q3_24": lambda: poisson_q3(24),
    "elasticity_q3_20": elasticity_q3,
    "elasticity_q3_12": lambda: elasticity_q3(12),
    "elasticity_q1_128_scrambled": lambda: scrambled(elasticity_q1_128(), seed=1),
}

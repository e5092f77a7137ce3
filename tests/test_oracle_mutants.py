"""The oracle's pins catch plausible mistakes: each case plants one slip in a
copy of fe_oracle.c (a transposed operand, a wrong sign, a dropped term or
factor, a wrong index), compiles that copy and runs the pin file against it;
at least one pin must fail. The oracle source itself is not changed. Every
slip changes the computed result (an unsymmetrised trial strain, for one,
would not: sigma(u) : eps(v) only sees the symmetric part of grad u, since
eps(v) is symmetric and tr grad u = div u; nor would mirrored bilinear weights
in the node keys: the keys only match nodes between cells, and any injective
orientation-free key gives the same list_dofs numbering)."""
import concurrent.futures
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "fe_oracle.c")
PINS = os.path.join(ROOT, "tests", "test_oracle_pins.py")

# (what is planted, text in fe_oracle.c, replacement, occurrences replaced: 0 = all)
MUTANTS = [
    ("J^-1 transposed in grad phi", "s += T->dphi[q][a][d] * Ji[d][k];", "s += T->dphi[q][a][d] * Ji[k][d];", 0),
    ("Jacobian transposed", "s += xv[3 * v + k] * T->dN[q][v][d];", "s += xv[3 * v + d] * T->dN[q][v][k];", 0),
    ("sign of one entry of J^-1", "Ji[1][2] = (J[0][2] * J[1][0] - J[0][0] * J[1][2]) / det;",
     "Ji[1][2] = (J[0][0] * J[1][2] - J[0][2] * J[1][0]) / det;", 0),
    ("det J dropped from the weight", "double dJw = det * T->w[q];", "double dJw = T->w[q];", 0),
    ("lambda term on every entry of sigma", "+ (k == l ? lambda * tr : 0.0);", "+ lambda * tr;", 0),
    ("sign of the lambda term", "su[k][l] = 2.0 * mu * eu[k][l] + (k == l ? lambda * tr : 0.0);",
     "su[k][l] = 2.0 * mu * eu[k][l] - (k == l ? lambda * tr : 0.0);", 0),
    ("factor 2 of the mu term dropped", "su[k][l] = 2.0 * mu * eu[k][l] +", "su[k][l] = mu * eu[k][l] +", 0),
    ("shape function dropped from the Poisson RHS", "fe[a] += f * T->phi[q][a] * dJw;", "fe[a] += f * dJw;", 0),
    ("Gauss weights of [-1,1] not halved", "w[n - 1 - i] = 0.5 * wt;", "w[n - 1 - i] = wt;", 0),
    ("compress keeps the last duplicate", "      values[nnz - 1] += coo[i].val;", "      values[nnz - 1] = coo[i].val;", 1),
    ("Stokes coupling missing from the pressure rows", "          Ke[(nv + c) * nl + (j * nb + b)] += bq;",
     "          (void)bq;", 0),
    ("Lagrange derivative: removed factor kept", "        if (s == m || s == r) continue;", "        if (s == m) continue;", 0),
    ("Stokes coupling sign", "double bq = -T->psi[q][c] * g[b][j] * dJw;", "double bq = T->psi[q][c] * g[b][j] * dJw;", 0),
    ("DG neighbour's reference point: one Newton step only",
     "  for (int it = 0; it < 100; ++it) {\n    double y[3], J[3][3], Ji[3][3];",
     "  for (int it = 0; it < 1; ++it) {\n    double y[3], J[3][3], Ji[3][3];", 0),
    ("DG normal sign flipped", "n[3] = {sgn * nd[0] / len, sgn * nd[1] / len, sgn * nd[2] / len};",
     "n[3] = {-sgn * nd[0] / len, -sgn * nd[1] / len, -sgn * nd[2] / len};", 0),
    ("DG mean without the factor 1/2", "const double half = interior ? 0.5 : 1.0, pen = gamma / area;",
     "const double half = 1.0, pen = gamma / area;", 0),
    ("DG jump sign dropped on one side", "+ pen * ga * gb * phi[sa][a] * phi[sb][b]);",
     "+ pen * ga * phi[sa][a] * phi[sb][b]);", 0),
    ("DG tau term with the other side's derivative", "- tau * gb * phi[sb][b] * half * gn[sa][a]",
     "- tau * gb * phi[sb][b] * half * gn[sb][a]", 0),
    ("DG penalty not divided by the facet area", "pen = gamma / area;", "pen = gamma;", 0),
    ("node keys: vef corners left in the cell's local order",
     "    while (j >= 0 && k->g[j] > gg) { k->g[j + 1] = k->g[j]; k->w[j + 1] = k->w[j]; --j; }",
     "    while (0) { k->g[j + 1] = k->g[j]; k->w[j + 1] = k->w[j]; --j; }", 0),
    ("list_dofs: cell-interior nodes met last instead of first", "    int dkey = (dim == 3) ? 0 : dim + 1;",
     "    int dkey = dim;", 0),
    ("list_dofs: n-faces of one dimension by anchor before extrusion",
     "    keys[a] = (((int64_t)dkey * 8 + ext) * 8 + anc) * 4096 + a;",
     "    keys[a] = (((int64_t)dkey * 8 + anc) * 8 + ext) * 4096 + a;", 0),
    ("smallest det J: vertices not sampled", "for (int q = 0; q < 8; ++q) { jacobian(V, q, xv, J);",
     "for (int q = 0; q < 0; ++q) { jacobian(V, q, xv, J);", 0),
    ("smallest det J: corner table left at the Gauss points",
     "    tp_basis(1, xh, phi, &V->dN[q][0][0]);", "    (void)xh; (void)phi;", 0),
]


# the oracle's Python part (strong Dirichlet conditions, compliance): one
# text replacement in one function, applied in the pytest process by conftest
PY_MUTANTS = [
    ("lifting sign", "dirichlet_reduce", "(np.asarray(rhs, dtype=np.float64) - lift)",
     "(np.asarray(rhs, dtype=np.float64) + lift)"),
    ("constrained columns keep the global ids", "dirichlet_reduce", "out_col = lab[col[kept]]", "out_col = col[kept]"),
    ("prescribed value of the wrong fixed DOF", "dirichlet_reduce", "u_fixed[-1 - lab[col[fx]]]",
     "u_fixed[(-1 - lab[col[fx]] + 1) % u_fixed.size]"),
    ("fixed labels start at 0", "dirichlet_labels", "lab[fixed] = -1 - np.arange", "lab[fixed] = -np.arange"),
    ("compliance gradient sign", "compliance_solve", "grad = -cell_energies(", "grad = cell_energies("),
    ("compliance as u^T u", "compliance_solve", "c = float(b_r @ u_free)", "c = float(u_free @ u_free)"),
]


def _run_py(case):
    name, fn, old, new = case
    env = dict(os.environ, ORACLE_PY_MUTANT=f"{fn}|{old}|{new}")
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider", PINS, "-k",
                        "dirichlet or compliance"], cwd=ROOT, env=env, capture_output=True, text=True, timeout=900)
    return name, r.returncode


def test_pins_catch_planted_mistakes_python_part():
    workers = max(1, min(len(PY_MUTANTS), len(os.sched_getaffinity(0))))
    with concurrent.futures.ThreadPoolExecutor(workers) as ex:
        results = list(ex.map(_run_py, PY_MUTANTS))
    survivors = [name for name, rc in results if rc == 0]
    assert not survivors, f"pins pass with these planted mistakes: {survivors}"
    assert all(rc == 1 for _, rc in results), results


def _run(case, tmp):
    name, old, new, count = case
    src = open(SRC).read()
    assert old in src, f"planting site not found: {name}"
    mutant = src.replace(old, new) if count == 0 else src.replace(old, new, count)
    tag = str(abs(hash(name)))
    c_file = os.path.join(tmp, f"m{tag}.c")
    so = os.path.join(tmp, f"liboracle_m{tag}.so")
    with open(c_file, "w") as f:
        f.write(mutant)
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-D_DEFAULT_SOURCE", "-fPIC", "-shared", c_file, "-o", so, "-lm"])
    env = dict(os.environ, ORACLE_LIB=so)
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider", PINS], cwd=ROOT, env=env,
                       capture_output=True, text=True, timeout=900)
    return name, r.returncode


def test_pins_catch_planted_mistakes(tmp_path):
    workers = max(1, min(len(MUTANTS), len(os.sched_getaffinity(0))))
    with concurrent.futures.ThreadPoolExecutor(workers) as ex:
        results = list(ex.map(lambda c: _run(c, str(tmp_path)), MUTANTS))
    survivors = [name for name, rc in results if rc == 0]
    assert not survivors, f"pins pass with these planted mistakes: {survivors}"
    assert all(rc == 1 for _, rc in results), results  # 1 = tests failed (not a collection or usage error)

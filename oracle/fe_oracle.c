/*
 * fe_oracle.c -- plain, slow, obviously correct FP64 CPU oracle for the cell-wise
 * numerical integration and global assembly of grad-conforming Lagrangian Q_p
 * hexahedra (Poisson and linear elasticity), following the FEMPAR paper.
 *
 * TEST INFRASTRUCTURE ONLY. Only the tests, the smoke check and the CPU-baseline
 * leg of the benchmark may load this library. The product path (the CUDA library
 * in the package) shares no code, header, table or constant with this file.
 *
 * Everything is double precision, single threaded, with no blocking or fusion:
 *   - Gauss-Legendre rule on [0,1]: Sect. "Numerical integration" (an n-point
 *     rule integrates degree 2n-1 exactly; n = p+1 by default), tensorised.
 *   - 1D Lagrange basis on equidistant nodes x_s = s/p: Eq. lagbas; tensor product
 *     basis on the cube: Eq. lagbasmd; nodes in lexicographic order: Eq. nodes_set.
 *   - Geometry: trilinear map Phi_K from the 8 vertices, J = dPhi/dxhat,
 *     det J and J^{-1}: Sect. "Numerical integration", Eq. fematrix.
 *   - Physical gradients grad(phi) = gradhat(phihat) J^{-1}: Eq. shape_grad.
 *   - Poisson cell matrix: the element loop over (q, b, a) of the Listing
 *     "element_matrix_entries_computation" with a scalar cell conductivity.
 *   - Elasticity cell matrix: a(u,v) = int sigma(u):eps(v) with isotropic Hooke
 *     sigma = lambda tr(eps) I + 2 mu eps, eps from the Stokes example
 *     (Sect. "Weak form"); the paper gives no constitutive law, Hooke is the
 *     textbook reading.
 *   - Global DOF numbering: the list_dofs algorithm of Sect. "Global DOF
 *     numbering generation" (cell interior DOFs first, then the vefs of the cell
 *     in local order; a vef seen before copies its owner's ids).
 *   - Global assembly A_[a][b] = sum_K A^K_ab (Eq. assembly) by COO push-back,
 *     sort and "compress" summing duplicates (Sect. "Linear algebra").
 *
 * Parity pins (tests): closed-form Q1 unit-cube stiffness, Gauss exactness,
 * partition of unity, patch test, zero row sums, rigid-body modes, symmetry,
 * RHS sums, uniform-strain energy, and high-order brute-force quadrature on
 * affine cells. On distorted (non-affine) cells the Gauss sums have no closed
 * form; there the entries are fixed by the patch test, the rigid-body modes,
 * the uniform-strain energy, zero row sums, symmetry and the convergence of
 * the rule, each of which a dropped term, a wrong sign or index or a
 * transposed Jacobian breaks.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_OK 0
#define OR_ERR_ARG -1
#define OR_ERR_OOM -3
#define OR_ERR_NEG_JAC -4

#define MAXP 3
#define MAXQ1D 16
#define MAXNB ((MAXP + 1) * (MAXP + 1) * (MAXP + 1))
#define MAXNQ (MAXQ1D * MAXQ1D * MAXQ1D)

/* ------------------------------------------------------------------ */
/* Gauss-Legendre rule on [0,1] (Newton iteration on the Legendre      */
/* polynomial built by its three-term recurrence).                     */
/* ------------------------------------------------------------------ */
static void legendre_eval(int n, double t, double* pn, double* dpn) {
  double p0 = 1.0, p1 = t;
  if (n == 0) { *pn = 1.0; *dpn = 0.0; return; }
  for (int k = 1; k < n; ++k) {
    double p2 = ((2.0 * k + 1.0) * t * p1 - k * p0) / (k + 1.0);
    p0 = p1;
    p1 = p2;
  }
  *pn = p1;
  /* P_n'(t) = n (t P_n - P_{n-1}) / (t^2 - 1) */
  *dpn = n * (t * p1 - p0) / (t * t - 1.0);
}

int or_gauss_legendre(int n, double* x, double* w) {
  if (n < 1 || n > MAXQ1D) return OR_ERR_ARG;
  for (int i = 0; i < n; ++i) {
    double t = cos(M_PI * (i + 0.75) / (n + 0.5));
    for (int it = 0; it < 100; ++it) {
      double pn, dpn;
      legendre_eval(n, t, &pn, &dpn);
      double dt = pn / dpn;
      t -= dt;
      if (fabs(dt) < 1e-16) break;
    }
    double pn, dpn;
    legendre_eval(n, t, &pn, &dpn);
    double wt = 2.0 / ((1.0 - t * t) * dpn * dpn);
    /* ascending order on [0,1]: the cos guesses come out descending in t */
    x[n - 1 - i] = 0.5 * (t + 1.0);
    w[n - 1 - i] = 0.5 * wt;
  }
  return OR_OK;
}

/* ------------------------------------------------------------------ */
/* 1D Lagrange basis of order p on the equidistant nodes s/p (Eq. lagbas) */
/* ------------------------------------------------------------------ */
void or_lagrange_1d(int p, double x, double* val, double* der) {
  for (int m = 0; m <= p; ++m) {
    double xm = (double)m / p;
    double v = 1.0;
    for (int s = 0; s <= p; ++s) {
      if (s == m) continue;
      double xs = (double)s / p;
      v *= (x - xs) / (xm - xs);
    }
    /* derivative: sum over the removed factor r of the product of the others */
    double d = 0.0;
    for (int r = 0; r <= p; ++r) {
      if (r == m) continue;
      double xr = (double)r / p;
      double term = 1.0 / (xm - xr);
      for (int s = 0; s <= p; ++s) {
        if (s == m || s == r) continue;
        double xs = (double)s / p;
        term *= (x - xs) / (xm - xs);
      }
      d += term;
    }
    val[m] = v;
    der[m] = d;
  }
}

/* Tensor-product (Eq. lagbasmd) values and reference gradients of all
 * (p+1)^3 shape functions at the point xh; local node a = a0 + (p+1) a1 +
 * (p+1)^2 a2 (lexicographic, x fastest). */
static void tp_basis(int p, const double* xh, double* phi, double* dphi /* [nb][3] */) {
  double v[3][MAXP + 1], d[3][MAXP + 1];
  for (int k = 0; k < 3; ++k) or_lagrange_1d(p, xh[k], v[k], d[k]);
  int n1 = p + 1;
  for (int a2 = 0; a2 < n1; ++a2)
    for (int a1 = 0; a1 < n1; ++a1)
      for (int a0 = 0; a0 < n1; ++a0) {
        int a = a0 + n1 * a1 + n1 * n1 * a2;
        phi[a] = v[0][a0] * v[1][a1] * v[2][a2];
        dphi[3 * a + 0] = d[0][a0] * v[1][a1] * v[2][a2];
        dphi[3 * a + 1] = v[0][a0] * d[1][a1] * v[2][a2];
        dphi[3 * a + 2] = v[0][a0] * v[1][a1] * d[2][a2];
      }
}

/* Reference tables for one order and one tensor Gauss rule. */
typedef struct {
  int p, nq1d, nb, nq;
  double w[MAXNQ];
  double xq[MAXNQ][3];
  double phi[MAXNQ][MAXNB];
  double dphi[MAXNQ][MAXNB][3];
  double dN[MAXNQ][8][3]; /* trilinear geometry basis gradients */
  int nbp;                 /* pressure basis Q_{p-1} (Taylor-Hood), p >= 2 */
  double psi[MAXNQ][MAXNB];
} ref_tables;

static int make_tables(int p, int nq1d, ref_tables* T) {
  if (p < 1 || p > MAXP || nq1d < 1 || nq1d > MAXQ1D) return OR_ERR_ARG;
  double x1[MAXQ1D], w1[MAXQ1D];
  int rc = or_gauss_legendre(nq1d, x1, w1);
  if (rc) return rc;
  T->p = p;
  T->nq1d = nq1d;
  T->nb = (p + 1) * (p + 1) * (p + 1);
  T->nq = nq1d * nq1d * nq1d;
  for (int q2 = 0; q2 < nq1d; ++q2)
    for (int q1 = 0; q1 < nq1d; ++q1)
      for (int q0 = 0; q0 < nq1d; ++q0) {
        int q = q0 + nq1d * q1 + nq1d * nq1d * q2;
        T->xq[q][0] = x1[q0];
        T->xq[q][1] = x1[q1];
        T->xq[q][2] = x1[q2];
        T->w[q] = w1[q0] * w1[q1] * w1[q2];
        tp_basis(p, T->xq[q], T->phi[q], &T->dphi[q][0][0]);
        double gphi[8];
        tp_basis(1, T->xq[q], gphi, &T->dN[q][0][0]);
        if (p >= 2) {
          double dpsi[MAXNB][3];
          tp_basis(p - 1, T->xq[q], T->psi[q], &dpsi[0][0]);
        }
      }
  T->nbp = p >= 2 ? p * p * p : 0;
  return OR_OK;
}

/* Local DOFs of a cell: Poisson nb, elasticity 3 nb, Stokes (Taylor-Hood
 * Q_p velocity, Q_{p-1} pressure) 3 nb + p^3. */
static int local_size(int problem, const ref_tables* T) {
  if (problem == 1) return 3 * T->nb;
  if (problem == 2) return 3 * T->nb + T->nbp;
  return T->nb;
}

/* ------------------------------------------------------------------ */
/* Geometry at one quadrature point: J_kd = sum_v x_v[k] dN_v/dxhat_d,  */
/* its determinant and inverse (Eq. fematrix, Eq. shape_grad).          */
/* ------------------------------------------------------------------ */
static double det3(const double J[3][3]) {
  return J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1])
       - J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0])
       + J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]);
}

static void inv3(const double J[3][3], double det, double Ji[3][3]) {
  Ji[0][0] = (J[1][1] * J[2][2] - J[1][2] * J[2][1]) / det;
  Ji[0][1] = (J[0][2] * J[2][1] - J[0][1] * J[2][2]) / det;
  Ji[0][2] = (J[0][1] * J[1][2] - J[0][2] * J[1][1]) / det;
  Ji[1][0] = (J[1][2] * J[2][0] - J[1][0] * J[2][2]) / det;
  Ji[1][1] = (J[0][0] * J[2][2] - J[0][2] * J[2][0]) / det;
  Ji[1][2] = (J[0][2] * J[1][0] - J[0][0] * J[1][2]) / det;
  Ji[2][0] = (J[1][0] * J[2][1] - J[1][1] * J[2][0]) / det;
  Ji[2][1] = (J[0][1] * J[2][0] - J[0][0] * J[2][1]) / det;
  Ji[2][2] = (J[0][0] * J[1][1] - J[0][1] * J[1][0]) / det;
}

static void jacobian(const ref_tables* T, int q, const double* xv, double J[3][3]) {
  for (int k = 0; k < 3; ++k)
    for (int d = 0; d < 3; ++d) {
      double s = 0.0;
      for (int v = 0; v < 8; ++v) s += xv[3 * v + k] * T->dN[q][v][d];
      J[k][d] = s;
    }
}

/* Physical gradients of all shape functions at qp q: row vector
 * gradhat(phihat_a) times J^{-1} (Eq. shape_grad). Returns det J. */
static double physical_gradients(const ref_tables* T, int q, const double* xv, double g[][3]) {
  double J[3][3], Ji[3][3];
  jacobian(T, q, xv, J);
  double det = det3(J);
  if (!(det > 0.0)) return det;
  inv3(J, det, Ji);
  for (int a = 0; a < T->nb; ++a)
    for (int k = 0; k < 3; ++k) {
      double s = 0.0;
      for (int d = 0; d < 3; ++d) s += T->dphi[q][a][d] * Ji[d][k];
      g[a][k] = s;
    }
  return det;
}

/* ------------------------------------------------------------------ */
/* Cell matrix and vector                                               */
/* ------------------------------------------------------------------ */
/* Poisson: the (q, b, a) element loop with conductivity kappa; source f. */
static int cell_poisson(const ref_tables* T, const double* xv, double kappa, double f,
                        double* Ke, double* fe) {
  int nb = T->nb;
  double g[MAXNB][3];
  memset(Ke, 0, sizeof(double) * nb * nb);
  memset(fe, 0, sizeof(double) * nb);
  for (int q = 0; q < T->nq; ++q) {
    double det = physical_gradients(T, q, xv, g);
    if (!(det > 0.0)) return OR_ERR_NEG_JAC;
    double dJw = det * T->w[q];
    for (int b = 0; b < nb; ++b)
      for (int a = 0; a < nb; ++a) {
        double dot = g[a][0] * g[b][0] + g[a][1] * g[b][1] + g[a][2] * g[b][2];
        Ke[a * nb + b] += kappa * dot * dJw;
      }
    for (int a = 0; a < nb; ++a) fe[a] += f * T->phi[q][a] * dJw;
  }
  return OR_OK;
}

/* Elasticity: A^K_{(a,i),(b,j)} = int sigma(phi_b e_j) : eps(phi_a e_i), local
 * DOF index i*nb + a (component-major). Strain and stress are formed as full
 * 3x3 tensors and contracted, the plain definition. */
static int cell_elasticity(const ref_tables* T, const double* xv, double E, double nu,
                           const double* force, double* Ke, double* fe) {
  int nb = T->nb, nl = 3 * nb;
  double lambda = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu));
  double mu = E / (2.0 * (1.0 + nu));
  double g[MAXNB][3];
  memset(Ke, 0, sizeof(double) * nl * nl);
  memset(fe, 0, sizeof(double) * nl);
  for (int q = 0; q < T->nq; ++q) {
    double det = physical_gradients(T, q, xv, g);
    if (!(det > 0.0)) return OR_ERR_NEG_JAC;
    double dJw = det * T->w[q];
    for (int j = 0; j < 3; ++j)
      for (int b = 0; b < nb; ++b) {
        /* trial function u = phi_b e_j: grad u [k][l] = delta_kj d_l phi_b */
        double eu[3][3], su[3][3];
        for (int k = 0; k < 3; ++k)
          for (int l = 0; l < 3; ++l) {
            double gkl = (k == j) ? g[b][l] : 0.0;
            double glk = (l == j) ? g[b][k] : 0.0;
            eu[k][l] = 0.5 * (gkl + glk);
          }
        double tr = eu[0][0] + eu[1][1] + eu[2][2];
        for (int k = 0; k < 3; ++k)
          for (int l = 0; l < 3; ++l) su[k][l] = 2.0 * mu * eu[k][l] + (k == l ? lambda * tr : 0.0);
        for (int i = 0; i < 3; ++i)
          for (int a = 0; a < nb; ++a) {
            /* test function v = phi_a e_i */
            double s = 0.0;
            for (int k = 0; k < 3; ++k)
              for (int l = 0; l < 3; ++l) {
                double gkl = (k == i) ? g[a][l] : 0.0;
                double glk = (l == i) ? g[a][k] : 0.0;
                s += su[k][l] * 0.5 * (gkl + glk);
              }
            Ke[(i * nb + a) * nl + (j * nb + b)] += s * dJw;
          }
      }
    for (int i = 0; i < 3; ++i)
      for (int a = 0; a < nb; ++a) fe[i * nb + a] += force[i] * T->phi[q][a] * dJw;
  }
  return OR_OK;
}

/* Stokes (Example "Stokes problem"), Taylor-Hood: velocity u = phi_b e_j
 * (Q_p, local index j*nb + b), pressure psi_c (Q_{p-1}, local index 3nb + c).
 *   velocity-velocity  mu int eps(u) : eps(v)   (full 3x3 strain tensors)
 *   velocity-pressure  - int (div v) p
 *   pressure-velocity  - int q (div u)           (the symmetric reading)
 *   pressure-pressure  0
 * Right-hand side: int f . v on the velocity rows, 0 on the pressure rows. */
static int cell_stokes(const ref_tables* T, const double* xv, double mu, const double* force, double* Ke,
                       double* fe) {
  int nb = T->nb, nbp = T->nbp, nv = 3 * nb, nl = nv + nbp;
  if (nbp <= 0) return OR_ERR_ARG;
  double g[MAXNB][3];
  memset(Ke, 0, sizeof(double) * nl * nl);
  memset(fe, 0, sizeof(double) * nl);
  for (int q = 0; q < T->nq; ++q) {
    double det = physical_gradients(T, q, xv, g);
    if (!(det > 0.0)) return OR_ERR_NEG_JAC;
    double dJw = det * T->w[q];
    for (int j = 0; j < 3; ++j)
      for (int b = 0; b < nb; ++b) {
        double eu[3][3];
        for (int k = 0; k < 3; ++k)
          for (int l = 0; l < 3; ++l) eu[k][l] = 0.5 * (((k == j) ? g[b][l] : 0.0) + ((l == j) ? g[b][k] : 0.0));
        for (int i = 0; i < 3; ++i)
          for (int a = 0; a < nb; ++a) {
            double s = 0.0;
            for (int k = 0; k < 3; ++k)
              for (int l = 0; l < 3; ++l)
                s += eu[k][l] * 0.5 * (((k == i) ? g[a][l] : 0.0) + ((l == i) ? g[a][k] : 0.0));
            Ke[(i * nb + a) * nl + (j * nb + b)] += mu * s * dJw;
          }
        /* div(phi_b e_j) = d_j phi_b */
        for (int c = 0; c < nbp; ++c) {
          double bq = -T->psi[q][c] * g[b][j] * dJw;
          Ke[(j * nb + b) * nl + (nv + c)] += bq;
          Ke[(nv + c) * nl + (j * nb + b)] += bq;
        }
      }
    for (int i = 0; i < 3; ++i)
      for (int a = 0; a < nb; ++a) fe[i * nb + a] += force[i] * T->phi[q][a] * dJw;
  }
  return OR_OK;
}

static int cell_matrix_t(const ref_tables* T, int problem, const double* xv, double coef, double nu,
                         const double* force, double* Ke, double* fe) {
  if (problem == 0) return cell_poisson(T, xv, coef, force[0], Ke, fe);
  if (problem == 1) return cell_elasticity(T, xv, coef, nu, force, Ke, fe);
  if (problem == 2) return cell_stokes(T, xv, coef, force, Ke, fe);
  return OR_ERR_ARG;
}

int or_cell_matrix(int problem, int p, int nq1d, const double* xv, double coef, double nu,
                   const double* force, double* Ke, double* fe) {
  ref_tables* T = (ref_tables*)malloc(sizeof(ref_tables));
  if (!T) return OR_ERR_OOM;
  int rc = make_tables(p, nq1d, T);
  if (!rc) rc = cell_matrix_t(T, problem, xv, coef, nu, force, Ke, fe);
  free(T);
  return rc;
}

/* Smallest det J over the Gauss points of rule nq1d and over the 8 vertices. */
double or_min_det_jacobian(int nq1d, int64_t n_cells, const int32_t* cell_vertices, const double* coords) {
  ref_tables* T = (ref_tables*)malloc(sizeof(ref_tables));
  ref_tables* V = (ref_tables*)malloc(sizeof(ref_tables));
  if (!T || !V || make_tables(1, nq1d, T)) { free(T); free(V); return -1.0; }
  /* vertices: evaluate at the corners through a 2-point table whose points are moved to 0/1 */
  make_tables(1, 2, V);
  for (int q = 0; q < 8; ++q) {
    double xh[3] = {(double)(q & 1), (double)((q >> 1) & 1), (double)((q >> 2) & 1)};
    double phi[8];
    tp_basis(1, xh, phi, &V->dN[q][0][0]);
  }
  double mn = INFINITY;
  for (int64_t e = 0; e < n_cells; ++e) {
    double xv[24];
    for (int v = 0; v < 8; ++v)
      for (int k = 0; k < 3; ++k) xv[3 * v + k] = coords[3 * (int64_t)cell_vertices[8 * e + v] + k];
    double J[3][3];
    for (int q = 0; q < T->nq; ++q) { jacobian(T, q, xv, J); double d = det3(J); if (d < mn) mn = d; }
    for (int q = 0; q < 8; ++q) { jacobian(V, q, xv, J); double d = det3(J); if (d < mn) mn = d; }
  }
  free(T);
  free(V);
  return mn;
}

/* ------------------------------------------------------------------ */
/* Global DOF numbering (list_dofs)                                     */
/* ------------------------------------------------------------------ */
/* A node of a cell is owned by the n-face ("vef") whose extrusion bits are
 * the directions where 0 < alpha_d < p; nodes shared between cells are
 * matched by an orientation-free key: the corner vertices of the vef (global
 * ids, sorted) with the integer bilinear weights of the node with respect to
 * each corner. */
typedef struct {
  int32_t dim;
  int32_t g[4];
  int32_t w[4];
  int64_t rec; /* e * nb + a */
} nodekey;

static int cmp_key(const void* pa, const void* pb) {
  const nodekey* a = (const nodekey*)pa;
  const nodekey* b = (const nodekey*)pb;
  if (a->dim != b->dim) return a->dim < b->dim ? -1 : 1;
  for (int i = 0; i < 4; ++i) {
    if (a->g[i] != b->g[i]) return a->g[i] < b->g[i] ? -1 : 1;
    if (a->w[i] != b->w[i]) return a->w[i] < b->w[i] ? -1 : 1;
  }
  return 0;
}

static int same_node(const nodekey* a, const nodekey* b) {
  if (a->dim != b->dim) return 0;
  for (int i = 0; i < 4; ++i)
    if (a->g[i] != b->g[i] || a->w[i] != b->w[i]) return 0;
  return 1;
}

/* Reference node alpha -> (dim, extrusion bits, anchor bits). */
static void node_vef(int p, int a, int* dim, int* ext, int* anc, int al[3]) {
  int n1 = p + 1;
  al[0] = a % n1;
  al[1] = (a / n1) % n1;
  al[2] = a / (n1 * n1);
  *dim = 0; *ext = 0; *anc = 0;
  for (int d = 0; d < 3; ++d) {
    if (al[d] > 0 && al[d] < p) { *ext |= 1 << d; (*dim)++; }
    else if (al[d] == p) *anc |= 1 << d;
  }
}

/* Order of the local nodes in which list_dofs meets them: cell interior first,
 * then the vefs of the cell from the lowest to the highest dimension, within a
 * dimension by extrusion code then anchor code, and the nodes of one vef in
 * lexicographic order. */
static void traversal_order(int p, int* order) {
  int nb = (p + 1) * (p + 1) * (p + 1);
  int64_t keys[MAXNB];
  for (int a = 0; a < nb; ++a) {
    int dim, ext, anc, al[3];
    node_vef(p, a, &dim, &ext, &anc, al);
    int dkey = (dim == 3) ? 0 : dim + 1;
    keys[a] = (((int64_t)dkey * 8 + ext) * 8 + anc) * 4096 + a;
  }
  for (int a = 0; a < nb; ++a) order[a] = a;
  /* insertion sort on the keys (nb <= 64) */
  for (int i = 1; i < nb; ++i) {
    int x = order[i];
    int j = i - 1;
    while (j >= 0 && keys[order[j]] > keys[x]) { order[j + 1] = order[j]; --j; }
    order[j + 1] = x;
  }
}

static void make_key(int p, const int32_t* cv, int a, nodekey* k) {
  int dim, ext, anc, al[3];
  node_vef(p, a, &dim, &ext, &anc, al);
  k->dim = dim;
  for (int i = 0; i < 4; ++i) { k->g[i] = -1; k->w[i] = 0; }
  int nc = 1 << dim;
  int cnt = 0;
  for (int c = 0; c < 8 && cnt < nc; ++c) {
    /* corners of the vef: free bits only in extruded directions */
    int ok = 1;
    for (int d = 0; d < 3; ++d)
      if (!(ext >> d & 1) && ((c >> d & 1) != (anc >> d & 1))) ok = 0;
    if (!ok) continue;
    int w = 1;
    for (int d = 0; d < 3; ++d)
      if (ext >> d & 1) w *= (c >> d & 1) ? al[d] : (p - al[d]);
    k->g[cnt] = cv[c];
    k->w[cnt] = w;
    cnt++;
  }
  /* sort corners by global id */
  for (int i = 1; i < cnt; ++i) {
    int32_t gg = k->g[i], ww = k->w[i];
    int j = i - 1;
    while (j >= 0 && k->g[j] > gg) { k->g[j + 1] = k->g[j]; k->w[j + 1] = k->w[j]; --j; }
    k->g[j + 1] = gg;
    k->w[j + 1] = ww;
  }
}

/* Fills cell_dofs[n_cells][ncomp*nb] (local index i*nb + a) and returns the
 * number of global DOFs, or a negative error code. The ncomp components of a
 * node receive consecutive global ids. */
int64_t or_dof_numbering(int p, int ncomp, int64_t n_cells, const int32_t* cell_vertices, int32_t* cell_dofs) {
  if (p < 1 || p > MAXP || (ncomp != 1 && ncomp != 3)) return OR_ERR_ARG;
  int nb = (p + 1) * (p + 1) * (p + 1);
  int nint = (p - 1) * (p - 1) * (p - 1);
  int64_t nrec = n_cells * (int64_t)(nb - nint);
  nodekey* keys = (nodekey*)malloc(sizeof(nodekey) * (nrec > 0 ? nrec : 1));
  int64_t* node_of = (int64_t*)malloc(sizeof(int64_t) * (n_cells * nb > 0 ? n_cells * nb : 1));
  if (!keys || !node_of) { free(keys); free(node_of); return OR_ERR_OOM; }
  int64_t r = 0;
  for (int64_t e = 0; e < n_cells; ++e)
    for (int a = 0; a < nb; ++a) {
      int dim, ext, anc, al[3];
      node_vef(p, a, &dim, &ext, &anc, al);
      if (dim == 3) continue;
      make_key(p, cell_vertices + 8 * e, a, &keys[r]);
      keys[r].rec = e * nb + a;
      r++;
    }
  qsort(keys, (size_t)nrec, sizeof(nodekey), cmp_key);
  /* unique shared nodes: ids 0..nshared-1; cell-interior nodes get ids after */
  int64_t nshared = 0;
  for (int64_t i = 0; i < nrec; ++i) {
    if (i > 0 && !same_node(&keys[i], &keys[i - 1])) nshared++;
    node_of[keys[i].rec] = nshared;
  }
  if (nrec > 0) nshared++;
  free(keys);
  int64_t nnodes = nshared;
  for (int64_t e = 0; e < n_cells; ++e)
    for (int a = 0; a < nb; ++a) {
      int dim, ext, anc, al[3];
      node_vef(p, a, &dim, &ext, &anc, al);
      if (dim == 3) node_of[e * nb + a] = nnodes++;
    }
  int64_t* first = (int64_t*)malloc(sizeof(int64_t) * (nnodes > 0 ? nnodes : 1));
  if (!first) { free(node_of); return OR_ERR_OOM; }
  for (int64_t u = 0; u < nnodes; ++u) first[u] = -1;
  int order[MAXNB];
  traversal_order(p, order);
  int64_t next = 0;
  for (int64_t e = 0; e < n_cells; ++e) {
    for (int t = 0; t < nb; ++t) {
      int a = order[t];
      int64_t u = node_of[e * nb + a];
      if (first[u] < 0) { first[u] = next; next += ncomp; }
    }
    for (int a = 0; a < nb; ++a)
      for (int c = 0; c < ncomp; ++c)
        cell_dofs[e * (int64_t)ncomp * nb + c * nb + a] = (int32_t)(first[node_of[e * nb + a]] + c);
  }
  free(first);
  free(node_of);
  return next;
}

/* ------------------------------------------------------------------ */
/* Global assembly                                                      */
/* ------------------------------------------------------------------ */
static void cell_coords(const int32_t* cv, const double* coords, double* xv) {
  for (int v = 0; v < 8; ++v)
    for (int k = 0; k < 3; ++k) xv[3 * v + k] = coords[3 * (int64_t)cv[v] + k];
}

typedef struct {
  int64_t row;
  int64_t col;
  double val;
} coo_t;

static int cmp_coo(const void* pa, const void* pb) {
  const coo_t* a = (const coo_t*)pa;
  const coo_t* b = (const coo_t*)pb;
  if (a->row != b->row) return a->row < b->row ? -1 : 1;
  if (a->col != b->col) return a->col < b->col ? -1 : 1;
  return 0;
}

/* Assembles the full (unconstrained) matrix in CSR and the RHS.
 * Call with row_ptr == NULL to get the number of nonzeros only (the pattern
 * counts every pair of DOFs sharing a cell, also numerically zero ones).
 * Returns nnz (>= 0) or a negative error code. */
int64_t or_assemble_csr(int problem, int p, int nq1d, int64_t n_cells, const int32_t* cell_vertices,
                        const double* coords, const int32_t* cell_dofs, int64_t n_dofs,
                        const double* coef, double nu, const double* force,
                        int64_t* row_ptr, int32_t* col_idx, double* values, double* rhs) {
  ref_tables* T = (ref_tables*)malloc(sizeof(ref_tables));
  if (!T) return OR_ERR_OOM;
  int rc = make_tables(p, nq1d, T);
  if (rc) { free(T); return rc; }
  int nl = local_size(problem, T);
  int64_t ncoo = n_cells * (int64_t)nl * nl;
  coo_t* coo = (coo_t*)malloc(sizeof(coo_t) * (ncoo > 0 ? ncoo : 1));
  double* Ke = (double*)malloc(sizeof(double) * nl * nl);
  double* fe = (double*)malloc(sizeof(double) * nl);
  if (!coo || !Ke || !fe) { free(T); free(coo); free(Ke); free(fe); return OR_ERR_OOM; }
  if (rhs) memset(rhs, 0, sizeof(double) * n_dofs);
  int64_t t = 0;
  for (int64_t e = 0; e < n_cells; ++e) {
    double xv[24];
    cell_coords(cell_vertices + 8 * e, coords, xv);
    rc = cell_matrix_t(T, problem, xv, coef ? coef[e] : 1.0, nu, force, Ke, fe);
    if (rc) { free(T); free(coo); free(Ke); free(fe); return rc; }
    const int32_t* dofs = cell_dofs + e * nl;
    for (int a = 0; a < nl; ++a) {
      for (int b = 0; b < nl; ++b) {
        coo[t].row = dofs[a];
        coo[t].col = dofs[b];
        coo[t].val = Ke[a * nl + b];
        t++;
      }
      if (rhs) rhs[dofs[a]] += fe[a];
    }
  }
  qsort(coo, (size_t)ncoo, sizeof(coo_t), cmp_coo);
  /* compress: sum duplicates */
  int64_t nnz = 0;
  for (int64_t i = 0; i < ncoo; ++i) {
    if (i == 0 || coo[i].row != coo[i - 1].row || coo[i].col != coo[i - 1].col) {
      if (row_ptr) {
        col_idx[nnz] = (int32_t)coo[i].col;
        values[nnz] = coo[i].val;
      }
      nnz++;
    } else if (row_ptr) {
      values[nnz - 1] += coo[i].val;
    }
  }
  if (row_ptr) {
    for (int64_t r = 0; r <= n_dofs; ++r) row_ptr[r] = 0;
    int64_t k = 0;
    for (int64_t i = 0; i < ncoo; ++i)
      if (i == 0 || coo[i].row != coo[i - 1].row || coo[i].col != coo[i - 1].col) {
        row_ptr[coo[i].row + 1]++;
        k++;
      }
    for (int64_t r = 0; r < n_dofs; ++r) row_ptr[r + 1] += row_ptr[r];
  }
  free(T);
  free(coo);
  free(Ke);
  free(fe);
  return nnz;
}

/* Assembles only the requested rows (for large meshes, sampled parity).
 * out_ptr[n_req+1] gets the offsets of each row's (sorted) columns in
 * out_col/out_val, out_rhs[n_req] the RHS entries. Returns the total number
 * of entries; if it exceeds cap nothing is written past cap and the caller
 * must retry with a larger buffer. */
int64_t or_assemble_rows(int problem, int p, int nq1d, int64_t n_cells, const int32_t* cell_vertices,
                         const double* coords, const int32_t* cell_dofs, int64_t n_dofs,
                         const double* coef, double nu, const double* force,
                         int64_t n_req, const int64_t* rows, int64_t cap,
                         int64_t* out_ptr, int32_t* out_col, double* out_val, double* out_rhs) {
  ref_tables* T = (ref_tables*)malloc(sizeof(ref_tables));
  if (!T) return OR_ERR_OOM;
  int rc = make_tables(p, nq1d, T);
  if (rc) { free(T); return rc; }
  int nl = local_size(problem, T);
  /* DOF -> (cell, local) incidence, cells ascending, by counting sort */
  int64_t ninc = n_cells * nl;
  int64_t* ptr = (int64_t*)calloc((size_t)(n_dofs + 1), sizeof(int64_t));
  int64_t* inc = (int64_t*)malloc(sizeof(int64_t) * (ninc > 0 ? ninc : 1));
  double* Ke = (double*)malloc(sizeof(double) * nl * nl);
  double* fe = (double*)malloc(sizeof(double) * nl);
  coo_t* acc = (coo_t*)malloc(sizeof(coo_t) * 8 * nl);
  if (!ptr || !inc || !Ke || !fe || !acc) { free(T); free(ptr); free(inc); free(Ke); free(fe); free(acc); return OR_ERR_OOM; }
  for (int64_t i = 0; i < ninc; ++i) ptr[cell_dofs[i] + 1]++;
  for (int64_t r = 0; r < n_dofs; ++r) ptr[r + 1] += ptr[r];
  int64_t* fill = (int64_t*)malloc(sizeof(int64_t) * (n_dofs > 0 ? n_dofs : 1));
  if (!fill) { free(T); free(ptr); free(inc); free(Ke); free(fe); free(acc); return OR_ERR_OOM; }
  memcpy(fill, ptr, sizeof(int64_t) * n_dofs);
  for (int64_t i = 0; i < ninc; ++i) inc[fill[cell_dofs[i]]++] = i;
  free(fill);
  int64_t total = 0;
  for (int64_t q = 0; q < n_req; ++q) {
    int64_t r = rows[q];
    int64_t na = 0;
    double f = 0.0;
    for (int64_t s = ptr[r]; s < ptr[r + 1]; ++s) {
      int64_t e = inc[s] / nl;
      int li = (int)(inc[s] % nl);
      double xv[24];
      cell_coords(cell_vertices + 8 * e, coords, xv);
      rc = cell_matrix_t(T, problem, xv, coef ? coef[e] : 1.0, nu, force, Ke, fe);
      if (rc) { total = rc; goto done; }
      for (int b = 0; b < nl; ++b) {
        acc[na].row = r;
        acc[na].col = cell_dofs[e * nl + b];
        acc[na].val = Ke[li * nl + b];
        na++;
      }
      f += fe[li];
    }
    qsort(acc, (size_t)na, sizeof(coo_t), cmp_coo);
    out_ptr[q] = total;
    for (int64_t i = 0; i < na; ++i) {
      if (i > 0 && acc[i].col == acc[i - 1].col) {
        if (total - 1 < cap) out_val[total - 1] += acc[i].val;
      } else {
        if (total < cap) { out_col[total] = (int32_t)acc[i].col; out_val[total] = acc[i].val; }
        total++;
      }
    }
    out_rhs[q] = f;
  }
  out_ptr[n_req] = total;
done:
  free(T); free(ptr); free(inc); free(Ke); free(fe); free(acc);
  return total;
}

/* Per-cell compliance sensitivities g_K = u_K^T (A^K / coef_K) u_K, the
 * derivative of c = u^T A(coef) u with respect to coef_K for a fixed u, since
 * A is linear in the cell coefficients (Eq. assembly). */
int or_cell_energies(int problem, int p, int nq1d, int64_t n_cells, const int32_t* cell_vertices,
                     const double* coords, const int32_t* cell_dofs, double nu, const double* u, double* g) {
  ref_tables* T = (ref_tables*)malloc(sizeof(ref_tables));
  if (!T) return OR_ERR_OOM;
  int rc = make_tables(p, nq1d, T);
  if (rc) { free(T); return rc; }
  int nl = local_size(problem, T);
  double* Ke = (double*)malloc(sizeof(double) * nl * nl);
  double* fe = (double*)malloc(sizeof(double) * nl);
  double zero[3] = {0.0, 0.0, 0.0};
  if (!Ke || !fe) { free(T); free(Ke); free(fe); return OR_ERR_OOM; }
  for (int64_t e = 0; e < n_cells; ++e) {
    double xv[24];
    cell_coords(cell_vertices + 8 * e, coords, xv);
    rc = cell_matrix_t(T, problem, xv, 1.0, nu, zero, Ke, fe);
    if (rc) break;
    const int32_t* dofs = cell_dofs + e * nl;
    double s = 0.0;
    for (int a = 0; a < nl; ++a)
      for (int b = 0; b < nl; ++b) s += u[dofs[a]] * Ke[a * nl + b] * u[dofs[b]];
    g[e] = s;
  }
  free(T); free(Ke); free(fe);
  return rc;
}

/* ------------------------------------------------------------------ */
/* Interior penalty DG for the Poisson problem (Sect. "Non-conforming   */
/* methods", Eq. ip_dg_formulations, Eq. mean_and_jump_ops, Eq.         */
/* local_to_face_matrix). DOFs are cell-local: DOF a of cell K is       */
/* K*nb + a. Local face f = 2 d + s lies on xhat_d = s; its parameters  */
/* are the other two reference coordinates in increasing axis order.    */
/* ------------------------------------------------------------------ */
static void face_point(int f, double s, double t, double xh[3]) {
  int d = f / 2, d1 = d == 0 ? 1 : 0, d2 = d == 2 ? 1 : 2;
  xh[d] = (double)(f % 2);
  xh[d1] = s;
  xh[d2] = t;
}

static void map_point(const double* xv, const double xh[3], double x[3]) {
  double N[8], dN[8][3];
  tp_basis(1, xh, N, &dN[0][0]);
  for (int k = 0; k < 3; ++k) {
    x[k] = 0.0;
    for (int v = 0; v < 8; ++v) x[k] += N[v] * xv[3 * v + k];
  }
}

static void jacobian_at(const double* xv, const double xh[3], double J[3][3]) {
  double N[8], dN[8][3];
  tp_basis(1, xh, N, &dN[0][0]);
  for (int k = 0; k < 3; ++k)
    for (int d = 0; d < 3; ++d) {
      J[k][d] = 0.0;
      for (int v = 0; v < 8; ++v) J[k][d] += xv[3 * v + k] * dN[v][d];
    }
}

/* Reference point of the physical point x in the cell (Newton on the
 * trilinear map from the cell centre). */
static int inverse_map(const double* xv, const double x[3], double xh[3]) {
  xh[0] = xh[1] = xh[2] = 0.5;
  for (int it = 0; it < 100; ++it) {
    double y[3], J[3][3], Ji[3][3];
    map_point(xv, xh, y);
    jacobian_at(xv, xh, J);
    double det = det3(J);
    if (!(fabs(det) > 0.0)) return OR_ERR_NEG_JAC;
    inv3(J, det, Ji);
    double step = 0.0;
    for (int d = 0; d < 3; ++d) {
      double dx = 0.0;
      for (int k = 0; k < 3; ++k) dx += Ji[d][k] * (x[k] - y[k]);
      xh[d] += dx;
      step += fabs(dx);
    }
    if (step < 1e-15) return OR_OK;
  }
  return OR_OK;
}

/* Values and physical gradients of the nb shape functions at xh. */
static void basis_phys(int p, const double* xv, const double xh[3], double* phi, double g[][3]) {
  double dphi[MAXNB][3], J[3][3], Ji[3][3];
  tp_basis(p, xh, phi, &dphi[0][0]);
  jacobian_at(xv, xh, J);
  inv3(J, det3(J), Ji);
  int nb = (p + 1) * (p + 1) * (p + 1);
  for (int a = 0; a < nb; ++a)
    for (int k = 0; k < 3; ++k) {
      g[a][k] = 0.0;
      for (int d = 0; d < 3; ++d) g[a][k] += dphi[a][d] * Ji[d][k];
    }
}

/* The 4 corner vertices of local face f (reference corners with xhat_d = s). */
static void face_vertices(const int32_t* cv, int f, int32_t out[4]) {
  int d = f / 2, s = f % 2, n = 0;
  for (int v = 0; v < 8; ++v)
    if (((v >> d) & 1) == s) out[n++] = cv[v];
}

typedef struct {
  int32_t key[4];
  int64_t cell;
  int face;
} face_rec;

static int cmp_face(const void* pa, const void* pb) {
  const face_rec* a = (const face_rec*)pa;
  const face_rec* b = (const face_rec*)pb;
  for (int i = 0; i < 4; ++i)
    if (a->key[i] != b->key[i]) return a->key[i] < b->key[i] ? -1 : 1;
  if (a->cell != b->cell) return a->cell < b->cell ? -1 : 1;
  return 0;
}

static int cmp_i32(const void* pa, const void* pb) {
  int32_t a = *(const int32_t*)pa, b = *(const int32_t*)pb;
  return a < b ? -1 : (a > b ? 1 : 0);
}

/* Assembles the IP-DG system: the cell terms int grad u . grad v and int f v,
 * the interior facets (K+, the lower cell id, and K-) with the four blocks of
 * Eq. local_to_face_matrix (row: test function, column: trial function),
 * the boundary facets with the degenerate one-sided block, and on the
 * right-hand side the weak Dirichlet terms for u_D(x) = ud[0] + ud[1..3] . x.
 * The normal and the surface element come from the cross product of the face
 * tangents; the reference point of a facet point in K- is found by inverting
 * K-'s trilinear map. n_dofs = n_cells (p+1)^3. Call with row_ptr == NULL to
 * get nnz only. Returns nnz or a negative error code. */
int64_t or_dg_assemble(int p, int64_t n_cells, const int32_t* cell_vertices, const double* coords, double tau,
                       double gamma, double f, const double* ud, int64_t* row_ptr, int32_t* col_idx, double* values,
                       double* rhs) {
  ref_tables* T = (ref_tables*)malloc(sizeof(ref_tables));
  if (!T) return OR_ERR_OOM;
  int rc = make_tables(p, p + 1, T);
  if (rc) { free(T); return rc; }
  const int nb = T->nb, n1 = p + 1;
  double gx[MAXQ1D], gw[MAXQ1D];
  or_gauss_legendre(n1, gx, gw);
  face_rec* fr = (face_rec*)malloc(sizeof(face_rec) * (n_cells > 0 ? 6 * n_cells : 1));
  /* entries: nb^2 per cell, 4 nb^2 per interior and nb^2 per boundary facet;
   * 2 F_int + F_bnd = 6 n_cells and F_int <= 3 n_cells give at most 13 n_cells nb^2 */
  int64_t cap = n_cells * (int64_t)nb * nb * 13 + 1;
  coo_t* coo = (coo_t*)malloc(sizeof(coo_t) * cap);
  double* Ke = (double*)malloc(sizeof(double) * nb * nb);
  double* fe = (double*)malloc(sizeof(double) * nb);
  double* M = (double*)malloc(sizeof(double) * 4 * nb * nb);
  if (!fr || !coo || !Ke || !fe || !M) { free(T); free(fr); free(coo); free(Ke); free(fe); free(M); return OR_ERR_OOM; }
  const int64_t n_dofs = n_cells * nb;
  if (rhs) memset(rhs, 0, sizeof(double) * n_dofs);
  int64_t t = 0;
  for (int64_t e = 0; e < n_cells && !rc; ++e) {
    double xv[24];
    cell_coords(cell_vertices + 8 * e, coords, xv);
    rc = cell_poisson(T, xv, 1.0, f, Ke, fe);
    for (int a = 0; a < nb && !rc; ++a) {
      for (int b = 0; b < nb; ++b) {
        coo[t].row = e * nb + a; coo[t].col = e * nb + b; coo[t].val = Ke[a * nb + b]; t++;
      }
      if (rhs) rhs[e * nb + a] += fe[a];
    }
    for (int lf = 0; lf < 6; ++lf) {
      face_rec* r = &fr[6 * e + lf];
      face_vertices(cell_vertices + 8 * e, lf, r->key);
      qsort(r->key, 4, sizeof(int32_t), cmp_i32);
      r->cell = e;
      r->face = lf;
    }
  }
  if (!rc) qsort(fr, (size_t)(6 * n_cells), sizeof(face_rec), cmp_face);
  for (int64_t i = 0; i < 6 * n_cells && !rc; ++i) {
    const int interior = i + 1 < 6 * n_cells && memcmp(fr[i].key, fr[i + 1].key, sizeof(fr[i].key)) == 0;
    int64_t K[2] = {fr[i].cell, interior ? fr[i + 1].cell : -1};
    double xvp[24], xvm[24];
    cell_coords(cell_vertices + 8 * K[0], coords, xvp);
    if (interior) cell_coords(cell_vertices + 8 * K[1], coords, xvm);
    const int lf = fr[i].face, d = lf / 2, d1 = d == 0 ? 1 : 0, d2 = d == 2 ? 1 : 2;
    const double sgn = (d == 1 ? -1.0 : 1.0) * (lf % 2 ? 1.0 : -1.0);
    /* two passes: the facet area |F|, then the entries */
    double area = 0.0;
    const int ns = interior ? 2 : 1;
    memset(M, 0, sizeof(double) * 4 * nb * nb);
    for (int pass = 0; pass < 2; ++pass)
      for (int qs = 0; qs < n1; ++qs)
        for (int qt = 0; qt < n1; ++qt) {
          double xh[3], x[3], J[3][3];
          face_point(lf, gx[qs], gx[qt], xh);
          map_point(xvp, xh, x);
          jacobian_at(xvp, xh, J);
          double t1[3] = {J[0][d1], J[1][d1], J[2][d1]}, t2[3] = {J[0][d2], J[1][d2], J[2][d2]};
          double nd[3] = {t1[1] * t2[2] - t1[2] * t2[1], t1[2] * t2[0] - t1[0] * t2[2], t1[0] * t2[1] - t1[1] * t2[0]};
          double len = sqrt(nd[0] * nd[0] + nd[1] * nd[1] + nd[2] * nd[2]);
          double dS = len * gw[qs] * gw[qt], n[3] = {sgn * nd[0] / len, sgn * nd[1] / len, sgn * nd[2] / len};
          if (pass == 0) { area += dS; continue; }
          double phi[2][MAXNB], g[2][MAXNB][3], gn[2][MAXNB];
          basis_phys(p, xvp, xh, phi[0], g[0]);
          if (interior) {
            double xm[3];
            inverse_map(xvm, x, xm);
            basis_phys(p, xvm, xm, phi[1], g[1]);
          }
          for (int s = 0; s < ns; ++s)
            for (int a = 0; a < nb; ++a) gn[s][a] = g[s][a][0] * n[0] + g[s][a][1] * n[1] + g[s][a][2] * n[2];
          const double half = interior ? 0.5 : 1.0, pen = gamma / area;
          for (int sa = 0; sa < ns; ++sa)
            for (int sb = 0; sb < ns; ++sb) {
              const double ga = sa == 0 ? 1.0 : -1.0, gb = sb == 0 ? 1.0 : -1.0;
              double* Mb = M + (sa * 2 + sb) * nb * nb;
              for (int a = 0; a < nb; ++a)
                for (int b = 0; b < nb; ++b)
                  Mb[a * nb + b] += dS * (-ga * phi[sa][a] * half * gn[sb][b] - tau * gb * phi[sb][b] * half * gn[sa][a]
                                          + pen * ga * gb * phi[sa][a] * phi[sb][b]);
            }
          if (!interior && rhs) {
            double u = ud[0] + ud[1] * x[0] + ud[2] * x[1] + ud[3] * x[2];
            for (int a = 0; a < nb; ++a) rhs[K[0] * nb + a] += dS * (-tau * u * gn[0][a] + pen * u * phi[0][a]);
          }
        }
    for (int sa = 0; sa < ns; ++sa)
      for (int sb = 0; sb < ns; ++sb)
        for (int a = 0; a < nb; ++a)
          for (int b = 0; b < nb; ++b) {
            coo[t].row = K[sa] * nb + a; coo[t].col = K[sb] * nb + b; coo[t].val = M[(sa * 2 + sb) * nb * nb + a * nb + b]; t++;
          }
    if (interior) ++i;
  }
  int64_t nnz = 0;
  if (!rc) {
    qsort(coo, (size_t)t, sizeof(coo_t), cmp_coo);
    if (row_ptr) for (int64_t r = 0; r <= n_dofs; ++r) row_ptr[r] = 0;
    for (int64_t i = 0; i < t; ++i) {
      if (i == 0 || coo[i].row != coo[i - 1].row || coo[i].col != coo[i - 1].col) {
        if (row_ptr) { col_idx[nnz] = (int32_t)coo[i].col; values[nnz] = coo[i].val; row_ptr[coo[i].row + 1]++; }
        nnz++;
      } else if (row_ptr) {
        values[nnz - 1] += coo[i].val;
      }
    }
    if (row_ptr) for (int64_t r = 0; r < n_dofs; ++r) row_ptr[r + 1] += row_ptr[r];
  }
  free(T); free(fr); free(coo); free(Ke); free(fe); free(M);
  return rc ? rc : nnz;
}

// Host-side setup of an FE space (runs once, untimed): reference tables,
// global DOF numbering, CSR sparsity pattern and the cell-to-nonzero assembly
// permutation consumed by the scatter kernel.
#include <algorithm>
#include <exception>
#include <functional>
#include <cmath>
#include <cstring>
#include <thread>
#include <unordered_map>

#include "fe_internal.h"

namespace feasm {

// ---------------------------------------------------------------------------
// Gauss-Legendre rule with n points on [0,1] (paper, Sect. "Numerical
// integration": an n-point rule is exact up to degree 2n-1). Roots of P_n by
// Newton's method from Chebyshev-like initial guesses; weights from P_n'.
static void gauss_rule_01(int n, double* x, double* w) {
  for (int k = 0; k < n; ++k) {
    // k-th root counted from the left end of [-1,1]
    double t = -std::cos(M_PI * (4.0 * k + 3.0) / (4.0 * n + 2.0));
    double dp = 1.0;
    for (int iter = 0; iter < 64; ++iter) {
      double pm1 = 1.0, p = t;  // P_0, P_1
      for (int m = 2; m <= n; ++m) {
        double pn = ((2.0 * m - 1.0) * t * p - (m - 1.0) * pm1) / m;
        pm1 = p;
        p = pn;
      }
      if (n == 1) { p = t; pm1 = 1.0; }
      dp = n * (pm1 - t * p) / (1.0 - t * t);
      double step = p / dp;
      t -= step;
      if (std::fabs(step) <= 1e-17) break;
    }
    // recompute the derivative at the converged root
    double pm1 = 1.0, p = t;
    for (int m = 2; m <= n; ++m) {
      double pn = ((2.0 * m - 1.0) * t * p - (m - 1.0) * pm1) / m;
      pm1 = p;
      p = pn;
    }
    if (n == 1) pm1 = 1.0;
    dp = n * (pm1 - t * p) / (1.0 - t * t);
    x[k] = 0.5 * (1.0 + t);
    w[k] = 1.0 / ((1.0 - t * t) * dp * dp);  // (2 / ((1-t^2) P_n'^2)) / 2
  }
}

// Lagrange polynomials of order p on the nodes 0, 1/p, ..., 1 (Eq. lagbas):
// values and first derivatives at x, via barycentric weights.
static void lagrange_01(int p, double x, double* val, double* der) {
  double nodes[kMaxOrder + 1], bw[kMaxOrder + 1];
  for (int m = 0; m <= p; ++m) nodes[m] = double(m) / p;
  for (int m = 0; m <= p; ++m) {
    double d = 1.0;
    for (int s = 0; s <= p; ++s)
      if (s != m) d *= nodes[m] - nodes[s];
    bw[m] = 1.0 / d;
  }
  for (int m = 0; m <= p; ++m) {
    double prod = 1.0, dsum = 0.0;
    for (int s = 0; s <= p; ++s) {
      if (s == m) continue;
      // derivative of the running product: d(prod * (x - x_s)) = dsum*(x-x_s) + prod
      dsum = dsum * (x - nodes[s]) + prod;
      prod *= x - nodes[s];
    }
    val[m] = bw[m] * prod;
    der[m] = bw[m] * dsum;
  }
}

void gauss_rule(int n, double* x, double* w) { gauss_rule_01(n, x, w); }

void lagrange_1d_table(int p, int nq1d, double* val, double* der) {
  double g[kMaxQ1d], gw[kMaxQ1d];
  gauss_rule_01(nq1d, g, gw);
  for (int q = 0; q < nq1d; ++q) lagrange_01(p, g[q], val + q * (p + 1), der + q * (p + 1));
}

void build_ref_tables(int p, int nq1d, RefTables* t) {
  t->p = p;
  t->nq1d = nq1d;
  const int n1 = p + 1;
  t->nb = n1 * n1 * n1;
  t->nq = nq1d * nq1d * nq1d;
  double g[kMaxQ1d], gw[kMaxQ1d];
  gauss_rule_01(nq1d, g, gw);
  t->w.assign(t->nq, 0.0);
  t->xq.assign(3 * t->nq, 0.0);
  t->phi.assign(size_t(t->nq) * t->nb, 0.0);
  t->dphi.assign(size_t(t->nq) * t->nb * 3, 0.0);
  for (int q = 0; q < t->nq; ++q) {
    const int qi[3] = {q % nq1d, (q / nq1d) % nq1d, q / (nq1d * nq1d)};
    double lv[3][kMaxOrder + 1], ld[3][kMaxOrder + 1];
    t->w[q] = gw[qi[0]] * gw[qi[1]] * gw[qi[2]];
    for (int d = 0; d < 3; ++d) {
      t->xq[3 * q + d] = g[qi[d]];
      lagrange_01(p, g[qi[d]], lv[d], ld[d]);
    }
    for (int a = 0; a < t->nb; ++a) {
      const int ai[3] = {a % n1, (a / n1) % n1, a / (n1 * n1)};
      const double v0 = lv[0][ai[0]], v1 = lv[1][ai[1]], v2 = lv[2][ai[2]];
      t->phi[size_t(q) * t->nb + a] = v0 * v1 * v2;
      double* dp = &t->dphi[(size_t(q) * t->nb + a) * 3];
      dp[0] = ld[0][ai[0]] * v1 * v2;
      dp[1] = v0 * ld[1][ai[1]] * v2;
      dp[2] = v0 * v1 * ld[2][ai[2]];
    }
  }
}

// ---------------------------------------------------------------------------
// Global DOF numbering (paper, Sect. "Global DOF numbering generation",
// list_dofs): cells in order; in each cell first the DOFs of nodes interior to
// the cell, then the vefs (vertices, edges, faces; within a dimension by
// extrusion bits then anchor bits), each vef's nodes in lexicographic order.
// A node met before keeps the ids it got in its owner cell. Shared nodes are
// identified by the vef's corner vertices and the node's integer bilinear
// weights on them, which does not depend on how a cell orients the vef.

namespace {

struct NodeId {
  int32_t corner[4];
  int32_t weight[4];
  int8_t dim;
  bool operator==(const NodeId& o) const {
    return dim == o.dim && std::memcmp(corner, o.corner, sizeof(corner)) == 0 &&
           std::memcmp(weight, o.weight, sizeof(weight)) == 0;
  }
};

struct NodeIdHash {
  size_t operator()(const NodeId& k) const {
    uint64_t h = 1469598103934665603ull ^ uint64_t(k.dim);
    for (int i = 0; i < 4; ++i) {
      h = (h ^ uint64_t(uint32_t(k.corner[i]))) * 1099511628211ull;
      h = (h ^ uint64_t(uint32_t(k.weight[i]))) * 1099511628211ull;
    }
    return size_t(h ^ (h >> 29));
  }
};

struct LocalNode {
  int a;          // lexicographic index
  int dim;        // dimension of the owning vef (3 = cell interior)
  int ext, anc;   // extrusion and anchor bits of the owning vef
  int alpha[3];
};

std::vector<LocalNode> local_nodes_in_visit_order(int p) {
  const int n1 = p + 1;
  std::vector<LocalNode> v;
  for (int a = 0; a < n1 * n1 * n1; ++a) {
    LocalNode ln{};
    ln.a = a;
    ln.alpha[0] = a % n1;
    ln.alpha[1] = (a / n1) % n1;
    ln.alpha[2] = a / (n1 * n1);
    for (int d = 0; d < 3; ++d) {
      const int al = ln.alpha[d];
      if (al != 0 && al != p) { ln.ext |= 1 << d; ++ln.dim; }
      if (al == p) ln.anc |= 1 << d;
    }
    v.push_back(ln);
  }
  auto rank = [](const LocalNode& n) { return n.dim == 3 ? -1 : n.dim; };
  std::stable_sort(v.begin(), v.end(), [&](const LocalNode& x, const LocalNode& y) {
    if (rank(x) != rank(y)) return rank(x) < rank(y);
    if (x.ext != y.ext) return x.ext < y.ext;
    if (x.anc != y.anc) return x.anc < y.anc;
    return x.a < y.a;
  });
  return v;
}

NodeId node_identity(int p, const LocalNode& ln, const int32_t* cv) {
  NodeId id;
  std::memset(&id, 0, sizeof(id));
  for (int i = 0; i < 4; ++i) id.corner[i] = -1;
  id.dim = int8_t(ln.dim);
  int n = 0;
  // enumerate the 2^dim corners: free bits in the extruded directions
  for (int c = 0; c < 8; ++c) {
    if ((c & ~ln.ext & 7) != (ln.anc & ~ln.ext & 7)) continue;
    int wgt = 1;
    for (int d = 0; d < 3; ++d)
      if (ln.ext >> d & 1) wgt *= (c >> d & 1) ? ln.alpha[d] : p - ln.alpha[d];
    id.corner[n] = cv[c];
    id.weight[n] = wgt;
    ++n;
  }
  // canonical order: ascending vertex id
  for (int i = 0; i < n; ++i)
    for (int j = i + 1; j < n; ++j)
      if (id.corner[j] < id.corner[i]) {
        std::swap(id.corner[i], id.corner[j]);
        std::swap(id.weight[i], id.weight[j]);
      }
  return id;
}

}  // namespace

static int number_dofs(int p, int ncomp, int64_t n_cells, const int32_t* cv, std::vector<int32_t>* cell_dofs,
                       int64_t* n_dofs, std::string* err) {
  const int n1 = p + 1, nb = n1 * n1 * n1, nl = ncomp * nb;
  const std::vector<LocalNode> visit = local_nodes_in_visit_order(p);
  std::unordered_map<NodeId, int64_t, NodeIdHash> first_id;
  first_id.reserve(size_t(n_cells) * (p == 1 ? 1 : 8) + 16);
  cell_dofs->assign(size_t(n_cells) * nl, -1);
  int64_t next = 0;
  for (int64_t e = 0; e < n_cells; ++e) {
    const int32_t* c = cv + 8 * e;
    int32_t* out = cell_dofs->data() + size_t(e) * nl;
    for (const LocalNode& ln : visit) {
      int64_t base;
      if (ln.dim == 3) {
        base = next;
        next += ncomp;
      } else {
        auto ins = first_id.emplace(node_identity(p, ln, c), next);
        if (ins.second) next += ncomp;
        base = ins.first->second;
      }
      for (int k = 0; k < ncomp; ++k) out[k * nb + ln.a] = int32_t(base + k);
    }
    if (next > INT32_MAX) {
      *err = "more than 2^31-1 DOFs";
      return FE_ERR_UNSUPPORTED;
    }
  }
  *n_dofs = next;
  return FE_OK;
}

// ---------------------------------------------------------------------------
// Sparsity pattern and assembly permutation. Row r collects the cells around
// DOF r ("slots", ascending cell id). Every pair (slot s, local column m) is a
// contribution to nonzero (r, cell_dofs[e_s][m]); contributions are sorted by
// column and, within one nonzero, by slot, i.e. by ascending cell. The code of
// a contribution is (head << 15) | (s << 8) | m, where head marks the first
// contribution of each nonzero; the scatter kernel reads
// K^{e_s}[local row of r in e_s][m]. The codes of a row start on a 16-byte
// boundary (each row's block is padded to a multiple of 8 codes). The same
// blocks also hold, slot-major, the index within the row of the nonzero that
// each (slot, local column) contributes to ("pos", bit 15 set on the first
// contribution of each nonzero in slot order), for the slot-wise scatter.
static void parallel_for(int64_t n, int nthreads, const std::function<void(int, int64_t, int64_t)>& body);

int build_host_setup(int p, int problem, int64_t n_cells, int64_t n_vertices, const int32_t* cell_vertices,
                     HostSetup* hs, std::string* err) {
  const int ncomp = problem == FE_POISSON ? 1 : 3;
  const int nb = (p + 1) * (p + 1) * (p + 1), nbp = problem == FE_STOKES ? p * p * p : 0;
  const int nl = ncomp * nb + nbp;
  for (int64_t i = 0; i < 8 * n_cells; ++i)
    if (cell_vertices[i] < 0 || cell_vertices[i] >= n_vertices) {
      *err = "cell_vertices entry out of range";
      return FE_ERR_INVALID_ARG;
    }
  // a hexahedron has 8 distinct vertices (a repeated one would give a cell two
  // local DOFs with one global id, which the assembly maps do not allow)
  for (int64_t e = 0; e < n_cells; ++e) {
    const int32_t* v = cell_vertices + 8 * e;
    for (int a = 0; a < 8; ++a)
      for (int b = a + 1; b < 8; ++b)
        if (v[a] == v[b]) {
          *err = "cell " + std::to_string(e) + " repeats a vertex";
          return FE_ERR_INVALID_ARG;
        }
  }
  if (n_cells * nl > INT32_MAX) {
    *err = "n_cells * n_loc exceeds int32";
    return FE_ERR_UNSUPPORTED;
  }
  int64_t n_dofs = 0;
  int rc = number_dofs(p, ncomp, n_cells, cell_vertices, &hs->cell_dofs, &n_dofs, err);
  if (rc) return rc;
  hs->n_first = n_dofs;
  if (problem == FE_STOKES) {
    // Taylor-Hood: the pressure field (Q_{p-1}) numbered by list_dofs after all
    // velocity DOFs; cell DOFs are the velocity ones (3 nb), then the pressure ones
    std::vector<int32_t> cdp;
    int64_t np = 0;
    rc = number_dofs(p - 1, 1, n_cells, cell_vertices, &cdp, &np, err);
    if (rc) return rc;
    if (n_dofs + np > INT32_MAX) {
      *err = "more than 2^31-1 DOFs";
      return FE_ERR_UNSUPPORTED;
    }
    std::vector<int32_t> cd(size_t(n_cells) * nl);
    for (int64_t e = 0; e < n_cells; ++e) {
      std::copy(hs->cell_dofs.begin() + e * ncomp * nb, hs->cell_dofs.begin() + (e + 1) * ncomp * nb,
                cd.begin() + e * nl);
      for (int c = 0; c < nbp; ++c) cd[e * nl + ncomp * nb + c] = int32_t(n_dofs + cdp[e * nbp + c]);
    }
    hs->cell_dofs.swap(cd);
    n_dofs += np;
  }
  return build_pattern(nl, nb, problem == FE_ELASTICITY ? 3 : 1, n_cells, hs->cell_dofs.data(), nullptr, n_dofs,
                       hs, err);
}

int build_pattern(int nl, int nb, int ncomp, int64_t n_cells, const int32_t* cell_dofs, const int32_t* label,
                  int64_t n_rows, HostSetup* hs, std::string* err) {
  // row of a global DOF: itself, or its label (negative = fixed, no row or column)
  auto row_of = [label](int32_t d) -> int32_t { return label ? label[d] : d; };
  hs->n_dofs = n_rows;
  const int64_t nd = n_rows;
  const int64_t ninc = n_cells * nl;
  // slots by counting sort (cell-major scan keeps cells ascending per row)
  hs->slot_ptr.assign(nd + 1, 0);
  for (int64_t i = 0; i < ninc; ++i) {
    const int32_t r = row_of(cell_dofs[i]);
    if (r >= 0) hs->slot_ptr[r + 1]++;
  }
  int max_slots = 0;
  for (int64_t r = 0; r < nd; ++r) max_slots = std::max<int64_t>(max_slots, hs->slot_ptr[r + 1]);
  if (max_slots * nl > 32767) {
    *err = "a row's contributions exceed 16-bit positions";
    return FE_ERR_UNSUPPORTED;
  }
  if (max_slots > kMaxSlots) {
    *err = "more than 127 cells around one DOF";
    return FE_ERR_UNSUPPORTED;
  }
  hs->max_slots = max_slots;
  for (int64_t r = 0; r < nd; ++r) hs->slot_ptr[r + 1] += hs->slot_ptr[r];
  hs->slots.assign(hs->slot_ptr[nd], 0);
  {
    std::vector<int64_t> fill(hs->slot_ptr.begin(), hs->slot_ptr.end() - 1);
    for (int64_t i = 0; i < ninc; ++i) {
      const int32_t r = row_of(cell_dofs[i]);
      if (r >= 0) hs->slots[fill[r]++] = int32_t(i);
    }
  }
  const int nthreads = std::max(1u, std::min(64u, std::thread::hardware_concurrency()));
  // pass 1: nonzeros per row (stamp arrays per thread)
  std::vector<int64_t> row_nnz(nd, 0);
  parallel_for(nd, nthreads, [&](int, int64_t r0, int64_t r1) {
    std::vector<int32_t> stamp(nd, -1);
    for (int64_t r = r0; r < r1; ++r) {
      int64_t k = 0;
      for (int64_t s = hs->slot_ptr[r]; s < hs->slot_ptr[r + 1]; ++s) {
        const int64_t e = hs->slots[s] / nl;
        const int32_t* dofs = cell_dofs + e * nl;
        for (int m = 0; m < nl; ++m) {
          const int32_t c = row_of(dofs[m]);
          if (c >= 0 && stamp[c] != int32_t(r)) { stamp[c] = int32_t(r); ++k; }
        }
      }
      row_nnz[r] = k;
    }
  });
  hs->row_ptr.assign(nd + 1, 0);
  hs->code_ptr.assign(nd + 1, 0);
  for (int64_t r = 0; r < nd; ++r) {
    hs->row_ptr[r + 1] = hs->row_ptr[r] + row_nnz[r];
    hs->code_ptr[r + 1] = hs->code_ptr[r] + (((hs->slot_ptr[r + 1] - hs->slot_ptr[r]) * nl + 7) & ~int64_t(7));
  }
  hs->nnz = hs->row_ptr[nd];
  hs->max_row_nnz = 0;
  for (int64_t r = 0; r < nd; ++r) hs->max_row_nnz = std::max(hs->max_row_nnz, row_nnz[r]);
  hs->n_codes = hs->code_ptr[nd];
  hs->n_contrib = hs->slot_ptr[nd] * nl;
  if (hs->nnz > (int64_t(1) << 40)) {
    *err = "too many nonzeros";
    return FE_ERR_UNSUPPORTED;
  }
  // Contributions of fixed columns (label only) are left out of the codes and
  // sent, in the slot-major positions, to the lane's private dummy accumulator
  // of the slot-wise scatter: entry acc_stride + (m mod 32) of the row.
  const int64_t acc_stride = (hs->max_row_nnz + 3) & ~int64_t(3);
  hs->pos_ok = acc_stride + 32 <= 0x7fff;
  hs->col.assign(hs->nnz, 0);
  hs->cnt.assign(hs->nnz, 0);
  hs->codes.assign(hs->n_codes, 0);
  if (label) hs->ncode.assign(nd, 0); else hs->ncode.clear();
  // 64 entries of padding: the scatter's lanes read whole 32-wide chunks of a
  // cell row's positions, past the end of the last row's block
  hs->pos.assign(hs->n_codes + 64, 0);
  // pass 2: sorted contributions per row
  parallel_for(nd, nthreads, [&](int, int64_t r0, int64_t r1) {
    std::vector<uint64_t> keys;
    keys.reserve(size_t(max_slots) * nl);
    for (int64_t r = r0; r < r1; ++r) {
      keys.clear();
      const int64_t s0 = hs->slot_ptr[r], ns = hs->slot_ptr[r + 1] - s0;
      for (int64_t s = 0; s < ns; ++s) {
        const int64_t e = hs->slots[s0 + s] / nl;
        const int32_t* dofs = cell_dofs + e * nl;
        for (int m = 0; m < nl; ++m) {
          const int32_t c = row_of(dofs[m]);
          if (c >= 0)
            keys.push_back((uint64_t(uint32_t(c)) << 16) | (uint64_t(s) << 8) | uint64_t(m));
          else if (hs->pos_ok)
            hs->pos[hs->code_ptr[r] + s * nl + m] = uint16_t(acc_stride + (m & 31));
        }
      }
      std::sort(keys.begin(), keys.end());
      if (label) hs->ncode[r] = int32_t(keys.size());
      int64_t k = hs->row_ptr[r] - 1;
      int64_t c = hs->code_ptr[r];
      int64_t prev = -1;
      for (uint64_t key : keys) {
        const int64_t col = int64_t(key >> 16);
        uint16_t head = 0;
        if (col != prev) {
          ++k;
          hs->col[k] = int32_t(col);
          prev = col;
          head = 0x8000;
        }
        hs->cnt[k]++;
        hs->codes[c++] = uint16_t((key & 0xffff) | head);
        const int64_t s_m = int64_t((key >> 8) & 0xff) * nl + int64_t(key & 0xff);
        hs->pos[hs->code_ptr[r] + s_m] = uint16_t((k - hs->row_ptr[r]) | (head ? 0x8000 : 0));
      }
    }
  });
  // The ncomp rows of one node (consecutive rows, components in order) lie in
  // the same cells, at local rows i * nb + a, and so share their column
  // pattern and positions; the scatter then treats them together.
  hs->node_rows = false;
  if (ncomp > 1 && nd % ncomp == 0) {
    bool ok = true;
    for (int64_t n = 0; n < nd / ncomp && ok; ++n) {
      const int64_t r0 = n * ncomp, ns = hs->slot_ptr[r0 + 1] - hs->slot_ptr[r0];
      const int64_t len = hs->row_ptr[r0 + 1] - hs->row_ptr[r0];
      for (int i = 1; i < ncomp && ok; ++i) {
        const int64_t r = r0 + i;
        ok = hs->slot_ptr[r + 1] - hs->slot_ptr[r] == ns && hs->row_ptr[r + 1] - hs->row_ptr[r] == len;
        for (int64_t t = 0; t < ns && ok; ++t)
          ok = hs->slots[hs->slot_ptr[r] + t] == hs->slots[hs->slot_ptr[r0] + t] + i * nb;
      }
    }
    hs->node_rows = ok;
  }
  return FE_OK;
}

// Runs body(t, a, b) over [0, n) in chunks on up to nthreads threads. An
// exception thrown by a chunk (std::bad_alloc when host memory runs out) is
// carried to the calling thread and rethrown there after every thread has
// joined, so that the entry point's handler turns it into a status code; a
// chunk whose thread cannot be started runs on the calling thread.
static void parallel_for(int64_t n, int nthreads, const std::function<void(int, int64_t, int64_t)>& body) {
  if (n <= 0) return;
  nthreads = int(std::max<int64_t>(1, std::min<int64_t>(nthreads, n / 1024 + 1)));
  const int64_t chunk = (n + nthreads - 1) / nthreads;
  std::vector<std::exception_ptr> errors(static_cast<size_t>(nthreads));
  auto run = [&](int t, int64_t a, int64_t b) {
    try {
      body(t, a, b);
    } catch (...) {
      errors[size_t(t)] = std::current_exception();
    }
  };
  std::vector<std::thread> th;
  for (int t = 0; t < nthreads; ++t) {
    const int64_t a = t * chunk, b = std::min(n, a + chunk);
    if (a >= b) break;
    try {
      th.emplace_back(run, t, a, b);
    } catch (...) {
      run(t, a, b);
    }
  }
  for (auto& x : th) x.join();
  for (auto& e : errors)
    if (e) std::rethrow_exception(e);
}

}  // namespace feasm

// ---------------------------------------------------------------------------
// Cell order for memory locality: cells sorted by the Morton (Z-order) code of
// their vertex centroids, quantised to 21 bits per axis over the bounding box
// of the centroids; equal codes keep the input order.

namespace {

// The 21 low bits of v spread to every third bit of a 63-bit word.
uint64_t spread3(uint64_t v) {
  v &= 0x1fffffull;
  v = (v | (v << 32)) & 0x1f00000000ffffull;
  v = (v | (v << 16)) & 0x1f0000ff0000ffull;
  v = (v | (v << 8)) & 0x100f00f00f00f00full;
  v = (v | (v << 4)) & 0x10c30c30c30c30c3ull;
  v = (v | (v << 2)) & 0x1249249249249249ull;
  return v;
}

}  // namespace

static int locality_order(const fe_mesh_desc* mesh, int64_t* order) {
  if (!mesh || mesh->n_cells < 0 || mesh->n_vertices < 0)
    return feasm::set_error(FE_ERR_INVALID_ARG, "invalid mesh descriptor");
  const int64_t nc = mesh->n_cells, nv = mesh->n_vertices;
  if (nc == 0) return FE_OK;
  if (!order || !mesh->cell_vertices || !mesh->coords)
    return feasm::set_error(FE_ERR_INVALID_ARG, "NULL argument");
  std::vector<double> cen(size_t(nc) * 3);
  double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
  for (int64_t e = 0; e < nc; ++e) {
    double c[3] = {0.0, 0.0, 0.0};
    for (int v = 0; v < 8; ++v) {
      const int32_t id = mesh->cell_vertices[e * 8 + v];
      if (id < 0 || id >= nv) return feasm::set_error(FE_ERR_INVALID_ARG, "cell_vertices entry out of range");
      for (int k = 0; k < 3; ++k) c[k] += mesh->coords[int64_t(id) * 3 + k];
    }
    for (int k = 0; k < 3; ++k) {
      c[k] *= 0.125;
      if (!std::isfinite(c[k])) return feasm::set_error(FE_ERR_INVALID_ARG, "non-finite vertex coordinate");
      cen[size_t(e) * 3 + k] = c[k];
      lo[k] = std::min(lo[k], c[k]);
      hi[k] = std::max(hi[k], c[k]);
    }
  }
  const double top = double((1 << 21) - 1);
  std::vector<std::pair<uint64_t, int64_t>> key(static_cast<size_t>(nc));
  for (int64_t e = 0; e < nc; ++e) {
    uint64_t code = 0;
    for (int k = 0; k < 3; ++k) {
      const double span = hi[k] - lo[k];
      const double t = span > 0.0 ? (cen[size_t(e) * 3 + k] - lo[k]) / span : 0.0;
      const uint64_t q = uint64_t(std::min(top, std::max(0.0, std::floor(t * top))));
      code |= spread3(q) << k;
    }
    key[size_t(e)] = {code, e};
  }
  std::sort(key.begin(), key.end());
  for (int64_t i = 0; i < nc; ++i) order[i] = key[size_t(i)].second;
  return FE_OK;
}

int fe_mesh_locality_order(const fe_mesh_desc* mesh, int64_t* order) {
  return feasm::no_throw("fe_mesh_locality_order", [&] { return locality_order(mesh, order); });
}

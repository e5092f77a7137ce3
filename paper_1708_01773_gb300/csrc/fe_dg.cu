// Interior penalty DG for the Poisson problem (paper, Sect. "Non-conforming
// methods", Eq. ip_dg_formulations, Eq. mean_and_jump_ops, Eq.
// local_to_face_matrix): discontinuous Q_p, cell-local DOFs K*nb + a.
//
// GB300 form: the cell integrals come from the Poisson cell kernels of an
// internal fe_space of the same order (FP64 or FP32 form); the facet
// integrals from k_dg_facets (one block per facet: its four nb x nb
// blocks, or one for a boundary facet, through small products over the face
// nodes, where the shape functions do not vanish; FP64 geometry, products in
// FP64 for the FP64 form and in FP32 for the FP32 forms); k_dg_rows then writes each cell's
// block row of the CSR matrix in one pass, the diagonal block being the cell
// matrix plus the cell's six facet diagonal blocks in face order, the others
// copies of facet off-diagonal blocks (fixed order: deterministic).
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <cstring>
#include <map>
#include <new>
#include <string>
#include <type_traits>
#include <vector>

#include "fe_device.cuh"
#include "fe_launch.h"

namespace feasm {
namespace dg {

constexpr int kSelf = 6;  // block slot code of the cell itself (0..5: the neighbour through that face)

}  // namespace dg
}  // namespace feasm

struct fe_dg {
  fe_space* s = nullptr;     // Poisson space of the same order: cell integrals, geometry, tables
  int p = 0, nb = 0;
  int64_t n_cells = 0, n_dofs = 0, nnz = 0;
  bool host_only = false;
  // interior facets: cells K+ < K-, their local faces, and for each corner (s, t)
  // of K+'s face (s, t in {0,1}, corner index s + 2t) the local vertex of K- there
  std::vector<int32_t> fplus, fminus;
  std::vector<uint8_t> fpf, fmf, fcorner;  // fcorner [n_int][4]
  std::vector<int32_t> bcell;
  std::vector<uint8_t> bface;
  // per cell: the code of each local face (interior facet i on side s: 2 i + s;
  // boundary facet j: -1 - j) and the block slots of its row in column order
  std::vector<int32_t> face_code;  // [cells][6]
  std::vector<uint8_t> slots;      // [cells][7]: face through which the neighbour is reached, or kSelf
  std::vector<uint8_t> nslot;      // [cells]
  std::vector<int64_t> row_ptr;
  std::vector<int32_t> col;
  // device
  int32_t* d_fplus = nullptr;
  int32_t* d_fminus = nullptr;
  uint8_t* d_fpf = nullptr;
  uint8_t* d_fmf = nullptr;
  uint8_t* d_fcorner = nullptr;
  int32_t* d_bcell = nullptr;
  uint8_t* d_bface = nullptr;
  int32_t* d_face_code = nullptr;
  uint8_t* d_slots = nullptr;
  uint8_t* d_nslot = nullptr;
  int64_t* d_row_ptr = nullptr;
  int32_t* d_col = nullptr;
  double* d_ones = nullptr;    // unit coefficients of the cell integrals
  double* d_fblk = nullptr;    // interior facet blocks [n_int][2][2][nb][nb]
  double* d_bblk = nullptr;    // boundary facet blocks [n_bnd][nb][nb]
  double* d_gx = nullptr;      // face Gauss rule on [0,1], p+1 points
  double* d_gw = nullptr;
};

namespace {

// local vertex of the corner (s, t) of local face f: xhat_d = f % 2, s along
// the lower and t along the higher of the two other axes
int face_corner_vertex(int f, int s, int t) {
  const int d = f / 2, d1 = d == 0 ? 1 : 0, d2 = d == 2 ? 1 : 2;
  return ((f % 2) << d) | (s << d1) | (t << d2);
}

int setup_dg(fe_dg* g, const fe_mesh_desc* mesh, std::string* err) {
  const int64_t nc = mesh->n_cells;
  const int nb = g->nb;
  g->face_code.assign(size_t(nc) * 6, 0);
  std::map<std::array<int32_t, 4>, std::pair<int32_t, int>> open;  // sorted face key -> (cell, face)
  for (int64_t e = 0; e < nc; ++e) {
    const int32_t* cv = mesh->cell_vertices + 8 * e;
    for (int f = 0; f < 6; ++f) {
      std::array<int32_t, 4> key;
      for (int c = 0; c < 4; ++c) key[c] = cv[face_corner_vertex(f, c & 1, c >> 1)];
      std::sort(key.begin(), key.end());
      auto it = open.find(key);
      if (it == open.end()) {
        open.emplace(key, std::make_pair(int32_t(e), f));
        continue;
      }
      // second cell on this face: an interior facet, K+ = the earlier (lower) cell
      const int32_t kp = it->second.first;
      const int fp = it->second.second;
      open.erase(it);
      const int32_t i = int32_t(g->fplus.size());
      g->fplus.push_back(kp);
      g->fminus.push_back(int32_t(e));
      g->fpf.push_back(uint8_t(fp));
      g->fmf.push_back(uint8_t(f));
      const int32_t* cvp = mesh->cell_vertices + 8 * int64_t(kp);
      for (int c = 0; c < 4; ++c) {
        const int32_t v = cvp[face_corner_vertex(fp, c & 1, c >> 1)];
        int lv = -1;
        for (int w = 0; w < 8; ++w)
          if (cv[w] == v) lv = w;
        if (lv < 0) {
          *err = "facet vertices do not match";
          return FE_ERR_INVALID_ARG;
        }
        g->fcorner.push_back(uint8_t(lv));
      }
      g->face_code[size_t(kp) * 6 + fp] = 2 * i;
      g->face_code[size_t(e) * 6 + f] = 2 * i + 1;
    }
  }
  // what stays open is on the boundary (ascending cell, face)
  std::vector<std::pair<int32_t, int>> bnd;
  for (auto& kv : open) bnd.push_back(kv.second);
  std::sort(bnd.begin(), bnd.end());
  for (auto& b : bnd) {
    const int32_t j = int32_t(g->bcell.size());
    g->bcell.push_back(b.first);
    g->bface.push_back(uint8_t(b.second));
    g->face_code[size_t(b.first) * 6 + b.second] = -1 - j;
  }
  // block slots of each cell's rows (cells ascending) and the CSR pattern
  g->slots.assign(size_t(nc) * 7, 0);
  g->nslot.assign(nc, 0);
  g->row_ptr.assign(size_t(nc) * nb + 1, 0);
  for (int64_t e = 0; e < nc; ++e) {
    std::vector<std::pair<int32_t, int>> blk{{int32_t(e), feasm::dg::kSelf}};
    for (int f = 0; f < 6; ++f) {
      const int32_t code = g->face_code[size_t(e) * 6 + f];
      if (code < 0) continue;
      const int32_t i = code >> 1;
      blk.push_back({(code & 1) ? g->fplus[i] : g->fminus[i], f});
    }
    std::sort(blk.begin(), blk.end());
    g->nslot[e] = uint8_t(blk.size());
    for (size_t j = 0; j < blk.size(); ++j) g->slots[size_t(e) * 7 + j] = uint8_t(blk[j].second);
    for (int a = 0; a < nb; ++a)
      g->row_ptr[size_t(e) * nb + a + 1] = int64_t(blk.size()) * nb;
    for (int a = 0; a < nb; ++a)
      for (auto& b : blk)
        for (int c = 0; c < nb; ++c) g->col.push_back(int32_t(int64_t(b.first) * nb + c));
  }
  for (size_t r = 0; r + 1 < g->row_ptr.size(); ++r) g->row_ptr[r + 1] += g->row_ptr[r];
  g->nnz = g->row_ptr.back();
  if (g->nnz > INT32_MAX * int64_t(8)) {
    *err = "too many nonzeros";
    return FE_ERR_UNSUPPORTED;
  }
  return FE_OK;
}

}  // namespace

namespace feasm {
namespace dg {

struct FacetParams {
  int64_t n_int, n_bnd;
  const double* xv;  // [cells][8][3]
  const int32_t* fplus;
  const int32_t* fminus;
  const uint8_t* fpf;
  const uint8_t* fmf;
  const uint8_t* fcorner;
  const int32_t* bcell;
  const uint8_t* bface;
  const double* gx;  // face Gauss points [n1] on [0,1]
  const double* gw;
  double tau, gamma;
  void* fblk;  // [n_int][4][nb][nb], double (FP64 form) or float
  void* bblk;  // [n_bnd][nb][nb]
  int* err;
};

// 1D Lagrange polynomials on the nodes m/P and their derivatives at x.
template <int P>
__device__ __forceinline__ void lagrange(double x, double* v, double* d) {
#pragma unroll
  for (int m = 0; m <= P; ++m) {
    double val = 1.0, der = 0.0;
#pragma unroll
    for (int s = 0; s <= P; ++s) {
      if (s == m) continue;
      const double den = double(m - s) / P;
      der = der * ((x - double(s) / P) / den) + val / den;
      val *= (x - double(s) / P) / den;
    }
    v[m] = val;
    d[m] = der;
  }
}

// Shared memory of k_dg_facets for order P: the products' operands and
// results in TB (FP64 form: double; FP32 forms: float), the rest double.
template <int P, typename TB>
struct FacetLayout {
  static constexpr int N1 = P + 1, NB = N1 * N1 * N1, NQF = N1 * N1, NBF = N1 * N1;
  static constexpr size_t S = sizeof(TB);
  static constexpr size_t GN = 0;                                        // [2][NQF][NB]   grad phi . n
  static constexpr size_t PF = GN + size_t(2) * NQF * NB * S;            // [2][NQF][NBF]  dS phi (face nodes)
  static constexpr size_t FF = PF + size_t(2) * NQF * NBF * S;           // [2][NQF][NBF]  phi (face nodes)
  static constexpr size_t X1 = FF + size_t(2) * NQF * NBF * S;           // [4][NBF][NB]
  static constexpr size_t YY = X1 + size_t(4) * NBF * NB * S;            // [4][NBF][NBF]
  static constexpr size_t NRM = (YY + size_t(4) * NBF * NBF * S + 15) & ~size_t(15);  // [NQF][3]
  static constexpr size_t DS = NRM + size_t(NQF) * 3 * 8;                // [NQF]
  static constexpr size_t CN = DS + size_t(NQF) * 8 + 8;                 // [2][NQF][3]    cof^T n / det
  static constexpr size_t VD = CN + size_t(2) * NQF * 3 * 8;             // [2][NQF][2][3][N1] Lagrange values, derivatives
  static constexpr size_t COF0 = VD + size_t(2) * NQF * 6 * N1 * 8;      // [NQF][10] side 0: cofactors, det
  static constexpr size_t CIDX = COF0 + size_t(NQF) * 10 * 8;            // int [2][NB] compact face index or -1
  static constexpr size_t BYTES = CIDX + size_t(2) * NB * sizeof(int);
};

// One block per facet (interior facets first, then boundary facets).
//   1. per quadrature point of side 0: the physical normal and surface element
//      from cof(J+) nhat = det J+ J+^{-T} nhat; the facet area |F|;
//   2. per (side, point): the reference point (side 1: the bilinear blend of
//      the reference corners that carry K+'s face corners, with the coordinate
//      normal to K-'s face set exactly), FP64 geometry, the normal derivatives
//      of all shape functions and the values of the (p+1)^2 face nodes (the
//      other shape functions vanish on the face);
//   3. the products X_{sa,sb} = sum_q dS phi^{sa}_{a'} (grad phi^{sb}_b . n)
//      (a' a face node of side sa) and Y_{sa,sb} = sum_q dS phi^{sa}_{a'} phi^{sb}_{b'};
//   4. block (sa, sb), row a, column b:
//      -s_a/2 X_{sa,sb}[a'][b] - tau s_b/2 X_{sb,sa}[b'][a] + gamma/|F| s_a s_b Y_{sa,sb}[a'][b']
//      (terms whose face node is missing are zero; boundary facets: one side,
//      s = 1 and the factor 1/2 dropped), Eq. local_to_face_matrix.
// FP32 forms (TB = float): geometry, normals and shape data in FP64, rounded
// to FP32 on the integer bits for steps 3 and 4, blocks stored in FP32.
template <int P, typename TB>
__global__ void __launch_bounds__(128) k_dg_facets(FacetParams fp) {
  using L = FacetLayout<P, TB>;
  constexpr bool F32 = std::is_same<TB, float>::value;
  auto cvt = [](double x) -> TB {
    if constexpr (F32) return d2f_rn(x); else return x;
  };
  constexpr int N1 = L::N1, NB = L::NB, NQF = L::NQF, NBF = L::NBF;
  extern __shared__ __align__(16) unsigned char sm[];
  TB* gn = reinterpret_cast<TB*>(sm + L::GN);
  TB* pf = reinterpret_cast<TB*>(sm + L::PF);
  TB* ff = reinterpret_cast<TB*>(sm + L::FF);
  TB* x1 = reinterpret_cast<TB*>(sm + L::X1);
  TB* yy = reinterpret_cast<TB*>(sm + L::YY);
  double* nrm = reinterpret_cast<double*>(sm + L::NRM);
  double* dS = reinterpret_cast<double*>(sm + L::DS);
  double* s_area = dS + NQF;
  int* cidx = reinterpret_cast<int*>(sm + L::CIDX);
  const int t = threadIdx.x;
  for (int64_t id = blockIdx.x; id < fp.n_int + fp.n_bnd; id += gridDim.x) {
    const bool interior = id < fp.n_int;
    const int64_t i = interior ? id : id - fp.n_int;
    const int ns = interior ? 2 : 1;
    const int face[2] = {interior ? int(fp.fpf[i]) : int(fp.bface[i]), interior ? int(fp.fmf[i]) : 0};
    const int64_t cell[2] = {interior ? int64_t(fp.fplus[i]) : int64_t(fp.bcell[i]),
                             interior ? int64_t(fp.fminus[i]) : 0};
    // compact index of each side's face nodes (node index along the face normal = the face's side)
    for (int it = t; it < ns * NB; it += blockDim.x) {
      const int s = it / NB, a = it % NB, d = face[s] / 2;
      const int ad = (a / (d == 0 ? 1 : (d == 1 ? N1 : N1 * N1))) % N1;
      int c = -1;
      if (ad == (face[s] % 2) * P) {
        const int d1 = d == 0 ? 1 : 0, d2 = d == 2 ? 1 : 2;
        const int st1 = d1 == 0 ? 1 : (d1 == 1 ? N1 : N1 * N1), st2 = d2 == 0 ? 1 : (d2 == 1 ? N1 : N1 * N1);
        c = (a / st1) % N1 + N1 * ((a / st2) % N1);
      }
      cidx[s * NB + a] = c;
    }
    double* cnv = reinterpret_cast<double*>(sm + L::CN);
    double* vd = reinterpret_cast<double*>(sm + L::VD);
    double* cof0 = reinterpret_cast<double*>(sm + L::COF0);
    // 1. side 0 per point: geometry, normal, surface element; then |F|
    // 2a. per (side, point): geometry (side 0 from step 1), cof^T n / det, Lagrange data
    for (int pass = 0; pass < 2; ++pass) {
      for (int it = t; it < (pass == 0 ? 1 : ns) * NQF; it += blockDim.x) {
        const int side = it / NQF, q = it % NQF, qs = q % N1, qt = q / N1;
        const double s = fp.gx[qs], tt = fp.gx[qt];
        double xh[3];
        if (side == 0) {
          const int d = face[0] / 2, d1 = d == 0 ? 1 : 0, d2 = d == 2 ? 1 : 2;
          xh[d] = double(face[0] % 2);
          xh[d1] = s;
          xh[d2] = tt;
        } else {
          const double Lw[4] = {(1 - s) * (1 - tt), s * (1 - tt), (1 - s) * tt, s * tt};
          xh[0] = xh[1] = xh[2] = 0.0;
#pragma unroll
          for (int c = 0; c < 4; ++c) {
            const int v = fp.fcorner[4 * i + c];
#pragma unroll
            for (int k = 0; k < 3; ++k) xh[k] += Lw[c] * double((v >> k) & 1);
          }
          xh[face[1] / 2] = double(face[1] % 2);
        }
        double cof[9], det;
        if (pass == 1 && side == 0) {
#pragma unroll
          for (int k = 0; k < 9; ++k) cof[k] = cof0[q * 10 + k];
          det = cof0[q * 10 + 9];
        } else {
          double xv[24], a[21];
#pragma unroll
          for (int k = 0; k < 24; ++k) xv[k] = fp.xv[cell[side] * 24 + k];
#pragma unroll
          for (int k = 0; k < 3; ++k) trilinear_coefficients(xv, k, a);
          geometry_at(a, xh[0], xh[1], xh[2], cof, &det);
          if (!(det > 0.0)) atomicOr(fp.err, kErrNegJacobian);
        }
        if (pass == 0) {
          const int d = face[0] / 2;
          const double sg = face[0] % 2 ? 1.0 : -1.0;
          const double nd[3] = {sg * cof[d], sg * cof[3 + d], sg * cof[6 + d]};
          const double len = sqrt(nd[0] * nd[0] + nd[1] * nd[1] + nd[2] * nd[2]);
          dS[q] = len * fp.gw[qs] * fp.gw[qt];
#pragma unroll
          for (int k = 0; k < 3; ++k) nrm[q * 3 + k] = nd[k] / len;
#pragma unroll
          for (int k = 0; k < 9; ++k) cof0[q * 10 + k] = cof[k];
          cof0[q * 10 + 9] = det;
          continue;
        }
        const double rdet = 1.0 / det;
#pragma unroll
        for (int d = 0; d < 3; ++d)
          cnv[(side * NQF + q) * 3 + d] =
              (cof[d] * nrm[q * 3] + cof[3 + d] * nrm[q * 3 + 1] + cof[6 + d] * nrm[q * 3 + 2]) * rdet;
        double* V = vd + (side * NQF + q) * 6 * N1;  // V[k][m] at k*N1 + m, D at (3 + k)*N1 + m
#pragma unroll
        for (int k = 0; k < 3; ++k) lagrange<P>(xh[k], V + k * N1, V + (3 + k) * N1);
      }
      __syncthreads();
      if (pass == 0 && t == 0) {
        double ar = 0.0;
        for (int q = 0; q < NQF; ++q) ar += dS[q];
        *s_area = ar;
      }
      __syncthreads();
    }
    // 2b. per (side, point, node): normal derivative; value and dS value on face nodes
    for (int it = t; it < ns * NQF * NB; it += blockDim.x) {
      const int side = it / (NQF * NB), q = (it / NB) % NQF, b = it % NB;
      const int b0 = b % N1, b1 = (b / N1) % N1, b2 = b / (N1 * N1);
      const double* V = vd + (side * NQF + q) * 6 * N1;
      const double* D = V + 3 * N1;
      const double* cn = cnv + (side * NQF + q) * 3;
      const double v0 = V[b0], v1 = V[N1 + b1], v2 = V[2 * N1 + b2];
      gn[(side * NQF + q) * NB + b] = cvt(cn[0] * D[b0] * v1 * v2 + cn[1] * v0 * D[N1 + b1] * v2 + cn[2] * v0 * v1 * D[2 * N1 + b2]);
      const int c = cidx[side * NB + b];
      if (c >= 0) {
        const double ph = v0 * v1 * v2;
        ff[(side * NQF + q) * NBF + c] = cvt(ph);
        pf[(side * NQF + q) * NBF + c] = cvt(dS[q] * ph);
      }
    }
    __syncthreads();
    // 3. X_{sa,sb} scaled by -s_a/2 (boundary: -1) and Y_{sa,sb} scaled by s_a s_b
    const TB half = interior ? TB(0.5) : TB(1);
    for (int it = t; it < ns * ns * NBF * NB; it += blockDim.x) {
      const int blk = it / (NBF * NB), sa = blk >> 1, sb = blk & 1, c = (it / NB) % NBF, b = it % NB;
      TB v = TB(0);
      for (int q = 0; q < NQF; ++q) v = fma(pf[(sa * NQF + q) * NBF + c], gn[(sb * NQF + q) * NB + b], v);
      x1[(blk * NBF + c) * NB + b] = (sa ? half : -half) * v;
    }
    for (int it = t; it < ns * ns * NBF * NBF; it += blockDim.x) {
      const int blk = it / (NBF * NBF), sa = blk >> 1, sb = blk & 1, c = (it / NBF) % NBF, e = it % NBF;
      TB v = TB(0);
      for (int q = 0; q < NQF; ++q) v = fma(pf[(sa * NQF + q) * NBF + c], ff[(sb * NQF + q) * NBF + e], v);
      yy[(blk * NBF + c) * NBF + e] = sa == sb ? v : -v;
    }
    __syncthreads();
    // 4. the facet blocks: X term, tau times the transposed X term of the
    //    swapped block, gamma/|F| times the Y term (entries with no face node:
    //    zero, no arithmetic)
    const TB pen = cvt(fp.gamma / *s_area), tau = cvt(fp.tau);
    TB* fblk = static_cast<TB*>(fp.fblk);
    TB* bblk = static_cast<TB*>(fp.bblk);
    for (int it = t; it < ns * ns * NB * NB; it += blockDim.x) {
      const int blk = it / (NB * NB), sa = blk >> 1, sb = blk & 1, a = (it / NB) % NB, b = it % NB;
      const int ca = cidx[sa * NB + a], cb = cidx[sb * NB + b];
      TB v = TB(0);
      if (ca >= 0) v = x1[(blk * NBF + ca) * NB + b];
      if (cb >= 0) v = fma(tau, x1[(((sb << 1) | sa) * NBF + cb) * NB + a], v);
      if (ca >= 0 && cb >= 0) v = fma(pen, yy[(blk * NBF + ca) * NBF + cb], v);
      if (interior)
        fblk[(i * 4 + blk) * NB * NB + a * NB + b] = v;
      else
        bblk[i * NB * NB + a * NB + b] = v;
    }
    __syncthreads();
  }
}

}  // namespace dg
}  // namespace feasm

namespace feasm {
namespace dg {

struct RowParams {
  int64_t n_cells;
  int nb, nlp;
  const void* ke;  // cell matrices [cells][nb][nlp], T
  const double* fe;
  const int32_t* face_code;
  const uint8_t* slots;
  const uint8_t* nslot;
  const int64_t* row_ptr;
  const void* fblk;  // facet blocks in T (the facet kernel's storage type)
  const void* bblk;
  double* values;
  double* rhs;
};

// One block per cell: every entry (block slot j, row a, column b) of the
// cell's block row. The diagonal block is the cell matrix plus the diagonal
// blocks of the cell's six facets in face order; a neighbour's block is the
// facet's off-diagonal block (rows: this cell's side). T is the storage of the
// cell and facet blocks: FP64, or FP32, whose seven terms are summed as an
// FP32 pair (TwoSum) and rounded once to FP64, and whose single terms convert
// exactly on the integer bits.
// Exact FP32 -> FP64 on the integer bits: the short path for zeros and normal
// numbers, the general one otherwise.
__device__ __forceinline__ double to_f64(float x) {
  return f32_zero_or_normal(x) ? f32_to_f64_normal(x) : f32_to_f64_exact(x);
}

template <int NB, typename T>
__global__ void __launch_bounds__(256) k_dg_rows(RowParams rp) {
  constexpr bool F32 = std::is_same<T, float>::value;
  const T* ke = static_cast<const T*>(rp.ke);
  const T* fblk = static_cast<const T*>(rp.fblk);
  const T* bblk = static_cast<const T*>(rp.bblk);
  for (int64_t e = blockIdx.x; e < rp.n_cells; e += gridDim.x) {
    const int ns = rp.nslot[e];
    for (int it = threadIdx.x; it < ns * NB * NB; it += blockDim.x) {
      const int j = it / (NB * NB), a = (it / NB) % NB, b = it % NB;
      const int slot = rp.slots[e * 7 + j];
      double v;
      if (slot == kSelf) {
        T hi = ke[(e * NB + a) * int64_t(rp.nlp) + b], lo = T(0);
#pragma unroll
        for (int f = 0; f < 6; ++f) {
          const int32_t code = rp.face_code[e * 6 + f];
          const T x = code >= 0 ? fblk[(int64_t(code >> 1) * 4 + 3 * (code & 1)) * NB * NB + a * NB + b]
                                : bblk[int64_t(-1 - code) * NB * NB + a * NB + b];
          if constexpr (F32) {
            const T sum = hi + x, bp = sum - hi;
            lo += (hi - (sum - bp)) + (x - bp);
            hi = sum;
          } else {
            hi += x;
          }
        }
        if constexpr (F32) v = to_f64(hi) + to_f64(lo); else v = hi;
      } else {
        const int32_t code = rp.face_code[e * 6 + slot];
        const int side = code & 1;  // this cell's side; the neighbour is on the other
        const T x = fblk[(int64_t(code >> 1) * 4 + 2 * side + (1 - side)) * NB * NB + a * NB + b];
        if constexpr (F32) v = to_f64(x); else v = x;
      }
      rp.values[rp.row_ptr[e * NB + a] + j * NB + b] = v;
    }
    if (rp.rhs)
      for (int a = threadIdx.x; a < NB; a += blockDim.x) rp.rhs[e * NB + a] = rp.fe[e * NB + a];
  }
}

template <int P>
cudaError_t launch(const fe_dg* g, double tau, double gamma, double* values, double* rhs, fe_precision prec,
                   const double* gx, const double* gw, cudaStream_t st) {
  constexpr int NB = (P + 1) * (P + 1) * (P + 1);
  int nsm = 152;
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, g->s->device);
  FacetParams fp;
  fp.n_int = int64_t(g->fplus.size());
  fp.n_bnd = int64_t(g->bcell.size());
  fp.xv = g->s->d_xv;
  fp.fplus = g->d_fplus;
  fp.fminus = g->d_fminus;
  fp.fpf = g->d_fpf;
  fp.fmf = g->d_fmf;
  fp.fcorner = g->d_fcorner;
  fp.bcell = g->d_bcell;
  fp.bface = g->d_bface;
  fp.gx = gx;
  fp.gw = gw;
  fp.tau = tau;
  fp.gamma = gamma;
  fp.fblk = g->d_fblk;
  fp.bblk = g->d_bblk;
  fp.err = g->s->d_err;
  const int64_t nf = fp.n_int + fp.n_bnd;
  const int fblocks = int(std::min<int64_t>(std::max<int64_t>(nf, 1), int64_t(nsm) * 16));
  if (nf > 0 && prec == FE_PREC_FP64) {
    constexpr size_t smem = FacetLayout<P, double>::BYTES;
    cudaError_t e = cudaFuncSetAttribute(k_dg_facets<P, double>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    if (e != cudaSuccess) return e;
    k_dg_facets<P, double><<<fblocks, 128, smem, st>>>(fp);
  } else if (nf > 0) {
    constexpr size_t smem = FacetLayout<P, float>::BYTES;
    cudaError_t e = cudaFuncSetAttribute(k_dg_facets<P, float>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    if (e != cudaSuccess) return e;
    k_dg_facets<P, float><<<fblocks, 128, smem, st>>>(fp);
  }
  RowParams rp;
  rp.n_cells = g->n_cells;
  rp.nb = NB;
  rp.nlp = g->s->nlp;
  rp.ke = g->s->d_ke;
  rp.fe = g->s->d_fe;
  rp.face_code = g->d_face_code;
  rp.slots = g->d_slots;
  rp.nslot = g->d_nslot;
  rp.row_ptr = g->d_row_ptr;
  rp.fblk = g->d_fblk;
  rp.bblk = g->d_bblk;
  rp.values = values;
  rp.rhs = rhs;
  const int blocks = int(std::min<int64_t>(g->n_cells, int64_t(nsm) * 8));
  if (prec == FE_PREC_FP64)
    k_dg_rows<NB, double><<<blocks, 256, 0, st>>>(rp);
  else
    k_dg_rows<NB, float><<<blocks, 256, 0, st>>>(rp);
  return cudaGetLastError();
}

}  // namespace dg
}  // namespace feasm

namespace {

template <typename T>
cudaError_t upload_vec(T** dst, const std::vector<T>& src) {
  *dst = nullptr;
  if (src.empty()) return cudaSuccess;
  cudaError_t e = cudaMalloc(reinterpret_cast<void**>(dst), src.size() * sizeof(T));
  if (e != cudaSuccess) return e;
  return cudaMemcpy(*dst, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice);
}

void free_dg(fe_dg* g) {
  void* ptrs[] = {g->d_fplus, g->d_fminus, g->d_fpf, g->d_fmf, g->d_fcorner, g->d_bcell, g->d_bface, g->d_face_code,
                  g->d_slots, g->d_nslot, g->d_row_ptr, g->d_col, g->d_ones, g->d_fblk, g->d_bblk, g->d_gx, g->d_gw};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  if (g->s) fe_space_destroy(g->s);
}

int dg_create(const fe_mesh_desc* mesh, int order, bool host_only, fe_dg** out) {
  if (!out) return feasm::set_error(FE_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (order < 1 || order > 3) return feasm::set_error(FE_ERR_INVALID_ARG, "order must be 1..3");
  fe_dg* g = new (std::nothrow) fe_dg();
  if (!g) return feasm::set_error(FE_ERR_OOM, "host allocation failed");
  int rc = host_only ? fe_space_create_host(mesh, order, 0, FE_POISSON, 0.0, &g->s)
                     : fe_space_create(mesh, order, 0, FE_POISSON, 0.0, &g->s);
  if (rc) {
    delete g;
    return rc;
  }
  g->p = order;
  g->nb = (order + 1) * (order + 1) * (order + 1);
  g->n_cells = mesh->n_cells;
  g->n_dofs = mesh->n_cells * g->nb;
  g->host_only = host_only;
  if (g->n_dofs > INT32_MAX) {
    fe_space_destroy(g->s);
    delete g;
    return feasm::set_error(FE_ERR_UNSUPPORTED, "more than 2^31-1 DG DOFs");
  }
  std::string err;
  try {
    rc = setup_dg(g, mesh, &err);
  } catch (const std::bad_alloc&) {
    rc = FE_ERR_OOM;
    err = "host allocation failed during DG setup";
  }
  if (rc) {
    fe_space_destroy(g->s);
    delete g;
    return feasm::set_error(rc, err.c_str());
  }
  if (!host_only) {
    std::vector<double> gx(order + 1), gw(order + 1), ones(std::max<int64_t>(1, g->n_cells), 1.0);
    feasm::gauss_rule(order + 1, gx.data(), gw.data());
    const size_t nbb = size_t(g->nb) * g->nb;
    cudaError_t e = upload_vec(&g->d_fplus, g->fplus);
    if (e == cudaSuccess) e = upload_vec(&g->d_fminus, g->fminus);
    if (e == cudaSuccess) e = upload_vec(&g->d_fpf, g->fpf);
    if (e == cudaSuccess) e = upload_vec(&g->d_fmf, g->fmf);
    if (e == cudaSuccess) e = upload_vec(&g->d_fcorner, g->fcorner);
    if (e == cudaSuccess) e = upload_vec(&g->d_bcell, g->bcell);
    if (e == cudaSuccess) e = upload_vec(&g->d_bface, g->bface);
    if (e == cudaSuccess) e = upload_vec(&g->d_face_code, g->face_code);
    if (e == cudaSuccess) e = upload_vec(&g->d_slots, g->slots);
    if (e == cudaSuccess) e = upload_vec(&g->d_nslot, g->nslot);
    if (e == cudaSuccess) e = upload_vec(&g->d_row_ptr, g->row_ptr);
    if (e == cudaSuccess) e = upload_vec(&g->d_col, g->col);
    if (e == cudaSuccess) e = upload_vec(&g->d_ones, ones);
    if (e == cudaSuccess) e = upload_vec(&g->d_gx, gx);
    if (e == cudaSuccess) e = upload_vec(&g->d_gw, gw);
    if (e == cudaSuccess && !g->fplus.empty())
      e = cudaMalloc(&g->d_fblk, g->fplus.size() * 4 * nbb * sizeof(double));
    if (e == cudaSuccess && !g->bcell.empty()) e = cudaMalloc(&g->d_bblk, g->bcell.size() * nbb * sizeof(double));
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
      free_dg(g);
      delete g;
      return feasm::set_error(e == cudaErrorMemoryAllocation ? FE_ERR_OOM : FE_ERR_CUDA, cudaGetErrorString(e));
    }
    std::vector<int32_t>().swap(g->col);  // kept on the device only
  }
  *out = g;
  return FE_OK;
}

}  // namespace

extern "C" {

int fe_dg_create(const fe_mesh_desc* mesh, int order, fe_dg** out) { return dg_create(mesh, order, false, out); }
int fe_dg_create_host(const fe_mesh_desc* mesh, int order, fe_dg** out) { return dg_create(mesh, order, true, out); }

int fe_dg_sizes(const fe_dg* g, int64_t* n_dofs, int64_t* nnz, int64_t* n_interior, int64_t* n_boundary) {
  if (!g) return feasm::set_error(FE_ERR_INVALID_ARG, "NULL argument");
  if (n_dofs) *n_dofs = g->n_dofs;
  if (nnz) *nnz = g->nnz;
  if (n_interior) *n_interior = int64_t(g->fplus.size());
  if (n_boundary) *n_boundary = int64_t(g->bcell.size());
  return FE_OK;
}

int fe_dg_csr_pattern_host(const fe_dg* g, int64_t* row_ptr, int32_t* col_idx) {
  if (!g || !row_ptr || (!col_idx && g->nnz)) return feasm::set_error(FE_ERR_INVALID_ARG, "NULL argument");
  if (!g->host_only) return feasm::set_error(FE_ERR_INVALID_ARG, "the pattern is kept on the host for host-only DG spaces; use fe_dg_csr_pattern");
  std::memcpy(row_ptr, g->row_ptr.data(), g->row_ptr.size() * sizeof(int64_t));
  if (g->nnz) std::memcpy(col_idx, g->col.data(), g->col.size() * sizeof(int32_t));
  return FE_OK;
}

int fe_dg_csr_pattern(const fe_dg* g, int64_t* row_ptr, int32_t* col_idx, void* stream) {
  if (!g || !row_ptr || (!col_idx && g->nnz)) return feasm::set_error(FE_ERR_INVALID_ARG, "NULL argument");
  if (g->host_only) return feasm::set_error(FE_ERR_INVALID_ARG, "host-only DG space");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  cudaError_t e = cudaMemcpyAsync(row_ptr, g->d_row_ptr, (g->n_dofs + 1) * sizeof(int64_t), cudaMemcpyDeviceToDevice, st);
  if (e == cudaSuccess && g->nnz)
    e = cudaMemcpyAsync(col_idx, g->d_col, g->nnz * sizeof(int32_t), cudaMemcpyDeviceToDevice, st);
  return e == cudaSuccess ? FE_OK : feasm::set_error(FE_ERR_CUDA, cudaGetErrorString(e));
}

int fe_dg_facets_host(const fe_dg* g, int32_t* plus, int32_t* minus, uint8_t* plus_face, uint8_t* minus_face,
                      int32_t* bnd_cell, uint8_t* bnd_face) {
  if (!g) return feasm::set_error(FE_ERR_INVALID_ARG, "NULL argument");
  const size_t ni = g->fplus.size(), nbd = g->bcell.size();
  if (plus && ni) std::memcpy(plus, g->fplus.data(), ni * sizeof(int32_t));
  if (minus && ni) std::memcpy(minus, g->fminus.data(), ni * sizeof(int32_t));
  if (plus_face && ni) std::memcpy(plus_face, g->fpf.data(), ni);
  if (minus_face && ni) std::memcpy(minus_face, g->fmf.data(), ni);
  if (bnd_cell && nbd) std::memcpy(bnd_cell, g->bcell.data(), nbd * sizeof(int32_t));
  if (bnd_face && nbd) std::memcpy(bnd_face, g->bface.data(), nbd);
  return FE_OK;
}

int fe_dg_assemble(fe_dg* g, double tau, double gamma, double source, double* csr_values, double* rhs,
                   fe_precision prec, void* stream) {
  if (!g) return feasm::set_error(FE_ERR_INVALID_ARG, "NULL argument");
  if (g->host_only) return feasm::set_error(FE_ERR_INVALID_ARG, "host-only DG space cannot compute");
  if (prec != FE_PREC_FP64 && prec != FE_PREC_FP32 && prec != FE_PREC_BF16)
    return feasm::set_error(FE_ERR_INVALID_ARG, "unknown precision");
  if (g->nnz && !csr_values) return feasm::set_error(FE_ERR_INVALID_ARG, "NULL csr_values");
  if (!(gamma > 0.0)) return feasm::set_error(FE_ERR_INVALID_ARG, "gamma must be positive");
  if (g->n_cells == 0) return FE_OK;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const double f[3] = {source, 0.0, 0.0};
  if (int rc = feasm::cell_stage(g->s, g->d_ones, f, prec, st)) return rc;
  cudaError_t e;
  switch (g->p) {
    case 1: e = feasm::dg::launch<1>(g, tau, gamma, csr_values, rhs, prec, g->d_gx, g->d_gw, st); break;
    case 2: e = feasm::dg::launch<2>(g, tau, gamma, csr_values, rhs, prec, g->d_gx, g->d_gw, st); break;
    default: e = feasm::dg::launch<3>(g, tau, gamma, csr_values, rhs, prec, g->d_gx, g->d_gw, st); break;
  }
  return e == cudaSuccess ? FE_OK : feasm::set_error(FE_ERR_CUDA, cudaGetErrorString(e));
}

void fe_dg_destroy(fe_dg* g) {
  if (!g) return;
  if (g->host_only) {
    if (g->s) fe_space_destroy(g->s);
  } else {
    free_dg(g);
  }
  delete g;
}

}  // extern "C"

// Interior penalty DG for the Poisson problem (paper, Sect. "Non-conforming
// methods", Eq. ip_dg_formulations, Eq. mean_and_jump_ops, Eq.
// local_to_face_matrix): discontinuous Q_p, cell-local DOFs K*nb + a.
//
// GB300 form: the cell integrals come from the Poisson cell kernels of an
// internal fe_space of the same order (FP64 or FP32 form); the facet
// integrals from k_dg_facets (persistent blocks, one facet at a time: its
// four nb x nb blocks, or one for a boundary facet, through small products
// over the face nodes, where the shape functions do not vanish; one warp forms
// the next facet's FP64 point data while the others form the products, in
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
      // K+'s face corners (s, t) = (0,0), (1,0), (0,1), (1,1) on K-'s reference
      // corners: a symmetry of the square, i.e. corner (1,1) = (1,0) + (0,1) - (0,0)
      // in every reference coordinate (the facet kernel relies on it)
      const uint8_t* fc = g->fcorner.data() + g->fcorner.size() - 4;
      for (int k = 0; k < 3; ++k) {
        const int b[4] = {(fc[0] >> k) & 1, (fc[1] >> k) & 1, (fc[2] >> k) & 1, (fc[3] >> k) & 1};
        if (b[3] != b[1] + b[2] - b[0]) {
          *err = "facet corners of the two cells are not related by a symmetry of the square";
          return FE_ERR_INVALID_ARG;
        }
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

// 1D Lagrange polynomials on the nodes m/P and their derivatives at x, in T.
template <int P, typename T>
__device__ __forceinline__ void lagrange(T x, T* v, T* d) {
#pragma unroll
  for (int m = 0; m <= P; ++m) {
    T val = T(1), der = T(0);
#pragma unroll
    for (int s = 0; s <= P; ++s) {
      if (s == m) continue;
      const T den = T(m - s) / T(P);
      der = der * ((x - T(s) / T(P)) / den) + val / den;
      val *= (x - T(s) / T(P)) / den;
    }
    v[m] = val;
    d[m] = der;
  }
}

// Shared memory of k_dg_facets for order P. The per-facet point data are
// double-buffered (the point warp fills facet n+1's while the other warps use
// facet n's): the sides' trilinear coefficients and |F| in double; cof^T n /
// det, the 1D Lagrange data, the surface elements (TB) and the face-node
// indices. The products' operands and results (TB: FP64 form double, FP32
// forms float) belong to the product warps alone.
template <int P, typename TB>
struct FacetLayout {
  static constexpr int N1 = P + 1, NB = N1 * N1 * N1, NQF = N1 * N1, NBF = N1 * N1;
  static constexpr size_t S = sizeof(TB);
  // one point-data buffer
  static constexpr size_t B_ACO = 0;                                      // double [2][21]
  static constexpr size_t B_AREA = B_ACO + size_t(2) * 21 * 8;           // double |F|
  static constexpr size_t B_CN = B_AREA + 8;                              // TB [2][NQF][3]
  static constexpr size_t B_VD = B_CN + size_t(2) * NQF * 3 * S;          // TB [2][NQF][2][3][N1]
  static constexpr size_t B_DS = B_VD + size_t(2) * NQF * 6 * N1 * S;     // TB [NQF]
  static constexpr size_t B_CIDX = (B_DS + size_t(NQF) * S + 3) & ~size_t(3);  // int [2][NB]
  static constexpr size_t B_BYTES = (B_CIDX + size_t(2) * NB * 4 + 15) & ~size_t(15);
  static constexpr size_t PT = 0;                                         // two buffers
  static constexpr size_t GN = PT + 2 * B_BYTES;                          // [2][NQF][NB]   grad phi . n
  static constexpr size_t PF = GN + size_t(2) * NQF * NB * S;             // [2][NQF][NBF]  dS phi (face nodes)
  static constexpr size_t FF = PF + size_t(2) * NQF * NBF * S;            // [2][NQF][NBF]  phi (face nodes)
  static constexpr size_t X1 = FF + size_t(2) * NQF * NBF * S;            // [4][NBF][NB]
  static constexpr size_t YY = X1 + size_t(4) * NBF * NB * S;             // [4][NBF][NBF]
  static constexpr size_t BYTES = YY + size_t(4) * NBF * NBF * S;
};

// The facet named by id (interior facets first, then boundary facets).
struct FacetRef {
  bool interior;
  int64_t i;  // index among the interior or the boundary facets
  int ns;     // sides
  int face[2];
  int64_t cell[2];
};

__device__ __forceinline__ FacetRef facet_ref(const FacetParams& fp, int64_t id) {
  FacetRef f;
  f.interior = id < fp.n_int;
  f.i = f.interior ? id : id - fp.n_int;
  f.ns = f.interior ? 2 : 1;
  f.face[0] = f.interior ? int(fp.fpf[f.i]) : int(fp.bface[f.i]);
  f.face[1] = f.interior ? int(fp.fmf[f.i]) : 0;
  f.cell[0] = f.interior ? int64_t(fp.fplus[f.i]) : int64_t(fp.bcell[f.i]);
  f.cell[1] = f.interior ? int64_t(fp.fminus[f.i]) : 0;
  return f;
}

// Point data of facet id into buffer b (all 32 lanes of the point warp):
// each side's compact face-node index (node index along the face normal =
// the face's side) and trilinear coefficients; then one lane per (side,
// point) (2 (p+1)^2 <= 32): the reference point (side 1: each coordinate s,
// 1 - s, t, 1 - t or the face's side, read off the reference corners of K-
// that carry K+'s face corners), FP64 geometry, the physical normal and
// surface element of the point from cof(J+) nhat = det J+ J+^{-T} nhat
// (side-0 lanes; shuffled to the side-1 lane of the same point), |F| (a
// butterfly sum over the side-0 lanes), cof^T n / det and the 1D Lagrange
// data.
template <int P, typename TB>
__device__ __forceinline__ void facet_points(const FacetParams& fp, int64_t id, unsigned char* b, int lane) {
  using L = FacetLayout<P, TB>;
  constexpr bool F32 = std::is_same<TB, float>::value;
  constexpr int N1 = L::N1, NB = L::NB, NQF = L::NQF;
  static_assert(2 * NQF <= 32, "one lane per (side, point)");
  auto cvt = [](double x) -> TB {
    if constexpr (F32) return d2f_rn(x); else return x;
  };
  double* aco = reinterpret_cast<double*>(b + L::B_ACO);
  TB* cnv = reinterpret_cast<TB*>(b + L::B_CN);
  TB* vd = reinterpret_cast<TB*>(b + L::B_VD);
  TB* dsw = reinterpret_cast<TB*>(b + L::B_DS);
  int* cidx = reinterpret_cast<int*>(b + L::B_CIDX);
  const FacetRef f = facet_ref(fp, id);
  for (int it = lane; it < f.ns * NB; it += 32) {
    const int s = it / NB, a = it % NB, d = f.face[s] / 2;
    const int ad = (a / (d == 0 ? 1 : (d == 1 ? N1 : N1 * N1))) % N1;
    int c = -1;
    if (ad == (f.face[s] % 2) * P) {
      const int d1 = d == 0 ? 1 : 0, d2 = d == 2 ? 1 : 2;
      const int st1 = d1 == 0 ? 1 : (d1 == 1 ? N1 : N1 * N1), st2 = d2 == 0 ? 1 : (d2 == 1 ? N1 : N1 * N1);
      c = (a / st1) % N1 + N1 * ((a / st2) % N1);
    }
    cidx[s * NB + a] = c;
  }
  if (lane < 3 * f.ns) trilinear_coefficients(fp.xv + f.cell[lane / 3] * 24, lane % 3, aco + (lane / 3) * 21);
  __syncwarp();
    const bool act = lane < f.ns * NQF;
    const int side = act ? lane / NQF : 0, q = lane % NQF, qs = q % N1, qt = q / N1;
    const double s = fp.gx[qs], tt = fp.gx[qt];
    // (selects, not indexing by the face's direction, so that xh, cof and
    // nd stay in registers)
    double xh[3];
    if (side == 0) {
      const int d = f.face[0] / 2;
      const double fv = double(f.face[0] % 2);
      xh[0] = d == 0 ? fv : s;
      xh[1] = d == 1 ? fv : (d == 0 ? s : tt);
      xh[2] = d == 2 ? fv : tt;
    } else {
      // the corners of K+'s face sit on K-'s reference corners v0 (s, t) =
      // (0, 0), v1 (1, 0), v2 (0, 1), v3 = v1 + v2 - v0 (a symmetry of the
      // square, checked at setup), so each reference coordinate of K-'s
      // point is v0 + (v1 - v0) s + (v2 - v0) t: one of s, 1 - s, t, 1 - t
      // or the face's side
      const int v0 = fp.fcorner[4 * f.i], v1 = fp.fcorner[4 * f.i + 1], v2 = fp.fcorner[4 * f.i + 2];
      const double sm1 = 1.0 - s, tm1 = 1.0 - tt;
      const int d = f.face[1] / 2;
      const double fv = double(f.face[1] % 2);
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        const int b0 = (v0 >> k) & 1, d1 = ((v1 >> k) & 1) - b0, d2 = ((v2 >> k) & 1) - b0;
        xh[k] = k == d ? fv : (d1 > 0 ? s : d1 < 0 ? sm1 : d2 > 0 ? tt : d2 < 0 ? tm1 : double(b0));
      }
    }
    double cof[9], det;
    geometry_at(aco + side * 21, xh[0], xh[1], xh[2], cof, &det);
    if (act && !(det > 0.0)) atomicOr(fp.err, kErrNegJacobian);
    // the normal of point q: cof(J+) nhat on the side-0 lane q
    const int d = f.face[0] / 2;
    const double sg = f.face[0] % 2 ? 1.0 : -1.0;
    double nd[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      nd[k] = sg * (d == 0 ? cof[3 * k] : (d == 1 ? cof[3 * k + 1] : cof[3 * k + 2]));
      nd[k] = __shfl_sync(kFull, nd[k], q);
    }
    const double l2 = nd[0] * nd[0] + nd[1] * nd[1] + nd[2] * nd[2];
    const double rl = rsqrt(l2), len = l2 * rl;
    const double dsq = len * fp.gw[qs] * fp.gw[qt];
    double ar = lane < NQF ? dsq : 0.0;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) ar += __shfl_xor_sync(kFull, ar, off);
    if (act) {
      const double rdet = 1.0 / det;
      const double n0 = nd[0] * rl, n1 = nd[1] * rl, n2 = nd[2] * rl;
#pragma unroll
      for (int k = 0; k < 3; ++k) cnv[lane * 3 + k] = cvt((cof[k] * n0 + cof[3 + k] * n1 + cof[6 + k] * n2) * rdet);
      // the 1D shape data; FP32 forms with p <= 2 evaluate them in FP32 at the
      // rounded reference point (nodes 0, 1/2, 1 exact, every Gauss point
      // and its mirror at least 0.11 from a node); for p = 3 a 4-point Gauss
      // abscissa lies 0.003 from the node 1/3, so x - 1/3 is formed in FP64
      TB* vt = vd + lane * 6 * N1;  // V[k][m] at k*N1 + m, D at (3 + k)*N1 + m
      if constexpr (F32 && P <= 2) {
#pragma unroll
        for (int k = 0; k < 3; ++k) lagrange<P, float>(d2f_rn(xh[k]), vt + k * N1, vt + (3 + k) * N1);
      } else {
        double V[3][N1], D[3][N1];
#pragma unroll
        for (int k = 0; k < 3; ++k) lagrange<P, double>(xh[k], V[k], D[k]);
#pragma unroll
        for (int k = 0; k < 3; ++k)
#pragma unroll
          for (int m = 0; m < N1; ++m) {
            vt[k * N1 + m] = cvt(V[k][m]);
            vt[(3 + k) * N1 + m] = cvt(D[k][m]);
          }
      }
      if (side == 0) dsw[q] = cvt(dsq);
    }
    if (lane == 0) *reinterpret_cast<double*>(b + L::B_AREA) = ar;
}

__device__ __forceinline__ void product_barrier() { asm volatile("bar.sync 1, 96;" ::: "memory"); }

// One block of 128 threads per facet at a time, persistent, with warp roles:
//   warp 3      the point data of the block's next facet (facet_points) into
//               the other buffer;
//   warps 0-2   with facet n's point data:
//     3. per (side, point) row and node column: the normal derivative of every
//        shape function and the values of the (p+1)^2 face nodes (the other
//        shape functions vanish on the face);
//     4. the products X_{sa,sb} = sum_q dS phi^{sa}_{a'} (grad phi^{sb}_b . n)
//        (a' a face node of side sa) and Y_{sa,sb} = sum_q dS phi^{sa}_{a'} phi^{sb}_{b'};
//     5. block (sa, sb), row a, column b:
//        -s_a/2 X_{sa,sb}[a'][b] - tau s_b/2 X_{sb,sa}[b'][a] + gamma/|F| s_a s_b Y_{sa,sb}[a'][b']
//        (terms whose face node is missing are zero; boundary facets: one side,
//        s = 1 and the factor 1/2 dropped), Eq. local_to_face_matrix;
//     named barrier 1 (96 threads) between the steps.
// One block barrier per facet hands the buffers over; every thread runs the
// same facet loop, so each barrier sees all of its threads. FP32 forms (TB =
// float): geometry, normals, |F| and the 1D shape data (for p = 3; p <= 2
// forms them in FP32) in FP64, rounded to FP32 on the integer bits; steps 3
// to 5 in FP32, blocks stored in FP32. GB300 issues FP64 at 2 lanes per clock
// per SM: the point warp's FP64 chain is the part the roles overlap.
template <int P, typename TB>
__global__ void __launch_bounds__(128) k_dg_facets(FacetParams fp) {
  using L = FacetLayout<P, TB>;
  constexpr bool F32 = std::is_same<TB, float>::value;
  auto cvt = [](double x) -> TB {
    if constexpr (F32) return d2f_rn(x); else return x;
  };
  constexpr int N1 = L::N1, NB = L::NB, NQF = L::NQF, NBF = L::NBF;
  constexpr int NW = 3, NBJ = (NB + 31) / 32;
  extern __shared__ __align__(16) unsigned char sm[];
  TB* gn = reinterpret_cast<TB*>(sm + L::GN);
  TB* pf = reinterpret_cast<TB*>(sm + L::PF);
  TB* ff = reinterpret_cast<TB*>(sm + L::FF);
  TB* x1 = reinterpret_cast<TB*>(sm + L::X1);
  TB* yy = reinterpret_cast<TB*>(sm + L::YY);
  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  const int64_t n_fac = fp.n_int + fp.n_bnd;
  // steps 3 and 5 give each product warp whole rows and each lane the columns
  // b = lane + 32 j; the tensor-product digits of those columns, once
  int bd[NBJ][3];
#pragma unroll
  for (int j = 0; j < NBJ; ++j) {
    const int bb = lane + 32 * j;
    bd[j][0] = bb % N1;
    bd[j][1] = N1 + (bb / N1) % N1;
    bd[j][2] = 2 * N1 + (bb / (N1 * N1)) % N1;
  }
  if (warp == 3 && blockIdx.x < n_fac) facet_points<P, TB>(fp, blockIdx.x, sm + L::PT, lane);
  __syncthreads();
  int buf = 0;
  for (int64_t id = blockIdx.x; id < n_fac; id += gridDim.x, buf ^= 1) {
    if (warp == 3) {
      const int64_t nx = id + gridDim.x;
      if (nx < n_fac) facet_points<P, TB>(fp, nx, sm + L::PT + (buf ^ 1) * L::B_BYTES, lane);
    } else {
      const unsigned char* b = sm + L::PT + buf * L::B_BYTES;
      const TB* cnv = reinterpret_cast<const TB*>(b + L::B_CN);
      const TB* vd = reinterpret_cast<const TB*>(b + L::B_VD);
      const TB* dsw = reinterpret_cast<const TB*>(b + L::B_DS);
      const int* cidx = reinterpret_cast<const int*>(b + L::B_CIDX);
      const double area = *reinterpret_cast<const double*>(b + L::B_AREA);
      const FacetRef f = facet_ref(fp, id);
      const int ns = f.ns;
      // the face-node index of the lane's columns on each side
      int cbl[2][NBJ];
#pragma unroll
      for (int j = 0; j < NBJ; ++j) {
        const int bb = lane + 32 * j;
        cbl[0][j] = bb < NB ? cidx[bb] : -1;
        cbl[1][j] = bb < NB && ns == 2 ? cidx[NB + bb] : -1;
      }
      // 3. row (side, point), column node b: normal derivative; value and dS
      //    value on face nodes
      for (int r = warp; r < ns * NQF; r += NW) {
        const int side = r / NQF, q = r % NQF;
        const TB* V = vd + r * 6 * N1;  // values at 0..3 N1, derivatives 3 N1 further
        const TB c0 = cnv[r * 3], c1 = cnv[r * 3 + 1], c2 = cnv[r * 3 + 2], dq = dsw[q];
  #pragma unroll
        for (int j = 0; j < NBJ; ++j) {
          const int b = lane + 32 * j;
          if (b < NB) {
            const TB v0 = V[bd[j][0]], v1 = V[bd[j][1]], v2 = V[bd[j][2]];
            const TB d0 = V[3 * N1 + bd[j][0]], d1 = V[3 * N1 + bd[j][1]], d2 = V[3 * N1 + bd[j][2]];
            gn[r * NB + b] = c0 * d0 * v1 * v2 + c1 * v0 * d1 * v2 + c2 * v0 * v1 * d2;
            const int c = side ? cbl[1][j] : cbl[0][j];
            if (c >= 0) {
              const TB ph = v0 * v1 * v2;
              ff[r * NBF + c] = ph;
              pf[r * NBF + c] = dq * ph;
            }
          }
        }
      }
      product_barrier();
      // 4. X_{sa,sb} scaled by -s_a/2 (boundary: -1), row (block, face node c),
      //    column b; Y_{sa,sb} scaled by s_a s_b
      const TB half = f.interior ? TB(0.5) : TB(1);
      for (int r = warp; r < ns * ns * NBF; r += NW) {
        const int blk = r / NBF, c = r % NBF, sa = blk >> 1, sb = blk & 1;
        TB pq[NQF];
  #pragma unroll
        for (int q = 0; q < NQF; ++q) pq[q] = pf[(sa * NQF + q) * NBF + c];
        const TB* g = gn + sb * NQF * NB;
        const TB sc = sa ? half : -half;
  #pragma unroll
        for (int j = 0; j < NBJ; ++j) {
          const int b = lane + 32 * j;
          if (b < NB) {
            TB v = TB(0);
  #pragma unroll
            for (int q = 0; q < NQF; ++q) v = fma(pq[q], g[q * NB + b], v);
            x1[r * NB + b] = sc * v;
          }
        }
      }
      for (int it = t; it < ns * ns * NBF * NBF; it += 32 * NW) {
        const int blk = it / (NBF * NBF), sa = blk >> 1, sb = blk & 1, c = (it / NBF) % NBF, e = it % NBF;
        TB v = TB(0);
  #pragma unroll
        for (int q = 0; q < NQF; ++q) v = fma(pf[(sa * NQF + q) * NBF + c], ff[(sb * NQF + q) * NBF + e], v);
        yy[(blk * NBF + c) * NBF + e] = sa == sb ? v : -v;
      }
      product_barrier();
      // 5. the facet blocks, row (block, a), column b: X term, tau times the
      //    transposed X term of the swapped block, gamma/|F| times the Y term
      //    (entries with no face node: zero, no arithmetic)
      const TB pen = cvt(fp.gamma / area), tau = cvt(fp.tau);
      for (int r = warp; r < ns * ns * NB; r += NW) {
        const int blk = r / NB, a = r % NB, sa = blk >> 1, sb = blk & 1;
        const int ca = cidx[sa * NB + a];
        const TB* xr = x1 + (blk * NBF + (ca >= 0 ? ca : 0)) * NB;
        const TB* xt = x1 + ((sb << 1) | sa) * NBF * NB + a;
        const TB* yr = yy + (blk * NBF + (ca >= 0 ? ca : 0)) * NBF;
        TB* out = f.interior ? static_cast<TB*>(fp.fblk) + ((f.i * 4 + blk) * NB + a) * NB
                           : static_cast<TB*>(fp.bblk) + (f.i * NB + a) * NB;
  #pragma unroll
        for (int j = 0; j < NBJ; ++j) {
          const int b = lane + 32 * j;
          if (b < NB) {
            const int cb = sb ? cbl[1][j] : cbl[0][j];
            TB v = ca >= 0 ? xr[b] : TB(0);
            if (cb >= 0) {
              v = fma(tau, xt[cb * NB], v);
              if (ca >= 0) v = fma(pen, yr[cb], v);
            }
            out[b] = v;
          }
        }
      }
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
// exactly on the integer bits. The block locations and the CSR row starts are
// resolved once per cell into shared memory.
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
  // per cell, resolved once: the diagonal block of its facet on face f, the
  // source block of slot j (nullptr: the diagonal) and the CSR row starts
  __shared__ const T* s_diag[6];
  __shared__ const T* s_blk[7];
  __shared__ int64_t s_rp[NB];
  const int t = threadIdx.x;
  for (int64_t e = blockIdx.x; e < rp.n_cells; e += gridDim.x) {
    const int ns = rp.nslot[e];
    if (t < 6) {
      const int32_t code = rp.face_code[e * 6 + t];
      s_diag[t] = code >= 0 ? fblk + (int64_t(code >> 1) * 4 + 3 * (code & 1)) * NB * NB
                            : bblk + int64_t(-1 - code) * NB * NB;
    } else if (t >= 32 && t < 32 + ns) {
      const int j = t - 32, slot = rp.slots[e * 7 + j];
      const T* src = nullptr;
      if (slot != kSelf) {
        const int32_t code = rp.face_code[e * 6 + slot];
        const int side = code & 1;  // this cell's side; the neighbour is on the other
        src = fblk + (int64_t(code >> 1) * 4 + 2 * side + (1 - side)) * NB * NB;
      }
      s_blk[j] = src;
    }
    for (int a = t; a < NB; a += blockDim.x) s_rp[a] = rp.row_ptr[e * NB + a];
    __syncthreads();
    for (int it = t; it < ns * NB * NB; it += blockDim.x) {
      const int j = it / (NB * NB), ab = it % (NB * NB), a = ab / NB, b = ab % NB;
      const T* src = s_blk[j];
      double v;
      if (src == nullptr) {
        T hi = ke[(e * NB + a) * int64_t(rp.nlp) + b], lo = T(0);
#pragma unroll
        for (int f = 0; f < 6; ++f) {
          const T x = s_diag[f][ab];
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
        if constexpr (F32) v = to_f64(src[ab]); else v = src[ab];
      }
      rp.values[s_rp[a] + j * NB + b] = v;
    }
    if (rp.rhs)
      for (int a = t; a < NB; a += blockDim.x) rp.rhs[e * NB + a] = rp.fe[e * NB + a];
    __syncthreads();
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
  // a persistent grid of the resident blocks (one wave; facets cost alike)
  auto facets = [&](auto kern, size_t smem) -> cudaError_t {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    int per_sm = 1;
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 128, smem);
    if (e != cudaSuccess) return e;
    const int fblocks = int(std::min<int64_t>(nf, int64_t(nsm) * std::max(per_sm, 1)));
    kern<<<fblocks, 128, smem, st>>>(fp);
    return cudaSuccess;
  };
  if (nf > 0) {
    const cudaError_t e = prec == FE_PREC_FP64 ? facets(k_dg_facets<P, double>, FacetLayout<P, double>::BYTES)
                                               : facets(k_dg_facets<P, float>, FacetLayout<P, float>::BYTES);
    if (e != cudaSuccess) return e;
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

int fe_dg_create(const fe_mesh_desc* mesh, int order, fe_dg** out) {
  return feasm::no_throw("fe_dg_create", [&] { return dg_create(mesh, order, false, out); });
}
int fe_dg_create_host(const fe_mesh_desc* mesh, int order, fe_dg** out) {
  return feasm::no_throw("fe_dg_create_host", [&] { return dg_create(mesh, order, true, out); });
}

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

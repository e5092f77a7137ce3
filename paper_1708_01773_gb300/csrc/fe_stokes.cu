// Stokes cell integration for the Taylor-Hood pair of the paper's Stokes
// driver (Example "Stokes problem"; Sect. "Driver example for the Stokes
// problem"): velocity Q_P (3 components), pressure Q_{P-1}, (P+1)^3 Gauss
// points. With the cofactor gradients gh_a = cof(J) gradhat(phihat_a), so
// that grad(phi_a) = gh_a / det J (Eq. shape_grad), and gw_a = (w/det J) gh_a:
//   G_ab[k][l] = sum_q (w_q / det J_q) gh_{a,k} gh_{b,l}
//   velocity-velocity  A_(a,i),(b,j) = mu/2 (delta_ij tr G_ab + G_ab[j][i])
//                      (mu int eps(u):eps(v), the elasticity contraction with
//                      lambda = 0)
//   coupling           B_c,(b,j) = -sum_q w_q psi_c(x_q) gh_{b,j}  (det J
//                      cancels), stored in the pressure rows and, transposed,
//                      in the pressure columns of the velocity rows
//   pressure-pressure  0
//   cell vector        f_i sum_q w_q det J_q phihat_a on the velocity rows, 0
//                      on the pressure rows (FP64)
// One block per cell (persistent loop; the layout allows CPB cells per
// block); Q2/Q1 in FP32 runs a warp-specialised variant (k_cell_stokes_ws)
// whose FP64 steps run one cell ahead on a warp of their own. Q2/Q1 cell
// matrices are staged in shared memory and copied out with coalesced 16-byte
// stores. The geometry is FP64. The velocity
// block is symmetric: only node pairs a <= b are summed, each writing both
// blocks. The FP64 form keeps everything in FP64; the FP32 form rounds the
// cofactors to FP32 on the integer bits, forms w/det J in FP32, and sums the
// Gram entries in FP32 per slab of (P+1)^2 points with compensated (Kahan)
// addition of the slab sums.
#include <cuda_runtime.h>

#include <algorithm>
#include <type_traits>

#include "fe_device.cuh"
#include "fe_launch.h"

namespace feasm {
namespace stokes {

constexpr int kThreads = 256;

struct Params {
  int64_t n_cells;
  const double* xv;    // [cells][8][3]
  const double* w;     // [nq]
  const double* xq;    // [nq][3]
  const double* phi;   // [nq][nb]
  const double* dphi;  // [nq][nb][3]
  const float* dphi32;
  const double* psi;   // [nq][nbp]
  const double* coef;  // mu per cell
  double f[3];
  void* ke;
  double* fe;
  int* err;
};

template <int P, typename T>
struct Layout {
  static constexpr int N1 = P + 1, NB = N1 * N1 * N1, NQ = NB, NBP = P * P * P, NV = 3 * NB, NL = NV + NBP;
  static constexpr int NLP = (NL + 3) & ~3;
  static constexpr int NPAIR = NB * (NB + 1) / 2;  // node pairs a <= b
  // Q2/Q1: the cell matrices are staged in shared memory and written out with
  // coalesced 16-byte stores (the symmetric half's transposed entries would
  // otherwise be stride-NLP stores, one sector per lane); Q3/Q2 matrices do not
  // fit and are stored directly. Cells integrated together by one block: one
  // (measured with this kernel on Q2/Q1 FP32: 4 blocks of one cell per SM,
  // 0.77 ms, against 2 blocks of two cells, 0.87 ms, and 0.95 ms for
  // unstaged stores; that case now runs k_cell_stokes_ws, 0.64 ms).
  static constexpr bool STAGE = P == 2;
  static constexpr int CPB = 1;
  static constexpr int GS = NQ * 3 * NB;  // gradient entries per cell
  // shared memory, per cell c < CPB: xv[c][24], a[c][24], wdet[c][NQ] (double);
  // cof[c][NQ][9], wod[c][NQ], wq[c][NQ], mu/2 [c] (T); gh[c][NQ][3][NB] and
  // gw[c][NQ][3][NB] = (w/det) gh (T); then, shared by the cells, the pressure
  // basis psi[NQ][NBP] (T) and the node pairs a <= b
  static constexpr size_t OFF_A = size_t(CPB) * 24 * sizeof(double);
  static constexpr size_t OFF_WDET = OFF_A + size_t(CPB) * 24 * sizeof(double);
  static constexpr size_t OFF_COF = OFF_WDET + size_t(CPB) * NQ * sizeof(double);
  static constexpr size_t OFF_WOD = OFF_COF + size_t(CPB) * NQ * 9 * sizeof(T);
  static constexpr size_t OFF_WQ = OFF_WOD + size_t(CPB) * NQ * sizeof(T);
  static constexpr size_t OFF_MU = OFF_WQ + size_t(CPB) * NQ * sizeof(T);
  static constexpr size_t OFF_GH = (OFF_MU + CPB * sizeof(T) + 15) & ~size_t(15);
  static constexpr size_t OFF_GW = OFF_GH + size_t(CPB) * GS * sizeof(T);
  static constexpr size_t OFF_PSI = OFF_GW + size_t(CPB) * GS * sizeof(T);
  static constexpr size_t OFF_PAIR = OFF_PSI + size_t(NQ) * NBP * sizeof(T);
  static constexpr size_t OFF_KS = (OFF_PAIR + size_t(NPAIR) * sizeof(uint16_t) + 15) & ~size_t(15);
  static constexpr size_t BYTES = OFF_KS + (STAGE ? size_t(CPB) * NL * NLP * sizeof(T) : 0);
};

template <int P, typename T>
__global__ void __launch_bounds__(kThreads) k_cell_stokes(Params p) {
  using L = Layout<P, T>;
  constexpr int N1 = L::N1, NB = L::NB, NQ = L::NQ, NBP = L::NBP, NV = L::NV, NL = L::NL, NLP = L::NLP;
  constexpr int CPB = L::CPB, GS = L::GS, NPAIR = L::NPAIR;
  constexpr bool F32 = std::is_same<T, float>::value;
  extern __shared__ __align__(16) unsigned char sm[];
  double* xv = reinterpret_cast<double*>(sm);
  double* a = reinterpret_cast<double*>(sm + L::OFF_A);
  double* wdet = reinterpret_cast<double*>(sm + L::OFF_WDET);
  T* cof = reinterpret_cast<T*>(sm + L::OFF_COF);
  T* wod = reinterpret_cast<T*>(sm + L::OFF_WOD);
  T* wq = reinterpret_cast<T*>(sm + L::OFF_WQ);
  T* smu = reinterpret_cast<T*>(sm + L::OFF_MU);
  T* gh = reinterpret_cast<T*>(sm + L::OFF_GH);
  T* gw = reinterpret_cast<T*>(sm + L::OFF_GW);
  T* spsi = reinterpret_cast<T*>(sm + L::OFF_PSI);
  uint16_t* pairs = reinterpret_cast<uint16_t*>(sm + L::OFF_PAIR);
  T* K = static_cast<T*>(p.ke);
  T* Ks = reinterpret_cast<T*>(sm + L::OFF_KS);
  // destination of cell c's matrix: the staging buffer or the cell-matrix scratch
  auto kdst = [&](int64_t e0, int c) -> T* {
    if constexpr (L::STAGE) return Ks + size_t(c) * NL * NLP;
    else return K + (e0 + c) * int64_t(NL) * NLP;
  };
  const int t = threadIdx.x;
  for (int i = t; i < NQ * NBP; i += kThreads) spsi[i] = T(p.psi[i]);
  if (t == 0) {
    int n = 0;
    for (int a0 = 0; a0 < NB; ++a0)
      for (int b0 = a0; b0 < NB; ++b0) pairs[n++] = uint16_t(a0 << 8 | b0);
  }
  for (int64_t e0 = int64_t(blockIdx.x) * CPB; e0 < p.n_cells; e0 += int64_t(gridDim.x) * CPB) {
    const int nc = int(p.n_cells - e0 < CPB ? p.n_cells - e0 : CPB);
    for (int i = t; i < nc * 24; i += kThreads) xv[i] = p.xv[e0 * 24 + i];
    __syncthreads();
    if (t < 3 * nc) trilinear_coefficients(xv + (t / 3) * 24, t % 3, a + (t / 3) * 24);
    __syncthreads();
    // 1. geometry per (cell, quadrature point), FP64
    for (int i = t; i < nc * NQ; i += kThreads) {
      const int c = i / NQ, q = i % NQ;
      double cf[9], det;
      geometry_at(a + c * 24, p.xq[3 * q], p.xq[3 * q + 1], p.xq[3 * q + 2], cf, &det);
      if (!(det > 0.0)) atomicOr(p.err, kErrNegJacobian);
      const double w = p.w[q];
      wdet[i] = w * det;
      if constexpr (F32) {
        // FP32 form: conversions on the integer bits, the quotient in FP32
        const float w32 = d2f_rn(w);
        wod[i] = w32 / d2f_rn(det);
        wq[i] = w32;
#pragma unroll
        for (int k = 0; k < 9; ++k) cof[i * 9 + k] = d2f_rn(cf[k]);
      } else {
        wod[i] = w / det;
        wq[i] = w;
#pragma unroll
        for (int k = 0; k < 9; ++k) cof[i * 9 + k] = cf[k];
      }
    }
    if (t < nc) {
      const double mh = 0.5 * p.coef[e0 + t];
      if constexpr (F32) smu[t] = d2f_rn(mh); else smu[t] = mh;
    }
    __syncthreads();
    // 2. cofactor gradients gh[c][q][k][a] = sum_d cof[c][q][k][d] gradhat_d phihat_a(x_q), gw = (w/det) gh
    for (int i = t; i < nc * NQ * NB; i += kThreads) {
      const int c = i / (NQ * NB), r = i % (NQ * NB), q = r / NB, b = r % NB;
      T g[3];
      if constexpr (F32) {
        g[0] = p.dphi32[3 * r]; g[1] = p.dphi32[3 * r + 1]; g[2] = p.dphi32[3 * r + 2];
      } else {
        g[0] = p.dphi[3 * r]; g[1] = p.dphi[3 * r + 1]; g[2] = p.dphi[3 * r + 2];
      }
      const T* cq = cof + (c * NQ + q) * 9;
      const T wv = wod[c * NQ + q];
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        const T v = cq[3 * k] * g[0] + cq[3 * k + 1] * g[1] + cq[3 * k + 2] * g[2];
        gh[c * GS + (q * 3 + k) * NB + b] = v;
        gw[c * GS + (q * 3 + k) * NB + b] = wv * v;
      }
    }
    __syncthreads();
    // 3. velocity-velocity block, one (cell, node pair a <= b) per item; the
    //    block is symmetric (A_(b,j),(a,i) = A_(a,i),(b,j)), so (a, b) and (b, a)
    //    are written from the same sums
    for (int i = t; i < nc * NPAIR; i += kThreads) {
      const int c = i / NPAIR, pr = pairs[i % NPAIR], an = pr >> 8, bn = pr & 255;
      const T* ghc = gh + c * GS;
      const T* gwc = gw + c * GS;
      T S[3][3], C[3][3];
#pragma unroll
      for (int k = 0; k < 3; ++k)
#pragma unroll
        for (int l = 0; l < 3; ++l) { S[k][l] = T(0); C[k][l] = T(0); }
      for (int s0 = 0; s0 < NQ; s0 += N1 * N1) {
        T G[3][3];
#pragma unroll
        for (int k = 0; k < 3; ++k)
#pragma unroll
          for (int l = 0; l < 3; ++l) G[k][l] = T(0);
        for (int q = s0; q < s0 + N1 * N1; ++q) {
          T ga[3], gb[3];
#pragma unroll
          for (int k = 0; k < 3; ++k) {
            ga[k] = gwc[(q * 3 + k) * NB + an];
            gb[k] = ghc[(q * 3 + k) * NB + bn];
          }
#pragma unroll
          for (int k = 0; k < 3; ++k)
#pragma unroll
            for (int l = 0; l < 3; ++l) G[k][l] = fma(ga[k], gb[l], G[k][l]);
        }
#pragma unroll
        for (int k = 0; k < 3; ++k)
#pragma unroll
          for (int l = 0; l < 3; ++l) {
            if constexpr (F32) kahan_add(S[k][l], C[k][l], G[k][l]); else S[k][l] += G[k][l];
          }
      }
      const T tr = S[0][0] + S[1][1] + S[2][2], mh = smu[c];
      T* Ke = kdst(e0, c);
#pragma unroll
      for (int ii = 0; ii < 3; ++ii)
#pragma unroll
        for (int jj = 0; jj < 3; ++jj) {
          T v = S[jj][ii];
          if (ii == jj) v += tr;
          v *= mh;
          Ke[size_t(ii * NB + an) * NLP + jj * NB + bn] = v;
          if (an != bn) Ke[size_t(jj * NB + bn) * NLP + ii * NB + an] = v;
        }
    }
    // 4. pressure coupling, one (cell, pressure node, velocity node) per item
    for (int i = t; i < nc * NBP * NB; i += kThreads) {
      const int c = i / (NBP * NB), r = i % (NBP * NB), cp = r / NB, bn = r % NB;
      const T* ghc = gh + c * GS;
      const T* wqc = wq + c * NQ;
      T S[3] = {T(0), T(0), T(0)}, C[3] = {T(0), T(0), T(0)};
      for (int s0 = 0; s0 < NQ; s0 += N1 * N1) {
        T G[3] = {T(0), T(0), T(0)};
        for (int q = s0; q < s0 + N1 * N1; ++q) {
          const T wp = wqc[q] * spsi[q * NBP + cp];
#pragma unroll
          for (int k = 0; k < 3; ++k) G[k] = fma(wp, ghc[(q * 3 + k) * NB + bn], G[k]);
        }
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          if constexpr (F32) kahan_add(S[k], C[k], G[k]); else S[k] += G[k];
        }
      }
      T* Ke = kdst(e0, c);
#pragma unroll
      for (int jj = 0; jj < 3; ++jj) {
        Ke[size_t(jj * NB + bn) * NLP + NV + cp] = -S[jj];
        Ke[size_t(NV + cp) * NLP + jj * NB + bn] = -S[jj];
      }
    }
    // 5. pressure-pressure blocks
    for (int i = t; i < nc * NBP * NBP; i += kThreads) {
      const int c = i / (NBP * NBP), r = i % (NBP * NBP);
      kdst(e0, c)[size_t(NV + r / NBP) * NLP + NV + r % NBP] = T(0);
    }
    // 6. cell vectors (FP64), one (cell, node) per item
    for (int i = t; i < nc * NB; i += kThreads) {
      const int c = i / NB, an = i % NB;
      double s = 0.0;
      for (int q = 0; q < NQ; ++q) s = fma(wdet[c * NQ + q], p.phi[q * NB + an], s);
      double* fe = p.fe + (e0 + c) * NL;
#pragma unroll
      for (int ii = 0; ii < 3; ++ii) fe[ii * NB + an] = p.f[ii] * s;
    }
    for (int i = t; i < nc * NBP; i += kThreads) p.fe[(e0 + i / NBP) * NL + NV + i % NBP] = 0.0;
    if constexpr (L::STAGE) {
      // 7. staged cell matrices -> scratch, 16-byte coalesced (the cells of a group
      //    are consecutive: one contiguous range; row padding is copied as is)
      __syncthreads();
      constexpr int N16 = int(size_t(NL) * NLP * sizeof(T) / 16);
      const uint4* src = reinterpret_cast<const uint4*>(Ks);
      uint4* dst = reinterpret_cast<uint4*>(K + e0 * int64_t(NL) * NLP);
      for (int i = t; i < nc * N16; i += kThreads) dst[i] = src[i];
    }
    __syncthreads();
  }
}

// Warp-specialised Q2/Q1 FP32 cell kernel (one cell per block iteration,
// persistent grid). The FP64 steps of a cell (geometry at its 27 points, the
// cell vector) are one warp's work and would otherwise hold the block at a
// barrier, so they get a warp of their own, one cell ahead:
//   warp 7      cell vector of cell n (FP64, from w det J of buffer n % 2),
//               then the geometry of the block's next cell into buffer
//               (n + 1) % 2: trilinear coefficients, FP64 cofactors and det J
//               per point, FP32 cofactors, w / det J, w, w det J, mu / 2;
//   warps 0-6   gh / gw of cell n from buffer n % 2; the node pairs a <= b
//               and the pressure coupling in one item loop; the staged cell
//               matrix out with 16-byte stores (named barrier 1 between the
//               steps, 224 threads).
// One block barrier per cell hands the buffers over. Arithmetic per entry as
// in k_cell_stokes (FP32 slab sums with Kahan addition of the slab sums).
struct WsLayout {
  static constexpr int N1 = 3, NB = 27, NQ = 27, NBP = 8, NV = 81, NL = 89, NLP = 92;
  static constexpr int NPAIR = NB * (NB + 1) / 2, NCPL = NBP * NB, GS = NQ * 3 * NB;
  static constexpr int kCompute = 224;  // warps 0-6
  // one geometry buffer: a[24] (double), wdet[NQ] (double), cof[NQ][9], wod[NQ], wq[NQ], mu/2 (float)
  static constexpr size_t G_A = 0, G_WDET = 24 * 8, G_COF = G_WDET + NQ * 8, G_WOD = G_COF + NQ * 9 * 4,
                          G_WQ = G_WOD + NQ * 4, G_MU = G_WQ + NQ * 4, G_BYTES = (G_MU + 4 + 15) & ~size_t(15);
  static constexpr size_t OFF_GEO = 0;
  static constexpr size_t OFF_GH = OFF_GEO + 2 * G_BYTES;
  static constexpr size_t OFF_GW = OFF_GH + size_t(GS) * 4;
  static constexpr size_t OFF_PSI = OFF_GW + size_t(GS) * 4;
  static constexpr size_t OFF_PAIR = OFF_PSI + size_t(NQ) * NBP * 4;
  static constexpr size_t OFF_KS = (OFF_PAIR + size_t(NPAIR) * 2 + 15) & ~size_t(15);
  static constexpr size_t BYTES = OFF_KS + size_t(NL) * NLP * 4;
};

__device__ __forceinline__ void ws_compute_barrier() { asm volatile("bar.sync 1, 224;" ::: "memory"); }

// geometry of cell e into buffer g (all 32 lanes of the geometry warp)
__device__ __forceinline__ void ws_geometry(const Params& p, int64_t e, unsigned char* g, int lane) {
  using L = WsLayout;
  double* a = reinterpret_cast<double*>(g + L::G_A);
  double* wdet = reinterpret_cast<double*>(g + L::G_WDET);
  float* cof = reinterpret_cast<float*>(g + L::G_COF);
  float* wod = reinterpret_cast<float*>(g + L::G_WOD);
  float* wq = reinterpret_cast<float*>(g + L::G_WQ);
  float* smu = reinterpret_cast<float*>(g + L::G_MU);
  if (lane < 3) trilinear_coefficients(p.xv + e * 24, lane, a);
  __syncwarp();
  if (lane < L::NQ) {
    const int q = lane;
    double cf[9], det;
    geometry_at(a, p.xq[3 * q], p.xq[3 * q + 1], p.xq[3 * q + 2], cf, &det);
    if (!(det > 0.0)) atomicOr(p.err, kErrNegJacobian);
    const double w = p.w[q];
    wdet[q] = w * det;
    // conversions on the integer bits, the quotient in FP32
    const float w32 = d2f_rn(w);
    wod[q] = w32 / d2f_rn(det);
    wq[q] = w32;
#pragma unroll
    for (int k = 0; k < 9; ++k) cof[q * 9 + k] = d2f_rn(cf[k]);
  }
  if (lane == 0) *smu = d2f_rn(0.5 * p.coef[e]);
}

__global__ void __launch_bounds__(kThreads) k_cell_stokes_ws(Params p) {
  using L = WsLayout;
  constexpr int NB = L::NB, NQ = L::NQ, NBP = L::NBP, NV = L::NV, NL = L::NL, NLP = L::NLP;
  constexpr int NPAIR = L::NPAIR, NSLAB = L::N1 * L::N1;
  extern __shared__ __align__(16) unsigned char sm[];
  float* gh = reinterpret_cast<float*>(sm + L::OFF_GH);
  float* gw = reinterpret_cast<float*>(sm + L::OFF_GW);
  float* spsi = reinterpret_cast<float*>(sm + L::OFF_PSI);
  uint16_t* pairs = reinterpret_cast<uint16_t*>(sm + L::OFF_PAIR);
  float* Ks = reinterpret_cast<float*>(sm + L::OFF_KS);
  float* K = static_cast<float*>(p.ke);
  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  const int64_t e_first = blockIdx.x;
  if (e_first >= p.n_cells) return;
  if (warp == 7) {
    ws_geometry(p, e_first, sm + L::OFF_GEO, lane);
  } else {
    for (int i = t; i < NQ * NBP; i += L::kCompute) spsi[i] = float(p.psi[i]);
    // the pressure-pressure block is zero and no later step writes there
    for (int i = t; i < NBP * NBP; i += L::kCompute) Ks[(NV + i / NBP) * NLP + NV + i % NBP] = 0.0f;
    if (t == 0) {
      int n = 0;
      for (int a0 = 0; a0 < NB; ++a0)
        for (int b0 = a0; b0 < NB; ++b0) pairs[n++] = uint16_t(a0 << 8 | b0);
    }
  }
  __syncthreads();
  int cur = 0;
  for (int64_t e = e_first; e < p.n_cells; e += gridDim.x, cur ^= 1) {
    unsigned char* gcur = sm + L::OFF_GEO + cur * L::G_BYTES;
    if (warp == 7) {
      // cell vector of cell e (FP64), then the geometry of the next cell
      const double* wdet = reinterpret_cast<const double*>(gcur + L::G_WDET);
      if (lane < NB) {
        double s = 0.0;
        for (int q = 0; q < NQ; ++q) s = fma(wdet[q], p.phi[q * NB + lane], s);
        double* fe = p.fe + e * NL;
#pragma unroll
        for (int ii = 0; ii < 3; ++ii) fe[ii * NB + lane] = p.f[ii] * s;
      }
      if (lane < NBP) p.fe[e * NL + NV + lane] = 0.0;
      const int64_t en = e + gridDim.x;
      if (en < p.n_cells) ws_geometry(p, en, sm + L::OFF_GEO + (cur ^ 1) * L::G_BYTES, lane);
    } else {
      const float* cof = reinterpret_cast<const float*>(gcur + L::G_COF);
      const float* wod = reinterpret_cast<const float*>(gcur + L::G_WOD);
      const float* wq = reinterpret_cast<const float*>(gcur + L::G_WQ);
      const float mh = *reinterpret_cast<const float*>(gcur + L::G_MU);
      // gh[q][k][a] = sum_d cof[q][k][d] gradhat_d phihat_a(x_q), gw = (w/det) gh
      for (int i = t; i < NQ * NB; i += L::kCompute) {
        const int q = i / NB, b = i % NB;
        const float g0 = p.dphi32[3 * i], g1 = p.dphi32[3 * i + 1], g2 = p.dphi32[3 * i + 2];
        const float* cq = cof + q * 9;
        const float wv = wod[q];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          const float v = cq[3 * k] * g0 + cq[3 * k + 1] * g1 + cq[3 * k + 2] * g2;
          gh[(q * 3 + k) * NB + b] = v;
          gw[(q * 3 + k) * NB + b] = wv * v;
        }
      }
      ws_compute_barrier();
      // node pairs a <= b (both symmetric entries), then the pressure coupling
      for (int i = t; i < NPAIR + L::NCPL; i += L::kCompute) {
        if (i < NPAIR) {
          const int pr = pairs[i], an = pr >> 8, bn = pr & 255;
          float S[3][3], C[3][3];
#pragma unroll
          for (int k = 0; k < 3; ++k)
#pragma unroll
            for (int l = 0; l < 3; ++l) { S[k][l] = 0.0f; C[k][l] = 0.0f; }
#pragma unroll 1
          for (int s0 = 0; s0 < NQ; s0 += NSLAB) {
            float G[3][3];
#pragma unroll
            for (int k = 0; k < 3; ++k)
#pragma unroll
              for (int l = 0; l < 3; ++l) G[k][l] = 0.0f;
#pragma unroll
            for (int q = s0; q < s0 + NSLAB; ++q) {
              float ga[3], gb[3];
#pragma unroll
              for (int k = 0; k < 3; ++k) {
                ga[k] = gw[(q * 3 + k) * NB + an];
                gb[k] = gh[(q * 3 + k) * NB + bn];
              }
#pragma unroll
              for (int k = 0; k < 3; ++k)
#pragma unroll
                for (int l = 0; l < 3; ++l) G[k][l] = fmaf(ga[k], gb[l], G[k][l]);
            }
#pragma unroll
            for (int k = 0; k < 3; ++k)
#pragma unroll
              for (int l = 0; l < 3; ++l) kahan_add(S[k][l], C[k][l], G[k][l]);
          }
          const float tr = S[0][0] + S[1][1] + S[2][2];
#pragma unroll
          for (int ii = 0; ii < 3; ++ii)
#pragma unroll
            for (int jj = 0; jj < 3; ++jj) {
              float v = S[jj][ii];
              if (ii == jj) v += tr;
              v *= mh;
              Ks[(ii * NB + an) * NLP + jj * NB + bn] = v;
              if (an != bn) Ks[(jj * NB + bn) * NLP + ii * NB + an] = v;
            }
        } else {
          const int r = i - NPAIR, cp = r / NB, bn = r % NB;
          float S[3] = {0.0f, 0.0f, 0.0f}, C[3] = {0.0f, 0.0f, 0.0f};
#pragma unroll 1
          for (int s0 = 0; s0 < NQ; s0 += NSLAB) {
            float G[3] = {0.0f, 0.0f, 0.0f};
#pragma unroll
            for (int q = s0; q < s0 + NSLAB; ++q) {
              const float wp = wq[q] * spsi[q * NBP + cp];
#pragma unroll
              for (int k = 0; k < 3; ++k) G[k] = fmaf(wp, gh[(q * 3 + k) * NB + bn], G[k]);
            }
#pragma unroll
            for (int k = 0; k < 3; ++k) kahan_add(S[k], C[k], G[k]);
          }
#pragma unroll
          for (int jj = 0; jj < 3; ++jj) {
            Ks[(jj * NB + bn) * NLP + NV + cp] = -S[jj];
            Ks[(NV + cp) * NLP + jj * NB + bn] = -S[jj];
          }
        }
      }
      ws_compute_barrier();
      // staged cell matrix -> scratch, 16-byte coalesced (row padding copied as is)
      constexpr int N16 = NL * NLP * 4 / 16;
      const uint4* src = reinterpret_cast<const uint4*>(Ks);
      uint4* dst = reinterpret_cast<uint4*>(K + e * int64_t(NL) * NLP);
      for (int i = t; i < N16; i += L::kCompute) dst[i] = src[i];
    }
    __syncthreads();
  }
}

template <int P, typename T>
cudaError_t launch(const fe_space* s, const Params& prm, cudaStream_t st) {
  using L = Layout<P, T>;
  constexpr bool WS = P == 2 && std::is_same<T, float>::value;  // Q2/Q1 FP32: the warp-specialised kernel
  void (*kern)(Params);
  if constexpr (WS) kern = k_cell_stokes_ws; else kern = k_cell_stokes<P, T>;
  const size_t bytes = WS ? WsLayout::BYTES : L::BYTES;
  const int64_t groups = WS ? s->n_cells : (s->n_cells + L::CPB - 1) / L::CPB;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(bytes));
  if (e != cudaSuccess) return e;
  int per_sm = 0, nsm = 152;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kThreads, bytes);
  if (e != cudaSuccess) return e;
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, s->device);
  const int blocks = int(std::min<int64_t>(groups, int64_t(nsm) * std::max(1, per_sm)));
  kern<<<blocks, kThreads, bytes, st>>>(prm);
  return cudaGetLastError();
}

}  // namespace stokes

cudaError_t launch_cell_stokes(const fe_space* s, const double* coef, const double force[3], fe_precision prec,
                               cudaStream_t st) {
  if (s->n_cells == 0) return cudaSuccess;
  if (s->nl != 3 * s->nb + s->nbp || s->nq != s->nb) return cudaErrorInvalidValue;
  stokes::Params p;
  p.n_cells = s->n_cells;
  p.xv = s->d_xv;
  p.w = s->d_w;
  p.xq = s->d_xq;
  p.phi = s->d_phi;
  p.dphi = s->d_dphi;
  p.dphi32 = s->d_dphi32;
  p.psi = s->d_psi;
  p.coef = coef;
  for (int k = 0; k < 3; ++k) p.f[k] = force[k];
  p.ke = s->d_ke;
  p.fe = s->d_fe;
  p.err = s->d_err;
  const bool f64 = prec == FE_PREC_FP64;
  switch (s->order) {
    case 2: return f64 ? stokes::launch<2, double>(s, p, st) : stokes::launch<2, float>(s, p, st);
    case 3: return f64 ? stokes::launch<3, double>(s, p, st) : stokes::launch<3, float>(s, p, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace feasm

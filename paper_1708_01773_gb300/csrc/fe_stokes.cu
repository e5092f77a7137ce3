// Stokes cell integration for the Taylor-Hood pair of the paper's Stokes
// driver (Example "Stokes problem"; Sect. "Driver example for the Stokes
// problem"): velocity Q_P (3 components), pressure Q_{P-1}, (P+1)^3 Gauss
// points. With the cofactor gradients gh_a = cof(J) gradhat(phihat_a), so
// that grad(phi_a) = gh_a / det J (Eq. shape_grad):
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
// One block per cell (persistent loop); the geometry is FP64; the FP64 form
// keeps everything in FP64, the FP32 form rounds the cofactor gradients to FP32
// and sums the Gram entries in FP32 per slab of (P+1)^2 points with
// compensated (Kahan) addition of the slab sums.
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
  // shared memory: xv[24], a[21], wdet[NQ] (double); cof[NQ][9], wod[NQ], wq[NQ] (T); gh[NQ][3][NB] (T);
  // the pressure basis psi[NQ][NBP] (T)
  static constexpr size_t OFF_A = 24 * sizeof(double);
  static constexpr size_t OFF_WDET = OFF_A + 24 * sizeof(double);
  static constexpr size_t OFF_COF = OFF_WDET + NQ * sizeof(double);
  static constexpr size_t OFF_WOD = OFF_COF + size_t(NQ) * 9 * sizeof(T);
  static constexpr size_t OFF_WQ = OFF_WOD + NQ * sizeof(T);
  static constexpr size_t OFF_GH = (OFF_WQ + NQ * sizeof(T) + 15) & ~size_t(15);
  static constexpr size_t OFF_PSI = OFF_GH + size_t(NQ) * 3 * NB * sizeof(T);
  static constexpr size_t BYTES = OFF_PSI + size_t(NQ) * NBP * sizeof(T);
};

template <int P, typename T>
__global__ void __launch_bounds__(kThreads) k_cell_stokes(Params p) {
  using L = Layout<P, T>;
  constexpr int N1 = L::N1, NB = L::NB, NQ = L::NQ, NBP = L::NBP, NV = L::NV, NL = L::NL, NLP = L::NLP;
  constexpr bool F32 = std::is_same<T, float>::value;
  extern __shared__ __align__(16) unsigned char sm[];
  double* xv = reinterpret_cast<double*>(sm);
  double* a = reinterpret_cast<double*>(sm + L::OFF_A);
  double* wdet = reinterpret_cast<double*>(sm + L::OFF_WDET);
  T* cof = reinterpret_cast<T*>(sm + L::OFF_COF);
  T* wod = reinterpret_cast<T*>(sm + L::OFF_WOD);
  T* wq = reinterpret_cast<T*>(sm + L::OFF_WQ);
  T* gh = reinterpret_cast<T*>(sm + L::OFF_GH);
  T* spsi = reinterpret_cast<T*>(sm + L::OFF_PSI);
  T* K = static_cast<T*>(p.ke);
  const int t = threadIdx.x;
  for (int i = t; i < NQ * NBP; i += kThreads) spsi[i] = T(p.psi[i]);
  for (int64_t e = blockIdx.x; e < p.n_cells; e += gridDim.x) {
    if (t < 24) xv[t] = p.xv[e * 24 + t];
    __syncthreads();
    if (t < 3) trilinear_coefficients(xv, t, a);
    __syncthreads();
    // 1. geometry per quadrature point (FP64)
    if (t < NQ) {
      double c[9], det;
      geometry_at(a, p.xq[3 * t], p.xq[3 * t + 1], p.xq[3 * t + 2], c, &det);
      if (!(det > 0.0)) atomicOr(p.err, kErrNegJacobian);
      const double w = p.w[t];
      wdet[t] = w * det;
      wod[t] = T(w / det);
      wq[t] = T(w);
#pragma unroll
      for (int k = 0; k < 9; ++k) cof[t * 9 + k] = T(c[k]);
    }
    __syncthreads();
    // 2. cofactor gradients gh[q][k][a] = sum_d cof[q][k][d] gradhat_d phihat_a(x_q)
    for (int i = t; i < NQ * NB; i += kThreads) {
      const int q = i / NB, b = i % NB;
      T g[3];
      if constexpr (F32) {
        g[0] = p.dphi32[3 * i]; g[1] = p.dphi32[3 * i + 1]; g[2] = p.dphi32[3 * i + 2];
      } else {
        g[0] = p.dphi[3 * i]; g[1] = p.dphi[3 * i + 1]; g[2] = p.dphi[3 * i + 2];
      }
      const T* cq = cof + q * 9;
#pragma unroll
      for (int k = 0; k < 3; ++k) gh[(q * 3 + k) * NB + b] = cq[3 * k] * g[0] + cq[3 * k + 1] * g[1] + cq[3 * k + 2] * g[2];
    }
    __syncthreads();
    const T mu_half = T(0.5 * p.coef[e]);
    T* Ke = K + e * int64_t(NL) * NLP;
    // 3. velocity-velocity block, one node pair per item
    for (int i = t; i < NB * NB; i += kThreads) {
      const int an = i / NB, bn = i % NB;
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
          const T wv = wod[q];
          T ga[3], gb[3];
#pragma unroll
          for (int k = 0; k < 3; ++k) {
            ga[k] = wv * gh[(q * 3 + k) * NB + an];
            gb[k] = gh[(q * 3 + k) * NB + bn];
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
      const T tr = S[0][0] + S[1][1] + S[2][2];
#pragma unroll
      for (int ii = 0; ii < 3; ++ii)
#pragma unroll
        for (int jj = 0; jj < 3; ++jj) {
          T v = S[jj][ii];
          if (ii == jj) v += tr;
          Ke[size_t(ii * NB + an) * NLP + jj * NB + bn] = mu_half * v;
        }
    }
    // 4. pressure coupling, one (pressure node, velocity node) pair per item
    for (int i = t; i < NBP * NB; i += kThreads) {
      const int c = i / NB, bn = i % NB;
      T S[3] = {T(0), T(0), T(0)}, C[3] = {T(0), T(0), T(0)};
      for (int s0 = 0; s0 < NQ; s0 += N1 * N1) {
        T G[3] = {T(0), T(0), T(0)};
        for (int q = s0; q < s0 + N1 * N1; ++q) {
          const T wp = wq[q] * spsi[q * NBP + c];
#pragma unroll
          for (int k = 0; k < 3; ++k) G[k] = fma(wp, gh[(q * 3 + k) * NB + bn], G[k]);
        }
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          if constexpr (F32) kahan_add(S[k], C[k], G[k]); else S[k] += G[k];
        }
      }
#pragma unroll
      for (int jj = 0; jj < 3; ++jj) {
        Ke[size_t(jj * NB + bn) * NLP + NV + c] = -S[jj];
        Ke[size_t(NV + c) * NLP + jj * NB + bn] = -S[jj];
      }
    }
    // 5. pressure-pressure block
    for (int i = t; i < NBP * NBP; i += kThreads) Ke[size_t(NV + i / NBP) * NLP + NV + i % NBP] = T(0);
    // 6. cell vector (FP64)
    if (t < NB) {
      double s = 0.0;
      for (int q = 0; q < NQ; ++q) s = fma(wdet[q], p.phi[q * NB + t], s);
      double* fe = p.fe + e * NL;
#pragma unroll
      for (int ii = 0; ii < 3; ++ii) fe[ii * NB + t] = p.f[ii] * s;
    } else if (t < NB + NBP) {
      p.fe[e * NL + NV + (t - NB)] = 0.0;
    }
    __syncthreads();
  }
}

template <int P, typename T>
cudaError_t launch(const fe_space* s, const Params& prm, cudaStream_t st) {
  using L = Layout<P, T>;
  auto kern = k_cell_stokes<P, T>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(L::BYTES));
  if (e != cudaSuccess) return e;
  int per_sm = 0, nsm = 152;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kThreads, L::BYTES);
  if (e != cudaSuccess) return e;
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, s->device);
  const int blocks = int(std::min<int64_t>(s->n_cells, int64_t(nsm) * std::max(1, per_sm)));
  kern<<<blocks, kThreads, L::BYTES, st>>>(prm);
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

// CUDA kernels of libfeasm (sm_103a): cell integration (geometry, physical
// gradients, cell-matrix contraction, cell vectors), the deterministic
// segmented scatter into CSR, and the compliance adjoint.
#include <cuda_bf16.h>

#include <type_traits>

#include "fe_launch.h"

namespace feasm {

constexpr int kCellThreads = 256;
constexpr int kScatterWarps = 8;

int cells_per_block(int nb) {
  const int pairs = nb * nb;
  return pairs >= kCellThreads ? 1 : kCellThreads / pairs;
}

// Shared memory of k_cell: vertex coordinates [cpb][24], trilinear
// coefficients [cpb][21], per-point geometry [cpb][nq][11] (cofactor matrix,
// w/det, w*det) in FP64, for the FP32/BF16 forms an FP32 copy [cpb][nq][12]
// of the cofactors and w/det, and the cofactor-scaled reference gradients
// [cpb][nq][3][nb] in the operand type.
long cell_smem_bytes(int nb, int nq, fe_precision prec, int cpb) {
  const long tsz = prec == FE_PREC_FP64 ? 8 : 4;
  long bytes = long(cpb) * (24 + 21) * 8 + long(cpb) * nq * 11 * 8 + long(cpb) * nq * 3 * nb * tsz;
  if (prec != FE_PREC_FP64) bytes += long(cpb) * nq * 12 * 4;
  return bytes <= 227 * 1024 ? bytes : -1;
}

struct CellParams {
  int64_t n_cells;
  int nq, cpb, qblock;
  const double* xv;
  const double* w;
  const double* xq;
  const double* phi;
  const double* dphi;
  const float* dphi32;
  const double* coef;
  double f[3];
  double lam_hat, mu_hat;
  void* ke;
  double* fe;
  int* err;
};

__device__ __forceinline__ float round_bf16(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }

// Trilinear map Phi(x) = a0 + a1 x + a2 y + a3 z + a4 xy + a5 xz + a6 yz + a7 xyz
// (the Q1 geometry of the cell written in monomials). Its Jacobian at a
// point, the cofactor matrix and the determinant, all FP64:
//   J[k][d] = dPhi_k / dxhat_d,  cof[k][d] = cofactor of J[k][d],
//   det J = sum_d J[0][d] cof[0][d],  J^{-T} = cof / det.
__device__ __forceinline__ void geometry_at(const double* a, double x, double y, double z, double cof[9],
                                            double* det) {
  double J[3][3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const double a1 = a[0 + k], a2 = a[3 + k], a3 = a[6 + k], a4 = a[9 + k], a5 = a[12 + k], a6 = a[15 + k],
                 a7 = a[18 + k];
    J[k][0] = a1 + a4 * y + a5 * z + a7 * (y * z);
    J[k][1] = a2 + a4 * x + a6 * z + a7 * (x * z);
    J[k][2] = a3 + a5 * x + a6 * y + a7 * (x * y);
  }
  cof[0] = J[1][1] * J[2][2] - J[1][2] * J[2][1];
  cof[1] = J[1][2] * J[2][0] - J[1][0] * J[2][2];
  cof[2] = J[1][0] * J[2][1] - J[1][1] * J[2][0];
  cof[3] = J[0][2] * J[2][1] - J[0][1] * J[2][2];
  cof[4] = J[0][0] * J[2][2] - J[0][2] * J[2][0];
  cof[5] = J[0][1] * J[2][0] - J[0][0] * J[2][1];
  cof[6] = J[0][1] * J[1][2] - J[0][2] * J[1][1];
  cof[7] = J[0][2] * J[1][0] - J[0][0] * J[1][2];
  cof[8] = J[0][0] * J[1][1] - J[0][1] * J[1][0];
  *det = J[0][0] * cof[0] + J[0][1] * cof[1] + J[0][2] * cof[2];
}

// Monomial coefficients a1..a7 (3 components each) from the 8 vertices in
// x-fastest order.
__device__ __forceinline__ void trilinear_coefficients(const double* x, int k, double* a) {
  const double x0 = x[k], x1 = x[3 + k], x2 = x[6 + k], x3 = x[9 + k], x4 = x[12 + k], x5 = x[15 + k],
               x6 = x[18 + k], x7 = x[21 + k];
  const double d10 = x1 - x0, d32 = x3 - x2, d54 = x5 - x4, d76 = x7 - x6, d20 = x2 - x0, d64 = x6 - x4;
  a[0 + k] = d10;
  a[3 + k] = d20;
  a[6 + k] = x4 - x0;
  a[9 + k] = d32 - d10;
  a[12 + k] = d54 - d10;
  a[15 + k] = d64 - d20;
  a[18 + k] = (d76 - d54) - (d32 - d10);
}

// Compensated (Kahan) addition of a block partial into (sum, carry).
template <typename T>
__device__ __forceinline__ void kahan_add(T& sum, T& carry, T part) {
  const T y = part - carry;
  const T t = sum + y;
  carry = (t - sum) - y;
  sum = t;
}

// One block integrates `cpb` cells. Steps (paper: Eq. fematrix, Eq.
// shape_grad, the element loop of the Listing
// "element_matrix_entries_computation"):
//   1. geometry at every quadrature point (FP64),
//   2. cofactor gradients gh_a = cof(J) gradhat(phihat_a), so that
//      grad(phi_a) = gh_a / det J,
//   3. G^{ij}_{ab} = sum_q (w_q / det J_q) gh_{a,i} gh_{b,j}, and
//      Poisson   K_ab = kappa sum_i G^{ii}_{ab},
//      elasticity K_(a,i),(b,j) = E (lam^ G^{ij}_ab + mu^ G^{ji}_ab + mu^ d_ij sum_k G^{kk}_ab),
//   4. cell vector f_(a,i) = f_i sum_q w_q det J_q phihat_a(x_q).
// PREC 0: FP64 throughout. PREC 1: FP32 gradients and products; the sum over
// quadrature points runs in blocks of `qblock` points (one z-slab of the
// tensor rule) whose FP32 partials are added with Kahan compensation. PREC 2:
// BF16-rounded operands, FP32 products and sums. Cell matrices are stored
// row-major with row stride NLP (16-byte aligned rows).
// cell_block integrates cells e0 .. e0 + ncell - 1 (ncell <= prm.cpb) with the
// whole thread block, using `smem` (cell_smem_bytes) as scratch; k_cell runs
// one such block per thread block, the batched driver any number of them.
template <int P, int NC, int PREC>
__device__ __forceinline__ void cell_block(const CellParams& prm, int64_t e0, int ncell, double* smem) {
  constexpr int NB = (P + 1) * (P + 1) * (P + 1);
  constexpr int NL = NC * NB;
  constexpr int NLP = (NL + 3) & ~3;
  using T = typename std::conditional<PREC == 0, double, float>::type;
  const int cpb = prm.cpb, nq = prm.nq;
  double* sx = smem;
  double* sa = sx + cpb * 24;
  double* geo = sa + cpb * 21;
  float* geo32 = reinterpret_cast<float*>(geo + cpb * nq * 11);
  T* g = reinterpret_cast<T*>(PREC == 0 ? reinterpret_cast<float*>(geo + cpb * nq * 11) : geo32 + cpb * nq * 12);
  const int tid = threadIdx.x;

  for (int i = tid; i < ncell * 24; i += blockDim.x) sx[i] = prm.xv[e0 * 24 + i];
  __syncthreads();
  for (int i = tid; i < ncell * 3; i += blockDim.x) trilinear_coefficients(sx + (i / 3) * 24, i % 3, sa + (i / 3) * 21);
  __syncthreads();
  for (int i = tid; i < ncell * nq; i += blockDim.x) {
    const int c = i / nq, q = i % nq;
    double cof[9], det;
    geometry_at(sa + c * 21, prm.xq[3 * q], prm.xq[3 * q + 1], prm.xq[3 * q + 2], cof, &det);
    if (!(det > 0.0)) atomicOr(prm.err, kErrNegJacobian);
    const double wq = prm.w[q];
    double* gm = geo + size_t(i) * 11;
#pragma unroll
    for (int t = 0; t < 9; ++t) gm[t] = cof[t];
    gm[9] = wq / det;
    gm[10] = wq * det;
    if (PREC != 0) {
      float* g32 = geo32 + size_t(i) * 12;
#pragma unroll
      for (int t = 0; t < 9; ++t) g32[t] = float(cof[t]);
      g32[9] = float(wq / det);
    }
  }
  __syncthreads();
  for (int i = tid; i < ncell * nq * NB; i += blockDim.x) {
    const int a = i % NB, cq = i / NB, q = cq % nq;
    T* gg = g + size_t(cq) * 3 * NB;
    if (PREC == 0) {
      const double* gm = geo + size_t(cq) * 11;
      const double* dp = prm.dphi + (size_t(q) * NB + a) * 3;
#pragma unroll
      for (int k = 0; k < 3; ++k) gg[k * NB + a] = gm[3 * k] * dp[0] + gm[3 * k + 1] * dp[1] + gm[3 * k + 2] * dp[2];
    } else {
      const float* gm = geo32 + size_t(cq) * 12;
      const float* dp = prm.dphi32 + (size_t(q) * NB + a) * 3;
      const float d0 = dp[0], d1 = dp[1], d2 = dp[2];
#pragma unroll
      for (int k = 0; k < 3; ++k) gg[k * NB + a] = T(fmaf(gm[3 * k + 2], d2, fmaf(gm[3 * k + 1], d1, gm[3 * k] * d0)));
    }
  }
  __syncthreads();
  const int qb = PREC == 1 ? prm.qblock : nq;
  for (int i = tid; i < ncell * NB * NB; i += blockDim.x) {
    const int c = i / (NB * NB), ab = i % (NB * NB), a = ab / NB, b = ab % NB;
    const T* gc = g + size_t(c) * nq * 3 * NB;
    const double* gm = geo + size_t(c) * nq * 11;
    const float* gm32 = geo32 + size_t(c) * nq * 12;
    const int64_t e = e0 + c;
    const double coef = prm.coef[e];
    T* K = reinterpret_cast<T*>(prm.ke) + e * NL * NLP;
    if (NC == 1) {
      T sum = T(0), carry = T(0);
      for (int q0 = 0; q0 < nq; q0 += qb) {
        T part = T(0);
        const int q1 = q0 + qb < nq ? q0 + qb : nq;
        for (int q = q0; q < q1; ++q) {
          const T* gq = gc + size_t(q) * 3 * NB;
          const T s = PREC == 0 ? T(gm[q * 11 + 9]) : T(gm32[q * 12 + 9]);
#pragma unroll
          for (int k = 0; k < 3; ++k) {
            T ga = s * gq[k * NB + a], gb = gq[k * NB + b];
            if (PREC == 2) { ga = round_bf16(ga); gb = round_bf16(gb); }
            part += ga * gb;
          }
        }
        if (PREC == 1) kahan_add(sum, carry, part); else sum += part;
      }
      K[a * NLP + b] = T(coef) * sum;
    } else {
      T S[3][3], C[3][3];
#pragma unroll
      for (int i2 = 0; i2 < 3; ++i2)
#pragma unroll
        for (int j2 = 0; j2 < 3; ++j2) S[i2][j2] = C[i2][j2] = T(0);
      for (int q0 = 0; q0 < nq; q0 += qb) {
        T G[3][3];
#pragma unroll
        for (int i2 = 0; i2 < 3; ++i2)
#pragma unroll
          for (int j2 = 0; j2 < 3; ++j2) G[i2][j2] = T(0);
        const int q1 = q0 + qb < nq ? q0 + qb : nq;
        for (int q = q0; q < q1; ++q) {
          const T* gq = gc + size_t(q) * 3 * NB;
          const T s = PREC == 0 ? T(gm[q * 11 + 9]) : T(gm32[q * 12 + 9]);
          T ga[3], gb[3];
#pragma unroll
          for (int k = 0; k < 3; ++k) {
            ga[k] = s * gq[k * NB + a];
            gb[k] = gq[k * NB + b];
            if (PREC == 2) { ga[k] = round_bf16(ga[k]); gb[k] = round_bf16(gb[k]); }
          }
#pragma unroll
          for (int i2 = 0; i2 < 3; ++i2)
#pragma unroll
            for (int j2 = 0; j2 < 3; ++j2) G[i2][j2] += ga[i2] * gb[j2];
        }
#pragma unroll
        for (int i2 = 0; i2 < 3; ++i2)
#pragma unroll
          for (int j2 = 0; j2 < 3; ++j2) {
            if (PREC == 1) kahan_add(S[i2][j2], C[i2][j2], G[i2][j2]); else S[i2][j2] += G[i2][j2];
          }
      }
      const T lh = T(prm.lam_hat), mh = T(prm.mu_hat), E = T(coef);
      const T tr = S[0][0] + S[1][1] + S[2][2];
#pragma unroll
      for (int i2 = 0; i2 < 3; ++i2)
#pragma unroll
        for (int j2 = 0; j2 < 3; ++j2) {
          T v = lh * S[i2][j2] + mh * S[j2][i2];
          if (i2 == j2) v += mh * tr;
          K[size_t(i2 * NB + a) * NLP + j2 * NB + b] = E * v;
        }
    }
  }
  for (int i = tid; i < ncell * NB; i += blockDim.x) {
    const int c = i / NB, a = i % NB;
    const double* gm = geo + size_t(c) * nq * 11;
    double f = 0.0;
    for (int q = 0; q < nq; ++q) f += gm[q * 11 + 10] * prm.phi[size_t(q) * NB + a];
    double* fe = prm.fe + (e0 + c) * NL;
#pragma unroll
    for (int k = 0; k < NC; ++k) fe[k * NB + a] = prm.f[k] * f;
  }
}

template <int P, int NC, int PREC>
__global__ void __launch_bounds__(kCellThreads) k_cell(CellParams prm) {
  extern __shared__ __align__(16) double smem[];
  const int64_t e0 = int64_t(blockIdx.x) * prm.cpb;
  const int ncell = int(prm.n_cells - e0 < prm.cpb ? prm.n_cells - e0 : prm.cpb);
  cell_block<P, NC, PREC>(prm, e0, ncell, smem);
}

template <int P, int NC, int PREC>
static cudaError_t launch_cell_t(const fe_space* s, const CellParams& prm, long smem, cudaStream_t st) {
  auto kern = k_cell<P, NC, PREC>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
  if (e != cudaSuccess) return e;
  const int64_t blocks = (s->n_cells + prm.cpb - 1) / prm.cpb;
  kern<<<dim3(unsigned(blocks)), kCellThreads, size_t(smem), st>>>(prm);
  return cudaGetLastError();
}

template <int P, int NC>
static cudaError_t launch_cell_p(const fe_space* s, const CellParams& prm, long smem, fe_precision prec,
                                 cudaStream_t st) {
  switch (prec) {
    case FE_PREC_FP64: return launch_cell_t<P, NC, 0>(s, prm, smem, st);
    case FE_PREC_FP32: return launch_cell_t<P, NC, 1>(s, prm, smem, st);
    default: return launch_cell_t<P, NC, 2>(s, prm, smem, st);
  }
}

cudaError_t launch_cell_integration(const fe_space* s, const double* coef, const double force[3],
                                    fe_precision prec, cudaStream_t st) {
  if (s->n_cells == 0) return cudaSuccess;
  CellParams prm;
  prm.n_cells = s->n_cells;
  prm.nq = s->nq;
  prm.cpb = cells_per_block(s->nb);
  prm.qblock = s->nq1d * s->nq1d;
  prm.xv = s->d_xv;
  prm.w = s->d_w;
  prm.xq = s->d_xq;
  prm.phi = s->d_phi;
  prm.dphi = s->d_dphi;
  prm.dphi32 = s->d_dphi32;
  prm.coef = coef;
  for (int k = 0; k < 3; ++k) prm.f[k] = force[k];
  prm.lam_hat = s->nu / ((1.0 + s->nu) * (1.0 - 2.0 * s->nu));
  prm.mu_hat = 1.0 / (2.0 * (1.0 + s->nu));
  prm.ke = s->d_ke;
  prm.fe = s->d_fe;
  prm.err = s->d_err;
  const long smem = cell_smem_bytes(s->nb, s->nq, prec, prm.cpb);
  if (smem < 0) return cudaErrorInvalidConfiguration;
  const int key = s->order * 10 + s->ncomp;
  switch (key) {
    case 11: return launch_cell_p<1, 1>(s, prm, smem, prec, st);
    case 13: return launch_cell_p<1, 3>(s, prm, smem, prec, st);
    case 21: return launch_cell_p<2, 1>(s, prm, smem, prec, st);
    case 23: return launch_cell_p<2, 3>(s, prm, smem, prec, st);
    case 31: return launch_cell_p<3, 1>(s, prm, smem, prec, st);
    case 33: return launch_cell_p<3, 3>(s, prm, smem, prec, st);
    default: return cudaErrorInvalidValue;
  }
}

// ---------------------------------------------------------------------------
// Deterministic scatter (Eq. assembly). One warp assembles one CSR row r at a
// time. The row's contributions are its codes, sorted by destination nonzero
// (columns ascending) and, within a nonzero, by ascending cell; a code
// (head << 15 | s << 8 | m) names entry m of the cell-matrix row of DOF r in
// the row's s-th cell ("slot"), head marking the first contribution of a
// nonzero.
//
// Exact FP64 accumulation without FP64 arithmetic. The FP64 pipe of this GPU
// is a small fraction of its FP32/INT32 rate, so each nonzero is summed in
// 64-bit integer fixed point: every term is split into sign, exponent and
// integer mantissa, the mantissas are aligned to the largest exponent of the
// nonzero (the largest term's leading bit at bit 57, so that up to 32 terms
// cannot overflow) and added as int64, and the integer sum is rounded once to
// the nearest double. Bits lost in the alignment are below 2^-57 of the
// largest term, so the result is at least as accurate as sequential FP64
// additions, is independent of the order of the terms, and is bitwise
// reproducible. A nonzero with a single FP32 term takes the exact FP32->FP64
// conversion, done on the integer bits.
template <typename TK>
struct FxTraits;
template <>
struct FxTraits<float> {
  // value = mant * 2^(ex - 150), mant < 2^24; aligned mantissa MSB at bit 57
  static constexpr int kShift0 = 34, kScale = 184;
  __device__ static __forceinline__ void split(float x, uint64_t& m, int& ex, bool& neg) {
    const uint32_t u = __float_as_uint(x);
    neg = (u >> 31) != 0;
    int e = int((u >> 23) & 0xffu);
    uint32_t mm = u & 0x7fffffu;
    if (e) mm |= 0x800000u; else e = 1;
    m = mm;
    ex = e;
  }
};
template <>
struct FxTraits<double> {
  // value = mant * 2^(ex - 1075), mant < 2^53; aligned mantissa MSB at bit 57
  static constexpr int kShift0 = 5, kScale = 1080;
  __device__ static __forceinline__ void split(double x, uint64_t& m, int& ex, bool& neg) {
    const uint64_t u = uint64_t(__double_as_longlong(x));
    neg = (u >> 63) != 0;
    int e = int((u >> 52) & 0x7ffu);
    uint64_t mm = u & 0xfffffffffffffull;
    if (e) mm |= 1ull << 52; else e = 1;
    m = mm;
    ex = e;
  }
};

// Rounds the integer S * 2^scale to the nearest double (ties to even).
__device__ __forceinline__ double fx_to_double(int64_t S, int scale) {
  if (S == 0) return 0.0;
  const bool neg = S < 0;
  const uint64_t mag = neg ? uint64_t(-S) : uint64_t(S);
  int lz = __clzll(static_cast<long long>(mag));
  const uint64_t norm = mag << lz;
  uint64_t mant = norm >> 11;
  const uint32_t rem = uint32_t(norm & 0x7ffu);
  if (rem > 0x400u || (rem == 0x400u && (mant & 1u))) ++mant;
  if (mant >> 53) {
    mant >>= 1;
    --lz;
  }
  const int biased = 63 - lz + scale + 1023;
  if (biased <= 0) return neg ? -0.0 : 0.0;
  if (biased >= 2047) return neg ? -__longlong_as_double(0x7ff0000000000000ll) : __longlong_as_double(0x7ff0000000000000ll);
  const uint64_t bits = (uint64_t(neg) << 63) | (uint64_t(biased) << 52) | (mant & 0xfffffffffffffull);
  return __longlong_as_double(static_cast<long long>(bits));
}

// Exact FP32 -> FP64 conversion on the integer bits (normal numbers and zero).
__device__ __forceinline__ bool f32_to_f64_bits(float x, double& out) {
  const uint32_t u = __float_as_uint(x);
  const uint32_t e = (u >> 23) & 0xffu;
  if ((u & 0x7fffffffu) == 0) {
    out = (u >> 31) ? -0.0 : 0.0;
    return true;
  }
  if (e == 0 || e == 0xffu) return false;
  const uint64_t bits = (uint64_t(u >> 31) << 63) | (uint64_t(e + 896u) << 52) | (uint64_t(u & 0x7fffffu) << 29);
  out = __longlong_as_double(static_cast<long long>(bits));
  return true;
}

// Sum of n terms produced by get(t), t = 0..n-1, accumulated exactly as above.
template <typename TK, typename Get>
__device__ __forceinline__ double fx_sum(int n, Get get) {
  using Tr = FxTraits<TK>;
  if (n == 1) {
    const TK x = get(0);
    if (sizeof(TK) == 8) return double(x);
    double d;
    if (f32_to_f64_bits(float(x), d)) return d;
  }
  int emax = 1;
  for (int t = 0; t < n; ++t) {
    uint64_t m;
    int ex;
    bool ng;
    Tr::split(get(t), m, ex, ng);
    if (m != 0 && ex > emax) emax = ex;
  }
  int64_t S = 0;
  for (int t = 0; t < n; ++t) {
    uint64_t m;
    int ex;
    bool ng;
    Tr::split(get(t), m, ex, ng);
    const int sh = Tr::kShift0 - (emax - ex);
    const uint64_t a = sh >= 0 ? (m << sh) : (sh > -64 ? (m >> (-sh)) : 0ull);
    S += ng ? -int64_t(a) : int64_t(a);
  }
  return fx_to_double(S, emax - Tr::kScale);
}

// k_scatter_rows copies the row's cell-matrix rows (padded to NLP entries,
// 16-byte vector loads) and its codes (16-byte aligned blocks) into a
// per-warp region of shared memory, finds the segment starts from the head
// flags with one ballot per 32 codes, then gives each lane one nonzero: the
// lane sums its segment from shared memory and stores values[k] (consecutive
// k across the lanes: coalesced). The RHS entry of the row is the exact sum of
// its cells' FP64 cell-vector entries.
//
// k_scatter (one lane per nonzero, direct gathers from global memory, using
// the per-nonzero counts, same arithmetic) serves meshes whose largest row does
// not fit the shared-memory region or that have more than 32 cells around a DOF.
struct ScatterParams {
  int64_t n_rows;
  int nl, nlp;
  const int64_t* row_ptr;
  const uint8_t* cnt;
  const int64_t* code_ptr;
  const uint16_t* codes;
  const uint16_t* pos;
  const int64_t* slot_ptr;
  const int32_t* slots;
  const void* ke;
  const double* fe;
  double* values;
  double* rhs;
  int ke_bytes, code_bytes, warp_bytes, acc_stride;
};

constexpr unsigned kFull = 0xffffffffu;

template <typename TK>
__global__ void __launch_bounds__(kScatterWarps * 32) k_scatter(ScatterParams p) {
  __shared__ int64_t sbase[kScatterWarps][kMaxSlots + 1];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const TK* ke = reinterpret_cast<const TK*>(p.ke);
  for (int64_t r = int64_t(blockIdx.x) * kScatterWarps + warp; r < p.n_rows;
       r += int64_t(gridDim.x) * kScatterWarps) {
    const int64_t s0 = p.slot_ptr[r];
    const int ns = int(p.slot_ptr[r + 1] - s0);
    for (int s = lane; s < ns; s += 32) sbase[warp][s] = int64_t(p.slots[s0 + s]) * p.nlp;
    __syncwarp();
    if (p.rhs != nullptr && lane == 0)
      p.rhs[r] = fx_sum<double>(ns, [&](int t) { return p.fe[p.slots[s0 + t]]; });
    const int64_t k0 = p.row_ptr[r], k1 = p.row_ptr[r + 1];
    int64_t c = p.code_ptr[r];
    for (int64_t kb = k0; kb < k1; kb += 32) {
      const int64_t k = kb + lane;
      const int n = k < k1 ? int(p.cnt[k]) : 0;
      int incl = n;
#pragma unroll
      for (int off = 1; off < 32; off <<= 1) {
        const int t = __shfl_up_sync(kFull, incl, off);
        if (lane >= off) incl += t;
      }
      const int total = __shfl_sync(kFull, incl, 31);
      const uint16_t* cp = p.codes + c + (incl - n);
      if (k < k1) {
        p.values[k] = fx_sum<TK>(n, [&](int t) {
          const unsigned code = cp[t];
          return ke[sbase[warp][(code >> 8) & 127u] + (code & 255u)];
        });
      }
      c += total;
    }
    __syncwarp();
  }
}

template <typename TK>
__global__ void __launch_bounds__(kScatterWarps * 32) k_scatter_rows(ScatterParams p) {
  extern __shared__ __align__(16) unsigned char sm[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  unsigned char* region = sm + size_t(warp) * p.warp_bytes;
  TK* ske = reinterpret_cast<TK*>(region);
  uint16_t* scode = reinterpret_cast<uint16_t*>(region + p.ke_bytes);
  uint16_t* sseg = reinterpret_cast<uint16_t*>(region + p.ke_bytes + p.code_bytes);
  const int vper = p.nlp * int(sizeof(TK)) / 16;  // 16-byte vectors per cell-matrix row
  const uint4* ke4 = reinterpret_cast<const uint4*>(p.ke);
  const unsigned lt_mask = (1u << lane) - 1u;
  for (int64_t r = int64_t(blockIdx.x) * kScatterWarps + warp; r < p.n_rows;
       r += int64_t(gridDim.x) * kScatterWarps) {
    const int64_t s0 = p.slot_ptr[r];
    const int ns = int(p.slot_ptr[r + 1] - s0);
    const int64_t k0 = p.row_ptr[r];
    const int64_t c0 = p.code_ptr[r];
    const int nc = ns * p.nl;
    const int my_slot = lane < ns ? p.slots[s0 + lane] : 0;
    const uint4* c4 = reinterpret_cast<const uint4*>(p.codes + c0);
    const int nc8 = (nc + 7) >> 3;
    for (int i = lane; i < nc8; i += 32) reinterpret_cast<uint4*>(scode)[i] = __ldg(c4 + i);
    const int nv = ns * vper;
    for (int base = 0; base < nv; base += 32) {
      const int i = base + lane;
      const int s = min(i / vper, ns - 1);
      const int sid = __shfl_sync(kFull, my_slot, s);
      if (i < nv) reinterpret_cast<uint4*>(ske)[i] = __ldg(ke4 + int64_t(sid) * vper + (i - s * vper));
    }
    if (p.rhs != nullptr) {
      // the same exact fixed-point sum, the terms spread over the lanes
      uint64_t m = 0;
      int ex = 1;
      bool ng = false;
      if (lane < ns) FxTraits<double>::split(p.fe[my_slot], m, ex, ng);
      const int emax = __reduce_max_sync(kFull, m != 0 ? ex : 1);
      const int sh = FxTraits<double>::kShift0 - (emax - ex);
      const uint64_t a = sh >= 0 ? (m << sh) : (sh > -64 ? (m >> (-sh)) : 0ull);
      int64_t S = ng ? -int64_t(a) : int64_t(a);
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) S += __shfl_xor_sync(kFull, S, off);
      if (lane == 0) p.rhs[r] = fx_to_double(S, emax - FxTraits<double>::kScale);
    }
    __syncwarp();
    int heads = 0;
    for (int cb = 0; cb < nc; cb += 32) {
      const int i = cb + lane;
      const bool h = i < nc && (scode[i] & 0x8000u) != 0;
      const unsigned m = __ballot_sync(kFull, h);
      if (h) sseg[heads + __popc(m & lt_mask)] = uint16_t(i);
      heads += __popc(m);
    }
    if (lane == 0) sseg[heads] = uint16_t(nc);
    __syncwarp();
    for (int k = lane; k < heads; k += 32) {
      const int a = sseg[k], b = sseg[k + 1];
      p.values[k0 + k] = fx_sum<TK>(b - a, [&](int t) {
        const unsigned code = scode[a + t];
        return ske[((code >> 8) & 127u) * p.nlp + (code & 255u)];
      });
    }
    __syncwarp();
  }
}

// Exact RHS entry of row r: the cells' FP64 cell-vector entries, one per lane
// (lanes < ns), summed in integer fixed point across the warp.
__device__ __forceinline__ void rhs_row(const ScatterParams& p, int64_t r, int ns, int my_slot, int lane) {
  uint64_t m = 0;
  int ex = 1;
  bool ng = false;
  if (lane < ns) FxTraits<double>::split(p.fe[my_slot], m, ex, ng);
  const int emax = __reduce_max_sync(kFull, m != 0 ? ex : 1);
  const int sh = FxTraits<double>::kShift0 - (emax - ex);
  const uint64_t a = sh >= 0 ? (m << sh) : (sh > -64 ? (m >> (-sh)) : 0ull);
  int64_t S = ng ? -int64_t(a) : int64_t(a);
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) S += __shfl_xor_sync(kFull, S, off);
  if (lane == 0) p.rhs[r] = fx_to_double(S, emax - FxTraits<double>::kScale);
}

// Exact FP32 -> FP64 conversion of any finite float on the integer bits
// (denormals included), without the FP64 pipe.
__device__ __forceinline__ double f32_to_f64_exact(float x) {
  double d;
  if (f32_to_f64_bits(x, d)) return d;
  uint64_t m;
  int ex;
  bool ng;
  FxTraits<float>::split(x, m, ex, ng);
  return fx_to_double(ng ? -int64_t(m) : int64_t(m), ex - 150);
}

// FP32 -> FP64 bits for zero and normal numbers (exponent rebias by 1023 - 127
// = 896 on the shifted exponent/mantissa field); `ok` is cleared for
// denormals, infinities and NaNs, which take the general path.
__device__ __forceinline__ double f32_to_f64_fast(float x, bool& ok) {
  const uint32_t u = __float_as_uint(x);
  const uint32_t mag = u & 0x7fffffffu;
  const uint32_t e = mag >> 23;
  ok = ok && (mag == 0 || (e != 0 && e != 0xffu));
  const uint64_t body = mag == 0 ? 0ull : ((uint64_t(mag) << 29) + (uint64_t(896) << 52));
  return __longlong_as_double(static_cast<long long>((uint64_t(u >> 31) << 63) | body));
}

// Aligned integer mantissa for the two-term sum below: m * 2^sh, with the bits
// shifted out (sh < 0) folded into a sticky lowest bit.
__device__ __forceinline__ uint64_t fx_align_sticky(uint64_t m, int sh) {
  if (sh >= 0) return m << sh;
  if (sh <= -64) return m != 0 ? 1ull : 0ull;
  const uint64_t kept = m >> (-sh);
  return kept | ((m & ((1ull << (-sh)) - 1ull)) != 0 ? 1ull : 0ull);
}

// hi + lo of a double-float accumulator, rounded once to the nearest double:
// both parts convert exactly on the integer bits, and one FP64 addition
// (only where lo is non-zero) rounds their exact sum.
__device__ __forceinline__ double df_to_double(float hi, float lo) {
  bool ok = true;
  double dh = f32_to_f64_fast(hi, ok);
  if (lo == 0.f && ok) return dh;
  double dl = f32_to_f64_fast(lo, ok);
  if (!ok) {
    dh = f32_to_f64_exact(hi);
    dl = f32_to_f64_exact(lo);
  }
  return __dadd_rn(dh, dl);
}

// Slot-wise scatter for FP32 cell matrices (the FP32 and BF16 forms). One warp
// per CSR row r: for each cell around DOF r in ascending order ("slot"), the
// lanes read that cell's matrix row (coalesced) and the slot-major positions
// pos[s][m] of its entries among the row's nonzeros, and add each entry into
// a per-row double-float accumulator (hi, lo) in shared memory with Knuth's
// TwoSum (the rounding error of every addition is kept exactly in lo). The
// entries of one cell row go to distinct nonzeros, so the lanes never collide;
// a __syncwarp between slots orders the additions, so every nonzero sums its
// terms in ascending cell order. The accumulator is rounded once to FP64
// (df_to_double) and stored coalesced. Lanes past the end of a cell row
// (m >= NL) read padding and add zero into a private dummy accumulator, so the
// inner loop has no divergent branches (the position array and the
// cell-matrix scratch are allocated with enough padding for those reads).
// Global loads of up to SB slots are issued before their additions, and the
// row descriptors (pointers, slot ids) of the warp's next row are fetched
// while the current row is reduced.
template <int NL, bool IDX32>
__global__ void __launch_bounds__(kScatterWarps * 32, 5) k_scatter_slots(ScatterParams p) {
  constexpr int CH = (NL + 31) / 32;
  constexpr int SB = CH >= 3 ? 4 : 8;
  extern __shared__ __align__(16) unsigned char sm[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  float2* acc = reinterpret_cast<float2*>(sm + size_t(warp) * p.warp_bytes);
  const int dummy = p.acc_stride + lane;
  const float* ke = reinterpret_cast<const float*>(p.ke) + lane;
  const int64_t stride = int64_t(gridDim.x) * kScatterWarps;
  int64_t r = int64_t(blockIdx.x) * kScatterWarps + warp;
  int64_t s0 = 0, k0 = 0, c0 = 0;
  int ns = 0, nnz = 0, my_slot = 0;
  if (r < p.n_rows) {
    s0 = p.slot_ptr[r];
    ns = int(p.slot_ptr[r + 1] - s0);
    k0 = p.row_ptr[r];
    nnz = int(p.row_ptr[r + 1] - k0);
    c0 = p.code_ptr[r];
    my_slot = lane < ns ? p.slots[s0 + lane] : 0;
  }
  for (; r < p.n_rows; r += stride) {
    // first-level descriptors of the next row (independent loads)
    const int64_t rn = r + stride;
    int64_t s0n = 0, s1n = 0, k0n = 0, k1n = 0, c0n = 0;
    if (rn < p.n_rows) {
      s0n = p.slot_ptr[rn];
      s1n = p.slot_ptr[rn + 1];
      k0n = p.row_ptr[rn];
      k1n = p.row_ptr[rn + 1];
      c0n = p.code_ptr[rn];
    }
    const uint16_t* pos = p.pos + c0 + lane;
    for (int k = lane; k < nnz; k += 32) acc[k] = make_float2(0.f, 0.f);
    if (p.rhs != nullptr) rhs_row(p, r, ns, my_slot, lane);
    __syncwarp();
    for (int sb0 = 0; sb0 < ns; sb0 += SB) {
      float x[SB][CH];
      int kk[SB][CH];
#pragma unroll
      for (int t = 0; t < SB; ++t) {
        const int s = sb0 + t < ns ? sb0 + t : ns - 1;
        const int sid = __shfl_sync(kFull, my_slot, s);
        const float* krow = IDX32 ? ke + uint32_t(sid) * uint32_t(p.nlp) : ke + int64_t(sid) * p.nlp;
        const uint16_t* prow = pos + s * NL;
#pragma unroll
        for (int c = 0; c < CH; ++c) {
          x[t][c] = __ldg(krow + c * 32);
          const int k = int(__ldg(prow + c * 32));
          kk[t][c] = (c < CH - 1 || c * 32 + lane < NL) ? k : dummy;
        }
      }
#pragma unroll
      for (int t = 0; t < SB; ++t) {
        if (sb0 + t < ns) {
#pragma unroll
          for (int c = 0; c < CH; ++c) {
            const int k = kk[t][c];
            const float v = (c < CH - 1 || c * 32 + lane < NL) ? x[t][c] : 0.f;
            const float2 a = acc[k];
            const float sum = a.x + v;
            const float bp = sum - a.x;
            const float err = (a.x - (sum - bp)) + (v - bp);
            acc[k] = make_float2(sum, a.y + err);
          }
          __syncwarp();
        }
      }
    }
    // second-level descriptor of the next row (its slot ids)
    const int nsn = int(s1n - s0n);
    const int my_slot_n = (rn < p.n_rows && lane < nsn) ? p.slots[s0n + lane] : 0;
    for (int k = lane; k < nnz; k += 32) {
      const float2 a = acc[k];
      p.values[k0 + k] = df_to_double(a.x, a.y);
    }
    __syncwarp();
    s0 = s0n;
    ns = nsn;
    k0 = k0n;
    nnz = int(k1n - k0n);
    c0 = c0n;
    my_slot = my_slot_n;
  }
}

static int align16(long x) { return int((x + 15) & ~15L); }

cudaError_t launch_scatter(const fe_space* s, fe_precision prec, double* values, double* rhs, cudaStream_t st) {
  if (s->hs.n_dofs == 0) return cudaSuccess;
  ScatterParams p;
  p.n_rows = s->hs.n_dofs;
  p.nl = s->nl;
  p.nlp = s->nlp;
  p.row_ptr = s->d_row_ptr;
  p.cnt = s->d_cnt;
  p.code_ptr = s->d_code_ptr;
  p.codes = s->d_codes;
  p.pos = s->d_pos;
  p.slot_ptr = s->d_slot_ptr;
  p.slots = s->d_slots;
  p.ke = s->d_ke;
  p.fe = s->d_fe;
  p.values = values;
  p.rhs = rhs;
  const int tk = prec == FE_PREC_FP64 ? 8 : 4;
  p.ke_bytes = align16(long(s->hs.max_slots) * s->nlp * tk);
  p.code_bytes = align16(((long(s->hs.max_slots) * s->nl + 7) & ~7L) * 2);
  const int rows_warp_bytes = p.ke_bytes + p.code_bytes + align16((s->hs.max_row_nnz + 1) * 2);
  const long smem = long(rows_warp_bytes) * kScatterWarps;
  int nsm = 152;
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, s->device);
  const int64_t need = (p.n_rows + kScatterWarps - 1) / kScatterWarps;
  auto launch = [&](auto kern, long bytes) -> cudaError_t {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(bytes));
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kScatterWarps * 32, size_t(bytes));
    if (e != cudaSuccess) return e;
    const int blocks = int(std::min<int64_t>(need, int64_t(nsm) * std::max(1, per_sm)));
    kern<<<blocks, kScatterWarps * 32, size_t(bytes), st>>>(p);
    return cudaGetLastError();
  };
  if (prec != FE_PREC_FP64 && s->hs.max_slots <= 32) {
    p.acc_stride = int((s->hs.max_row_nnz + 3) & ~int64_t(3));
    p.warp_bytes = (p.acc_stride + 32) * 8;  // accumulators + one dummy per lane
    const long bytes = long(p.warp_bytes) * kScatterWarps;
    if (bytes <= 200 * 1024) {
      const bool idx32 = int64_t(s->n_cells) * s->nl * s->nlp < (int64_t(1) << 32);
      switch (s->nl * 2 + (idx32 ? 1 : 0)) {
        case 16: return launch(k_scatter_slots<8, false>, bytes);
        case 17: return launch(k_scatter_slots<8, true>, bytes);
        case 48: return launch(k_scatter_slots<24, false>, bytes);
        case 49: return launch(k_scatter_slots<24, true>, bytes);
        case 54: return launch(k_scatter_slots<27, false>, bytes);
        case 55: return launch(k_scatter_slots<27, true>, bytes);
        case 128: return launch(k_scatter_slots<64, false>, bytes);
        case 129: return launch(k_scatter_slots<64, true>, bytes);
        case 162: return launch(k_scatter_slots<81, false>, bytes);
        case 163: return launch(k_scatter_slots<81, true>, bytes);
        case 384: return launch(k_scatter_slots<192, false>, bytes);
        case 385: return launch(k_scatter_slots<192, true>, bytes);
        default: break;
      }
    }
  }
  p.warp_bytes = rows_warp_bytes;
  if (smem <= 200 * 1024 && s->hs.max_slots <= 32) {
    return prec == FE_PREC_FP64 ? launch(k_scatter_rows<double>, smem) : launch(k_scatter_rows<float>, smem);
  }
  const int blocks = int(std::min<int64_t>(need, int64_t(nsm) * 8));
  if (prec == FE_PREC_FP64)
    k_scatter<double><<<blocks, kScatterWarps * 32, 0, st>>>(p);
  else
    k_scatter<float><<<blocks, kScatterWarps * 32, 0, st>>>(p);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Compliance adjoint: one thread per cell. For fixed u the sensitivity of
// c = u^T A u to the cell coefficient is the cell energy of u per unit
// coefficient, evaluated per quadrature point from grad u (Eq. fematrix,
// Eq. shape_grad) without forming A^K:
//   Poisson    |grad u|^2,
//   elasticity lam^ (div u)^2 + 2 mu^ eps(u):eps(u),
// times w_q det J_q. T is the arithmetic of the strain (FP64 or FP32); the
// geometry and the sums over points are FP64.
struct AdjParams {
  int64_t n_cells;
  int nq;
  const double* xv;
  const double* w;
  const double* xq;
  const double* dphi;
  const int32_t* cell_dofs;
  const double* u;
  const double* coef;
  double grad_scale, lam_hat, mu_hat;
  double* g;
  double* partials;
  int* err;
};

constexpr int kAdjThreads = kAdjointBlock;

template <int P, int NC, typename T>
__global__ void __launch_bounds__(kAdjThreads) k_adjoint(AdjParams p) {
  constexpr int NB = (P + 1) * (P + 1) * (P + 1);
  constexpr int NL = NC * NB;
  __shared__ double red[kAdjThreads];
  const int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  double energy = 0.0;
  if (e < p.n_cells) {
    double x[24], a[21];
#pragma unroll
    for (int i = 0; i < 24; ++i) x[i] = p.xv[e * 24 + i];
#pragma unroll
    for (int k = 0; k < 3; ++k) trilinear_coefficients(x, k, a);
    T ue[NL];
#pragma unroll
    for (int l = 0; l < NL; ++l) ue[l] = T(p.u[p.cell_dofs[e * NL + l]]);
    for (int q = 0; q < p.nq; ++q) {
      double cof[9], det;
      geometry_at(a, p.xq[3 * q], p.xq[3 * q + 1], p.xq[3 * q + 2], cof, &det);
      if (!(det > 0.0)) atomicOr(p.err, kErrNegJacobian);
      // reference gradient of each component of u
      T gr[NC][3];
#pragma unroll
      for (int c = 0; c < NC; ++c) gr[c][0] = gr[c][1] = gr[c][2] = T(0);
      const double* dq = p.dphi + size_t(q) * NB * 3;
#pragma unroll 4
      for (int b = 0; b < NB; ++b) {
        const T d0 = T(dq[3 * b]), d1 = T(dq[3 * b + 1]), d2 = T(dq[3 * b + 2]);
#pragma unroll
        for (int c = 0; c < NC; ++c) {
          const T uc = ue[c * NB + b];
          gr[c][0] += uc * d0;
          gr[c][1] += uc * d1;
          gr[c][2] += uc * d2;
        }
      }
      // physical gradient: (grad u)_{c,k} = sum_d gr[c][d] cof[k][d] / det
      const double inv = 1.0 / det;
      T cs[9];
#pragma unroll
      for (int t = 0; t < 9; ++t) cs[t] = T(cof[t] * inv);
      T gu[NC][3];
#pragma unroll
      for (int c = 0; c < NC; ++c)
#pragma unroll
        for (int k = 0; k < 3; ++k) gu[c][k] = gr[c][0] * cs[3 * k] + gr[c][1] * cs[3 * k + 1] + gr[c][2] * cs[3 * k + 2];
      double dens;
      if (NC == 1) {
        dens = double(gu[0][0] * gu[0][0] + gu[0][1] * gu[0][1] + gu[0][2] * gu[0][2]);
      } else {
        const T div = gu[0][0] + gu[1 % NC][1] + gu[2 % NC][2];
        T ee = T(0);
#pragma unroll
        for (int k = 0; k < 3; ++k)
#pragma unroll
          for (int l = 0; l < 3; ++l) {
            const T eps = T(0.5) * (gu[k % NC][l] + gu[l % NC][k]);
            ee += eps * eps;
          }
        dens = p.lam_hat * double(div * div) + 2.0 * p.mu_hat * double(ee);
      }
      energy += p.w[q] * det * dens;
    }
    p.g[e] = p.grad_scale * energy;
  }
  if (p.partials != nullptr) {
    red[threadIdx.x] = (e < p.n_cells) ? p.coef[e] * energy : 0.0;
    __syncthreads();
    for (int off = kAdjThreads / 2; off > 0; off >>= 1) {
      if (threadIdx.x < off) red[threadIdx.x] += red[threadIdx.x + off];
      __syncthreads();
    }
    if (threadIdx.x == 0) p.partials[blockIdx.x] = red[0];
  }
}

// Sums the per-block partials in a fixed order (one block).
__global__ void k_sum_partials(const double* partials, int n, double* out) {
  __shared__ double red[256];
  double s = 0.0;
  for (int i = threadIdx.x; i < n; i += 256) s += partials[i];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int off = 128; off > 0; off >>= 1) {
    if (threadIdx.x < off) red[threadIdx.x] += red[threadIdx.x + off];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = red[0];
}

template <int P, int NC>
static cudaError_t launch_adj_p(const AdjParams& prm, bool fp32, int blocks, cudaStream_t st) {
  if (fp32)
    k_adjoint<P, NC, float><<<blocks, kAdjThreads, 0, st>>>(prm);
  else
    k_adjoint<P, NC, double><<<blocks, kAdjThreads, 0, st>>>(prm);
  return cudaGetLastError();
}

cudaError_t launch_adjoint(const fe_space* s, const double* u, const double* coef, double grad_scale, double* g,
                           double* compliance, fe_precision prec, cudaStream_t st) {
  if (s->n_cells == 0) return cudaSuccess;
  AdjParams prm;
  prm.n_cells = s->n_cells;
  prm.nq = s->nq;
  prm.xv = s->d_xv;
  prm.w = s->d_w;
  prm.xq = s->d_xq;
  prm.dphi = s->d_dphi;
  prm.cell_dofs = s->d_cell_dofs;
  prm.u = u;
  prm.coef = coef;
  prm.grad_scale = grad_scale;
  prm.lam_hat = s->nu / ((1.0 + s->nu) * (1.0 - 2.0 * s->nu));
  prm.mu_hat = 1.0 / (2.0 * (1.0 + s->nu));
  prm.g = g;
  prm.err = s->d_err;
  const int blocks = int((s->n_cells + kAdjThreads - 1) / kAdjThreads);
  const bool want_c = compliance != nullptr && coef != nullptr;
  prm.partials = want_c ? s->d_partials : nullptr;
  if (want_c && blocks > s->n_partials) return cudaErrorInvalidValue;
  const bool fp32 = prec != FE_PREC_FP64;
  cudaError_t e;
  switch (s->order * 10 + s->ncomp) {
    case 11: e = launch_adj_p<1, 1>(prm, fp32, blocks, st); break;
    case 13: e = launch_adj_p<1, 3>(prm, fp32, blocks, st); break;
    case 21: e = launch_adj_p<2, 1>(prm, fp32, blocks, st); break;
    case 23: e = launch_adj_p<2, 3>(prm, fp32, blocks, st); break;
    case 31: e = launch_adj_p<3, 1>(prm, fp32, blocks, st); break;
    case 33: e = launch_adj_p<3, 3>(prm, fp32, blocks, st); break;
    default: return cudaErrorInvalidValue;
  }
  if (e != cudaSuccess || !want_c) return e;
  k_sum_partials<<<1, 256, 0, st>>>(s->d_partials, blocks, compliance);
  return cudaGetLastError();
}

cudaError_t launch_adjoint_with_scratch(const fe_space* s, const double* u, const double* coef, double grad_scale,
                                        double* g, double* compliance, fe_precision prec, double* partials,
                                        int max_partials, cudaStream_t st) {
  if (s->n_cells == 0) return cudaSuccess;
  AdjParams prm;
  prm.n_cells = s->n_cells;
  prm.nq = s->nq;
  prm.xv = s->d_xv;
  prm.w = s->d_w;
  prm.xq = s->d_xq;
  prm.dphi = s->d_dphi;
  prm.cell_dofs = s->d_cell_dofs;
  prm.u = u;
  prm.coef = coef;
  prm.grad_scale = grad_scale;
  prm.lam_hat = s->nu / ((1.0 + s->nu) * (1.0 - 2.0 * s->nu));
  prm.mu_hat = 1.0 / (2.0 * (1.0 + s->nu));
  prm.g = g;
  prm.err = s->d_err;
  const int blocks = int((s->n_cells + kAdjThreads - 1) / kAdjThreads);
  const bool want_c = compliance != nullptr && coef != nullptr;
  prm.partials = want_c ? partials : nullptr;
  if (want_c && blocks > max_partials) return cudaErrorInvalidValue;
  const bool fp32 = prec != FE_PREC_FP64;
  cudaError_t e;
  switch (s->order * 10 + s->ncomp) {
    case 11: e = launch_adj_p<1, 1>(prm, fp32, blocks, st); break;
    case 13: e = launch_adj_p<1, 3>(prm, fp32, blocks, st); break;
    case 21: e = launch_adj_p<2, 1>(prm, fp32, blocks, st); break;
    case 23: e = launch_adj_p<2, 3>(prm, fp32, blocks, st); break;
    case 31: e = launch_adj_p<3, 1>(prm, fp32, blocks, st); break;
    case 33: e = launch_adj_p<3, 3>(prm, fp32, blocks, st); break;
    default: return cudaErrorInvalidValue;
  }
  if (e != cudaSuccess || !want_c) return e;
  k_sum_partials<<<1, 256, 0, st>>>(partials, blocks, compliance);
  return cudaGetLastError();
}

}  // namespace feasm

// Device-side building blocks shared by the kernels of libfeasm
// (fe_kernels.cu) and the batched persistent driver (fe_batch.cu): cell
// integration of a block of cells, exact FP64 accumulation helpers, and the
// parameter blocks of both phases.
#pragma once

#include <cuda_bf16.h>

#include <type_traits>

#include "fe_launch.h"

namespace feasm {

constexpr int kCellThreads = 256;
constexpr int kScatterWarps = 8;


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


// Exact RHS entry of row r: the cells' FP64 cell-vector entries, one per lane
// (lanes < ns), summed in integer fixed point across the warp.
__device__ __forceinline__ void rhs_row_value(const ScatterParams& p, int64_t r, double my_fe, int lane) {
  uint64_t m = 0;
  int ex = 1;
  bool ng = false;
  FxTraits<double>::split(my_fe, m, ex, ng);
  const int emax = __reduce_max_sync(kFull, m != 0 ? ex : 1);
  const int sh = FxTraits<double>::kShift0 - (emax - ex);
  const uint64_t a = sh >= 0 ? (m << sh) : (sh > -64 ? (m >> (-sh)) : 0ull);
  int64_t S = ng ? -int64_t(a) : int64_t(a);
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) S += __shfl_xor_sync(kFull, S, off);
  if (lane == 0) p.rhs[r] = fx_to_double(S, emax - FxTraits<double>::kScale);
}

__device__ __forceinline__ void rhs_row(const ScatterParams& p, int64_t r, int ns, int my_slot, int lane) {
  rhs_row_value(p, r, lane < ns ? p.fe[my_slot] : 0.0, lane);
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


}  // namespace feasm

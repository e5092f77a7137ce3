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
  int nq, cpb, qblock, nq1d;
  const double* xv;
  const double* w;
  const double* xq;
  const double* phi;
  const float2* phi2;  // [nq][nb] phihat as FP32 hi + lo (hi + lo == phihat to ~2^-48)
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
// Two values rounded to BF16 (nearest even) by one paired conversion.
__device__ __forceinline__ void round_bf16_pair(float& x, float& y) {
  const __nv_bfloat162 h = __floats2bfloat162_rn(x, y);
  x = __low2float(h);
  y = __high2float(h);
}

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

// One block integrates `cpb` cells in FP64 (paper: Eq. fematrix, Eq.
// shape_grad, the element loop of the element-matrix computation):
//   1. geometry at every quadrature point,
//   2. cofactor gradients gh_a = cof(J) gradhat(phihat_a), so that
//      grad(phi_a) = gh_a / det J,
//   3. G^{ij}_{ab} = sum_q (w_q / det J_q) gh_{a,i} gh_{b,j}, and
//      Poisson   K_ab = kappa sum_i G^{ii}_{ab},
//      elasticity K_(a,i),(b,j) = E (lam^ G^{ij}_ab + mu^ G^{ji}_ab + mu^ d_ij sum_k G^{kk}_ab),
//   4. cell vector f_(a,i) = f_i sum_q w_q det J_q phihat_a(x_q).
// Cell matrices are stored row-major with row stride NLP (16-byte aligned
// rows). Shared memory: vertex coordinates [cpb][24], trilinear coefficients
// [cpb][21], per-point geometry [cpb][nq][11] (cofactors, w/det, w*det), the
// cofactor gradients [cpb][nq][3][nb].
template <int P, int NC>
__device__ __forceinline__ void cell_block_fp64(const CellParams& prm, int64_t e0, int ncell, double* smem) {
  constexpr int NB = (P + 1) * (P + 1) * (P + 1);
  constexpr int NL = NC * NB;
  constexpr int NLP = (NL + 3) & ~3;
  const int cpb = prm.cpb, nq = prm.nq;
  double* sx = smem;
  double* sa = sx + cpb * 24;
  double* geo = sa + cpb * 21;
  double* g = geo + cpb * nq * 11;
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
  }
  __syncthreads();
  for (int i = tid; i < ncell * nq * NB; i += blockDim.x) {
    const int a = i % NB, cq = i / NB, q = cq % nq;
    double* gg = g + size_t(cq) * 3 * NB;
    const double* gm = geo + size_t(cq) * 11;
    const double* dp = prm.dphi + (size_t(q) * NB + a) * 3;
#pragma unroll
    for (int k = 0; k < 3; ++k) gg[k * NB + a] = gm[3 * k] * dp[0] + gm[3 * k + 1] * dp[1] + gm[3 * k + 2] * dp[2];
  }
  __syncthreads();
  for (int i = tid; i < ncell * NB * NB; i += blockDim.x) {
    const int c = i / (NB * NB), ab = i % (NB * NB), a = ab / NB, b = ab % NB;
    const double* gc = g + size_t(c) * nq * 3 * NB;
    const double* gm = geo + size_t(c) * nq * 11;
    const int64_t e = e0 + c;
    const double coef = prm.coef[e];
    double* K = reinterpret_cast<double*>(prm.ke) + e * NL * NLP;
    if (NC == 1) {
      double sum = 0.0;
      for (int q = 0; q < nq; ++q) {
        const double* gq = gc + size_t(q) * 3 * NB;
        const double s = gm[q * 11 + 9];
#pragma unroll
        for (int k = 0; k < 3; ++k) sum += (s * gq[k * NB + a]) * gq[k * NB + b];
      }
      K[a * NLP + b] = coef * sum;
    } else {
      double S[3][3];
#pragma unroll
      for (int i2 = 0; i2 < 3; ++i2)
#pragma unroll
        for (int j2 = 0; j2 < 3; ++j2) S[i2][j2] = 0.0;
      for (int q = 0; q < nq; ++q) {
        const double* gq = gc + size_t(q) * 3 * NB;
        const double s = gm[q * 11 + 9];
        double ga[3], gb[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          ga[k] = s * gq[k * NB + a];
          gb[k] = gq[k * NB + b];
        }
#pragma unroll
        for (int i2 = 0; i2 < 3; ++i2)
#pragma unroll
          for (int j2 = 0; j2 < 3; ++j2) S[i2][j2] += ga[i2] * gb[j2];
      }
      const double lh = prm.lam_hat, mh = prm.mu_hat;
      const double tr = S[0][0] + S[1][1] + S[2][2];
#pragma unroll
      for (int i2 = 0; i2 < 3; ++i2)
#pragma unroll
        for (int j2 = 0; j2 < 3; ++j2) {
          double v = lh * S[i2][j2] + mh * S[j2][i2];
          if (i2 == j2) v += mh * tr;
          K[size_t(i2 * NB + a) * NLP + j2 * NB + b] = coef * v;
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


// fx_sum of N terms held in registers (zeros pad a shorter list): the same
// fixed-point sum and rounding, so the same result, without a second pass
// over memory.
template <int N>
__device__ __forceinline__ double fx_sum_regs(const double (&v)[N]) {
  using Tr = FxTraits<double>;
  int emax = 1;
#pragma unroll
  for (int t = 0; t < N; ++t) {
    uint64_t m;
    int ex;
    bool ng;
    Tr::split(v[t], m, ex, ng);
    if (m != 0 && ex > emax) emax = ex;
  }
  int64_t S = 0;
#pragma unroll
  for (int t = 0; t < N; ++t) {
    uint64_t m;
    int ex;
    bool ng;
    Tr::split(v[t], m, ex, ng);
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
  const int32_t* ncode;  // codes per row (constrained patterns), or nullptr: slots * nl
  unsigned long long* sched;  // [2] item counters of the dynamic schedule, zero between launches
  const void* ke;
  const double* fe;
  double* values;
  double* rhs;
  int ke_bytes, code_bytes, warp_bytes, acc_stride;
};

constexpr unsigned kFull = 0xffffffffu;

// Dynamic assignment of work items (CSR rows, or the rows of one node) to the
// warps of a scatter launch. A warp takes `grab` consecutive items at a time
// from a counter in device memory (one atomicAdd by lane 0) and holds its next
// grab in reserve, so that the atomic's latency hides behind the current
// items. Rows differ in cost (a node lies in 1, 2, 4 or 8 cells, in a pattern
// that repeats every few tens of rows and shifts wherever rows are dropped);
// any static cyclic schedule lets that pattern line up with the warp index
// for some meshes and warp counts, so that a few warps collect the expensive
// rows. Taking items on demand balances the warps to within one grab, while
// the items in flight still form one contiguous window of rows. Every warp
// calls finish() once at the end; the last one resets both counters (next
// item, finished warps) to zero for the next launch on the stream.
struct ItemStream {
  unsigned long long* ctr;
  int64_t n, u, end, nxt;
  int grab;
  __device__ __forceinline__ int64_t take(int lane) const {
    unsigned long long b = 0;
    if (lane == 0) b = atomicAdd(ctr, static_cast<unsigned long long>(grab));
    return static_cast<int64_t>(__shfl_sync(kFull, b, 0));
  }
  __device__ __forceinline__ ItemStream(unsigned long long* c, int64_t n_items, int grab_size, int lane)
      : ctr(c), n(n_items), grab(grab_size) {
    u = take(lane);
    end = u + grab < n ? u + grab : n;
    nxt = take(lane);
  }
  __device__ __forceinline__ bool valid() const { return u < n; }
  // the item after the current one (>= n: no more); takes a new reserve grab when needed
  __device__ __forceinline__ void advance(int lane) {
    if (u + 1 < end) {
      ++u;
    } else {
      u = nxt;
      end = u + grab < n ? u + grab : n;
      nxt = u < n ? take(lane) : u;
    }
  }
  __device__ __forceinline__ void finish(int64_t n_warps, int lane) const {
    if (lane == 0) {
      __threadfence();
      if (atomicAdd(ctr + 1, 1ull) == static_cast<unsigned long long>(n_warps - 1)) {
        atomicExch(ctr, 0ull);
        atomicExch(ctr + 1, 0ull);
      }
    }
  }
};


// Exact FP32 -> FP64 conversion on the integer bits (denormals included),
// without the FP64 pipe; infinities and NaNs take the hardware conversion.
static __device__ __noinline__ double f2d_slow(float x) { return double(x); }
__device__ __forceinline__ double f32_to_f64_exact(float x) {
  double d;
  if (f32_to_f64_bits(x, d)) return d;
  if ((__float_as_uint(x) & 0x7f800000u) == 0x7f800000u) return f2d_slow(x);
  uint64_t m;
  int ex;
  bool ng;
  FxTraits<float>::split(x, m, ex, ng);
  return fx_to_double(ng ? -int64_t(m) : int64_t(m), ex - 150);
}

// FP32 -> FP64, exact, for zero and normal numbers, in 32-bit integer
// operations: the high word is the sign, the exponent rebiased by
// 1023 - 127 = 896 and the top 20 mantissa bits, i.e. sign | ((|x| >> 3) +
// (896 << 20)); the low word holds the last 3 mantissa bits, |x| << 29.
__device__ __forceinline__ double f32_to_f64_normal(float x) {
  const uint32_t u = __float_as_uint(x), mag = u & 0x7fffffffu, sgn = u & 0x80000000u;
  const uint32_t hw = mag == 0 ? sgn : (sgn | ((mag >> 3) + 0x38000000u));
  return __hiloint2double(int(hw), int(mag << 29));
}

// True for zero and FP32-normal x (exponent field 1..254).
__device__ __forceinline__ bool f32_zero_or_normal(float x) {
  const uint32_t mag = __float_as_uint(x) & 0x7fffffffu;
  return mag == 0 || mag - 0x00800000u < 0x7f000000u;
}

// hi + lo of a double-float accumulator, rounded once to the nearest double:
// both parts convert exactly on the integer bits and one FP64 addition rounds
// their exact sum (lo == 0 keeps hi, sign of zero included). Branch-free; a
// warp vote sends the whole warp to the general conversion in the rare case of
// a denormal part. All 32 lanes of the warp must call it.
__device__ __forceinline__ double df_to_double(float hi, float lo) {
  double dh, dl;
  if (__all_sync(kFull, f32_zero_or_normal(hi) && f32_zero_or_normal(lo))) {
    dh = f32_to_f64_normal(hi);
    dl = f32_to_f64_normal(lo);
  } else {
    dh = f32_to_f64_exact(hi);
    dl = f32_to_f64_exact(lo);
  }
  const double sum = __dadd_rn(dh, dl);
  return lo == 0.f ? dh : sum;
}


// FP64 -> FP32 round to nearest even on the integer bits (zero and
// FP32-normal results; values that would under- or overflow FP32 take the
// hardware conversion, out of line). Keeps the conversions of the FP64 geometry off the FP64 pipe.
static __device__ __noinline__ float d2f_slow(double x) { return __double2float_rn(x); }
__device__ __forceinline__ float d2f_rn(double x) {
  const uint64_t u = uint64_t(__double_as_longlong(x));
  const int e = int((u >> 52) & 0x7ffu) - 896;
  if (e <= 0 || e >= 255) {
    if ((u << 1) == 0) return __uint_as_float(uint32_t(u >> 63) << 31);
    return d2f_slow(x);  // out of line: FP64-pipe instructions on a predicated path still occupy the pipe
  }
  const uint64_t mant = u & 0xfffffffffffffull;
  uint32_t body = (uint32_t(e) << 23) | uint32_t(mant >> 29);
  const uint32_t rem = uint32_t(mant & 0x1fffffffu);
  if (rem > 0x10000000u || (rem == 0x10000000u && (body & 1u))) ++body;  // carries into the exponent
  return __uint_as_float((uint32_t(u >> 63) << 31) | body);
}

// FP64 -> FP32 round to nearest even on the 32-bit words of x, branch-free, for
// a result that is zero or an FP32 normal number; `odd` is set for inputs
// outside that range (the tile's geometry is then recomputed with the general
// conversions). A rounding at the top of the range that carries into infinity
// comes out exact without the flag.
__device__ __forceinline__ float d2f_fast(double x, bool& odd) {
  const uint32_t hi = uint32_t(__double2hiint(x)), lo = uint32_t(__double2loint(x));
  const uint32_t ahi = hi & 0x7fffffffu;
  const int e = int(ahi >> 20) - 896;
  const bool zero = (ahi | lo) == 0;
  odd |= (e <= 0 || e >= 255) && !zero;
  uint32_t body = (uint32_t(e) << 23) | ((ahi & 0xfffffu) << 3) | (lo >> 29);
  const uint32_t rem = lo & 0x1fffffffu;
  body += (rem > 0x10000000u || (rem == 0x10000000u && (body & 1u))) ? 1u : 0u;
  return __uint_as_float((hi & 0x80000000u) | (zero ? 0u : body));
}

// x - d2f_fast(x), the part of x below its FP32 rounding, itself rounded to
// FP32, on the 32-bit words: the low 29 mantissa bits minus the rounding
// carry, times 2^(exponent - 1075), normalised on the integer bits. For x with
// an FP32-normal rounding; `odd` is set where the result leaves the FP32
// normal range (the tile is then recomputed with the general conversions).
__device__ __forceinline__ float d2f_rest(double x, bool& odd) {
  const uint32_t hi = uint32_t(__double2hiint(x)), lo = uint32_t(__double2loint(x));
  const int E = int((hi & 0x7fffffffu) >> 20);
  const uint32_t rem = lo & 0x1fffffffu;
  const uint32_t body = ((hi & 0xfffffu) << 3) | (lo >> 29);
  const bool up = rem > 0x10000000u || (rem == 0x10000000u && (body & 1u));
  // r = rem - up 2^29, |r| <= 2^28; the value is r 2^(E - 1075), sign of x, negated if up
  const uint32_t m = up ? (0x20000000u - rem) : rem;
  const int lz = __clz(m | 1u);            // >= 3
  const int sh = lz - 8;                   // normalise the leading 1 to bit 23
  const int rs = sh < 0 ? -sh : 1;         // 25..29 significant bits: round to nearest even
  const uint32_t t = m >> rs, rb = m & ((1u << rs) - 1u), half = 1u << (rs - 1);
  const uint32_t rnd = t + ((rb > half || (rb == half && (t & 1u))) ? 1u : 0u);
  const bool carry = sh < 0 && (rnd >> 24) != 0;
  const uint32_t mm = sh >= 0 ? (m << sh) : (carry ? rnd >> 1 : rnd);
  const int er = E - 948 + (31 - lz) + (carry ? 1 : 0);  // biased exponent of m 2^(E - 1075)
  odd |= m != 0 && (er <= 0 || er >= 255);
  const uint32_t sgn = (hi & 0x80000000u) ^ (up ? 0x80000000u : 0u);
  return __uint_as_float(m == 0 ? 0u : (sgn | (uint32_t(er) << 23) | (mm & 0x7fffffu)));
}

// TF32 rounding of x (to nearest, ties away from zero), the hi part of the
// 3xTF32 split; the lo part is to_tf32(x - hi).
__device__ __forceinline__ float to_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

// Exact sum of N FP32 terms held in registers, rounded once to FP64 (the
// fixed-point accumulation of fx_sum), on the integer bits.
template <int N>
__device__ __forceinline__ double fx_sum_regs_f32(const float (&v)[N]) {
  using Tr = FxTraits<float>;
  int emax = 1;
#pragma unroll
  for (int t = 0; t < N; ++t) {
    uint64_t m;
    int ex;
    bool ng;
    Tr::split(v[t], m, ex, ng);
    if (m != 0 && ex > emax) emax = ex;
  }
  int64_t S = 0;
#pragma unroll
  for (int t = 0; t < N; ++t) {
    uint64_t m;
    int ex;
    bool ng;
    Tr::split(v[t], m, ex, ng);
    const int sh = Tr::kShift0 - (emax - ex);
    const uint64_t a = sh >= 0 ? (m << sh) : (sh > -64 ? (m >> (-sh)) : 0ull);
    S += ng ? -int64_t(a) : int64_t(a);
  }
  return fx_to_double(S, emax - Tr::kScale);
}

// Shared-memory layout of the FP32/BF16 cell block (byte offsets; host and
// device agree on it through this one function). Regions: vertex coordinates
// [cpb][24] and trilinear coefficients [cpb][21] (FP64), the Jacobian columns
// [cpb][3][n1d^2][3] (FP64), the products u v of the 1D points [n1d^2] (FP64),
// w det J as hi + lo [cpb][nq] (float2), FP32 cofactors and w/det J
// [cpb][nq][12], then the operands: for nb <= 27 the scaled and plain
// cofactor gradients as float4 [cpb][nq][nb] each, else the plain gradients
// [cpb][nq][3][nb] (float).
struct MixedLayout {
  long x, a, jc, uv, djw, geo32, ga, gb, bytes;
};
__host__ __device__ inline MixedLayout mixed_layout(int cpb, int nq, int n1d, int nb) {
  MixedLayout L;
  const long p2 = long(n1d) * n1d;
  L.x = 0;
  L.a = L.x + long(cpb) * 24 * 8;
  L.jc = L.a + long(cpb) * 21 * 8;
  L.uv = L.jc + long(cpb) * 9 * p2 * 8;
  L.djw = (L.uv + p2 * 8 + 15) & ~15l;
  L.geo32 = (L.djw + long(cpb) * nq * 8 + 15) & ~15l;
  L.ga = L.geo32 + long(cpb) * nq * 48;
  if (nb <= 27) {
    L.gb = L.ga + long(cpb) * nq * nb * 16;
    L.bytes = L.gb + long(cpb) * nq * nb * 16;
  } else {
    L.gb = L.ga;
    L.bytes = L.ga + long(cpb) * nq * 3 * nb * 4;
  }
  return L;
}

// One block integrates `cpb` cells for the FP32 (PREC 1) and BF16 (PREC 2)
// forms; same steps as cell_block_fp64, with the geometry FP64 and everything
// after it FP32:
//   * each Jacobian column of the trilinear map depends on two of the three
//     reference coordinates only (column d is linear in the other two and
//     bilinear in their product), so it is evaluated once per pair of 1D
//     points of the tensor rule, n1d^2 instead of n1d^3 times (FP64);
//   * per quadrature point: cofactors and det J (FP64), rounded once to FP32
//     on the integer bits; w/det J as the FP32 quotient of the rounded values;
//     w det J as an FP32 hi + lo pair;
//   * gradients gh_a = cof gradhat(phihat_a) in FP32, stored as (w/det) gh_a
//     and gh_a (rounded to BF16 for PREC 2), so that a product of one point
//     costs one load per side;
//   * PREC 1 sums the points in blocks of `qblock` (one z-slab of the rule)
//     with Kahan compensation between blocks; PREC 2 sums plainly;
//   * the cell vector sum_q (w det J)_q phihat_a(x_q) in double-float
//     arithmetic (products with fmaf error terms, TwoSum accumulation),
//     rounded once to FP64.
template <int P, int NC, int PREC>
__device__ __forceinline__ void cell_block_mixed(const CellParams& prm, int64_t e0, int ncell, double* smem) {
  constexpr int NB = (P + 1) * (P + 1) * (P + 1);
  constexpr int NL = NC * NB;
  constexpr int NLP = (NL + 3) & ~3;
  constexpr bool VEC = NB <= 27;
  const int cpb = prm.cpb, nq = prm.nq, n1d = prm.nq1d, p2 = n1d * n1d;
  const MixedLayout L = mixed_layout(cpb, nq, n1d, NB);
  unsigned char* base = reinterpret_cast<unsigned char*>(smem);
  double* sx = reinterpret_cast<double*>(base + L.x);
  double* sa = reinterpret_cast<double*>(base + L.a);
  double* sj = reinterpret_cast<double*>(base + L.jc);
  double* suv = reinterpret_cast<double*>(base + L.uv);
  float2* djw = reinterpret_cast<float2*>(base + L.djw);
  float* geo32 = reinterpret_cast<float*>(base + L.geo32);
  float4* gA = reinterpret_cast<float4*>(base + L.ga);
  float4* gB = reinterpret_cast<float4*>(base + L.gb);
  float* g = reinterpret_cast<float*>(base + L.ga);
  const int tid = threadIdx.x;

  for (int i = tid; i < ncell * 24; i += blockDim.x) sx[i] = prm.xv[e0 * 24 + i];
  __syncthreads();
  // trilinear coefficients; u v of the 1D point pairs (the 1D rule is the x
  // coordinates of the first n1d points)
  for (int i = tid; i < ncell * 3 + p2; i += blockDim.x) {
    if (i < ncell * 3) {
      trilinear_coefficients(sx + (i / 3) * 24, i % 3, sa + (i / 3) * 21);
    } else {
      const int pr = i - ncell * 3;
      suv[pr] = prm.xq[3 * (pr % n1d)] * prm.xq[3 * (pr / n1d)];
    }
  }
  __syncthreads();
  // Jacobian columns: J[k][d] at the pair (u, v) of the other two coordinates
  // (in axis order): d = 0: a1 + a4 y + a5 z + a7 yz; d = 1: a2 + a4 x + a6 z +
  // a7 xz; d = 2: a3 + a5 x + a6 y + a7 xy (coefficients a1..a7 at offsets
  // 0, 3, .., 18 of the component).
  for (int i = tid; i < ncell * 9 * p2; i += blockDim.x) {
    const int c = i / (9 * p2), r = i % (9 * p2), d = r / (3 * p2), rem = r % (3 * p2), pr = rem / 3, k = rem % 3;
    const double* a = sa + c * 21;
    const double u = prm.xq[3 * (pr % n1d)], v = prm.xq[3 * (pr / n1d)];
    const int o0 = 3 * d, ou = d == 2 ? 12 : 9, ov = d == 0 ? 12 : 15;
    sj[i] = fma(a[18 + k], suv[pr], fma(a[ov + k], v, fma(a[ou + k], u, a[o0 + k])));
  }
  __syncthreads();
  for (int i = tid; i < ncell * nq; i += blockDim.x) {
    const int c = i / nq, q = i % nq;
    const int ix = q % n1d, iy = (q / n1d) % n1d, iz = q / p2;
    const double* jc = sj + c * 9 * p2;
    double J[3][3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      J[k][0] = jc[(0 * p2 + iy + n1d * iz) * 3 + k];
      J[k][1] = jc[(1 * p2 + ix + n1d * iz) * 3 + k];
      J[k][2] = jc[(2 * p2 + ix + n1d * iy) * 3 + k];
    }
    double cof[9];
    cof[0] = J[1][1] * J[2][2] - J[1][2] * J[2][1];
    cof[1] = J[1][2] * J[2][0] - J[1][0] * J[2][2];
    cof[2] = J[1][0] * J[2][1] - J[1][1] * J[2][0];
    cof[3] = J[0][2] * J[2][1] - J[0][1] * J[2][2];
    cof[4] = J[0][0] * J[2][2] - J[0][2] * J[2][0];
    cof[5] = J[0][1] * J[2][0] - J[0][0] * J[2][1];
    cof[6] = J[0][1] * J[1][2] - J[0][2] * J[1][1];
    cof[7] = J[0][2] * J[1][0] - J[0][0] * J[1][2];
    cof[8] = J[0][0] * J[1][1] - J[0][1] * J[1][0];
    const double det = J[0][0] * cof[0] + J[0][1] * cof[1] + J[0][2] * cof[2];
    if (!(det > 0.0)) atomicOr(prm.err, kErrNegJacobian);
    const double wq = prm.w[q];
    float* g32 = geo32 + size_t(i) * 12;
#pragma unroll
    for (int t = 0; t < 9; ++t) g32[t] = d2f_rn(cof[t]);
    g32[9] = d2f_rn(wq) / d2f_rn(det);
    const double wd = wq * det;
    const float hi = d2f_rn(wd);
    djw[i] = make_float2(hi, d2f_rn(wd - f32_to_f64_exact(hi)));
  }
  __syncthreads();
  for (int i = tid; i < ncell * nq * NB; i += blockDim.x) {
    const int a = i % NB, cq = i / NB, q = cq % nq;
    const float4* gq4 = reinterpret_cast<const float4*>(geo32 + size_t(cq) * 12);
    const float4 c0 = gq4[0], c1 = gq4[1], c2 = gq4[2];
    const float* dp = prm.dphi32 + (size_t(q) * NB + a) * 3;
    const float d0 = dp[0], d1 = dp[1], d2 = dp[2];
    float g0 = fmaf(c0.z, d2, fmaf(c0.y, d1, c0.x * d0));
    float g1 = fmaf(c1.y, d2, fmaf(c1.x, d1, c0.w * d0));
    float g2 = fmaf(c2.x, d2, fmaf(c1.w, d1, c1.z * d0));
    if (VEC) {
      const float s = c2.y;
      float a0 = s * g0, a1 = s * g1, a2 = s * g2;
      if (PREC == 2) {
        round_bf16_pair(a0, a1);
        round_bf16_pair(a2, g0);
        round_bf16_pair(g1, g2);
      }
      gA[i] = make_float4(a0, a1, a2, 0.f);
      gB[i] = make_float4(g0, g1, g2, 0.f);
    } else {
      float* gg = g + size_t(cq) * 3 * NB;
      gg[a] = g0;
      gg[NB + a] = g1;
      gg[2 * NB + a] = g2;
    }
  }
  __syncthreads();
  const int qb = PREC == 1 ? prm.qblock : nq;
  if constexpr (NC == 1) {
    // Poisson: each thread sums a TA x TB tile of node pairs, so that one
    // point's loads (TA + TB gradients, w/det) serve TA TB products per
    // component; per pair the same slab-blocked (Kahan) sum as one pair per
    // thread.
    constexpr int TA = NB == 64 ? 4 : NB == 27 ? 3 : 2, TB = NB == 64 ? 2 : TA;  // 4 x 2 for Q3: fewer registers
    constexpr int NTA = NB / TA, NTB = NB / TB;
    static_assert(NB % TA == 0 && NB % TB == 0, "tile");
    for (int i = tid; i < ncell * NTA * NTB; i += blockDim.x) {
      const int c = i / (NTA * NTB), tt = i % (NTA * NTB), a0 = (tt / NTB) * TA, b0 = (tt % NTB) * TB;
      const int64_t e = e0 + c;
      const float coef = d2f_rn(prm.coef[e]);
      float sum[TA][TB], carry[TA][TB];
#pragma unroll
      for (int u = 0; u < TA; ++u)
#pragma unroll
        for (int v = 0; v < TB; ++v) sum[u][v] = carry[u][v] = 0.f;
      for (int q0 = 0; q0 < nq; q0 += qb) {
        float part[TA][TB];
#pragma unroll
        for (int u = 0; u < TA; ++u)
#pragma unroll
          for (int v = 0; v < TB; ++v) part[u][v] = 0.f;
        const int q1 = q0 + qb < nq ? q0 + qb : nq;
        for (int q = q0; q < q1; ++q) {
          float ga[3][TA], gb[3][TB];
          if (VEC) {
#pragma unroll
            for (int u = 0; u < TA; ++u) {
              const float4 A = gA[(size_t(c) * nq + q) * NB + a0 + u];
              ga[0][u] = A.x, ga[1][u] = A.y, ga[2][u] = A.z;
            }
#pragma unroll
            for (int v = 0; v < TB; ++v) {
              const float4 B = gB[(size_t(c) * nq + q) * NB + b0 + v];
              gb[0][v] = B.x, gb[1][v] = B.y, gb[2][v] = B.z;
            }
          } else {
            const float* gq = g + (size_t(c) * nq + q) * 3 * NB;
            const float sq = geo32[(size_t(c) * nq + q) * 12 + 9];
#pragma unroll
            for (int k = 0; k < 3; ++k) {
#pragma unroll
              for (int u = 0; u < TA; ++u) {
                ga[k][u] = sq * gq[k * NB + a0 + u];
                if (PREC == 2) ga[k][u] = round_bf16(ga[k][u]);
              }
#pragma unroll
              for (int v = 0; v < TB; ++v) {
                gb[k][v] = gq[k * NB + b0 + v];
                if (PREC == 2) gb[k][v] = round_bf16(gb[k][v]);
              }
            }
          }
#pragma unroll
          for (int k = 0; k < 3; ++k)
#pragma unroll
            for (int u = 0; u < TA; ++u)
#pragma unroll
              for (int v = 0; v < TB; ++v) part[u][v] = fmaf(ga[k][u], gb[k][v], part[u][v]);
        }
#pragma unroll
        for (int u = 0; u < TA; ++u)
#pragma unroll
          for (int v = 0; v < TB; ++v) {
            if (PREC == 1) kahan_add(sum[u][v], carry[u][v], part[u][v]); else sum[u][v] += part[u][v];
          }
      }
      float* K = reinterpret_cast<float*>(prm.ke) + e * NL * NLP;
#pragma unroll
      for (int u = 0; u < TA; ++u)
#pragma unroll
        for (int v = 0; v < TB; ++v) K[(a0 + u) * NLP + b0 + v] = coef * sum[u][v];
    }
  }
  for (int i = tid; i < (NC == 1 ? 0 : ncell * NB * NB); i += blockDim.x) {
    const int c = i / (NB * NB), ab = i % (NB * NB), a = ab / NB, b = ab % NB;
    const int64_t e = e0 + c;
    const float coef = d2f_rn(prm.coef[e]);
    float* K = reinterpret_cast<float*>(prm.ke) + e * NL * NLP;
    // (w/det) gh_a and gh_b of point q as float3
    auto load = [&](int q, float (&ga)[3], float (&gb)[3]) {
      if (VEC) {
        const float4 A = gA[(size_t(c) * nq + q) * NB + a], B = gB[(size_t(c) * nq + q) * NB + b];
        ga[0] = A.x, ga[1] = A.y, ga[2] = A.z;
        gb[0] = B.x, gb[1] = B.y, gb[2] = B.z;
      } else {
        const float* gq = g + (size_t(c) * nq + q) * 3 * NB;
        const float s = geo32[(size_t(c) * nq + q) * 12 + 9];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          ga[k] = s * gq[k * NB + a];
          gb[k] = gq[k * NB + b];
          if (PREC == 2) round_bf16_pair(ga[k], gb[k]);
        }
      }
    };
    if (NC == 1) {
      float sum = 0.f, carry = 0.f;
      for (int q0 = 0; q0 < nq; q0 += qb) {
        float part = 0.f;
        const int q1 = q0 + qb < nq ? q0 + qb : nq;
        for (int q = q0; q < q1; ++q) {
          float ga[3], gb[3];
          load(q, ga, gb);
#pragma unroll
          for (int k = 0; k < 3; ++k) part = fmaf(ga[k], gb[k], part);
        }
        if (PREC == 1) kahan_add(sum, carry, part); else sum += part;
      }
      K[a * NLP + b] = coef * sum;
    } else {
      float S[3][3], C[3][3];
#pragma unroll
      for (int i2 = 0; i2 < 3; ++i2)
#pragma unroll
        for (int j2 = 0; j2 < 3; ++j2) S[i2][j2] = C[i2][j2] = 0.f;
      for (int q0 = 0; q0 < nq; q0 += qb) {
        float G[3][3];
#pragma unroll
        for (int i2 = 0; i2 < 3; ++i2)
#pragma unroll
          for (int j2 = 0; j2 < 3; ++j2) G[i2][j2] = 0.f;
        const int q1 = q0 + qb < nq ? q0 + qb : nq;
        for (int q = q0; q < q1; ++q) {
          float ga[3], gb[3];
          load(q, ga, gb);
#pragma unroll
          for (int i2 = 0; i2 < 3; ++i2)
#pragma unroll
            for (int j2 = 0; j2 < 3; ++j2) G[i2][j2] = fmaf(ga[i2], gb[j2], G[i2][j2]);
        }
#pragma unroll
        for (int i2 = 0; i2 < 3; ++i2)
#pragma unroll
          for (int j2 = 0; j2 < 3; ++j2) {
            if (PREC == 1) kahan_add(S[i2][j2], C[i2][j2], G[i2][j2]); else S[i2][j2] += G[i2][j2];
          }
      }
      const float lh = d2f_rn(prm.lam_hat), mh = d2f_rn(prm.mu_hat);
      const float tr = S[0][0] + S[1][1] + S[2][2];
#pragma unroll
      for (int i2 = 0; i2 < 3; ++i2)
#pragma unroll
        for (int j2 = 0; j2 < 3; ++j2) {
          float v = lh * S[i2][j2] + mh * S[j2][i2];
          if (i2 == j2) v += mh * tr;
          K[size_t(i2 * NB + a) * NLP + j2 * NB + b] = coef * v;
        }
    }
  }
  for (int i = tid; i < ncell * NB; i += blockDim.x) {
    const int c = i / NB, a = i % NB;
    float sh = 0.f, sl = 0.f;
    for (int q = 0; q < nq; ++q) {
      const float2 w2 = djw[c * nq + q], p2v = prm.phi2[size_t(q) * NB + a];
      const float ph = w2.x * p2v.x;
      const float pe = fmaf(w2.x, p2v.x, -ph) + (w2.x * p2v.y + w2.y * p2v.x);
      const float sum = sh + ph;
      const float bp = sum - sh;
      const float err = (sh - (sum - bp)) + (ph - bp);
      sh = sum;
      sl += err + pe;
    }
    const double f = sl == 0.f ? f32_to_f64_exact(sh) : __dadd_rn(f32_to_f64_exact(sh), f32_to_f64_exact(sl));
    double* fe = prm.fe + (e0 + c) * NL;
#pragma unroll
    for (int k = 0; k < NC; ++k) fe[k * NB + a] = prm.f[k] * f;
  }
}

// Cell integration of one block of cells in the given precision.
template <int P, int NC, int PREC>
__device__ __forceinline__ void cell_block(const CellParams& prm, int64_t e0, int ncell, double* smem) {
  if constexpr (PREC == 0) {
    cell_block_fp64<P, NC>(prm, e0, ncell, smem);
  } else {
    cell_block_mixed<P, NC, PREC>(prm, e0, ncell, smem);
  }
}

// Read-only loads of the scatter: through the non-coherent read-only path,
// or, for data written earlier in the same launch by other blocks (the
// batched driver), bypassing L1 (ld.global.cg).
template <bool CG, typename T>
__device__ __forceinline__ T ld_ro(const T* p) {
  if constexpr (CG) return __ldcg(p); else return __ldg(p);
}

// One batch of the slot-wise double-float scatter of k_scatter_slots (see
// there): B slots from s_begin, R rows per item (R = 3: the rows of one node,
// local rows i * NL / R + a of each cell), accumulator rows of stride rs with
// a private dummy per lane at index `dummy`. The first contribution of a
// nonzero (flag bit 15 of pos; every entry of slot 0) stores (v, 0); later
// ones add with TwoSum.
template <int NL, int R, bool CG = false>
struct SlotScatter {
  static constexpr int CH = (NL + 31) / 32;
  static constexpr int NBR = NL / R;  // local-row offset between the rows of one node
  static constexpr int LOADS = CH * (R + 1);
  // slots per batch: 4 where the loads of a batch fit the registers (measured on
  // the Q1 node rows: 4 slots per batch at five blocks per SM beat 8 at four)
  static constexpr int SB = LOADS <= 8 ? 4 : LOADS <= 16 ? 2 : 1;

  // One batch of B slots starting at slot s_begin.
  template <int B, bool IDX32>
  __device__ __forceinline__ static void batch(const ScatterParams& p, const float* ke, const uint16_t* pos,
                                               int my_slot, int s_begin, float2* acc, int rs, int dummy, int lane) {
    float x[B][CH][R];
    int kk[B][CH];
#pragma unroll
    for (int t = 0; t < B; ++t) {
      const int s = s_begin + t;
      const int sid = __shfl_sync(kFull, my_slot, s);
      const float* krow = IDX32 ? ke + uint32_t(sid) * uint32_t(p.nlp) : ke + int64_t(sid) * p.nlp;
      const uint16_t* prow = pos + s * NL;
#pragma unroll
      for (int c = 0; c < CH; ++c) {
        const int k = int(ld_ro<CG>(prow + c * 32));
        kk[t][c] = (c < CH - 1 || c * 32 + lane < NL) ? k : dummy;
#pragma unroll
        for (int i = 0; i < R; ++i) x[t][c][i] = ld_ro<CG>(krow + i * NBR * p.nlp + c * 32);
      }
    }
#pragma unroll
    for (int t = 0; t < B; ++t) {
#pragma unroll
      for (int c = 0; c < CH; ++c) {
        const int raw = kk[t][c];
        const int k = raw & 0x7fff;
#pragma unroll
        for (int i = 0; i < R; ++i) {
          float2* ai = acc + i * rs;
          const float v = (c < CH - 1 || c * 32 + lane < NL) ? x[t][c][i] : 0.f;
          if (s_begin + t == 0) {
            ai[k] = make_float2(v, 0.f);
          } else {
            const float2 a = (raw & 0x8000) ? make_float2(0.f, 0.f) : ai[k];
            const float sum = a.x + v;
            const float bp = sum - a.x;
            const float err = (a.x - (sum - bp)) + (v - bp);
            ai[k] = make_float2(sum, a.y + err);
          }
        }
      }
      __syncwarp();
    }
  }
};


}  // namespace feasm

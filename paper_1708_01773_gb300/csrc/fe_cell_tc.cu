// Cell integration of Q2 linear elasticity on the 5th-generation tensor cores
// (tcgen05, sm_103a): the per-cell Gram contraction
//     G[(i,a),(j,b)] = sum_q (w_q / det J_q) gh_{a,i}(q) gh_{b,j}(q),
// gh_a = cof(J) gradhat(phihat_a) (Eq. shape_grad with J^{-T} = cof(J)/det J,
// Eq. fematrix), is one 128x96x32 MMA per cell (81 rows/columns used, 27
// quadrature points along K), operands staged in shared memory in the 128-byte
// swizzled K-major layout, the accumulator in tensor memory.
//
// FP32 form: 3xTF32 split (hi = tf32(x), lo = tf32(x - hi); products
// hi*hi + hi*lo + lo*hi) accumulated in FP32, with the 27 quadrature points
// split into two accumulators (points 0-15 and 16-31) that the epilogue adds.
// BF16 form: BF16 operands, one product, FP32 accumulation.
// The epilogue reads G from tensor memory into shared memory and forms
//     K_(a,i),(b,j) = E (lam^ G^{ij}_ab + mu^ G^{ji}_ab + mu^ d_ij sum_k G^{kk}_ab)
// (the isotropic Hooke law written on the Gram blocks), stored with 16-byte
// vector stores; the cell vector is formed in FP64. Geometry (Jacobian,
// cofactors, determinant) is FP64, as in the CUDA-core kernel.
#include <cuda_bf16.h>

#include "fe_launch.h"

namespace feasm {

namespace tc {

constexpr int NB = 27, NL = 81, NLP = 84, NQ = 27;
constexpr int M = 128, N = 96;
constexpr int GS = 85;  // row stride of the G staging area (odd: conflict-free column writes)
constexpr int OFF_AHI = 0, OFF_ALO = 16384, OFF_BHI = 32768, OFF_BLO = 45056;
constexpr int OPER_BYTES = 57344;
constexpr int OFF_G = 57344;
constexpr int OFF_GEO32 = (OFF_G + NL * GS * 4 + 15) & ~15;  // [2][27][12] float: cof (9), w/det
constexpr int OFF_DJW = OFF_GEO32 + 2 * NQ * 12 * 4;  // [2][27][2] float: w*det as hi + lo
constexpr int OFF_X = OFF_DJW + 2 * NQ * 8;          // [24] double
constexpr int OFF_A = OFF_X + 24 * 8;                // [21] double
constexpr int OFF_DPHI = (OFF_A + 21 * 8 + 15) & ~15;  // [27][27][3] float reference gradients
constexpr int OFF_PHI = (OFF_DPHI + NQ * NB * 3 * 4 + 15) & ~15;  // [27][27][2] float reference values, hi + lo
constexpr int OFF_BAR = (OFF_PHI + NQ * NB * 8 + 7) & ~7;  // mbarrier (8 bytes)
constexpr int OFF_TMEM = OFF_BAR + 8;                // tensor-memory base address, then the abort flag
constexpr int SMEM_USED = OFF_TMEM + 8;
// 1 KB of slack to align the base to the 1024-byte swizzle atom; the request is
// also kept above a third of the SM's shared memory so that at most two CTAs
// (2 x 256 tensor-memory columns) share an SM.
constexpr int SMEM_BYTES = (SMEM_USED + 1024) > 80 * 1024 ? (SMEM_USED + 1024) : 80 * 1024;
constexpr uint32_t TMEM_COLS = 256;
static_assert(OFF_GEO32 % 16 == 0 && OFF_DJW % 8 == 0 && SMEM_BYTES <= 227 * 1024, "layout");

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Byte offset of element (row, kbyte) in a K-major operand with 128-byte rows
// and the 128-byte swizzle: 8-row atoms of 1024 bytes, 16-byte chunk c of row
// r stored at chunk c ^ (r % 8).
__device__ __forceinline__ uint32_t swz(int row, int kbyte) {
  return uint32_t((row >> 3) * 1024 + (row & 7) * 128 + ((((kbyte >> 4) ^ row) & 7) << 4) + (kbyte & 15));
}

// Shared-memory matrix descriptor (tcgen05): start address >> 4, leading
// byte offset (unused for swizzled K-major), stride byte offset 1024 (one
// 8-row atom), descriptor version 1, 128-byte swizzle.
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
  uint64_t d = uint64_t((saddr & 0x3FFFFu) >> 4);
  d |= uint64_t(1) << 16;
  d |= uint64_t(1024 >> 4) << 32;
  d |= uint64_t(1) << 46;
  d |= uint64_t(2) << 61;
  return d;
}

// Instruction descriptor: FP32 accumulator, A/B format (TF32 = 2 for
// kind::tf32, BF16 = 1 for kind::f16), both K-major, N >> 3, M >> 4.
__host__ __device__ constexpr uint32_t instr_desc(int m, int n, uint32_t fmt) {
  return (1u << 4) | (fmt << 7) | (fmt << 10) | (uint32_t(n >> 3) << 17) | (uint32_t(m >> 4) << 24);
}

__device__ __forceinline__ void mma_tf32(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
      "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}

__device__ __forceinline__ void mma_bf16(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
      "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
               : "memory");
}

__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}

// 16 consecutive accumulator columns of this thread's lane; the wait is tied
// to the registers so no use can be scheduled before it.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr)
      : "memory");
  asm volatile("tcgen05.wait::ld.sync.aligned;\n"
               : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]),
                 "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]), "+r"(r[14]),
                 "+r"(r[15])
               :
               : "memory");
#pragma unroll
  for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(r[j]);
}

__device__ __forceinline__ float to_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

// hi + lo (FP32 pair) rounded once to FP64: both parts convert exactly, one
// FP64 addition rounds their sum.
__device__ __forceinline__ double feasm_df_to_double(float hi, float lo) {
  return __dadd_rn(double(hi), double(lo));
}

// Same FP64 geometry as the CUDA-core kernel (trilinear map in monomials).
__device__ __forceinline__ void tri_coef(const double* x, int k, double* a) {
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

__device__ __forceinline__ void cof_det(const double* a, double x, double y, double z, double cof[9], double* det) {
  double J[3][3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    J[k][0] = a[0 + k] + a[9 + k] * y + a[12 + k] * z + a[18 + k] * (y * z);
    J[k][1] = a[3 + k] + a[9 + k] * x + a[15 + k] * z + a[18 + k] * (x * z);
    J[k][2] = a[6 + k] + a[12 + k] * x + a[15 + k] * y + a[18 + k] * (x * y);
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

struct Params {
  int64_t n_cells;
  const double* xv;
  const double* w;
  const double* xq;
  const double* phi;
  const float* dphi32;
  const double* coef;
  double f[3];
  float lam_hat, mu_hat;
  float* ke;
  double* fe;
  int* err;
};

// FP64 -> FP32 round to nearest even on the integer bits (normal results;
// values that would under- or overflow FP32 take the hardware conversion).
// Keeps the conversions of the FP64 geometry off the FP64 pipe.
__device__ __forceinline__ float d2f_rn(double x) {
  const uint64_t u = uint64_t(__double_as_longlong(x));
  const int e = int((u >> 52) & 0x7ffu) - 896;
  if (e <= 0 || e >= 255) return __double2float_rn(x);
  const uint64_t mant = u & 0xfffffffffffffull;
  uint32_t body = (uint32_t(e) << 23) | uint32_t(mant >> 29);
  const uint32_t rem = uint32_t(mant & 0x1fffffffu);
  if (rem > 0x10000000u || (rem == 0x10000000u && (body & 1u))) ++body;  // carries into the exponent
  return __uint_as_float((uint32_t(u >> 63) << 31) | body);
}

// Geometry of one cell by warps 0-1 (`t` = thread index 0..63, `xreg` this
// thread's vertex coordinate, t < 24): FP64 monomial coefficients, Jacobian,
// cofactors and determinant; one thread per quadrature point writes the FP32
// cofactors, w/det J in FP32 (geo32), and w det J split into FP32 hi + lo
// (djw). A non-positive det J sets the error word. Warps 0-1 synchronise on
// named barrier 1.
__device__ __forceinline__ void pair_geometry(const Params& p, int t, double xreg, double* X, double* A,
                                              float* geo32, float* djw) {
  if (t < 24) X[t] = xreg;
  asm volatile("bar.sync 1, 64;" ::: "memory");  // geometry role only (64 threads)
  if (t < 3) tri_coef(X, t, A);
  asm volatile("bar.sync 1, 64;" ::: "memory");
  if (t < NQ) {
    double cof[9], det;
    cof_det(A, p.xq[3 * t], p.xq[3 * t + 1], p.xq[3 * t + 2], cof, &det);
    if (!(det > 0.0)) atomicOr(p.err, kErrNegJacobian);
    const double wq = p.w[t];
#pragma unroll
    for (int k = 0; k < 9; ++k) geo32[t * 12 + k] = d2f_rn(cof[k]);
    geo32[t * 12 + 9] = float(wq) / d2f_rn(det);
    const double wd = wq * det;
    const float hi = d2f_rn(wd);
    djw[2 * t] = hi;
    djw[2 * t + 1] = d2f_rn(wd - double(hi));
  }
  asm volatile("bar.sync 1, 64;" ::: "memory");
}

// Persistent: each CTA loops over cells blockIdx.x, blockIdx.x + gridDim.x, ...
// Warp roles: warps 0-7 ("math") build the operands, issue the MMAs (thread 0),
// move the accumulators to shared memory and form the cell matrix and cell
// vector of cell n; warps 8-9 ("geometry") compute the FP64 geometry of cell
// n+1 meanwhile, into the other half of a double buffer. The two roles meet
// once per cell at a block barrier; inside the math role, named barrier 2
// (256 threads) orders its phases.
constexpr int MATH_THREADS = 256;
constexpr int ALL_THREADS = MATH_THREADS + 64;

__device__ __forceinline__ void math_sync() { asm volatile("bar.sync 2, 256;" ::: "memory"); }

template <bool BF16>
__global__ void __launch_bounds__(ALL_THREADS) k_cell_tc(Params p) {
  extern __shared__ unsigned char smem_raw[];
  unsigned char* sm = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const bool geo_role = tid >= MATH_THREADS;
  const int gt = tid - MATH_THREADS;  // thread index inside the geometry role
  float* G = reinterpret_cast<float*>(sm + OFF_G);
  float* geo32_0 = reinterpret_cast<float*>(sm + OFF_GEO32);
  float* djw_0 = reinterpret_cast<float*>(sm + OFF_DJW);
  double* X = reinterpret_cast<double*>(sm + OFF_X);
  double* A = reinterpret_cast<double*>(sm + OFF_A);
  const uint32_t sbase = smem_u32(sm);
  const uint32_t bar = sbase + OFF_BAR;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(sm + OFF_TMEM);
  int* abort_flag = reinterpret_cast<int*>(sm + OFF_TMEM + 4);

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(sbase + OFF_TMEM),
                 "r"(TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(1u) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    *abort_flag = 0;
  }
  float* sdphi = reinterpret_cast<float*>(sm + OFF_DPHI);
  float* sphi = reinterpret_cast<float*>(sm + OFF_PHI);
  double xnext = 0.0;
  if (!geo_role) {
    // zero the operand area once: padding rows/columns are never written again
    for (int i = tid; i < OPER_BYTES / 16; i += MATH_THREADS) reinterpret_cast<uint4*>(sm)[i] = make_uint4(0, 0, 0, 0);
    for (int i = tid; i < NQ * NB * 3; i += MATH_THREADS) sdphi[i] = p.dphi32[i];
    for (int i = tid; i < NQ * NB; i += MATH_THREADS) {
      const double v = p.phi[i];
      const float hi = __double2float_rn(v);
      sphi[2 * i] = hi;
      sphi[2 * i + 1] = __double2float_rn(v - double(hi));
    }
  } else {
    if (int64_t(blockIdx.x) < p.n_cells) {
      const double x0 = gt < 24 ? p.xv[int64_t(blockIdx.x) * 24 + gt] : 0.0;
      pair_geometry(p, gt, x0, X, A, geo32_0, djw_0);
    }
    if (gt < 24 && int64_t(blockIdx.x) + gridDim.x < p.n_cells)
      xnext = p.xv[(int64_t(blockIdx.x) + gridDim.x) * 24 + gt];
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = *tmem_slot;
  constexpr uint32_t IDESC = instr_desc(M, N, BF16 ? 1u : 2u);
  uint32_t phase = 0;
  int buf = 0;

  for (int64_t e = blockIdx.x; e < p.n_cells; e += gridDim.x, buf ^= 1) {
    if (geo_role) {
      // geometry of the next cell (FP64), then fetch the coordinates of the one after
      if (e + gridDim.x < p.n_cells) {
        pair_geometry(p, gt, xnext, X, A, geo32_0 + (buf ^ 1) * (NQ * 12), djw_0 + (buf ^ 1) * (2 * NQ));
        if (gt < 24 && e + 2 * int64_t(gridDim.x) < p.n_cells) xnext = p.xv[(e + 2 * int64_t(gridDim.x)) * 24 + gt];
      }
    } else {
      const float* geo32 = geo32_0 + buf * (NQ * 12);
      const float* djw = djw_0 + buf * (2 * NQ);
      // 1. operands: A[(i,a)][q] = (w/det) gh_{a,i}(q), B[(j,b)][q] = gh_{b,j}(q);
      //    one thread per (node a, point q) forms the three components i.
      for (int idx = tid; idx < NB * NQ; idx += MATH_THREADS) {
        const int a = idx / NQ, q = idx - a * NQ;
        const float* gq = geo32 + q * 12;
        const float* dp = sdphi + (q * NB + a) * 3;
        const float d0 = dp[0], d1 = dp[1], d2 = dp[2], sq = gq[9];
#pragma unroll
        for (int i = 0; i < 3; ++i) {
          const float g = fmaf(gq[3 * i + 2], d2, fmaf(gq[3 * i + 1], d1, gq[3 * i] * d0));
          const float av = sq * g;
          const int m = i * NB + a;
          if (BF16) {
            const uint32_t o = swz(m, q * 2);
            *reinterpret_cast<__nv_bfloat16*>(sm + OFF_AHI + o) = __float2bfloat16_rn(av);
            *reinterpret_cast<__nv_bfloat16*>(sm + OFF_BHI + o) = __float2bfloat16_rn(g);
          } else {
            const uint32_t o = swz(m, q * 4);
            const float ah = to_tf32(av), bh = to_tf32(g);
            *reinterpret_cast<float*>(sm + OFF_AHI + o) = ah;
            *reinterpret_cast<float*>(sm + OFF_ALO + o) = to_tf32(av - ah);
            *reinterpret_cast<float*>(sm + OFF_BHI + o) = bh;
            *reinterpret_cast<float*>(sm + OFF_BLO + o) = to_tf32(g - bh);
          }
        }
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      math_sync();
      // 2. one thread issues the MMAs; completion is signalled on the mbarrier
      if (tid == 0) {
        fence_after();
        const uint64_t ahi = sw128_desc(sbase + OFF_AHI), alo = sw128_desc(sbase + OFF_ALO);
        const uint64_t bhi = sw128_desc(sbase + OFF_BHI), blo = sw128_desc(sbase + OFF_BLO);
        if (BF16) {
#pragma unroll
          for (int ks = 0; ks < 2; ++ks) mma_bf16(tmem, ahi + 2 * ks, bhi + 2 * ks, IDESC, ks > 0);
        } else {
#pragma unroll
          for (int g = 0; g < 2; ++g)
#pragma unroll
            for (int k2 = 0; k2 < 2; ++k2) {
              const int ks = 2 * g + k2;
              const uint32_t d = tmem + uint32_t(g * N);
              mma_tf32(d, alo + 2 * ks, bhi + 2 * ks, IDESC, k2 > 0);
              mma_tf32(d, ahi + 2 * ks, blo + 2 * ks, IDESC, 1);
              mma_tf32(d, ahi + 2 * ks, bhi + 2 * ks, IDESC, 1);
            }
        }
        mma_commit(bar);
      }
      __syncwarp();
      // 3. bounded wait for the MMAs (about one second of clock cycles at most)
      bool done = false;
      {
        const long long t0 = clock64();
        while (!done) {
          done = mbar_try_wait(bar, phase);
          if (!done && clock64() - t0 > (1ll << 31)) break;
        }
      }
      done = __all_sync(0xffffffffu, done);  // tcgen05.ld below is warp-collective
      phase ^= 1u;
      if (!done) *abort_flag = 1;
      fence_after();
      // 4. accumulators -> shared staging of G (FP32): warp w reads lanes
      //    32 (w % 4) .. +31 (rows), column half w / 4
      if (done) {
        const int row = 32 * (warp & 3) + lane;
        const uint32_t lane_addr = tmem + (uint32_t(32 * (warp & 3)) << 16);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          const int col0 = ((warp >> 2) * 3 + c) * 16;
          float v[16];
          tmem_ld16(lane_addr + uint32_t(col0), v);
          if (!BF16) {
            float v2[16];
            tmem_ld16(lane_addr + uint32_t(N + col0), v2);
#pragma unroll
            for (int j = 0; j < 16; ++j) v[j] += v2[j];
          }
          if (row < NL) {
#pragma unroll
            for (int j = 0; j < 16; ++j)
              if (col0 + j < NL) G[row * GS + col0 + j] = v[j];
          }
        }
      }
      fence_before();
      math_sync();
      // 5. warps 1-7: K^e from the Gram blocks, one thread per node pair (a, b)
      //    (the nine G^{ij}_ab give the nine entries K_(a,i),(b,j): the
      //    transposed block and the trace come from the same values);
      //    consecutive threads take consecutive b (conflict-free reads,
      //    coalesced stores). Warp 0: the cell vector.
      if (*abort_flag == 0) {
        if (warp > 0) {
          const float E = float(p.coef[e]);
          const float lh = p.lam_hat * E, mh = p.mu_hat * E;
          float* K = p.ke + e * (NL * NLP);
          for (int idx = tid - 32; idx < NB * NB; idx += MATH_THREADS - 32) {
            const int a = idx / NB, b = idx - a * NB;
            float g[3][3];
#pragma unroll
            for (int i = 0; i < 3; ++i)
#pragma unroll
              for (int j = 0; j < 3; ++j) g[i][j] = G[(i * NB + a) * GS + j * NB + b];
            const float tr = g[0][0] + g[1][1] + g[2][2];
#pragma unroll
            for (int i = 0; i < 3; ++i)
#pragma unroll
              for (int j = 0; j < 3; ++j) {
                float v = lh * g[i][j] + mh * g[j][i];
                if (i == j) v += mh * tr;
                K[(i * NB + a) * NLP + j * NB + b] = v;
              }
          }
        } else if (lane < NB) {
          // f_a = sum_q (w det J)_q phihat_a(x_q), both factors as FP32 hi + lo,
          // products and sum in double-float arithmetic (error ~2^-46
          // relative), rounded once to FP64.
          float sh = 0.f, sl = 0.f;
          for (int q = 0; q < NQ; ++q) {
            const float ah = djw[2 * q], al = djw[2 * q + 1];
            const float bh = sphi[2 * (q * NB + lane)], bl = sphi[2 * (q * NB + lane) + 1];
            const float ph = ah * bh;
            const float pe = fmaf(ah, bh, -ph) + (ah * bl + al * bh);
            const float sum = sh + ph;
            const float bp = sum - sh;
            const float err = (sh - (sum - bp)) + (ph - bp);
            sh = sum;
            sl += err + pe;
          }
          const double f = feasm_df_to_double(sh, sl);
          double* fe = p.fe + e * NL;
#pragma unroll
          for (int k = 0; k < 3; ++k) fe[k * NB + lane] = p.f[k] * f;
        }
      }
    }
    // cell boundary: the next geometry is ready and the staging area is free
    __syncthreads();
    if (*abort_flag) {
      if (tid == 0) atomicOr(p.err, kErrTimeout);
      break;
    }
  }
  fence_before();
  __syncthreads();
  if (warp == 0) {
    fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
  }
}

}  // namespace tc

bool cell_tc_applicable(const fe_space* s, fe_precision prec) {
  return s->order == 2 && s->ncomp == 3 && s->nq1d == 3 && prec != FE_PREC_FP64;
}

cudaError_t launch_cell_tc(const fe_space* s, const double* coef, const double force[3], fe_precision prec,
                           cudaStream_t st) {
  if (s->n_cells == 0) return cudaSuccess;
  tc::Params p;
  p.n_cells = s->n_cells;
  p.xv = s->d_xv;
  p.w = s->d_w;
  p.xq = s->d_xq;
  p.phi = s->d_phi;
  p.dphi32 = s->d_dphi32;
  p.coef = coef;
  for (int k = 0; k < 3; ++k) p.f[k] = force[k];
  p.lam_hat = float(s->nu / ((1.0 + s->nu) * (1.0 - 2.0 * s->nu)));
  p.mu_hat = float(1.0 / (2.0 * (1.0 + s->nu)));
  p.ke = static_cast<float*>(s->d_ke);
  p.fe = s->d_fe;
  p.err = s->d_err;
  int nsm = 152;
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, s->device);
  auto run = [&](auto kern) -> cudaError_t {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, tc::SMEM_BYTES);
    if (e != cudaSuccess) return e;
    const int64_t grid = std::min<int64_t>(s->n_cells, int64_t(nsm) * 2);
    kern<<<unsigned(grid), tc::ALL_THREADS, tc::SMEM_BYTES, st>>>(p);
    return cudaGetLastError();
  };
  return prec == FE_PREC_BF16 ? run(tc::k_cell_tc<true>) : run(tc::k_cell_tc<false>);
}

}  // namespace feasm

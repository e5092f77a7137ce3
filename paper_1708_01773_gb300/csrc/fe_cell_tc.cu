// Cell integration of Q2 linear elasticity on the 5th-generation tensor cores
// (tcgen05, sm_103a): the per-cell Gram contraction
//     G[(i,a),(j,b)] = sum_q (w_q / det J_q) gh_{a,i}(q) gh_{b,j}(q),
// gh_a = cof(J) gradhat(phihat_a) (Eq. shape_grad with J^{-T} = cof(J)/det J,
// Eq. fematrix), is one 128x96x32 MMA group per cell (81 rows/columns used,
// 27 quadrature points along K). Both operands are the one matrix
// C[(i,a)][q] = sqrt(w_q / det J_q) gh_{a,i}(q), so that G = C C^T (B is the
// first 96 rows of A); C is staged in shared memory in the 128-byte swizzled
// K-major layout, the accumulator in tensor memory.
//
// FP32 form: 3xTF32 split (hi = tf32(x), lo = tf32(x - hi); products
// hi*hi + hi*lo + lo*hi) accumulated in FP32, the 27 points split into two
// accumulators (points 0-15 and 16-31) that the epilogue adds. BF16 form: BF16
// operand, one product, FP32 accumulation. The epilogue forms
//     K_(a,i),(b,j) = E (lam^ G^{ij}_ab + mu^ G^{ji}_ab + mu^ d_ij sum_k G^{kk}_ab)
// (the isotropic Hooke law written on the Gram blocks). Geometry (Jacobian,
// cofactors, determinant) is FP64; the cell vector is a double-float sum
// rounded once to FP64.
//
// One persistent CTA per SM runs a warp-specialised pipeline over its cells:
//   warp 0      allocates tensor memory; lane 0 issues the MMAs of cell n
//               into accumulator stage n % 2 once its operands are staged;
//   warps 1-4   FP64 geometry of cell n into geometry slot n % 4, warp
//               1 + n % 4 (four cells at a time, one per SM sub-partition:
//               each sub-partition has its own small share of the FP64 pipe,
//               and an FP64 warp instruction costs the same with 27 active
//               lanes as with 7, so a whole cell's points fill one warp);
//   warps 5-11  operands of cell n into operand stage n % 2 (one item per
//               thread), and the cell vector of cell n (idle threads);
//   warps 12-19 accumulators of cell n -> shared staging -> cell matrix.
// Hand-offs use mbarriers (full/empty per slot or stage); every wait is
// bounded (about one second of clock cycles), after which the role sets
// FE_ERR_TIMEOUT and leaves its loop; the MMA thread then waits (bounded) for
// its last MMAs to complete, and the CTA frees tensor memory and exits.
#include <cuda_bf16.h>

#include "fe_device.cuh"
#include "fe_pair_table.h"
#include "fe_sync.cuh"
#include "fe_tcgen05.cuh"

namespace feasm {

namespace tc {

constexpr int NB = 27, NL = 81, NLP = 84, NQ = 27;
constexpr int M = 128, N = 96;
constexpr int GS = 100;  // row stride of the G staging area (GS % 32 == 4: conflict-free 16-byte column writes)
// warp roles
constexpr int W_MMA = 0, W_GEO0 = 1, N_GEO = 4, W_OP0 = 5, N_OP = 7, W_EPI0 = 12, N_EPI = 8;
constexpr int THREADS = 32 * (W_EPI0 + N_EPI);
constexpr int OP_THREADS = 32 * N_OP, EPI_THREADS = 32 * N_EPI;
constexpr int GEO_SLOTS = 4;
// shared memory (offsets from a 1024-byte aligned base)
constexpr int STAGE_BYTES = 32768;  // C hi 16 KB, C lo 16 KB (128 rows of 128 bytes each)
constexpr int OFF_CHI = 0, OFF_CLO = 16384;
constexpr int OFF_G = 2 * STAGE_BYTES;
// geo32 [27][12] float, djw [27][2] float; a multiple of 16 bytes, since the
// operand warps read geo32 rows as float4
constexpr int GEO_SLOT_BYTES = (NQ * 12 * 4 + NQ * 2 * 4 + 15) & ~15;
constexpr int G_BYTES = NL * GS * 4;  // 32,400: a multiple of 16; two buffers
constexpr int OFF_GEO = (OFF_G + 2 * G_BYTES + 15) & ~15;
// per geometry warp: edge differences [3][4][3] and Jacobian columns [3][9][3] (double)
constexpr int GEO_WARP_DOUBLES = 36 + 81;
constexpr int OFF_EJ = (OFF_GEO + GEO_SLOTS * GEO_SLOT_BYTES + 15) & ~15;
constexpr int OFF_WT = OFF_EJ + N_GEO * GEO_WARP_DOUBLES * 8;              // [9][4] double bilinear weights
constexpr int OFF_DPHI = (OFF_WT + 36 * 8 + 15) & ~15;                     // [27][27][3] float
constexpr int OFF_PHI = (OFF_DPHI + NQ * NB * 3 * 4 + 15) & ~15;           // [27][27][2] float hi + lo
constexpr int OFF_KS = (OFF_PHI + NQ * NB * 8 + 15) & ~15;                 // [2][81][84] float cell-matrix staging
constexpr int KS_BYTES = NL * NLP * 4;                                      // 27,216: a multiple of 16
constexpr int OFF_PAIRS = OFF_KS + 2 * KS_BYTES;  // [PAIR_GROUPS][32] u16 node pairs (kPairTable)
constexpr int OFF_BAR = (OFF_PAIRS + PAIR_GROUPS * 32 * 2 + 7) & ~7;
// mbarriers: geo_full[4], geo_empty[4], op_full[2], op_empty[2], acc_full[2], acc_empty[2], drain
constexpr int BAR_GEO_FULL = 0, BAR_GEO_EMPTY = 4, BAR_OP_FULL = 8, BAR_OP_EMPTY = 10, BAR_ACC_FULL = 12,
              BAR_ACC_EMPTY = 14, BAR_DRAIN = 16, N_BARS = 17;
constexpr int OFF_TMEM = OFF_BAR + N_BARS * 8;  // tensor-memory base address, then the abort flag
constexpr int SMEM_USED = OFF_TMEM + 8;
constexpr int SMEM_BYTES = SMEM_USED + 1024;  // + alignment slack; > half of the SM: one CTA per SM
constexpr uint32_t TMEM_COLS = 512;            // two accumulator stages of 2 x 96 columns, at 0 and 256
static_assert(G_BYTES % 16 == 0 && OFF_GEO % 16 == 0 && GEO_SLOT_BYTES % 16 == 0 && OFF_DPHI % 16 == 0 && OFF_KS % 16 == 0 &&
                  KS_BYTES % 16 == 0 && OFF_BAR % 8 == 0 &&
                  SMEM_BYTES <= 227 * 1024,
              "layout");
static_assert(SMEM_BYTES > 114 * 1024, "one CTA per SM (512 tensor-memory columns)");
static_assert(GEO_SLOTS == N_GEO, "geometry warp w owns geometry slot w");

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

// Named-barrier OR-reduction over the `count` threads of barrier `id`.
template <int ID, int COUNT>
__device__ __forceinline__ bool bar_or(bool v) {
  uint32_t r;
  asm volatile(
      "{\n.reg .pred p, q;\nsetp.ne.u32 p, %1, 0;\nbar.red.or.pred q, %2, %3, p;\nselp.u32 %0, 1, 0, q;\n}\n"
      : "=r"(r)
      : "r"(uint32_t(v)), "n"(ID), "n"(COUNT)
      : "memory");
  return r != 0;
}

template <int ID, int COUNT>
__device__ __forceinline__ void bar_sync() {
  asm volatile("bar.sync %0, %1;" ::"n"(ID), "n"(COUNT) : "memory");
}

// Per-lane constants of a geometry warp. The Jacobian of the trilinear map
// is built from the 36 edge differences of the cell (direction d, edge c of
// the four parallel ones, component k): column d at reference point xi is
// the bilinear interpolation of the four edge differences of direction d in
// the other two coordinates (u, v) (in axis order), with weights
// (1-u)(1-v), u(1-v), (1-u)v, uv for edges c = 0..3 (bit 0 of c: u side,
// bit 1: v side). Column d depends on (u, v) only, so the 27 points need 9
// pairs per column: 81 entries (d, pair, k), 3 per lane. Lanes 0-26 then
// take one quadrature point each.
struct GeoLane {
  int src0[2], src1[2];  // edge-difference items: lanes holding the two vertex values
  int jw[3], je[3];      // Jacobian items: weight row and edge-difference base
  int q, j0, j1, j2;
  double wq;
  float wq32;
};

__device__ __forceinline__ GeoLane geo_lane(const Params& p, int lane) {
  GeoLane g;
#pragma unroll
  for (int r = 0; r < 2; ++r) {
    const int L = (32 * r + lane) < 36 ? 32 * r + lane : 0;
    const int d = L / 12, c = (L / 3) % 4, k = L % 3, bu = c & 1, bv = c >> 1;
    const int v0 = d == 0 ? 2 * bu + 4 * bv : d == 1 ? bu + 4 * bv : bu + 2 * bv;
    const int v1 = v0 + (d == 0 ? 1 : d == 1 ? 2 : 4);
    g.src0[r] = 3 * v0 + k;
    g.src1[r] = 3 * v1 + k;
  }
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    const int t = (32 * r + lane) < 81 ? 32 * r + lane : 0;
    const int d = t / 27, pr = (t % 27) / 3, k = t % 3;
    g.jw[r] = 4 * pr;
    g.je[r] = 12 * d + k;
  }
  g.q = lane < NQ ? lane : -1;
  const int q = lane < NQ ? lane : 0;
  const int ix = q % 3, iy = (q / 3) % 3, iz = q / 9;
  g.j0 = (0 + iy + 3 * iz) * 3;
  g.j1 = (9 + ix + 3 * iz) * 3;
  g.j2 = (18 + ix + 3 * iy) * 3;
  g.wq = p.w[q];
  g.wq32 = d2f_rn(g.wq);
  return g;
}

// FP64 geometry of one cell by one geometry warp (xreg = this lane's vertex
// coordinate for lanes < 24, vertex v component k at lane 3 v + k): edge
// differences (ED), Jacobian columns per point pair (JC), then per quadrature
// point the FP32 cofactors and w/det J (geo32) and w det J as FP32 hi + lo
// (djw). A non-positive det J sets the error word.
__device__ __forceinline__ void cell_geometry(const Params& p, const GeoLane& g, int lane, double xreg, double* ED,
                                              double* JC, const double* WT, float* geo32, float* djw) {
#pragma unroll
  for (int r = 0; r < 2; ++r) {
    const double x1 = __shfl_sync(0xffffffffu, xreg, g.src1[r]);
    const double x0 = __shfl_sync(0xffffffffu, xreg, g.src0[r]);
    if (32 * r + lane < 36) ED[32 * r + lane] = x1 - x0;
  }
  __syncwarp();
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    if (32 * r + lane < 81) {
      const double* w = WT + g.jw[r];
      const double* ed = ED + g.je[r];
      JC[32 * r + lane] = fma(w[3], ed[9], fma(w[2], ed[6], fma(w[1], ed[3], w[0] * ed[0])));
    }
  }
  __syncwarp();
  if (g.q >= 0) {
    const int q = g.q;
    double J[3][3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      J[k][0] = JC[g.j0 + k];
      J[k][1] = JC[g.j1 + k];
      J[k][2] = JC[g.j2 + k];
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
    if (!(det > 0.0)) atomicOr(p.err, kErrNegJacobian);
#pragma unroll
    for (int k = 0; k < 9; ++k) geo32[q * 12 + k] = d2f_rn(cof[k]);
    const float s = g.wq32 / d2f_rn(det);
    geo32[q * 12 + 9] = s;
    geo32[q * 12 + 10] = sqrtf(s);
    const double wd = g.wq * det;
    const float hi = d2f_rn(wd);
    djw[2 * q] = hi;
    djw[2 * q + 1] = d2f_rn(wd - f32_to_f64_exact(hi));
  }
}

// Cell vector of one cell, entry a: f_a = sum_q (w det J)_q phihat_a(x_q),
// both factors as FP32 hi + lo, products and sums in double-float arithmetic
// (three interleaved partial sums over q = 0, 1, 2 mod 3, then combined),
// rounded once to FP64 and scaled by the body force.
__device__ __forceinline__ void cell_vector(const Params& p, int64_t e, int a, const float* djw, const float* sphi) {
  float sh[3] = {0.f, 0.f, 0.f}, sl[3] = {0.f, 0.f, 0.f};
#pragma unroll
  for (int q = 0; q < NQ; ++q) {
    const int r = q % 3;
    const float ah = djw[2 * q], al = djw[2 * q + 1];
    const float bh = sphi[2 * (q * NB + a)], bl = sphi[2 * (q * NB + a) + 1];
    const float ph = ah * bh;
    const float pe = fmaf(ah, bh, -ph) + (ah * bl + al * bh);
    const float sum = sh[r] + ph;
    const float bp = sum - sh[r];
    const float err = (sh[r] - (sum - bp)) + (ph - bp);
    sh[r] = sum;
    sl[r] += err + pe;
  }
  float h = sh[0], l = sl[0];
#pragma unroll
  for (int r = 1; r < 3; ++r) {
    const float sum = h + sh[r];
    const float bp = sum - h;
    const float err = (h - (sum - bp)) + (sh[r] - bp);
    h = sum;
    l += err + sl[r];
  }
  const double f = __dadd_rn(f32_to_f64_exact(h), f32_to_f64_exact(l));  // h + l rounded once
  double* fe = p.fe + e * NL;
#pragma unroll
  for (int k = 0; k < 3; ++k) fe[k * NB + a] = p.f[k] * f;
}

// Operand of one cell from its geometry slot: C[(i,a)][q] =
// sqrt(w/det) gh_{a,i}(q); one thread per (node a, 4 points q0..q0+3) forms
// the three components and stores each K-chunk of the hi and lo arrays with
// one vector store (points q >= 27 are the zero padding of K).
template <bool BF16>
__device__ __forceinline__ void build_operands(unsigned char* st, const float* geo32, const float* sdphi, int t) {
  for (int idx = t; idx < NB * 7; idx += OP_THREADS) {
    // consecutive threads take consecutive nodes of one 4-point chunk: the
    // geometry-row loads are broadcasts, the reference-gradient loads
    // (stride 3 words) and the swizzled 16-byte stores (consecutive rows) are
    // conflict-free
    const int qc = idx / NB, a = idx - qc * NB, q0 = 4 * qc;
    float g[3][4], sq[4];
#pragma unroll
    for (int dq = 0; dq < 4; ++dq) {
      const int q = q0 + dq;
      if (q < NQ) {
        const float4* gq4 = reinterpret_cast<const float4*>(geo32 + q * 12);
        const float4 c0 = gq4[0], c1 = gq4[1], c2 = gq4[2];
        const float* dp = sdphi + (q * NB + a) * 3;
        const float d0 = dp[0], d1 = dp[1], d2 = dp[2];
        g[0][dq] = fmaf(c0.z, d2, fmaf(c0.y, d1, c0.x * d0));
        g[1][dq] = fmaf(c1.y, d2, fmaf(c1.x, d1, c0.w * d0));
        g[2][dq] = fmaf(c2.x, d2, fmaf(c1.w, d1, c1.z * d0));
        sq[dq] = c2.z;  // sqrt(w/det)
      } else {
        g[0][dq] = g[1][dq] = g[2][dq] = 0.f;
        sq[dq] = 0.f;
      }
    }
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      const int m = i * NB + a;
      if (BF16) {
        const uint32_t o = swz(m, q0 * 2);
        __nv_bfloat162 c0 = __floats2bfloat162_rn(sq[0] * g[i][0], sq[1] * g[i][1]);
        __nv_bfloat162 c1 = __floats2bfloat162_rn(sq[2] * g[i][2], sq[3] * g[i][3]);
        *reinterpret_cast<uint2*>(st + OFF_CHI + o) =
            make_uint2(*reinterpret_cast<uint32_t*>(&c0), *reinterpret_cast<uint32_t*>(&c1));
      } else {
        const uint32_t o = swz(m, q0 * 4);
        float ch[4], cl[4];
#pragma unroll
        for (int dq = 0; dq < 4; ++dq) {
          const float cv = sq[dq] * g[i][dq];
          ch[dq] = to_tf32(cv);
          cl[dq] = to_tf32(cv - ch[dq]);
        }
        *reinterpret_cast<float4*>(st + OFF_CHI + o) = make_float4(ch[0], ch[1], ch[2], ch[3]);
        *reinterpret_cast<float4*>(st + OFF_CLO + o) = make_float4(cl[0], cl[1], cl[2], cl[3]);
      }
    }
  }
}

template <bool BF16>
__global__ void __launch_bounds__(THREADS, 1) k_cell_tc(Params p) {
  extern __shared__ unsigned char smem_raw[];
  unsigned char* sm = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  float* G = reinterpret_cast<float*>(sm + OFF_G);
  float* sdphi = reinterpret_cast<float*>(sm + OFF_DPHI);
  float* sphi = reinterpret_cast<float*>(sm + OFF_PHI);
  const uint32_t sbase = smem_u32(sm);
  auto bar = [&](int i) { return sbase + OFF_BAR + 8u * uint32_t(i); };
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(sm + OFF_TMEM);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(sm + OFF_TMEM + 4);
  const int64_t n_mine = p.n_cells > blockIdx.x ? (p.n_cells - 1 - blockIdx.x) / gridDim.x + 1 : 0;

  if (warp == W_MMA) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(sbase + OFF_TMEM),
                 "r"(TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    for (int i = 0; i < GEO_SLOTS; ++i) {
      mbar_init(bar(BAR_GEO_FULL + i), 32);
      mbar_init(bar(BAR_GEO_EMPTY + i), OP_THREADS);
    }
    for (int i = 0; i < 2; ++i) {
      mbar_init(bar(BAR_OP_FULL + i), OP_THREADS);
      mbar_init(bar(BAR_OP_EMPTY + i), 1);
      mbar_init(bar(BAR_ACC_FULL + i), 1);
      mbar_init(bar(BAR_ACC_EMPTY + i), EPI_THREADS);
    }
    mbar_init(bar(BAR_DRAIN), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    *abort_flag = 0;
  }
  // zero both operand stages once (padding rows and columns are never written
  // again), load the reference tables
  for (int i = tid; i < 2 * STAGE_BYTES / 16; i += THREADS) reinterpret_cast<uint4*>(sm)[i] = make_uint4(0, 0, 0, 0);
  for (int i = tid; i < NQ * NB * 3; i += THREADS) sdphi[i] = p.dphi32[i];
  for (int i = tid; i < PAIR_GROUPS * 32; i += THREADS)
    reinterpret_cast<uint16_t*>(sm + OFF_PAIRS)[i] = kPairTable[i / 32][i % 32];
  if (tid < 36) {
    const int pr = tid / 4, c = tid % 4;
    const double u = p.xq[3 * (pr % 3)], v = p.xq[3 * (pr / 3)];
    reinterpret_cast<double*>(sm + OFF_WT)[tid] = ((c & 1) ? u : 1.0 - u) * ((c >> 1) ? v : 1.0 - v);
  }
  for (int i = tid; i < NQ * NB; i += THREADS) {
    const double v = p.phi[i];
    const float hi = __double2float_rn(v);
    sphi[2 * i] = hi;
    sphi[2 * i + 1] = __double2float_rn(v - double(hi));
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = *tmem_slot;
  bool failed = false;

  if (warp == W_MMA) {
    // ---------------------------------------------------------------- MMA issue
    if (lane == 0) {
      constexpr uint32_t IDESC = instr_desc(M, N, BF16 ? 1u : 2u);
      for (int64_t n = 0; n < n_mine && !failed; ++n) {
        const int st = int(n & 1);
        const uint32_t use = uint32_t((n >> 1) & 1);
        if (!mbar_wait(bar(BAR_OP_FULL + st), use) || !mbar_wait(bar(BAR_ACC_EMPTY + st), use ^ 1u)) {
          failed = true;
          break;
        }
        fence_after();
        const uint32_t sb = sbase + uint32_t(st * STAGE_BYTES);
        // A = C (128 rows), B = the first 96 rows of C: the same descriptors
        const uint64_t ahi = sw128_desc(sb + OFF_CHI), alo = sw128_desc(sb + OFF_CLO);
        const uint64_t bhi = ahi, blo = alo;
        const uint32_t dst = tmem + uint32_t(st * 256);
        if (BF16) {
#pragma unroll
          for (int ks = 0; ks < 2; ++ks) mma_bf16(dst, ahi + 2 * ks, bhi + 2 * ks, IDESC, ks > 0);
        } else {
#pragma unroll
          for (int g = 0; g < 2; ++g)
#pragma unroll
            for (int k2 = 0; k2 < 2; ++k2) {
              const int ks = 2 * g + k2;
              const uint32_t d = dst + uint32_t(g * N);
              mma_tf32(d, alo + 2 * ks, bhi + 2 * ks, IDESC, k2 > 0);
              mma_tf32(d, ahi + 2 * ks, blo + 2 * ks, IDESC, 1);
              mma_tf32(d, ahi + 2 * ks, bhi + 2 * ks, IDESC, 1);
            }
        }
        mma_commit(bar(BAR_OP_EMPTY + st));   // operands may be overwritten
        mma_commit(bar(BAR_ACC_FULL + st));   // accumulators ready for the epilogue
      }
      // Every MMA this thread issued completes before the tensor memory is
      // freed: on the normal path the epilogue has already waited for all of
      // them; after a timeout elsewhere the last cell's MMAs may still be in
      // flight, and this commit arrives only once they are done (bounded wait).
      mma_commit(bar(BAR_DRAIN));
      if (!mbar_wait(bar(BAR_DRAIN), 0)) failed = true;
    }
    __syncwarp();
  } else if (warp >= W_GEO0 && warp < W_GEO0 + N_GEO) {
    // ---------------------------------------------------------------- geometry
    const int gw = warp - W_GEO0;  // cells n = gw, gw + 4, ... into slot gw
    double* ED = reinterpret_cast<double*>(sm + OFF_EJ) + gw * GEO_WARP_DOUBLES;
    double* JC = ED + 36;
    const double* WT = reinterpret_cast<const double*>(sm + OFF_WT);
    const GeoLane g = geo_lane(p, lane);
    float* geo32 = reinterpret_cast<float*>(sm + OFF_GEO + gw * GEO_SLOT_BYTES);
    float* djw = geo32 + NQ * 12;
    double xnext = (lane < 24 && gw < n_mine) ? p.xv[(int64_t(blockIdx.x) + int64_t(gw) * gridDim.x) * 24 + lane] : 0.0;
    for (int64_t n = gw; n < n_mine; n += N_GEO) {
      const int64_t e = blockIdx.x + n * int64_t(gridDim.x);
      const uint32_t use = uint32_t((n / GEO_SLOTS) & 1);
      const bool ok = __all_sync(0xffffffffu, mbar_wait(bar(BAR_GEO_EMPTY + gw), use ^ 1u));
      if (!ok) {
        failed = true;
        break;
      }
      const double xcur = xnext;
      if (lane < 24 && n + N_GEO < n_mine) xnext = p.xv[(e + int64_t(N_GEO) * gridDim.x) * 24 + lane];
      cell_geometry(p, g, lane, xcur, ED, JC, WT, geo32, djw);
      mbar_arrive(bar(BAR_GEO_FULL + gw));
    }
  } else if (warp >= W_OP0 && warp < W_OP0 + N_OP) {
    // ---------------------------------------------------------------- operands
    const int t = tid - 32 * W_OP0;
    for (int64_t n = 0; n < n_mine; ++n) {
      const int slot = int(n % GEO_SLOTS), st = int(n & 1);
      const uint32_t guse = uint32_t((n / GEO_SLOTS) & 1), use = uint32_t((n >> 1) & 1);
      if (!mbar_wait(bar(BAR_GEO_FULL + slot), guse) || !mbar_wait(bar(BAR_OP_EMPTY + st), use ^ 1u)) {
        failed = true;
        break;
      }
      const float* geo32 = reinterpret_cast<const float*>(sm + OFF_GEO + slot * GEO_SLOT_BYTES);
      build_operands<BF16>(sm + st * STAGE_BYTES, geo32, sdphi, t);
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      mbar_arrive(bar(BAR_OP_FULL + st));
      // threads 192-218 have no operand item: they form the cell vector
      if (t >= 192 && t < 192 + NB) cell_vector(p, blockIdx.x + n * int64_t(gridDim.x), t - 192, geo32 + NQ * 12, sphi);
      mbar_arrive(bar(BAR_GEO_EMPTY + slot));
    }
  } else {
    // ---------------------------------------------------------------- epilogue
    // Software-pipelined: iteration n starts the accumulator loads of cell n,
    // forms K^e of cell n - 1 from G buffer (n - 1) % 2 while they are in
    // flight, stores cell n's G into buffer n % 2 and releases its
    // accumulators; one barrier per cell, then one thread sends K^e of cell
    // n - 1 with a bulk copy from staging buffer (n - 1) % 2.
    const int t = tid - 32 * W_EPI0;
    const int ew = warp - W_EPI0;  // 0..7: lane quadrant warp % 4, column half ew / 4
    const int row = 32 * (warp & 3) + lane;
    const int cbase = (ew >> 2) * 48;  // this warp's 48 of the 96 accumulator columns
    const uint16_t* pairs = reinterpret_cast<const uint16_t*>(sm + OFF_PAIRS);
    double coef_next = n_mine > 0 ? p.coef[blockIdx.x] : 0.0;
    float E_prev = 0.f;
    uint32_t ra[32], rb[32];
#pragma unroll
    for (int j = 0; j < 32; ++j) ra[j] = rb[j] = 0u;
    for (int64_t n = 0; n <= n_mine; ++n) {
      const bool drain = n < n_mine, form = n > 0;
      const int st = int(n & 1);
      const float E_cur = d2f_rn(coef_next);
      if (n + 1 < n_mine) coef_next = p.coef[blockIdx.x + (n + 1) * int64_t(gridDim.x)];
      const uint32_t lane_addr = tmem + uint32_t(st * 256) + (uint32_t(32 * (warp & 3)) << 16) + uint32_t(cbase);
      float* grow = G + st * (G_BYTES / 4) + (row < NL ? row : 0) * GS + cbase;
      if (drain) {
        bool ok = mbar_wait(bar(BAR_ACC_FULL + st), uint32_t((n >> 1) & 1));
        ok = __all_sync(0xffffffffu, ok);
        if (bar_or<3, EPI_THREADS>(!ok)) {
          failed = true;
          break;
        }
        fence_after();
        if (BF16) tmem_ld16_start(lane_addr, ra);
        else tmem_ld16x2_start(lane_addr, lane_addr + uint32_t(N), ra);
      }
      if (form) {
        // K^e of cell n - 1: one thread per node pair a <= b reads the nine
        // G^{ij}_ab and forms the nine entries K_(a,i),(b,j) (the transposed
        // block and the trace come from the same values), written to block
        // (a, b) and, K^e being symmetric, transposed to block (b, a), in a
        // shared staging copy of K^e in its global layout. Warp w takes the
        // pair groups w and w + 8 of kPairTable, whose lanes hit distinct
        // banks in the G loads and in both stores.
        const float* Gp = G + (st ^ 1) * (G_BYTES / 4);
        float* K = reinterpret_cast<float*>(sm + OFF_KS + (st ^ 1) * KS_BYTES);
        const float lh = p.lam_hat * E_prev, mh = p.mu_hat * E_prev;
        constexpr int ROUNDS = (PAIR_GROUPS + N_EPI - 1) / N_EPI;
        float g[ROUNDS][3][3];
        int ab[ROUNDS];
#pragma unroll
        for (int r = 0; r < ROUNDS; ++r) {
          const int grp = ew + N_EPI * r;
          ab[r] = grp < PAIR_GROUPS ? pairs[grp * 32 + lane] : 0xffff;
          const int a = ab[r] == 0xffff ? 0 : ab[r] >> 8, b = ab[r] == 0xffff ? 0 : ab[r] & 255;
#pragma unroll
          for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int j = 0; j < 3; ++j) g[r][i][j] = Gp[(i * NB + a) * GS + j * NB + b];
        }
#pragma unroll
        for (int r = 0; r < ROUNDS; ++r) {
          if (ab[r] != 0xffff) {
            const int a = ab[r] >> 8, b = ab[r] & 255;
            const float tr = g[r][0][0] + g[r][1][1] + g[r][2][2];
#pragma unroll
            for (int i = 0; i < 3; ++i)
#pragma unroll
              for (int j = 0; j < 3; ++j) {
                float v = lh * g[r][i][j] + mh * g[r][j][i];
                if (i == j) v += mh * tr;
                K[(i * NB + a) * NLP + j * NB + b] = v;
                if (a != b) K[(j * NB + b) * NLP + i * NB + a] = v;
              }
          }
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      }
      if (drain) {
        // cell n's accumulators -> G buffer n % 2 (FP32: the two 16-point
        // partial sums of 16 columns per load pair, the next pair in flight
        // while this one is stored)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          uint32_t(&cur)[32] = (c & 1) ? rb : ra;
          uint32_t(&nxt)[32] = (c & 1) ? ra : rb;
          tmem_wait32(cur);
          if (c < 2) {
            if (BF16) tmem_ld16_start(lane_addr + uint32_t(16 * (c + 1)), nxt);
            else tmem_ld16x2_start(lane_addr + uint32_t(16 * (c + 1)), lane_addr + uint32_t(N + 16 * (c + 1)), nxt);
          }
          if (row < NL) {
#pragma unroll
            for (int j = 0; j < 16; j += 4) {
              float4 v;
              if (BF16) {
                v = make_float4(__uint_as_float(cur[j]), __uint_as_float(cur[j + 1]), __uint_as_float(cur[j + 2]),
                                __uint_as_float(cur[j + 3]));
              } else {
                v = make_float4(__uint_as_float(cur[j]) + __uint_as_float(cur[16 + j]),
                                __uint_as_float(cur[j + 1]) + __uint_as_float(cur[17 + j]),
                                __uint_as_float(cur[j + 2]) + __uint_as_float(cur[18 + j]),
                                __uint_as_float(cur[j + 3]) + __uint_as_float(cur[19 + j]));
              }
              *reinterpret_cast<float4*>(grow + 16 * c + j) = v;
            }
          }
        }
        fence_before();
        mbar_arrive(bar(BAR_ACC_EMPTY + st));
      }
      // the bulk copy issued last iteration (cell n - 2) has read staging
      // buffer n % 2, which the next iteration overwrites
      if (t == 0) bulk_wait_read();
      bar_sync<3, EPI_THREADS>();
      if (form && t == 0)
        bulk_store(p.ke + (blockIdx.x + (n - 1) * int64_t(gridDim.x)) * (NL * NLP), sbase + OFF_KS + (st ^ 1) * KS_BYTES,
                   KS_BYTES);
      E_prev = E_cur;
    }
    if (t == 0) bulk_wait_all();
  }
  if (failed) {
    *abort_flag = 1;
    atomicOr(p.err, kErrTimeout);
  }
  fence_before();
  __syncthreads();
  if (warp == W_MMA) {
    fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
  }
}

}  // namespace tc

bool cell_tc_applicable(const fe_space* s, fe_precision prec) {
  return s->problem == FE_ELASTICITY && s->order == 2 && s->nq1d == 3 && prec != FE_PREC_FP64;
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
    const int64_t grid = std::min<int64_t>(s->n_cells, int64_t(nsm));
    kern<<<unsigned(grid), tc::THREADS, tc::SMEM_BYTES, st>>>(p);
    return cudaGetLastError();
  };
  return prec == FE_PREC_BF16 ? run(tc::k_cell_tc<true>) : run(tc::k_cell_tc<false>);
}

}  // namespace feasm

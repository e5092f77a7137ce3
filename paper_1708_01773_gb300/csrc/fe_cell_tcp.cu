// Cell integration of the Poisson problem for Q2 and Q3 (rule (p+1)^3) on the
// 5th-generation tensor cores (tcgen05, sm_103a).
//
// The cell matrix (Eq. fematrix with grad phi_a = cof(J) gradhat(phihat_a) /
// det J, Eq. shape_grad) is a Gram matrix over the points and the three
// gradient components:
//   K_ab = kappa sum_{i, q} C[a][(i, q)] C[b][(i, q)],
//   C[a][(i, q)] = sqrt(w_q / det J_q) sum_d cof(J_q)[i][d] gradhat_d(phihat_a)(x_q),
// i.e. K = kappa C C^T with C of nb rows and K = 3 nq columns. The rows of
// several cells are stacked into one 128-row operand (4 cells of 27 rows for
// Q2, 2 cells of 64 rows for Q3); one MMA group per K chunk forms the
// 128 x N product, of which the diagonal cell blocks are the cell matrices
// (the off-diagonal blocks are discarded). Both operands are the same matrix
// (B is its first N rows), staged in shared memory in the 128-byte swizzled
// K-major layout, one chunk of 128 bytes per row at a time (32 TF32 or 64
// BF16 values), the next chunk formed while the MMAs of the previous one run.
//
// FP32 form: 3xTF32 split (hi = tf32(x), lo = tf32(x - hi); products hi*hi +
// hi*lo + lo*hi), FP32 accumulation in tensor memory: the hi*hi products and
// the corrections in separate accumulators, a fresh pair per K chunk (4 MMA
// k-steps), each chunk's sum added by the warps into double-float sums in
// registers, so that no FP32 accumulator carries more than 4 additions of the
// large terms. BF16 form: BF16 operand, one product. Geometry (Jacobian,
// cofactors, determinant) is FP64; the cell vector is a double-float sum
// rounded once to FP64.
//
// One persistent CTA per SM (its shared memory exceeds half of the SM's; it
// holds all 512 tensor-memory columns) loops over tiles of cells. Per tile: FP64
// geometry of every point (one thread per point) and the cell vectors; then
// per K chunk the operand (all threads) and the MMAs (one thread, committed to
// the chunk's mbarrier); then the epilogue reads the diagonal blocks from
// tensor memory into shared memory and writes K^e = kappa G with 16-byte
// stores. Every mbarrier wait is bounded (about one second), after which the
// CTA sets FE_ERR_TIMEOUT, waits (bounded) for its issued MMAs and frees the
// tensor memory.
#include <cuda_bf16.h>

#include "fe_device.cuh"
#include "fe_sync.cuh"
#include "fe_tcgen05.cuh"

namespace feasm {
namespace tcp {

template <int P, bool BF16>
struct Cfg {
  static constexpr int NB = (P + 1) * (P + 1) * (P + 1);
  static constexpr int NQ = NB;                    // the (p+1)^3 Gauss rule
  static constexpr int NLP = (NB + 3) & ~3;        // row stride of a cell matrix
  static constexpr int CPT = 128 / NB;             // cells per tile: 4 (Q2), 2 (Q3)
  static constexpr int ROWS = CPT * NB;            // operand rows used: 108, 128
  static constexpr int N = (ROWS + 15) & ~15;      // MMA N: 112, 128
  static constexpr int KDIM = 3 * NQ;              // 81, 192
  static constexpr int ESZ = BF16 ? 2 : 4;
  static constexpr int KCH = 128 / ESZ;            // K values per chunk (one 128-byte row)
  static constexpr int NCH = (KDIM + KCH - 1) / KCH;
  static constexpr int EPV = 16 / ESZ;             // values per 16-byte vector
  static constexpr int PLANE = 128 * 128;          // one operand plane: 128 rows of 128 bytes
  static constexpr int STAGE = BF16 ? PLANE : 2 * PLANE;  // hi (and lo)
  static constexpr int GSTR = NLP + 4 * (P == 3);  // row stride of the staged cell blocks (floats)
  static constexpr int THREADS = 512;
  // shared memory, offsets from a 1024-byte aligned base
  static constexpr int al16(int x) { return (x + 15) & ~15; }
  static constexpr int OFF_OP = 0;                                          // 2 stages
  static constexpr int OFF_G = OFF_OP + 2 * STAGE;                          // [CPT][NB][GSTR] float
  static constexpr int OFF_DPHI = al16(OFF_G + CPT * NB * GSTR * 4);        // [NQ][NB][3] float
  static constexpr int OFF_PHI = al16(OFF_DPHI + NQ * NB * 3 * 4);          // [NQ][NB] float2 hi + lo
  static constexpr int OFF_GEO = al16(OFF_PHI + NQ * NB * 2 * 4);           // [ROWS points][12] float
  static constexpr int OFF_X = al16(OFF_GEO + ROWS * 12 * 4);               // [CPT][24] double
  static constexpr int OFF_A = al16(OFF_X + CPT * 24 * 8);                  // [CPT][21] double
  static constexpr int OFF_BAR = al16(OFF_A + CPT * 21 * 8);                // chunk[2], done, drain
  static constexpr int OFF_TMEM = OFF_BAR + 4 * 8;
  static constexpr int USED = OFF_TMEM + 8;
  // more than half of the SM's shared memory: one CTA (512 tensor-memory columns) per SM
  static constexpr int SMEM_BYTES = (USED + 1024 > 116 * 1024 ? USED + 1024 : 116 * 1024);
  static_assert(SMEM_BYTES <= 227 * 1024, "shared memory");
  static_assert(STAGE % 1024 == 0 && GSTR % 4 == 0, "alignment");
  static_assert(N <= 128, "accumulators of N <= 128 columns");
};

// accumulators of stage st: hi*hi products at column 256 st, the hi*lo and
// lo*hi corrections at 256 st + 128
constexpr uint32_t TMEM_COLS = 512;

struct Params {
  int64_t n_cells;
  const double* xv;
  const double* w;
  const double* xq;
  const float2* phi2;  // [nq][nb] phihat as FP32 hi + lo
  const float* dphi32; // [nq][nb][3]
  const double* coef;
  double f;            // source
  float* ke;
  double* fe;
  int* err;
};

// Operand chunk c of the current tile into the stage at `stage`: element
// (row r, k) = C[a][(i, q)] of cell r / NB, node a = r % NB, k = i NQ + q (the
// chunk's k = c KCH .. c KCH + KCH - 1), zero past ROWS rows or KDIM columns.
// One 16-byte vector per item; consecutive threads take consecutive rows, so
// that the swizzled stores of 8 rows fall in distinct banks.
template <int P, bool BF16>
__device__ __forceinline__ void build_chunk(unsigned char* stage, const float* geo, const float* sdphi, int c,
                                            int tid) {
  using C = Cfg<P, BF16>;
  for (int item = tid; item < 128 * 8; item += C::THREADS) {
    const int r = item & 127, g = item >> 7;
    const int cell = r / C::NB, a = r - cell * C::NB;
    float v[C::EPV];
#pragma unroll
    for (int e = 0; e < C::EPV; ++e) {
      const int k = c * C::KCH + g * C::EPV + e;
      float x = 0.f;
      if (r < C::ROWS && k < C::KDIM) {
        const int i = k / C::NQ, q = k - i * C::NQ;
        const float* gq = geo + (cell * C::NQ + q) * 12;
        const float* d = sdphi + (q * C::NB + a) * 3;
        x = gq[9] * fmaf(gq[3 * i + 2], d[2], fmaf(gq[3 * i + 1], d[1], gq[3 * i] * d[0]));
      }
      v[e] = x;
    }
    const uint32_t o = swz(r, g * 16);
    if constexpr (BF16) {
      uint32_t u[4];
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        __nv_bfloat162 h = __floats2bfloat162_rn(v[2 * e], v[2 * e + 1]);
        u[e] = *reinterpret_cast<uint32_t*>(&h);
      }
      *reinterpret_cast<uint4*>(stage + o) = make_uint4(u[0], u[1], u[2], u[3]);
    } else {
      float hi[4], lo[4];
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        hi[e] = to_tf32(v[e]);
        lo[e] = to_tf32(v[e] - hi[e]);
      }
      *reinterpret_cast<float4*>(stage + o) = make_float4(hi[0], hi[1], hi[2], hi[3]);
      *reinterpret_cast<float4*>(stage + C::PLANE + o) = make_float4(lo[0], lo[1], lo[2], lo[3]);
    }
  }
}

template <int P, bool BF16>
__global__ void __launch_bounds__(512, 1) k_cell_tcp(Params p) {
  using C = Cfg<P, BF16>;
  extern __shared__ unsigned char smem_raw[];
  unsigned char* sm = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  float* stg = reinterpret_cast<float*>(sm + C::OFF_G);
  float* sdphi = reinterpret_cast<float*>(sm + C::OFF_DPHI);
  float2* sphi = reinterpret_cast<float2*>(sm + C::OFF_PHI);
  float* geo = reinterpret_cast<float*>(sm + C::OFF_GEO);
  double* sx = reinterpret_cast<double*>(sm + C::OFF_X);
  double* sa = reinterpret_cast<double*>(sm + C::OFF_A);
  const uint32_t sbase = smem_u32(sm);
  const uint32_t bar_chunk0 = sbase + C::OFF_BAR, bar_drain = bar_chunk0 + 24;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(sm + C::OFF_TMEM);

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(sbase + C::OFF_TMEM),
                 "r"(TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    for (int i = 0; i < 4; ++i) mbar_init(bar_chunk0 + 8u * uint32_t(i), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  for (int i = tid; i < C::NQ * C::NB * 3; i += C::THREADS) sdphi[i] = p.dphi32[i];
  for (int i = tid; i < C::NQ * C::NB; i += C::THREADS) sphi[i] = p.phi2[i];
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = *tmem_slot;
  const int64_t n_tiles = (p.n_cells + C::CPT - 1) / C::CPT;
  uint32_t commits[2] = {0u, 0u};  // completed waits on each chunk barrier so far
  bool failed = false, issued = false;

  for (int64_t tile = blockIdx.x; tile < n_tiles && !failed; tile += gridDim.x) {
    const int64_t e0 = tile * C::CPT;
    const int ncell = int(p.n_cells - e0 < C::CPT ? p.n_cells - e0 : C::CPT);
    // ---- coordinates and trilinear coefficients of the tile's cells (a
    // missing last cell repeats the first: its results are not stored)
    for (int i = tid; i < C::CPT * 24; i += C::THREADS) {
      const int c = i / 24;
      sx[i] = p.xv[(e0 + (c < ncell ? c : 0)) * 24 + (i - c * 24)];
    }
    __syncthreads();
    if (tid < C::CPT * 3) trilinear_coefficients(sx + (tid / 3) * 24, tid % 3, sa + (tid / 3) * 21);
    __syncthreads();
    // ---- FP64 geometry, one thread per point of the tile
    if (tid < C::ROWS) {
      const int c = tid / C::NQ, q = tid - c * C::NQ;
      double cof[9], det;
      geometry_at(sa + c * 21, p.xq[3 * q], p.xq[3 * q + 1], p.xq[3 * q + 2], cof, &det);
      if (c < ncell && !(det > 0.0)) atomicOr(p.err, kErrNegJacobian);
      const double wq = p.w[q];
      float* g = geo + tid * 12;
#pragma unroll
      for (int k = 0; k < 9; ++k) g[k] = d2f_rn(cof[k]);
      g[9] = sqrtf(d2f_rn(wq) / d2f_rn(det));
      const double wd = wq * det;
      const float hi = d2f_rn(wd);
      g[10] = hi;
      g[11] = d2f_rn(wd - f32_to_f64_exact(hi));
    }
    __syncthreads();
    // ---- cell vectors: f_a = f sum_q (w det J)_q phihat_a(x_q), double-float
    // products and sums rounded once to FP64
    if (tid < C::ROWS) {
      const int c = tid / C::NB, a = tid - c * C::NB;
      if (c < ncell) {
        float sh = 0.f, sl = 0.f;
        for (int q = 0; q < C::NQ; ++q) {
          const float* g = geo + (c * C::NQ + q) * 12;
          const float wh = g[10], wl = g[11];
          const float2 b = sphi[q * C::NB + a];
          const float ph = wh * b.x;
          const float pe = fmaf(wh, b.x, -ph) + (wh * b.y + wl * b.x);
          const float sum = sh + ph;
          const float bp = sum - sh;
          const float er = (sh - (sum - bp)) + (ph - bp);
          sh = sum;
          sl += er + pe;
        }
        p.fe[(e0 + c) * C::NB + a] = p.f * __dadd_rn(f32_to_f64_exact(sh), f32_to_f64_exact(sl));
      }
    }
    // ---- operand chunks, MMAs and accumulator drains. Chunk c is formed in
    // stage c % 2 and multiplied into accumulator c % 2 (a fresh sum per chunk);
    // while the MMAs of chunk c + 1 run, the warps drain accumulator c % 2 into
    // double-float sums in registers, so that no FP32 accumulator carries more
    // than one chunk's 4 k-steps (the tensor cores' FP32 accumulation error
    // grows with the number of MMAs added into one sum).
    // Drain mapping: warp = 4 gi + qd reads tensor-memory lanes 32 qd .. (rows),
    // column groups g0 + gi, g0 + gi + 4 of 16 (the rows' own-cell columns).
    const int qd = warp & 3, gi = warp >> 2;
    const int r = 32 * qd + lane;
    const int rc = r / C::NB, ra = r - rc * C::NB;
    const int rlast = 32 * qd + 31 < C::ROWS - 1 ? 32 * qd + 31 : C::ROWS - 1;
    const int g0 = (C::NB * ((32 * qd) / C::NB)) / 16, g1 = (C::NB * (rlast / C::NB) + C::NB - 1) / 16;
    const bool drains = 32 * qd < C::ROWS;
    const uint32_t lane_addr = tmem + (uint32_t(32 * qd) << 16);
    float sh[2][16], sl[2][16];
#pragma unroll
    for (int t = 0; t < 2; ++t)
#pragma unroll
      for (int j = 0; j < 16; ++j) sh[t][j] = sl[t][j] = 0.f;
    auto issue = [&](int c) {  // thread 0: the MMAs of chunk c
      fence_after();
      constexpr uint32_t IDESC = instr_desc(128, C::N, BF16 ? 1u : 2u);
      const int st = c & 1;
      const uint32_t acc = tmem + uint32_t(st) * 256u, accc = acc + 128u;
      const uint32_t sb = sbase + uint32_t(C::OFF_OP + st * C::STAGE);
      const uint64_t ahi = sw128_desc(sb), alo = sw128_desc(sb + C::PLANE);
#pragma unroll
      for (int ks = 0; ks < 4; ++ks) {
        if (BF16) {
          mma_bf16(acc, ahi + 2 * ks, ahi + 2 * ks, IDESC, ks > 0 ? 1u : 0u);
        } else {
          mma_tf32(acc, ahi + 2 * ks, ahi + 2 * ks, IDESC, ks > 0 ? 1u : 0u);
          mma_tf32(accc, alo + 2 * ks, ahi + 2 * ks, IDESC, ks > 0 ? 1u : 0u);
          mma_tf32(accc, ahi + 2 * ks, alo + 2 * ks, IDESC, 1u);
        }
      }
      mma_commit(bar_chunk0 + 8u * uint32_t(st));
      issued = true;
    };
    build_chunk<P, BF16>(sm + C::OFF_OP, geo, sdphi, 0, tid);
    fence_proxy_async();
    __syncthreads();
    if (tid == 0) issue(0);
    for (int c = 0; c < C::NCH && !failed; ++c) {
      const int st = c & 1;
      if (c + 1 < C::NCH) {
        // stage and accumulator (c + 1) % 2 were freed by the drain of chunk c - 1
        build_chunk<P, BF16>(sm + C::OFF_OP + (st ^ 1) * C::STAGE, geo, sdphi, c + 1, tid);
        fence_proxy_async();
        __syncthreads();
        if (tid == 0) issue(c + 1);
      }
      const bool ok = mbar_wait(bar_chunk0 + 8u * uint32_t(st), (commits[st]) & 1u);
      ++commits[st];
      if (__syncthreads_or(!ok)) {
        failed = true;
        break;
      }
      fence_after();
      if (drains) {
#pragma unroll
        for (int t = 0; t < 2; ++t) {
          const int gg = g0 + gi + 4 * t;
          if (gg <= g1) {
            float v[16], vc[16];
            const uint32_t ta = lane_addr + uint32_t(st) * 256u + uint32_t(16 * gg);
            if (BF16) tmem_ld16(ta, v);
            else tmem_ld16x2(ta, ta + 128u, v, vc);
#pragma unroll
            for (int j = 0; j < 16; ++j) {  // the chunk's sum into the register sums (TwoSum)
              if (!BF16) v[j] += vc[j];
              const float sum = sh[t][j] + v[j];
              const float bp = sum - sh[t][j];
              sl[t][j] += (sh[t][j] - (sum - bp)) + (v[j] - bp);
              sh[t][j] = sum;
            }
          }
        }
      }
      fence_before();
      __syncthreads();
    }
    if (failed) break;
    // ---- epilogue: the rows' own-cell columns of the summed chunks into shared memory
    if (drains) {
#pragma unroll
      for (int t = 0; t < 2; ++t) {
        const int gg = g0 + gi + 4 * t;
        if (gg <= g1) {
#pragma unroll
          for (int j = 0; j < 16; ++j) {
            const int col = 16 * gg + j - C::NB * rc;
            if (r < C::ROWS && col >= 0 && col < C::NB) stg[(rc * C::NB + ra) * C::GSTR + col] = sh[t][j] + sl[t][j];
          }
        }
      }
    }
    fence_before();
    __syncthreads();
    // ---- K^e = kappa G of the tile's cells, 16-byte stores (zero padding columns)
    constexpr int V4 = C::NLP / 4;
    for (int item = tid; item < ncell * C::NB * V4; item += C::THREADS) {
      const int c = item / (C::NB * V4), rem = item - c * C::NB * V4, a = rem / V4, v = rem - a * V4;
      const float kappa = d2f_rn(p.coef[e0 + c]);
      const float* s = stg + (c * C::NB + a) * C::GSTR + 4 * v;
      float4 o;
      o.x = 4 * v + 0 < C::NB ? kappa * s[0] : 0.f;
      o.y = 4 * v + 1 < C::NB ? kappa * s[1] : 0.f;
      o.z = 4 * v + 2 < C::NB ? kappa * s[2] : 0.f;
      o.w = 4 * v + 3 < C::NB ? kappa * s[3] : 0.f;
      reinterpret_cast<float4*>(p.ke + (e0 + c) * (C::NB * C::NLP) + a * C::NLP)[v] = o;
    }
    __syncthreads();
  }
  // teardown: every MMA this CTA issued has completed before the tensor memory
  // is freed (bounded wait; on the normal path they all have already)
  if (tid == 0 && issued) {
    mma_commit(bar_drain);
    if (!mbar_wait(bar_drain, 0)) failed = true;
  }
  if (failed && tid == 0) atomicOr(p.err, kErrTimeout);
  fence_before();
  __syncthreads();
  if (warp == 0) {
    fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
  }
}

}  // namespace tcp

bool cell_tcp_applicable(const fe_space* s, fe_precision prec) {
  return s->problem == FE_POISSON && (s->order == 2 || s->order == 3) && s->nq1d == s->order + 1 &&
         prec != FE_PREC_FP64;
}

cudaError_t launch_cell_tcp(const fe_space* s, const double* coef, const double force[3], fe_precision prec,
                            cudaStream_t st) {
  if (s->n_cells == 0) return cudaSuccess;
  tcp::Params p;
  p.n_cells = s->n_cells;
  p.xv = s->d_xv;
  p.w = s->d_w;
  p.xq = s->d_xq;
  p.phi2 = reinterpret_cast<const float2*>(s->d_phi2);
  p.dphi32 = s->d_dphi32;
  p.coef = coef;
  p.f = force[0];
  p.ke = static_cast<float*>(s->d_ke);
  p.fe = s->d_fe;
  p.err = s->d_err;
  int nsm = 152;
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, s->device);
  auto run = [&](auto kern, int smem, int cpt) -> cudaError_t {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    const int64_t tiles = (s->n_cells + cpt - 1) / cpt;
    const int64_t grid = std::min<int64_t>(tiles, int64_t(nsm));
    kern<<<unsigned(grid), 512, size_t(smem), st>>>(p);
    return cudaGetLastError();
  };
  const bool bf = prec == FE_PREC_BF16;
  if (s->order == 2)
    return bf ? run(tcp::k_cell_tcp<2, true>, tcp::Cfg<2, true>::SMEM_BYTES, tcp::Cfg<2, true>::CPT)
              : run(tcp::k_cell_tcp<2, false>, tcp::Cfg<2, false>::SMEM_BYTES, tcp::Cfg<2, false>::CPT);
  return bf ? run(tcp::k_cell_tcp<3, true>, tcp::Cfg<3, true>::SMEM_BYTES, tcp::Cfg<3, true>::CPT)
            : run(tcp::k_cell_tcp<3, false>, tcp::Cfg<3, false>::SMEM_BYTES, tcp::Cfg<3, false>::CPT);
}

}  // namespace feasm

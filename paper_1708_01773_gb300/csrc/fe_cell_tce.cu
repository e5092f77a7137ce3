// Cell integration of Q3 linear elasticity (4^3 Gauss rule) on the
// 5th-generation tensor cores (tcgen05, sm_103a), BF16 and FP32 (3xTF32) forms.
//
// With C[(a,i)][q] = sqrt(w_q / det J_q) sum_d cof(J_q)[i][d] gradhat_d(phihat_a)(x_q)
// (Eq. shape_grad: grad phi_a = cof(J) gradhat(phihat_a) / det J), the Gram
//   G[(a,i)][(b,j)] = sum_q C[(a,i)][q] C[(b,j)][q] = G^{ij}_ab
// gives the cell matrix of Eq. fematrix with the isotropic Hooke law:
//   K_(i,a),(j,b) = E (lam^ G^{ij}_ab + mu^ G^{ji}_ab + mu^ d_ij sum_k G^{kk}_ab).
// C has 192 rows (64 nodes x 3 components) and K = 64 points. The rows are
// laid out node-major with a zero fourth component, r = 4 a + i (256 rows), so
// that the four rows of a node sit in four consecutive lanes of one warp in the
// accumulator read-out. One cell per MMA round: two M = 128 tiles (nodes 0-31,
// 32-63) times all N = 256 columns, accumulated in the 512 tensor-memory
// columns of the SM; K^e is 25 % padding in M and N, which costs nothing here
// (the cell matrix store bounds the kernel, 147 KB per cell).
//
// Operand: one 128-byte swizzled K-major row per chunk of K (64 BF16 or 32
// TF32 values), formed by all 512 threads from the FP32 geometry of the 64
// points and the 1D Lagrange values and derivatives (gradhat(phihat_a)(x_q) is
// a product of three 1D factors). FP32 form: hi = tf32(x), lo = tf32(x - hi),
// products hi*hi + lo*hi + hi*lo into one FP32 accumulator. Geometry (Jacobian,
// cofactors, determinant) is FP64, rounded once to FP32; the cell vector is a
// double-float sum rounded once to FP64.
//
// Read-out: warp w reads tensor-memory lanes 32 (w % 4).. of tile (w / 4) % 2,
// columns 128 (w / 8).. (32 column nodes b). For each b the four lanes of a node
// a exchange their G[(a, .)][(b, .)] values with four shuffles (two rotated
// transposes, a butterfly for the trace), form K^e rows (i, a) at columns
// (j, b), 8 column nodes at a time, stage them in shared memory and store
// 128-byte row segments. One persistent CTA per SM (all 512 tensor-memory
// columns); every mbarrier wait is bounded, after which the CTA sets
// FE_ERR_TIMEOUT, waits (bounded) for its issued MMAs and frees the tensor
// memory.
#include <cuda_bf16.h>

#include "fe_device.cuh"
#include "fe_sync.cuh"
#include "fe_tcgen05.cuh"

namespace feasm {
namespace tce {

constexpr int NB = 64, NQ = 64, NL = 192, ROWS = 256, THREADS = 512, WARPS = THREADS / 32;
constexpr uint32_t TMEM_COLS = 512;     // tile t accumulates at column 256 t
constexpr int STG_ROW = 97, STG_FLOATS = 24 * STG_ROW;  // read-out staging per warp

template <bool BF16>
struct Cfg {
  static constexpr int ESZ = BF16 ? 2 : 4;
  static constexpr int KCH = 128 / ESZ;          // points per chunk (one 128-byte row)
  static constexpr int NCH = NQ / KCH;           // 1 (BF16) or 2 (TF32)
  static constexpr int EPV = 16 / ESZ;           // values per 16-byte vector
  static constexpr int PLANE = ROWS * 128;       // one operand plane: 256 rows of 128 bytes
  static constexpr int STAGE = BF16 ? PLANE : 2 * PLANE;  // hi (and lo)
  static constexpr int al16(int x) { return (x + 15) & ~15; }
  static constexpr int OFF_OP = 0;                                   // NCH stages
  // the operand stages, reused as the read-out staging once the MMAs are done
  static constexpr int OP_BYTES = NCH * STAGE > WARPS * STG_FLOATS * 4 ? NCH * STAGE : WARPS * STG_FLOATS * 4;
  static constexpr int OFF_PHI = al16(OFF_OP + OP_BYTES);            // [NQ][NB] float2 hi + lo
  static constexpr int OFF_GEO = OFF_PHI + NQ * NB * 8;              // [NQ][12] float
  static constexpr int OFF_X = al16(OFF_GEO + NQ * 12 * 4);          // 24 double
  static constexpr int OFF_A = al16(OFF_X + 24 * 8);                 // 21 double
  static constexpr int OFF_T = al16(OFF_A + 21 * 8);                 // V[16], D[16] float
  static constexpr int OFF_JC = al16(OFF_T + 32 * 4);                // [48][3] double: Jacobian columns
  static constexpr int OFF_VP = al16(OFF_JC + 48 * 3 * 8);           // [THREADS] float2: cell-vector partials
  static constexpr int OFF_BAR = al16(OFF_VP + THREADS * 8);         // mma, drain
  static constexpr int OFF_TMEM = OFF_BAR + 2 * 8;
  static constexpr int USED = OFF_TMEM + 8;
  // more than half of the SM's shared memory: one CTA (512 tensor-memory columns) per SM
  static constexpr int SMEM_BYTES = (USED + 1024 > 116 * 1024 ? USED + 1024 : 116 * 1024);
  static_assert(SMEM_BYTES <= 227 * 1024, "shared memory");
  static_assert(STAGE % 1024 == 0, "alignment");
};

struct Params {
  int64_t n_cells;
  const double* xv;    // [n_cells][8][3]
  const double* w;     // [NQ]
  const double* xq;    // [NQ][3]
  const float2* phi2;  // [NQ][NB] phihat as FP32 hi + lo
  float v1[16], d1[16];  // 1D Lagrange values and derivatives at the Gauss points, [q][a]
  const double* coef;    // E per cell
  double f[3];           // body force
  float lam_hat, mu_hat;
  float* ke;
  double* fe;
  int* err;
};

// Operand vectors of node a, point block qv (EPV consecutive points from
// qv * EPV), rows 4 a + i, i = 0..2, into the chunk's stage: C[(a,i)][q] =
// g9_q sum_d cof_q[i][d] gradhat_d(phihat_a)(x_q), gradhat from the 1D factors.
template <bool BF16>
__device__ __forceinline__ void build_vectors(unsigned char* stage, const float* geo, const float* sv,
                                              const float* sd, int a, int qv) {
  using C = Cfg<BF16>;
  const int a0 = a & 3, a1 = (a >> 2) & 3, a2 = a >> 4;
  float x[3][C::EPV];
#pragma unroll
  for (int e = 0; e < C::EPV; ++e) {
    const int q = qv * C::EPV + e;
    const int q0 = q & 3, q1 = (q >> 2) & 3, q2 = q >> 4;
    const float v0 = sv[q0 * 4 + a0], v1 = sv[q1 * 4 + a1], v2 = sv[q2 * 4 + a2];
    const float g0 = sd[q0 * 4 + a0] * (v1 * v2), g1 = v0 * (sd[q1 * 4 + a1] * v2), g2 = (v0 * v1) * sd[q2 * 4 + a2];
    const float* gq = geo + q * 12;
#pragma unroll
    for (int i = 0; i < 3; ++i) x[i][e] = gq[9] * fmaf(gq[3 * i + 2], g2, fmaf(gq[3 * i + 1], g1, gq[3 * i] * g0));
  }
  const int kbyte = ((qv * C::EPV) % C::KCH) * C::ESZ;
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    const uint32_t o = swz(4 * a + i, kbyte);
    if constexpr (BF16) {
      uint32_t u[4];
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        __nv_bfloat162 h = __floats2bfloat162_rn(x[i][2 * e], x[i][2 * e + 1]);
        u[e] = *reinterpret_cast<uint32_t*>(&h);
      }
      *reinterpret_cast<uint4*>(stage + o) = make_uint4(u[0], u[1], u[2], u[3]);
    } else {
      float hi[4], lo[4];
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        hi[e] = to_tf32(x[i][e]);
        lo[e] = to_tf32(x[i][e] - hi[e]);
      }
      *reinterpret_cast<float4*>(stage + o) = make_float4(hi[0], hi[1], hi[2], hi[3]);
      *reinterpret_cast<float4*>(stage + C::PLANE + o) = make_float4(lo[0], lo[1], lo[2], lo[3]);
    }
  }
}

// The MMAs of chunk c of the current cell (thread 0): both M tiles against all
// 256 rows as B; the first product of chunk 0 starts each accumulator.
template <bool BF16>
__device__ __forceinline__ void issue_chunk(uint32_t tmem, uint32_t sop, int c) {
  using C = Cfg<BF16>;
  constexpr uint32_t IDESC = instr_desc(128, 256, BF16 ? 1u : 2u);
  const uint32_t sb = sop + uint32_t(c * C::STAGE);
  const uint64_t bhi = sw128_desc(sb), blo = sw128_desc(sb + C::PLANE);
#pragma unroll
  for (int t = 0; t < 2; ++t) {
    const uint32_t d = tmem + uint32_t(256 * t);
    const uint64_t ahi = sw128_desc(sb + uint32_t(t * 128 * 128)), alo = sw128_desc(sb + C::PLANE + uint32_t(t * 128 * 128));
#pragma unroll
    for (int ks = 0; ks < 4; ++ks) {
      const uint32_t acc = (c > 0 || ks > 0) ? 1u : 0u;
      if constexpr (BF16) {
        mma_bf16(d, ahi + 2 * ks, bhi + 2 * ks, IDESC, acc);
      } else {
        mma_tf32(d, ahi + 2 * ks, bhi + 2 * ks, IDESC, acc);
        mma_tf32(d, alo + 2 * ks, bhi + 2 * ks, IDESC, 1u);
        mma_tf32(d, ahi + 2 * ks, blo + 2 * ks, IDESC, 1u);
      }
    }
  }
}

template <bool BF16>
__global__ void __launch_bounds__(THREADS, 1) k_cell_tce(Params p) {
  using C = Cfg<BF16>;
  extern __shared__ unsigned char smem_raw[];
  unsigned char* sm = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  float2* sphi = reinterpret_cast<float2*>(sm + C::OFF_PHI);
  float* geo = reinterpret_cast<float*>(sm + C::OFF_GEO);
  double* sx = reinterpret_cast<double*>(sm + C::OFF_X);
  double* sa = reinterpret_cast<double*>(sm + C::OFF_A);
  float* sv = reinterpret_cast<float*>(sm + C::OFF_T);
  float* sd = sv + 16;
  double* jc = reinterpret_cast<double*>(sm + C::OFF_JC);
  float2* vpart = reinterpret_cast<float2*>(sm + C::OFF_VP);
  const uint32_t sbase = smem_u32(sm);
  const uint32_t sop = sbase + C::OFF_OP;
  const uint32_t bar_mma = sbase + C::OFF_BAR, bar_drain = bar_mma + 8;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(sm + C::OFF_TMEM);

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(sbase + C::OFF_TMEM),
                 "r"(TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    mbar_init(bar_mma, 1);
    mbar_init(bar_drain, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  for (int i = tid; i < NQ * NB; i += THREADS) sphi[i] = p.phi2[i];
  if (tid < 16) {
    sv[tid] = p.v1[tid];
    sd[tid] = p.d1[tid];
  }
  // The fourth-component rows (4 a + 3) of the operand are never written here:
  // whatever they hold (the read-out staging shares their shared memory) only
  // reaches accumulator rows (a, 3) and columns (b, 3), which are never read.
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = *tmem_slot;
  const float lam = p.lam_hat, mu = p.mu_hat;
  uint32_t n_mma = 0;  // completed waits on bar_mma
  bool failed = false, issued = false;

  // read-out roles: tensor-memory lane quadrant, tile, column half
  const int rq = warp & 3, rt = (warp >> 2) & 1, rh = warp >> 3;
  const uint32_t lane_addr = tmem + (uint32_t(32 * rq) << 16) + uint32_t(256 * rt + 128 * rh);
  const int ci = lane & 3;  // component of the lane's row (node 32 rt + 8 rq + lane / 4)
  // read-out exchange within the node's four lanes: source lanes of the rows
  // (a, i+2) and (a, i+1); staging row and the columns of components i, i+1, i+2
  const int qbase = lane & ~3, src_p = ci < 3 ? (ci + 2) % 3 : 0, src_n = ci < 3 ? (ci + 1) % 3 : 0;
  const int srow = (ci < 3 ? ci * 8 + (lane >> 2) : 0) * STG_ROW;
  const int cs = 32 * (ci < 3 ? ci : 0), cn = 32 * ((ci + 1) % 3), cp = 32 * ((ci + 2) % 3);
  // the warp's staging rows (24 K^e rows of 96 floats, stride 97: conflict-free)
  float* stg = reinterpret_cast<float*>(sm + C::OFF_OP) + warp * STG_FLOATS;

  double xnext = (tid < 24 && blockIdx.x < p.n_cells) ? p.xv[int64_t(blockIdx.x) * 24 + tid] : 0.0;
  for (int64_t cell = blockIdx.x; cell < p.n_cells && !failed; cell += gridDim.x) {
    // ---- coordinates (loaded during the previous cell), trilinear
    // coefficients, FP64 geometry at the 64 points
    if (tid < 24) sx[tid] = xnext;
    __syncthreads();
    if (tid < 3) trilinear_coefficients(sx, tid, sa);
    if (tid < 24 && cell + gridDim.x < p.n_cells) xnext = p.xv[(cell + gridDim.x) * 24 + tid];
    __syncthreads();
    // Jacobian column d at the 16 pairs of 1D points of the two other
    // directions (it does not depend on its own direction): 48 items
    if (tid < 48) {
      const int d = tid >> 4, u = tid & 3, v = (tid >> 2) & 3;
      const double s = p.xq[3 * u], t = p.xq[3 * v];  // 1D Gauss points
      const int c0 = 3 * d, cs = d == 2 ? 12 : 9, ct = d == 0 ? 12 : 15;
      const double st = s * t;
#pragma unroll
      for (int k = 0; k < 3; ++k) jc[tid * 3 + k] = sa[c0 + k] + sa[cs + k] * s + sa[ct + k] * t + sa[18 + k] * st;
    }
    __syncthreads();
    if (tid < NQ) {
      const int q = tid, q0 = q & 3, q1 = (q >> 2) & 3, q2 = q >> 4;
      const double* j0 = jc + (q1 + 4 * q2) * 3;        // column 0 at (y, z)
      const double* j1 = jc + (16 + q0 + 4 * q2) * 3;   // column 1 at (x, z)
      const double* j2 = jc + (32 + q0 + 4 * q1) * 3;   // column 2 at (x, y)
      const double J[3][3] = {{j0[0], j1[0], j2[0]}, {j0[1], j1[1], j2[1]}, {j0[2], j1[2], j2[2]}};
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
      const double wq = p.w[q];
      float* g = geo + q * 12;
#pragma unroll
      for (int k = 0; k < 9; ++k) g[k] = d2f_rn(cof[k]);
      g[9] = sqrtf(d2f_rn(wq) / d2f_rn(det));
      const double wd = wq * det;
      const float hi = d2f_rn(wd);
      g[10] = hi;
      g[11] = d2f_rn(wd - f32_to_f64_exact(hi));
    }
    __syncthreads();
    // ---- cell vector: f_(i,a) = f_i sum_q (w det J)_q phihat_a(x_q), double-float
    // products and sums (8 points per thread, then the 8 partial sums of a
    // node in order), rounded once to FP64
    {
      const int a = tid & (NB - 1), q0 = (tid >> 6) * 8;
      float sh = 0.f, sl = 0.f;
#pragma unroll
      for (int q = q0; q < q0 + 8; ++q) {
        const float* g = geo + q * 12;
        const float wh = g[10], wl = g[11];
        const float2 b = sphi[q * NB + a];
        const float ph = wh * b.x;
        const float pe = fmaf(wh, b.x, -ph) + (wh * b.y + wl * b.x);
        const float sum = sh + ph;
        const float bp = sum - sh;
        const float er = (sh - (sum - bp)) + (ph - bp);
        sh = sum;
        sl += er + pe;
      }
      vpart[tid] = make_float2(sh, sl);
    }
    __syncthreads();
    if (tid < NB) {
      const int a = tid;
      float sh = 0.f, sl = 0.f;
#pragma unroll
      for (int k = 0; k < THREADS / NB; ++k) {
        const float2 v = vpart[k * NB + a];
        const float sum = sh + v.x;
        const float bp = sum - sh;
        const float er = (sh - (sum - bp)) + (v.x - bp);
        sh = sum;
        sl += er + v.y;
      }
      const double s = __dadd_rn(f32_to_f64_exact(sh), f32_to_f64_exact(sl));
#pragma unroll
      for (int i = 0; i < 3; ++i) p.fe[cell * NL + i * NB + a] = p.f[i] * s;
    }
    // ---- operand chunks and MMAs (chunk 1 of the FP32 form is formed while
    // the MMAs of chunk 0 run)
    constexpr int VPC = C::KCH / C::EPV;  // vectors per node and chunk: 8
#pragma unroll 1
    for (int c = 0; c < C::NCH; ++c) {
      for (int item = tid; item < NB * VPC; item += THREADS) {
        const int a = item % NB, qv = c * VPC + item / NB;
        build_vectors<BF16>(sm + C::OFF_OP + c * C::STAGE, geo, sv, sd, a, qv);
      }
      fence_proxy_async();
      __syncthreads();
      if (tid == 0) {
        fence_after();
        issue_chunk<BF16>(tmem, sop, c);
        if (c == C::NCH - 1) mma_commit(bar_mma);
        issued = true;
      }
    }
    const bool ok = mbar_wait(bar_mma, n_mma & 1u);
    ++n_mma;
    if (__syncthreads_or(!ok)) {
      failed = true;
      break;
    }
    fence_after();
    // ---- read-out: K^e row (i, a) of the lane at columns (j, b), 8 column
    // nodes at a time, staged in shared memory (the operand stages, free once
    // the MMAs are done) and stored as 128-byte row segments
    const float E = d2f_rn(p.coef[cell]);
    const float lE = lam * E, mE = mu * E;
    float* kc = p.ke + cell * (NL * NL) + (32 * rt + 8 * rq) * NL + 32 * rh;
    const float lmE = lE + mE;
    // quarter qq + 1 is loaded from tensor memory while quarter qq is formed
    uint32_t rbuf[2][32];
    tmem_ld16x2_start(lane_addr, lane_addr + 16u, rbuf[0]);
    tmem_wait32(rbuf[0]);
#pragma unroll
    for (int qq = 0; qq < 4; ++qq) {
      uint32_t(&r)[32] = rbuf[qq & 1];
      if (qq < 3) tmem_ld16x2_start(lane_addr + uint32_t(32 * qq + 32), lane_addr + uint32_t(32 * qq + 48), rbuf[(qq + 1) & 1]);
#pragma unroll
      for (int bb = 0; bb < 8; ++bb) {
        // the lane's row (a, i) holds v_m = G[(a,i)][(b,m)]; it needs G[(a,j)][(b,i)]
        // from the lanes of rows (a, j) and the trace sum_k G[(a,k)][(b,k)]
        const float v0 = __uint_as_float(r[4 * bb]), v1 = __uint_as_float(r[4 * bb + 1]),
                    v2 = __uint_as_float(r[4 * bb + 2]);
        const float vs = ci == 0 ? v0 : ci == 1 ? v1 : ci == 2 ? v2 : 0.f;  // v_i
        const float vn = ci == 0 ? v1 : ci == 1 ? v2 : v0;                   // v_(i+1)
        const float vp = ci == 0 ? v2 : ci == 1 ? v0 : v1;                   // v_(i+2)
        float dsum = vs + __shfl_xor_sync(kFull, vs, 1);
        dsum += __shfl_xor_sync(kFull, dsum, 2);
        // the lane of row (a, i-1) sends its v_(i), that of row (a, i+1) its v_(i)
        const float tp = __shfl_sync(kFull, vn, qbase | src_p);  // G[(a,i+2)][(b,i)]
        const float tn = __shfl_sync(kFull, vp, qbase | src_n);  // G[(a,i+1)][(b,i)]
        if (ci < 3) {
          float* o = stg + srow + 8 * qq + bb;
          o[cs] = fmaf(lmE, vs, mE * dsum);
          o[cn] = fmaf(lE, vn, mE * tn);
          o[cp] = fmaf(lE, vp, mE * tp);
        }
      }
      if (qq < 3) tmem_wait32(rbuf[(qq + 1) & 1]);
    }
    __syncwarp();
    // the warp's 24 rows x 3 components x 32 column nodes: 72 coalesced 128-byte row segments
#pragma unroll
    for (int sgm = 0; sgm < 72; ++sgm) {
      const int rw = sgm / 3, j = sgm - 3 * rw;  // row within the warp (i * 8 + node), component
      const int i = rw >> 3;
      kc[(i * NB + rw % 8) * NL + j * NB + lane] = stg[rw * STG_ROW + j * 32 + lane];
    }
    fence_before();
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

}  // namespace tce

bool cell_tce_applicable(const fe_space* s, fe_precision prec) {
  return s->problem == FE_ELASTICITY && s->order == 3 && s->nq1d == 4 && prec != FE_PREC_FP64;
}

cudaError_t launch_cell_tce(const fe_space* s, const double* coef, const double force[3], fe_precision prec,
                            cudaStream_t st) {
  if (s->n_cells == 0) return cudaSuccess;
  tce::Params p;
  p.n_cells = s->n_cells;
  p.xv = s->d_xv;
  p.w = s->d_w;
  p.xq = s->d_xq;
  p.phi2 = reinterpret_cast<const float2*>(s->d_phi2);
  double v1[16], d1[16];
  lagrange_1d_table(3, 4, v1, d1);
  for (int i = 0; i < 16; ++i) {
    p.v1[i] = float(v1[i]);
    p.d1[i] = float(d1[i]);
  }
  p.coef = coef;
  for (int k = 0; k < 3; ++k) p.f[k] = force[k];
  p.lam_hat = float(s->nu / ((1.0 + s->nu) * (1.0 - 2.0 * s->nu)));
  p.mu_hat = float(1.0 / (2.0 * (1.0 + s->nu)));
  p.ke = static_cast<float*>(s->d_ke);
  p.fe = s->d_fe;
  p.err = s->d_err;
  int nsm = 152;
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, s->device);
  auto run = [&](auto kern, int smem) -> cudaError_t {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    const int64_t grid = std::min<int64_t>(s->n_cells, int64_t(nsm));
    kern<<<unsigned(grid), tce::THREADS, size_t(smem), st>>>(p);
    return cudaGetLastError();
  };
  return prec == FE_PREC_BF16 ? run(tce::k_cell_tce<true>, tce::Cfg<true>::SMEM_BYTES)
                              : run(tce::k_cell_tce<false>, tce::Cfg<false>::SMEM_BYTES);
}

}  // namespace feasm

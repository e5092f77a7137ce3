// CUDA kernels of libfeasm (sm_103a): cell integration (geometry, physical
// gradients, cell-matrix contraction, cell vectors), the deterministic
// segmented scatter into CSR, and the compliance adjoint.
#include "fe_device.cuh"

namespace feasm {


// Shared memory of k_cell: for FP64, vertex coordinates [cpb][24],
// trilinear coefficients [cpb][21], per-point geometry [cpb][nq][11]
// (cofactors, w/det, w*det) and the cofactor gradients [cpb][nq][3][nb]; for
// the FP32/BF16 forms the layout of mixed_layout. -1 if it exceeds an SM.
long cell_smem_bytes(int nb, int nq, fe_precision prec, int cpb) {
  long bytes;
  if (prec == FE_PREC_FP64) {
    bytes = long(cpb) * (24 + 21) * 8 + long(cpb) * nq * 11 * 8 + long(cpb) * nq * 3 * nb * 8;
  } else {
    int n1d = 1;
    while (n1d * n1d * n1d < nq) ++n1d;
    bytes = mixed_layout(cpb, nq, n1d, nb).bytes;
  }
  return bytes <= 227 * 1024 ? bytes : -1;
}

// Cells per block of k_cell: at least one node pair per thread, then doubled
// while the block has fewer than 128 quadrature points (the FP64 geometry
// runs one thread per point: 128 points fill four warps, one per SM
// sub-partition, each with its own share of the FP64 pipe) and the shared
// memory of every precision stays within 64 KB.
int cells_per_block(int nb, int nq) {
  const int pairs = nb * nb;
  int cpb = pairs >= kCellThreads ? 1 : kCellThreads / pairs;
  auto fits = [&](int c) {
    const long a = cell_smem_bytes(nb, nq, FE_PREC_FP64, c), b = cell_smem_bytes(nb, nq, FE_PREC_FP32, c);
    return a >= 0 && b >= 0 && a <= 64 * 1024 && b <= 64 * 1024;
  };
  while (cpb * nq < 128 && fits(2 * cpb)) cpb *= 2;
  return cpb;
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
  prm.cpb = cells_per_block(s->nb, s->nq);
  prm.qblock = s->nq1d * s->nq1d;
  prm.nq1d = s->nq1d;
  prm.xv = s->d_xv;
  prm.w = s->d_w;
  prm.xq = s->d_xq;
  prm.phi = s->d_phi;
  prm.phi2 = reinterpret_cast<const float2*>(s->d_phi2);
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
template <typename TK>
__global__ void __launch_bounds__(kScatterWarps * 32) k_scatter(ScatterParams p) {
  __shared__ int64_t sbase[kScatterWarps][kMaxSlots + 1];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const TK* ke = reinterpret_cast<const TK*>(p.ke);
  ItemStream items(p.sched, p.n_rows, 1, lane);
  for (; items.valid(); items.advance(lane)) {
    const int64_t r = items.u;
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
  items.finish(int64_t(gridDim.x) * kScatterWarps, lane);
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
  ItemStream items(p.sched, p.n_rows, 1, lane);
  for (; items.valid(); items.advance(lane)) {
    const int64_t r = items.u;
    const int64_t s0 = p.slot_ptr[r];
    const int ns = int(p.slot_ptr[r + 1] - s0);
    const int64_t k0 = p.row_ptr[r];
    const int64_t c0 = p.code_ptr[r];
    const int nc = p.ncode ? p.ncode[r] : ns * p.nl;
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
  items.finish(int64_t(gridDim.x) * kScatterWarps, lane);
}

// Slot-wise scatter for FP32 cell matrices (the FP32 and BF16 forms). One warp
// per work item: a CSR row r (R = 1), or the R = ncomp rows of one node, which
// lie in the same cells at local rows i * nb + a and share their column
// pattern (R = 3). For each cell around the DOF in ascending order ("slot"),
// the lanes read that cell's matrix row(s) (coalesced) and the slot-major
// positions pos[s][m] of the entries among the row's nonzeros (one position
// block serves all R rows). The first contribution of each nonzero (flag bit
// 15 of pos; every entry of slot 0) stores (v, 0) into the row's double-float
// accumulator in shared memory; later ones add with Knuth's TwoSum, whose
// rounding error is kept exactly in the low part. The entries of one cell row
// go to distinct nonzeros, so the lanes never collide; a __syncwarp between
// slots orders the additions, so every nonzero sums its terms in ascending cell
// order. Each accumulator is rounded once to FP64 (df_to_double) and stored
// coalesced. Lanes past the end of a cell row (m >= NL) read padding and touch
// a private dummy accumulator, so the inner loop has no divergent branches
// (the position array and the cell-matrix scratch are allocated with padding
// for those reads). Slots are processed in batches of 4, 2 or 1 (the
// largest that fits the slots left and the register budget), all loads of a
// batch issued before its additions; the item descriptors (pointers, slot ids)
// of the warp's next item are fetched while the current one is reduced. Items
// go to warps on demand, kSlotGrab at a time (ItemStream). The RHS entries are
// formed first, in a static pass of 32 consecutive items per warp, one item per
// lane (exact fixed-point sum of its cells' FP64 cell-vector entries).
constexpr int kSlotGrab = 4;  // items per grab of k_scatter_slots

template <int NL, int R, bool IDX32>
__global__ void __launch_bounds__(kScatterWarps * 32, NL >= 128 ? 4 : 5) k_scatter_slots(ScatterParams p) {
  using S = SlotScatter<NL, R>;
  extern __shared__ __align__(16) unsigned char sm[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  float2* acc = reinterpret_cast<float2*>(sm + size_t(warp) * p.warp_bytes);
  const int rs = p.acc_stride + 32;       // accumulator row: acc_stride nonzeros, then one dummy per lane
  const int dummy = p.acc_stride + lane;  // within each accumulator row
  const float* ke = reinterpret_cast<const float*>(p.ke) + lane;
  const bool want_rhs = p.rhs != nullptr;
  const int64_t n_items = p.n_rows / R;
  const int64_t n_warps = int64_t(gridDim.x) * kScatterWarps;
  ItemStream items(p.sched, n_items, kSlotGrab, lane);
  if (want_rhs) {
    // RHS entries first, statically: 32 consecutive items per warp pass, one per lane
    for (int64_t ub = (int64_t(blockIdx.x) * kScatterWarps + warp) * 32; ub < n_items; ub += n_warps * 32) {
      const int64_t uu = ub + lane;
      if (uu < n_items) {
        const int64_t ss = p.slot_ptr[uu * R];
        const int nss = int(p.slot_ptr[uu * R + 1] - ss);
        if (nss <= 8) {
          // all gathers issued at once, the sum from registers
          int sl[8];
#pragma unroll
          for (int t = 0; t < 8; ++t) sl[t] = t < nss ? p.slots[ss + t] : 0;
#pragma unroll
          for (int i = 0; i < R; ++i) {
            double v[8];
#pragma unroll
            for (int t = 0; t < 8; ++t) v[t] = t < nss ? p.fe[sl[t] + i * S::NBR] : 0.0;
            p.rhs[uu * R + i] = fx_sum_regs(v);
          }
        } else {
#pragma unroll
          for (int i = 0; i < R; ++i)
            p.rhs[uu * R + i] = fx_sum<double>(nss, [&](int t) { return p.fe[p.slots[ss + t] + i * S::NBR]; });
        }
      }
    }
  }
  int64_t u = items.u;
  int64_t s0 = 0, k0 = 0, c0 = 0;
  int ns = 0, nnz = 0, my_slot = 0;
  if (u < n_items) {
    const int64_t r = u * R;
    s0 = p.slot_ptr[r];
    ns = int(p.slot_ptr[r + 1] - s0);
    k0 = p.row_ptr[r];
    nnz = int(p.row_ptr[r + 1] - k0);
    c0 = p.code_ptr[r];
    my_slot = lane < ns ? p.slots[s0 + lane] : 0;
  }
  while (u < n_items) {
    // first-level descriptors of the next item (independent loads)
    items.advance(lane);
    const int64_t un = items.u, rn = un * R;
    int64_t s0n = 0, s1n = 0, k0n = 0, k1n = 0, c0n = 0;
    if (un < n_items) {
      s0n = p.slot_ptr[rn];
      s1n = p.slot_ptr[rn + 1];
      k0n = p.row_ptr[rn];
      k1n = p.row_ptr[rn + 1];
      c0n = p.code_ptr[rn];
    }
    const uint16_t* pos = p.pos + c0 + lane;
    int sb = 0;
    while (sb < ns) {
      const int left = ns - sb;
      if (S::SB >= 4 && left >= 4) {
        S::template batch<4, IDX32>(p, ke, pos, my_slot, sb, acc, rs, dummy, lane);
        sb += 4;
      } else if (S::SB >= 2 && left >= 2) {
        S::template batch<2, IDX32>(p, ke, pos, my_slot, sb, acc, rs, dummy, lane);
        sb += 2;
      } else {
        S::template batch<1, IDX32>(p, ke, pos, my_slot, sb, acc, rs, dummy, lane);
        sb += 1;
      }
    }
    // second-level descriptors of the next item (its slot ids)
    const int nsn = int(s1n - s0n);
    const int my_slot_n = (un < n_items && lane < nsn) ? p.slots[s0n + lane] : 0;
#pragma unroll
    for (int i = 0; i < R; ++i) {
      const int64_t ki = k0 + int64_t(i) * nnz;  // the rows of one node are consecutive and equally long
      const float2* ai = acc + i * rs;
      for (int kb = 0; kb < nnz; kb += 32) {
        const int k = kb + lane;
        const float2 a = ai[k < nnz ? k : dummy];
        const double v = df_to_double(a.x, a.y);
        if (k < nnz) p.values[ki + k] = v;
      }
    }
    __syncwarp();
    s0 = s0n;
    ns = nsn;
    k0 = k0n;
    nnz = int(k1n - k0n);
    c0 = c0n;
    my_slot = my_slot_n;
    u = un;
  }
  items.finish(n_warps, lane);
}

static int align16(long x) { return int((x + 15) & ~15L); }

ScatterPattern space_pattern(const fe_space* s) {
  ScatterPattern pt;
  pt.n_rows = s->hs.n_dofs;
  pt.nnz = s->hs.nnz;
  pt.max_row_nnz = s->hs.max_row_nnz;
  pt.max_slots = s->hs.max_slots;
  pt.node_rows = s->hs.node_rows;
  pt.pos_ok = s->hs.pos_ok;
  pt.row_ptr = s->d_row_ptr;
  pt.cnt = s->d_cnt;
  pt.code_ptr = s->d_code_ptr;
  pt.codes = s->d_codes;
  pt.pos = s->d_pos;
  pt.slot_ptr = s->d_slot_ptr;
  pt.slots = s->d_slots;
  pt.ncode = nullptr;
  pt.sched = s->d_sched;
  return pt;
}

cudaError_t launch_scatter(const fe_space* s, fe_precision prec, double* values, double* rhs, cudaStream_t st) {
  return launch_scatter_pattern(s, space_pattern(s), prec, values, rhs, st);
}

cudaError_t launch_scatter_rows(const fe_space* s, const ScatterPattern& pt, fe_precision prec, double* values,
                                double* rhs, int64_t r0, int64_t r1, cudaStream_t st) {
  // every row-indexed array is offset to r0; positions within values, codes,
  // slots and cell data are absolute, so the kernels run unchanged
  ScatterPattern q = pt;
  q.n_rows = r1 - r0;
  q.row_ptr = pt.row_ptr + r0;
  q.code_ptr = pt.code_ptr + r0;
  q.slot_ptr = pt.slot_ptr + r0;
  if (pt.ncode) q.ncode = pt.ncode + r0;
  return launch_scatter_pattern(s, q, prec, values, rhs ? rhs + r0 : nullptr, st);
}

cudaError_t launch_scatter_pattern(const fe_space* s, const ScatterPattern& pt, fe_precision prec, double* values,
                                   double* rhs, cudaStream_t st) {
  if (pt.n_rows == 0) return cudaSuccess;
  ScatterParams p;
  p.n_rows = pt.n_rows;
  p.nl = s->nl;
  p.nlp = s->nlp;
  p.row_ptr = pt.row_ptr;
  p.cnt = pt.cnt;
  p.code_ptr = pt.code_ptr;
  p.codes = pt.codes;
  p.pos = pt.pos;
  p.slot_ptr = pt.slot_ptr;
  p.slots = pt.slots;
  p.ncode = pt.ncode;
  p.sched = pt.sched;
  p.ke = s->d_ke;
  p.fe = s->d_fe;
  p.values = values;
  p.rhs = rhs;
  const int tk = prec == FE_PREC_FP64 ? 8 : 4;
  p.ke_bytes = align16(long(pt.max_slots) * s->nlp * tk);
  p.code_bytes = align16(((long(pt.max_slots) * s->nl + 7) & ~7L) * 2);
  const int rows_warp_bytes = p.ke_bytes + p.code_bytes + align16((pt.max_row_nnz + 1) * 2);
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
  if (prec != FE_PREC_FP64 && pt.max_slots <= 32 && pt.pos_ok) {
    const bool idx32 = int64_t(s->n_cells) * s->nl * s->nlp < (int64_t(1) << 32);
    p.acc_stride = int((pt.max_row_nnz + 3) & ~int64_t(3));
    // rows of one node together (3-component problems), else one row per warp
    // (measured: pays for Q1, 24-entry cell rows; for wider rows one row per warp is faster)
    const int R = (pt.node_rows && s->ncomp == 3 && s->nl <= 32) ? 3 : 1;  // 3: nl = 24 only
    p.warp_bytes = R * (p.acc_stride + 32) * 8;  // R accumulator rows, each with one dummy per lane
    const long bytes = long(p.warp_bytes) * kScatterWarps;
    if (bytes <= 200 * 1024) {
      switch (s->nl * 4 + (R == 3 ? 2 : 0) + (idx32 ? 1 : 0)) {
        case 32: return launch(k_scatter_slots<8, 1, false>, bytes);
        case 33: return launch(k_scatter_slots<8, 1, true>, bytes);
        case 96: return launch(k_scatter_slots<24, 1, false>, bytes);
        case 97: return launch(k_scatter_slots<24, 1, true>, bytes);
        case 98: return launch(k_scatter_slots<24, 3, false>, bytes);
        case 99: return launch(k_scatter_slots<24, 3, true>, bytes);
        case 108: return launch(k_scatter_slots<27, 1, false>, bytes);
        case 109: return launch(k_scatter_slots<27, 1, true>, bytes);
        case 256: return launch(k_scatter_slots<64, 1, false>, bytes);
        case 257: return launch(k_scatter_slots<64, 1, true>, bytes);
        case 324: return launch(k_scatter_slots<81, 1, false>, bytes);
        case 325: return launch(k_scatter_slots<81, 1, true>, bytes);
        case 356: return launch(k_scatter_slots<89, 1, false>, bytes);   // Stokes Q2/Q1
        case 357: return launch(k_scatter_slots<89, 1, true>, bytes);
        case 768: return launch(k_scatter_slots<192, 1, false>, bytes);
        case 769: return launch(k_scatter_slots<192, 1, true>, bytes);
        default: break;
      }
    }
  }
  p.warp_bytes = rows_warp_bytes;
  if (smem <= 200 * 1024 && pt.max_slots <= 32) {
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
  const float* dphi32;
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
    if constexpr (std::is_same<T, float>::value) {
      // FP32 strain, FP64 geometry and sums: the conversions run on the
      // integer bits, w/det J and the physical gradients in FP32, one FP64
      // multiply-add per point accumulates w det J times the energy density
      // (GB300's FP64 pipe is the limit of this kernel).
      float ue[NL];
#pragma unroll
      for (int l = 0; l < NL; ++l) ue[l] = d2f_rn(p.u[p.cell_dofs[e * NL + l]]);
      const float lh = d2f_rn(p.lam_hat), mh2 = 2.f * d2f_rn(p.mu_hat);
      for (int q = 0; q < p.nq; ++q) {
        double cof[9], det;
        geometry_at(a, p.xq[3 * q], p.xq[3 * q + 1], p.xq[3 * q + 2], cof, &det);
        if (!(det > 0.0)) atomicOr(p.err, kErrNegJacobian);
        float gr[NC][3];
#pragma unroll
        for (int c = 0; c < NC; ++c) gr[c][0] = gr[c][1] = gr[c][2] = 0.f;
        const float* dq = p.dphi32 + size_t(q) * NB * 3;
#pragma unroll 4
        for (int b = 0; b < NB; ++b) {
          const float d0 = dq[3 * b], d1 = dq[3 * b + 1], d2 = dq[3 * b + 2];
#pragma unroll
          for (int c = 0; c < NC; ++c) {
            const float uc = ue[c * NB + b];
            gr[c][0] = fmaf(uc, d0, gr[c][0]);
            gr[c][1] = fmaf(uc, d1, gr[c][1]);
            gr[c][2] = fmaf(uc, d2, gr[c][2]);
          }
        }
        const float rdet = 1.f / d2f_rn(det);
        float cs[9];
#pragma unroll
        for (int t = 0; t < 9; ++t) cs[t] = d2f_rn(cof[t]) * rdet;
        float gu[NC][3];
#pragma unroll
        for (int c = 0; c < NC; ++c)
#pragma unroll
          for (int k = 0; k < 3; ++k) gu[c][k] = gr[c][0] * cs[3 * k] + gr[c][1] * cs[3 * k + 1] + gr[c][2] * cs[3 * k + 2];
        float dens;
        if (NC == 1) {
          dens = gu[0][0] * gu[0][0] + gu[0][1] * gu[0][1] + gu[0][2] * gu[0][2];
        } else {
          const float div = gu[0][0] + gu[1 % NC][1] + gu[2 % NC][2];
          float ee = 0.f;
#pragma unroll
          for (int k = 0; k < 3; ++k)
#pragma unroll
            for (int l = 0; l < 3; ++l) {
              const float eps = 0.5f * (gu[k % NC][l] + gu[l % NC][k]);
              ee += eps * eps;
            }
          dens = lh * (div * div) + mh2 * ee;
        }
        energy = fma(p.w[q] * det, f32_to_f64_exact(dens), energy);
      }
      p.g[e] = p.grad_scale * energy;
    } else {
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
  return launch_adjoint_with_scratch(s, u, coef, grad_scale, g, compliance, prec, s->d_partials, s->n_partials, st);
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
  prm.dphi32 = s->d_dphi32;
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

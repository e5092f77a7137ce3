// Batched assembly: many independent FE spaces (any order, problem and size)
// in one persistent launch, replayed from a CUDA graph.
//
// Work list. Each space contributes "cell items" (blocks of cells to
// integrate) and "row items" (blocks of CSR rows to assemble). The list
// holds, in order, the cell items of spaces 0 and 1, the row items of space
// 0, the cell items of space 2, the row items of space 1, ..., so the
// memory-bound assembly of one space overlaps the integration of the next.
// Persistent thread blocks take items from a global counter. A row item waits
// (bounded) until all cells of its space are integrated: every cell item of
// that space sits earlier in the list, was taken by a running block and never
// waits itself, so the wait always ends; after about one second of clock
// cycles it gives up, sets FE_ERR_TIMEOUT in every space's error word and the
// block leaves.
//
// Cell items run the CUDA-core cell kernel of the space's order and problem;
// row items run the slot-wise double-float scatter (FP32 and BF16 forms) or
// the exact fixed-point scatter (FP64 form), one warp per row. A space whose
// cells fe_assemble integrates on the tensor cores in the requested precision
// (its kernel selection: by default Q2 elasticity, and the BF16 forms of Q3
// Poisson and Q3 elasticity) gets no cell items: its tcgen05 cell kernel runs
// as a launch of its own on the caller's stream just before the persistent
// launch (outside the graph, whose kernel arguments are fixed at capture,
// while the coefficient pointers change per call), and its row items do not
// wait. Results are deterministic and, space by space, the same as
// fe_assemble's with the tensor-core kernel for those spaces and with the
// CUDA-core kernel for the others.
//
// Autotuning. The first fe_batch_assemble of a precision times each candidate
// (cells per item, rows per item) twice on the caller's buffers, keeps the
// fastest, and captures the counter reset and the launch into a CUDA graph;
// later calls update the per-space descriptors (one small copy) and replay it.
#include <cuda_runtime.h>

#include <algorithm>
#include <memory>
#include <vector>

#include "fe_device.cuh"

namespace feasm {
namespace batch {

struct Space {
  CellParams cell;
  ScatterParams scat;
  int order, ncomp, nl, pad;
  int64_t n_cells, n_rows;
  int64_t wait_target;     // integrated cells a row item waits for (n_cells; more only under the test hook)
  long long wait_cycles;   // limit of that wait in clock cycles
};

constexpr long long kDefaultWaitCycles = 1ll << 31;  // about one second

struct Item {
  int32_t space, kind;  // kind 0: cells [begin, end), kind 1: rows [begin, end)
  int64_t begin, end;
};

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;

// One CSR row by one warp for FP32 cell matrices: the slot-wise double-float
// accumulation of k_scatter_slots (slot batches of 4, 2 or 1, first
// contributions stored, later ones added with TwoSum); loads bypass L1 (the
// cell matrices were written earlier in this launch by other blocks). The
// RHS entries are formed separately (rhs_rows).
template <int NL>
__device__ void row_slots(const ScatterParams& p, int64_t r, int lane, float2* acc) {
  using S = SlotScatter<NL, 1, true>;
  const int64_t s0 = p.slot_ptr[r];
  const int ns = int(p.slot_ptr[r + 1] - s0);
  const int64_t k0 = p.row_ptr[r];
  const int nnz = int(p.row_ptr[r + 1] - k0);
  const uint16_t* pos = p.pos + p.code_ptr[r] + lane;
  const int my_slot = lane < ns ? p.slots[s0 + lane] : 0;
  const float* ke = reinterpret_cast<const float*>(p.ke) + lane;
  const int rs = p.acc_stride + 32;
  const int dummy = p.acc_stride + lane;
  int sb = 0;
  while (sb < ns) {
    const int left = ns - sb;
    if (S::SB >= 4 && left >= 4) {
      S::template batch<4, false>(p, ke, pos, my_slot, sb, acc, rs, dummy, lane);
      sb += 4;
    } else if (S::SB >= 2 && left >= 2) {
      S::template batch<2, false>(p, ke, pos, my_slot, sb, acc, rs, dummy, lane);
      sb += 2;
    } else {
      S::template batch<1, false>(p, ke, pos, my_slot, sb, acc, rs, dummy, lane);
      sb += 1;
    }
  }
  for (int kb = 0; kb < nnz; kb += 32) {
    const int k = kb + lane;
    const float2 a = acc[k < nnz ? k : dummy];
    const double v = df_to_double(a.x, a.y);
    if (k < nnz) p.values[k0 + k] = v;
  }
  __syncwarp();
}

// RHS entries of rows r0, r0 + step, ... (< r1), one row per lane: the exact
// fixed-point sum of the row's cells' FP64 cell-vector entries.
__device__ void rhs_rows(const ScatterParams& p, int64_t r0, int64_t r1, int64_t step, int lane) {
  for (int64_t r = r0 + lane * step; r < r1; r += 32 * step) {
    const int64_t s0 = p.slot_ptr[r];
    const int ns = int(p.slot_ptr[r + 1] - s0);
    p.rhs[r] = fx_sum<double>(ns, [&](int t) { return __ldcg(p.fe + p.slots[s0 + t]); });
  }
}

// One CSR row by one warp for FP64 cell matrices: one lane per nonzero, each
// summing its destination-sorted contributions exactly (k_scatter's method).
__device__ void row_exact64(const ScatterParams& p, int64_t r, int lane, int64_t* sbase) {
  const int64_t s0 = p.slot_ptr[r];
  const int ns = int(p.slot_ptr[r + 1] - s0);
  for (int s = lane; s < ns; s += 32) sbase[s] = int64_t(p.slots[s0 + s]) * p.nlp;
  __syncwarp();
  const double* ke = reinterpret_cast<const double*>(p.ke);
  if (p.rhs != nullptr && lane == 0)
    p.rhs[r] = fx_sum<double>(ns, [&](int t) { return __ldcg(p.fe + p.slots[s0 + t]); });
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
      p.values[k] = fx_sum<double>(n, [&](int t) {
        const unsigned code = cp[t];
        return __ldcg(ke + sbase[(code >> 8) & 127u] + (code & 255u));
      });
    }
    c += total;
  }
  __syncwarp();
}

template <int PREC>
__device__ __forceinline__ void run_cells(const Space& S, int64_t e0, int ncell, double* smem) {
  switch (S.order * 10 + S.ncomp) {
    case 11: cell_block<1, 1, PREC>(S.cell, e0, ncell, smem); break;
    case 13: cell_block<1, 3, PREC>(S.cell, e0, ncell, smem); break;
    case 21: cell_block<2, 1, PREC>(S.cell, e0, ncell, smem); break;
    case 23: cell_block<2, 3, PREC>(S.cell, e0, ncell, smem); break;
    case 31: cell_block<3, 1, PREC>(S.cell, e0, ncell, smem); break;
    case 33: cell_block<3, 3, PREC>(S.cell, e0, ncell, smem); break;
    default: break;
  }
}

template <int PREC>
__device__ __forceinline__ void run_row(const Space& S, int64_t r, int lane, unsigned char* wsm, int64_t* sbase) {
  if (PREC == 0) {
    row_exact64(S.scat, r, lane, sbase);
    return;
  }
  float2* acc = reinterpret_cast<float2*>(wsm);
  switch (S.nl) {
    case 8: row_slots<8>(S.scat, r, lane, acc); break;
    case 24: row_slots<24>(S.scat, r, lane, acc); break;
    case 27: row_slots<27>(S.scat, r, lane, acc); break;
    case 64: row_slots<64>(S.scat, r, lane, acc); break;
    case 81: row_slots<81>(S.scat, r, lane, acc); break;
    case 192: row_slots<192>(S.scat, r, lane, acc); break;
    default: break;
  }
}

template <int PREC>
__global__ void __launch_bounds__(kThreads) k_batch(const Space* sp, int n_spaces, const Item* items, int n_items,
                                                    int* counters, int row_warp_bytes) {
  extern __shared__ __align__(16) double smem[];
  __shared__ int s_item;
  __shared__ int s_abort;
  __shared__ int64_t sbase[kWarps][kMaxSlots + 1];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  for (;;) {
    if (tid == 0) {
      s_item = atomicAdd(&counters[0], 1);
      s_abort = 0;
    }
    __syncthreads();
    const int it = s_item;
    if (it >= n_items) break;
    const Item item = items[it];
    const Space& S = sp[item.space];
    if (item.kind == 0) {
      for (int64_t e0 = item.begin; e0 < item.end; e0 += S.cell.cpb) {
        const int ncell = int(item.end - e0 < S.cell.cpb ? item.end - e0 : S.cell.cpb);
        run_cells<PREC>(S, e0, ncell, smem);
        __syncthreads();
      }
      __threadfence();
      __syncthreads();
      if (tid == 0) atomicAdd(&counters[1 + item.space], int(item.end - item.begin));
    } else {
      if (tid == 0) {
        const long long t0 = clock64();
        while (atomicAdd(&counters[1 + item.space], 0) < S.wait_target) {
          if (clock64() - t0 > S.wait_cycles) {
            s_abort = 1;
            break;
          }
          __nanosleep(256);
        }
      }
      __syncthreads();
      if (s_abort) {
        if (tid == 0)
          for (int i = 0; i < n_spaces; ++i) atomicOr(sp[i].cell.err, kErrTimeout);
        break;
      }
      __threadfence();
      unsigned char* wsm = reinterpret_cast<unsigned char*>(smem) + size_t(warp) * row_warp_bytes;
      if (PREC != 0 && S.scat.rhs != nullptr) rhs_rows(S.scat, item.begin + warp, item.end, kWarps, lane);
      for (int64_t r = item.begin + warp; r < item.end; r += kWarps) run_row<PREC>(S, r, lane, wsm, sbase[warp]);
    }
    __syncthreads();
  }
}

}  // namespace batch
}  // namespace feasm

using feasm::batch::Item;
using feasm::batch::Space;

struct fe_batch {
  std::vector<fe_space*> spaces;
  int device = 0;
  int cells_per_item = 0;  // 0 = autotuned multiple of each space's cells per block
  std::vector<Space> h_spaces;
  Space* d_spaces = nullptr;
  int* d_counters = nullptr;
  cudaStream_t cap_stream = nullptr;
  struct Plan {
    bool ready = false;
    int cell_mult = 1, rows_per_item = 256;
    Item* d_items = nullptr;
    int n_items = 0;
    size_t smem = 0;
    int grid = 0, row_warp_bytes = 0;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    std::vector<char> tensor;  // per space: cells integrated on the tensor cores (no cell items)
  } plan[3];
  int extra_cells = 0;       // test hook: row items wait for this many cells more than exist
};

namespace {

int row_warp_bytes_for(const fe_space* s, fe_precision prec) {
  if (prec == FE_PREC_FP64) return 0;
  return int(((s->hs.max_row_nnz + 3) & ~int64_t(3)) + 32) * 8;
}

template <int PREC>
cudaError_t occupancy(int* per_sm, size_t smem) {
  cudaError_t e = cudaFuncSetAttribute(feasm::batch::k_batch<PREC>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       int(smem));
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, feasm::batch::k_batch<PREC>,
                                                       feasm::batch::kThreads, smem);
}

// Builds the work list of one plan and uploads it.
std::vector<char> tensor_spaces(const fe_batch* b, fe_precision prec) {
  std::vector<char> t(b->spaces.size());
  for (size_t i = 0; i < t.size(); ++i) t[i] = feasm::cell_on_tensor_cores(b->spaces[i], prec) ? 1 : 0;
  return t;
}

int build_plan(fe_batch* b, fe_precision prec, int cell_mult, int rows_per_item, fe_batch::Plan* pl) {
  std::vector<Item> items;
  const int n = int(b->spaces.size());
  pl->tensor = tensor_spaces(b, prec);
  auto add_cells = [&](int i) {
    if (pl->tensor[i]) return;
    const fe_space* s = b->spaces[i];
    const int64_t step = int64_t(feasm::cells_per_block(s->nb, s->nq)) *
                         (b->cells_per_item > 0 ? std::max(1, b->cells_per_item / feasm::cells_per_block(s->nb, s->nq))
                                                : cell_mult);
    for (int64_t c = 0; c < s->n_cells; c += step) items.push_back(Item{i, 0, c, std::min(s->n_cells, c + step)});
  };
  auto add_rows = [&](int i) {
    const fe_space* s = b->spaces[i];
    for (int64_t r = 0; r < s->hs.n_dofs; r += rows_per_item)
      items.push_back(Item{i, 1, r, std::min(s->hs.n_dofs, r + rows_per_item)});
  };
  for (int i = 0; i < n; ++i) {
    add_cells(i);
    if (i >= 1) add_rows(i - 1);
  }
  if (n > 0) add_rows(n - 1);
  size_t smem = 0;
  int rwb = 0;
  for (const fe_space* s : b->spaces) {
    smem = std::max<size_t>(smem, size_t(feasm::cell_smem_bytes(s->nb, s->nq, prec, feasm::cells_per_block(s->nb, s->nq))));
    rwb = std::max(rwb, row_warp_bytes_for(s, prec));
  }
  smem = std::max<size_t>(smem, size_t(rwb) * feasm::batch::kWarps);
  smem = std::max<size_t>(smem, 16);
  int per_sm = 0;
  cudaError_t e = prec == FE_PREC_FP64 ? occupancy<0>(&per_sm, smem)
                  : prec == FE_PREC_FP32 ? occupancy<1>(&per_sm, smem)
                                         : occupancy<2>(&per_sm, smem);
  if (e != cudaSuccess) return feasm::set_error(FE_ERR_CUDA, cudaGetErrorString(e));
  if (per_sm < 1) return feasm::set_error(FE_ERR_UNSUPPORTED, "batched kernel does not fit an SM");
  int nsm = 152;
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, b->device);
  if (pl->d_items) cudaFree(pl->d_items);
  pl->d_items = nullptr;
  e = cudaMalloc(&pl->d_items, std::max<size_t>(1, items.size()) * sizeof(Item));
  if (e == cudaSuccess && !items.empty())
    e = cudaMemcpy(pl->d_items, items.data(), items.size() * sizeof(Item), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return feasm::set_error(FE_ERR_CUDA, cudaGetErrorString(e));
  pl->n_items = int(items.size());
  pl->smem = smem;
  pl->grid = nsm * per_sm;
  pl->row_warp_bytes = rwb;
  pl->cell_mult = cell_mult;
  pl->rows_per_item = rows_per_item;
  return FE_OK;
}

cudaError_t launch_plan(fe_batch* b, fe_precision prec, const fe_batch::Plan& pl, cudaStream_t st) {
  const int n = int(b->spaces.size());
  cudaError_t e = cudaMemsetAsync(b->d_counters, 0, sizeof(int) * (n + 1), st);
  if (e != cudaSuccess) return e;
  if (pl.n_items == 0) return cudaSuccess;
  switch (prec) {
    case FE_PREC_FP64:
      feasm::batch::k_batch<0><<<pl.grid, feasm::batch::kThreads, pl.smem, st>>>(b->d_spaces, n, pl.d_items, pl.n_items,
                                                                                b->d_counters, pl.row_warp_bytes);
      break;
    case FE_PREC_FP32:
      feasm::batch::k_batch<1><<<pl.grid, feasm::batch::kThreads, pl.smem, st>>>(b->d_spaces, n, pl.d_items, pl.n_items,
                                                                                b->d_counters, pl.row_warp_bytes);
      break;
    default:
      feasm::batch::k_batch<2><<<pl.grid, feasm::batch::kThreads, pl.smem, st>>>(b->d_spaces, n, pl.d_items, pl.n_items,
                                                                                b->d_counters, pl.row_warp_bytes);
  }
  return cudaGetLastError();
}

void free_plan(fe_batch::Plan* pl) {
  if (pl->exec) cudaGraphExecDestroy(pl->exec);
  if (pl->graph) cudaGraphDestroy(pl->graph);
  if (pl->d_items) cudaFree(pl->d_items);
  *pl = fe_batch::Plan();
}

// Times the candidate (cells per item, rows per item) plans on the caller's
// buffers, keeps the fastest, and captures it into a CUDA graph.
int tune_and_capture(fe_batch* b, fe_precision prec, cudaStream_t st) {
  fe_batch::Plan& pl = b->plan[prec];
  const int mults[] = {1, 4, 16};
  const int rows[] = {128, 1024};
  float best = -1.f;
  int best_m = 1, best_r = 256;
  if (b->cells_per_item > 0) {
    best_m = 1;
    best_r = 256;
  } else {
    cudaEvent_t a, z;
    cudaEventCreate(&a);
    cudaEventCreate(&z);
    for (int m : mults)
      for (int rr : rows) {
        fe_batch::Plan cand;
        int rc = build_plan(b, prec, m, rr, &cand);
        if (rc) {
          cudaEventDestroy(a);
          cudaEventDestroy(z);
          free_plan(&cand);
          return rc;
        }
        float ms = 0.f;
        for (int rep = 0; rep < 2; ++rep) {
          cudaEventRecord(a, st);
          cudaError_t e = launch_plan(b, prec, cand, st);
          cudaEventRecord(z, st);
          if (e == cudaSuccess) e = cudaEventSynchronize(z);
          if (e != cudaSuccess) {
            cudaEventDestroy(a);
            cudaEventDestroy(z);
            free_plan(&cand);
            return feasm::set_error(FE_ERR_CUDA, cudaGetErrorString(e));
          }
          cudaEventElapsedTime(&ms, a, z);
        }
        if (best < 0.f || ms < best) {
          best = ms;
          best_m = m;
          best_r = rr;
        }
        free_plan(&cand);
      }
    cudaEventDestroy(a);
    cudaEventDestroy(z);
  }
  int rc = build_plan(b, prec, best_m, best_r, &pl);
  if (rc) return rc;
  cudaError_t e = cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    cudaError_t le = launch_plan(b, prec, pl, b->cap_stream);
    e = cudaStreamEndCapture(b->cap_stream, &pl.graph);
    if (le != cudaSuccess) e = le;
  }
  if (e == cudaSuccess) e = cudaGraphInstantiate(&pl.exec, pl.graph, 0);
  if (e != cudaSuccess) return feasm::set_error(FE_ERR_CUDA, cudaGetErrorString(e));
  pl.ready = true;
  return FE_OK;
}

}  // namespace

extern "C" {

static int batch_create(fe_space* const* spaces, int n, int cells_per_item, fe_batch** out) {
  if (!out) return feasm::set_error(FE_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (n < 0 || (n > 0 && !spaces)) return feasm::set_error(FE_ERR_INVALID_ARG, "invalid space list");
  int device = 0;
  cudaError_t e = cudaGetDevice(&device);
  if (e != cudaSuccess) return feasm::set_error(FE_ERR_CUDA, cudaGetErrorString(e));
  for (int i = 0; i < n; ++i) {
    const fe_space* s = spaces[i];
    if (!s || s->host_only) return feasm::set_error(FE_ERR_INVALID_ARG, "NULL or host-only space in the batch");
    if (s->device != device) return feasm::set_error(FE_ERR_INVALID_ARG, "spaces of a batch must share the current device");
    if (s->hs.max_slots > 32) return feasm::set_error(FE_ERR_UNSUPPORTED, "batched scatter needs at most 32 cells per DOF");
    if (s->problem == FE_STOKES) return feasm::set_error(FE_ERR_UNSUPPORTED, "the batch takes Poisson and elasticity spaces");
    if (int64_t(s->n_cells) > INT32_MAX) return feasm::set_error(FE_ERR_UNSUPPORTED, "space too large for a batch");
  }
  std::unique_ptr<fe_batch, void (*)(fe_batch*)> owner(new fe_batch(), fe_batch_destroy);
  fe_batch* b = owner.get();
  b->spaces.assign(spaces, spaces + n);
  b->device = device;
  b->cells_per_item = cells_per_item;
  b->h_spaces.resize(n);
  for (int i = 0; i < n; ++i) {
    const fe_space* s = spaces[i];
    Space& S = b->h_spaces[i];
    S.order = s->order;
    S.ncomp = s->ncomp;
    S.nl = s->nl;
    S.pad = 0;
    S.n_cells = s->n_cells;
    S.n_rows = s->hs.n_dofs;
    S.wait_target = s->n_cells;
    S.wait_cycles = feasm::batch::kDefaultWaitCycles;
    feasm::CellParams& c = S.cell;
    c.n_cells = s->n_cells;
    c.nq = s->nq;
    c.cpb = feasm::cells_per_block(s->nb, s->nq);
    c.qblock = s->nq1d * s->nq1d;
    c.nq1d = s->nq1d;
    c.xv = s->d_xv;
    c.w = s->d_w;
    c.xq = s->d_xq;
    c.phi = s->d_phi;
    c.phi2 = reinterpret_cast<const float2*>(s->d_phi2);
    c.dphi = s->d_dphi;
    c.dphi32 = s->d_dphi32;
    c.coef = nullptr;
    c.f[0] = c.f[1] = c.f[2] = 0.0;
    c.lam_hat = s->nu / ((1.0 + s->nu) * (1.0 - 2.0 * s->nu));
    c.mu_hat = 1.0 / (2.0 * (1.0 + s->nu));
    c.ke = s->d_ke;
    c.fe = s->d_fe;
    c.err = s->d_err;
    feasm::ScatterParams& q = S.scat;
    q = feasm::ScatterParams();
    q.n_rows = s->hs.n_dofs;
    q.nl = s->nl;
    q.nlp = s->nlp;
    q.row_ptr = s->d_row_ptr;
    q.cnt = s->d_cnt;
    q.code_ptr = s->d_code_ptr;
    q.codes = s->d_codes;
    q.pos = s->d_pos;
    q.slot_ptr = s->d_slot_ptr;
    q.slots = s->d_slots;
    q.ke = s->d_ke;
    q.fe = s->d_fe;
    q.acc_stride = int((s->hs.max_row_nnz + 3) & ~int64_t(3));
  }
  e = cudaMalloc(&b->d_spaces, std::max(1, n) * sizeof(Space));
  if (e == cudaSuccess) e = cudaMalloc(&b->d_counters, sizeof(int) * (n + 1));
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking);
  if (e != cudaSuccess)
    return feasm::set_error(e == cudaErrorMemoryAllocation ? FE_ERR_OOM : FE_ERR_CUDA, cudaGetErrorString(e));
  *out = owner.release();
  return FE_OK;
}

int fe_batch_create(fe_space* const* spaces, int n, int cells_per_item, fe_batch** out) {
  return feasm::no_throw("fe_batch_create", [&] { return batch_create(spaces, n, cells_per_item, out); });
}

static int batch_assemble(fe_batch* b, const double* const* coefficients, const double* body_force,
                          double* const* csr_values, double* const* rhs, fe_precision prec, void* stream) {
  if (!b) return feasm::set_error(FE_ERR_INVALID_ARG, "batch is NULL");
  if (prec != FE_PREC_FP64 && prec != FE_PREC_FP32 && prec != FE_PREC_BF16)
    return feasm::set_error(FE_ERR_INVALID_ARG, "unknown precision");
  const int n = int(b->spaces.size());
  if (n == 0) return FE_OK;
  if (!coefficients || !csr_values || !body_force) return feasm::set_error(FE_ERR_INVALID_ARG, "NULL argument");
  for (int i = 0; i < n; ++i) {
    Space& S = b->h_spaces[i];
    if ((S.n_cells && !coefficients[i]) || (b->spaces[i]->hs.nnz && !csr_values[i]))
      return feasm::set_error(FE_ERR_INVALID_ARG, "NULL coefficients or csr_values");
    S.cell.coef = coefficients[i];
    for (int k = 0; k < 3; ++k) S.cell.f[k] = k < S.ncomp ? body_force[3 * i + k] : 0.0;
    S.scat.values = csr_values[i];
    S.scat.rhs = rhs ? rhs[i] : nullptr;
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  fe_batch::Plan& pl = b->plan[prec];
  const std::vector<char> tensor = tensor_spaces(b, prec);
  if (pl.ready && pl.tensor != tensor) free_plan(&pl);  // a space's kernel selection changed
  for (int i = 0; i < n; ++i) {
    Space& S = b->h_spaces[i];
    S.wait_target = (tensor[i] ? 0 : S.n_cells) + b->extra_cells;
  }
  cudaError_t e = cudaMemcpyAsync(b->d_spaces, b->h_spaces.data(), n * sizeof(Space), cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return feasm::set_error(FE_ERR_CUDA, cudaGetErrorString(e));
  // the tensor-core cell kernels first, on the same stream
  for (int i = 0; i < n; ++i) {
    if (!tensor[i] || b->spaces[i]->n_cells == 0) continue;
    double f[3] = {0.0, 0.0, 0.0};
    for (int k = 0; k < b->spaces[i]->ncomp && k < 3; ++k) f[k] = body_force[3 * i + k];
    e = feasm::launch_cell_tensor(b->spaces[i], coefficients[i], f, prec, st);
    if (e != cudaSuccess) return feasm::set_error(FE_ERR_CUDA, cudaGetErrorString(e));
  }
  if (!pl.ready) {
    const int rc = tune_and_capture(b, prec, st);
    if (rc) return rc;
  }
  e = cudaGraphLaunch(pl.exec, st);
  if (e != cudaSuccess) return feasm::set_error(FE_ERR_CUDA, cudaGetErrorString(e));
  return FE_OK;
}

int fe_batch_assemble(fe_batch* b, const double* const* coefficients, const double* body_force,
                      double* const* csr_values, double* const* rhs, fe_precision prec, void* stream) {
  return feasm::no_throw("fe_batch_assemble",
                         [&] { return batch_assemble(b, coefficients, body_force, csr_values, rhs, prec, stream); });
}

int fe_batch_set_wait(fe_batch* b, long long wait_cycles, int extra_cells) {
  if (!b) return feasm::set_error(FE_ERR_INVALID_ARG, "batch is NULL");
  if (wait_cycles < 0 || extra_cells < 0) return feasm::set_error(FE_ERR_INVALID_ARG, "negative wait or extra cells");
  b->extra_cells = extra_cells;
  for (size_t i = 0; i < b->h_spaces.size(); ++i) {
    Space& S = b->h_spaces[i];
    S.wait_cycles = wait_cycles > 0 ? wait_cycles : feasm::batch::kDefaultWaitCycles;
    S.wait_target = S.n_cells + extra_cells;  // (the tensor-core spaces' share is set per call)
  }
  return FE_OK;
}

void fe_batch_destroy(fe_batch* b) {
  if (!b) return;
  for (auto& pl : b->plan) free_plan(&pl);
  if (b->d_spaces) cudaFree(b->d_spaces);
  if (b->d_counters) cudaFree(b->d_counters);
  if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
  delete b;
}

}  // extern "C"

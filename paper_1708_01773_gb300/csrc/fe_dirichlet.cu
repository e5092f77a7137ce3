// Strong Dirichlet conditions (paper, Sect. "Strong imposition of boundary
// conditions", Eq. dirichlet_bc_discrete_problem): the DOFs split into free
// and fixed ones, each labelled separately; the global matrix keeps the rows
// and columns of free DOFs only, and the cell vectors are updated with
// -A^K_{a,fixed} u^D before assembly. Also the DOF node positions of a space.
//
// GB300 form: the constrained system has its own assembly permutation, built
// once on the host from the space's cell-to-DOF map with the fixed DOFs
// dropped (fe_setup.cpp, build_pattern), and runs through the same scatter
// kernels as the unconstrained one. The cell-vector update ("lifting") is a
// small kernel over the cells that touch a fixed DOF, between the cell
// integration and the scatter.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "fe_device.cuh"
#include "fe_launch.h"

struct fe_dirichlet {
  fe_space* s = nullptr;
  int64_t n_free = 0, n_fixed = 0;
  std::vector<int32_t> label;  // [n_dofs]: free id >= 0, or -1 - fixed id
  feasm::HostSetup hs;         // the constrained pattern (cell_dofs unused)
  std::vector<int32_t> lift_cell, lift_ptr, lift_fix;
  std::vector<uint8_t> lift_m;
  // device copies
  int64_t* d_row_ptr = nullptr;
  int32_t* d_col = nullptr;
  uint8_t* d_cnt = nullptr;
  int64_t* d_code_ptr = nullptr;
  uint16_t* d_codes = nullptr;
  uint16_t* d_pos = nullptr;
  int64_t* d_slot_ptr = nullptr;
  int32_t* d_slots = nullptr;
  int32_t* d_ncode = nullptr;
  int32_t* d_lift_cell = nullptr;
  int32_t* d_lift_ptr = nullptr;
  uint8_t* d_lift_m = nullptr;
  int32_t* d_lift_fix = nullptr;
  unsigned long long* d_sched = nullptr;  // scatter schedule counters of this pattern
  int32_t* d_label = nullptr;             // [n_dofs] labels (free id or -1 - fixed id)
};

namespace feasm {

// One thread per (listed cell, local row a): the thread forms
// sum_j A^e[a][m_j] u_j over the cell's fixed local columns in ascending j, in
// FP64 (FP32 cell-matrix entries convert exactly), and subtracts it from
// fe[e][a]. All its loads are independent of the result, so the threads of a
// block keep many in flight; the order of the sum is fixed (deterministic).
template <typename TK>
__global__ void __launch_bounds__(256) k_lift(LiftParams p) {
  const TK* __restrict__ ke = static_cast<const TK*>(p.ke);
  double* __restrict__ fe = p.fe;
  const int64_t total = p.n_cells * p.nl;
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < total;
       i += int64_t(gridDim.x) * blockDim.x) {
    const int64_t c = i / p.nl;
    const int a = int(i - c * p.nl);
    const int64_t e = __ldg(p.cell + c);
    const int j0 = __ldg(p.ptr + c), j1 = __ldg(p.ptr + c + 1);
    const TK* __restrict__ krow = ke + (e * p.nl + a) * int64_t(p.nlp);
    const double f0 = fe[e * p.nl + a];
    double acc = 0.0;
#pragma unroll 4
    for (int j = j0; j < j1; ++j)
      acc = fma(double(__ldg(krow + __ldg(p.m + j))), __ldg(p.u_fixed + __ldg(p.fix + j)), acc);
    fe[e * p.nl + a] = f0 - acc;
  }
}

cudaError_t launch_lift(const LiftParams& lp, fe_precision prec, cudaStream_t st) {
  if (lp.n_cells == 0) return cudaSuccess;
  int dev = 0, nsm = 152;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  const int64_t need = (lp.n_cells * lp.nl + 255) / 256;
  const int blocks = int(std::min<int64_t>(need, int64_t(nsm) * 8));
  if (prec == FE_PREC_FP64)
    k_lift<double><<<blocks, 256, 0, st>>>(lp);
  else
    k_lift<float><<<blocks, 256, 0, st>>>(lp);
  return cudaGetLastError();
}

}  // namespace feasm

namespace {

int cuda_fail(cudaError_t e, const char* what) {
  std::string m = std::string(what) + ": " + cudaGetErrorString(e);
  return feasm::set_error(e == cudaErrorMemoryAllocation ? FE_ERR_OOM : FE_ERR_CUDA, m.c_str());
}

template <typename T>
cudaError_t upload(T** dst, const std::vector<T>& src, size_t extra = 0) {
  *dst = nullptr;
  const size_t n = src.size() + extra;
  if (n == 0) return cudaSuccess;
  cudaError_t e = cudaMalloc(reinterpret_cast<void**>(dst), n * sizeof(T));
  if (e != cudaSuccess) return e;
  if (extra) {
    e = cudaMemset(*dst, 0, n * sizeof(T));
    if (e != cudaSuccess) return e;
  }
  if (src.empty()) return cudaSuccess;
  return cudaMemcpy(*dst, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice);
}

void free_device(fe_dirichlet* d) {
  void* ptrs[] = {d->d_row_ptr, d->d_col,   d->d_cnt,       d->d_code_ptr, d->d_codes,   d->d_pos,     d->d_slot_ptr,
                  d->d_slots,   d->d_ncode, d->d_lift_cell, d->d_lift_ptr, d->d_lift_m, d->d_lift_fix,
                  d->d_sched,   d->d_label};
  for (void* p : ptrs)
    if (p) cudaFree(p);
}

feasm::ScatterPattern pattern_of(const fe_dirichlet* d) {
  feasm::ScatterPattern pt;
  pt.n_rows = d->hs.n_dofs;
  pt.nnz = d->hs.nnz;
  pt.max_row_nnz = d->hs.max_row_nnz;
  pt.max_slots = d->hs.max_slots;
  pt.node_rows = d->hs.node_rows;
  pt.pos_ok = d->hs.pos_ok;
  pt.row_ptr = d->d_row_ptr;
  pt.cnt = d->d_cnt;
  pt.code_ptr = d->d_code_ptr;
  pt.codes = d->d_codes;
  pt.pos = d->d_pos;
  pt.slot_ptr = d->d_slot_ptr;
  pt.slots = d->d_slots;
  pt.ncode = d->d_ncode;
  pt.sched = d->d_sched;
  return pt;
}

}  // namespace

extern "C" {

static int dof_points_host(const fe_space* s, const fe_mesh_desc* mesh, double* points) {
  if (!s || !mesh || !points) return feasm::set_error(FE_ERR_INVALID_ARG, "NULL argument");
  if (mesh->n_cells != s->n_cells || mesh->n_vertices != s->n_vertices || (s->n_cells && !mesh->cell_vertices) ||
      (s->n_vertices && !mesh->coords))
    return feasm::set_error(FE_ERR_INVALID_ARG, "mesh does not match the space");
  const int p = s->order, n1 = p + 1, nb = s->nb, nl = s->nl;
  const int64_t nd = s->hs.n_dofs;
  for (int64_t i = 0; i < 8 * s->n_cells; ++i)
    if (mesh->cell_vertices[i] < 0 || mesh->cell_vertices[i] >= mesh->n_vertices)
      return feasm::set_error(FE_ERR_INVALID_ARG, "cell_vertices entry out of range");
  std::vector<uint8_t> done(nd, 0);
  for (int64_t e = 0; e < s->n_cells; ++e) {
    const int32_t* cv = mesh->cell_vertices + 8 * e;
    const int32_t* dofs = s->hs.cell_dofs.data() + e * nl;
    for (int a = 0; a < nb; ++a) {
      if (done[dofs[a]]) continue;
      // the node's reference position alpha / p, mapped by the trilinear Phi_K
      const double al[3] = {double(a % n1) / p, double((a / n1) % n1) / p, double(a / (n1 * n1)) / p};
      double x[3] = {0.0, 0.0, 0.0};
      for (int v = 0; v < 8; ++v) {
        double n = 1.0;
        for (int d = 0; d < 3; ++d) n *= (v >> d & 1) ? al[d] : 1.0 - al[d];
        for (int d = 0; d < 3; ++d) x[d] += n * mesh->coords[3 * int64_t(cv[v]) + d];
      }
      for (int k = 0; k < s->ncomp; ++k) {
        const int32_t g = dofs[k * nb + a];
        done[g] = 1;
        for (int d = 0; d < 3; ++d) points[3 * int64_t(g) + d] = x[d];
      }
    }
  }
  return FE_OK;
}

int fe_space_dof_points_host(const fe_space* s, const fe_mesh_desc* mesh, double* points) {
  return feasm::no_throw("fe_space_dof_points_host", [&] { return dof_points_host(s, mesh, points); });
}

static int dirichlet_create(fe_space* s, const uint8_t* fixed, fe_dirichlet** out) {
  if (!out) return feasm::set_error(FE_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (!s || (s->hs.n_dofs && !fixed)) return feasm::set_error(FE_ERR_INVALID_ARG, "NULL argument");
  fe_dirichlet* d = new (std::nothrow) fe_dirichlet();
  if (!d) return feasm::set_error(FE_ERR_OOM, "host allocation failed");
  d->s = s;
  const int64_t nd = s->hs.n_dofs;
  const int nl = s->nl;
  std::string err;
  int rc = FE_OK;
  try {
    // free DOFs 0, 1, ... and fixed DOFs -1, -2, ..., each in ascending global id
    d->label.resize(nd);
    for (int64_t g = 0; g < nd; ++g)
      d->label[g] = fixed[g] ? int32_t(-1 - d->n_fixed++) : int32_t(d->n_free++);
    rc = feasm::build_pattern(s->nl, s->nb, s->problem == FE_ELASTICITY ? 3 : 1, s->n_cells, s->hs.cell_dofs.data(),
                              d->label.data(), d->n_free, &d->hs, &err);
    // lifting lists: every cell with a fixed and a free DOF, its fixed local columns ascending
    d->lift_ptr.push_back(0);
    for (int64_t e = 0; e < s->n_cells && rc == FE_OK; ++e) {
      const int32_t* dofs = s->hs.cell_dofs.data() + e * nl;
      bool any_free = false;
      size_t first = d->lift_m.size();
      for (int m = 0; m < nl; ++m) {
        const int32_t l = d->label[dofs[m]];
        if (l < 0) {
          d->lift_m.push_back(uint8_t(m));
          d->lift_fix.push_back(-1 - l);
        } else {
          any_free = true;
        }
      }
      if (d->lift_m.size() > first && any_free) {
        d->lift_cell.push_back(int32_t(e));
        d->lift_ptr.push_back(int32_t(d->lift_m.size()));
      } else {
        d->lift_m.resize(first);
        d->lift_fix.resize(first);
      }
    }
  } catch (const std::bad_alloc&) {
    rc = FE_ERR_OOM;
    err = "host allocation failed during setup";
  }
  if (rc) {
    delete d;
    return feasm::set_error(rc, err.c_str());
  }
  if (!s->host_only) {
    const auto& hs = d->hs;
    cudaError_t e = upload(&d->d_row_ptr, hs.row_ptr);
    if (e == cudaSuccess) e = upload(&d->d_col, hs.col);
    if (e == cudaSuccess) e = upload(&d->d_cnt, hs.cnt);
    if (e == cudaSuccess) e = upload(&d->d_code_ptr, hs.code_ptr);
    if (e == cudaSuccess) e = upload(&d->d_codes, hs.codes);
    if (e == cudaSuccess) e = upload(&d->d_pos, hs.pos);
    if (e == cudaSuccess) e = upload(&d->d_slot_ptr, hs.slot_ptr);
    if (e == cudaSuccess) e = upload(&d->d_slots, hs.slots);
    if (e == cudaSuccess) e = upload(&d->d_ncode, hs.ncode);
    if (e == cudaSuccess) e = upload(&d->d_lift_cell, d->lift_cell);
    if (e == cudaSuccess) e = upload(&d->d_lift_ptr, d->lift_ptr);
    if (e == cudaSuccess) e = upload(&d->d_lift_m, d->lift_m);
    if (e == cudaSuccess) e = upload(&d->d_lift_fix, d->lift_fix);
    if (e == cudaSuccess) e = upload(&d->d_sched, std::vector<unsigned long long>(2, 0ull));
    if (e == cudaSuccess) e = upload(&d->d_label, d->label);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
      free_device(d);
      delete d;
      return cuda_fail(e, "fe_dirichlet_create upload");
    }
    // the large host arrays are no longer needed (row_ptr and col are kept for inspection)
    std::vector<uint8_t>().swap(d->hs.cnt);
    std::vector<uint16_t>().swap(d->hs.codes);
    std::vector<uint16_t>().swap(d->hs.pos);
    std::vector<int64_t>().swap(d->hs.code_ptr);
    std::vector<int32_t>().swap(d->hs.slots);
    std::vector<int32_t>().swap(d->hs.ncode);
  }
  *out = d;
  return FE_OK;
}

int fe_dirichlet_create(fe_space* s, const uint8_t* fixed, fe_dirichlet** out) {
  return feasm::no_throw("fe_dirichlet_create", [&] { return dirichlet_create(s, fixed, out); });
}

int fe_dirichlet_sizes(const fe_dirichlet* d, int64_t* n_free, int64_t* n_fixed, int64_t* nnz) {
  if (!d) return feasm::set_error(FE_ERR_INVALID_ARG, "NULL argument");
  if (n_free) *n_free = d->n_free;
  if (n_fixed) *n_fixed = d->n_fixed;
  if (nnz) *nnz = d->hs.nnz;
  return FE_OK;
}

int fe_dirichlet_labels_host(const fe_dirichlet* d, int32_t* labels) {
  if (!d || (!labels && !d->label.empty())) return feasm::set_error(FE_ERR_INVALID_ARG, "NULL argument");
  if (!d->label.empty()) std::memcpy(labels, d->label.data(), d->label.size() * sizeof(int32_t));
  return FE_OK;
}

int fe_dirichlet_csr_pattern_host(const fe_dirichlet* d, int64_t* row_ptr, int32_t* col_idx) {
  if (!d || !row_ptr || (!col_idx && d->hs.nnz)) return feasm::set_error(FE_ERR_INVALID_ARG, "NULL argument");
  std::memcpy(row_ptr, d->hs.row_ptr.data(), d->hs.row_ptr.size() * sizeof(int64_t));
  if (d->hs.nnz) std::memcpy(col_idx, d->hs.col.data(), d->hs.col.size() * sizeof(int32_t));
  return FE_OK;
}

int fe_dirichlet_csr_pattern(const fe_dirichlet* d, int64_t* row_ptr, int32_t* col_idx, void* stream) {
  if (!d || !row_ptr || (!col_idx && d->hs.nnz)) return feasm::set_error(FE_ERR_INVALID_ARG, "NULL argument");
  if (d->s->host_only) return feasm::set_error(FE_ERR_INVALID_ARG, "host-only space");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  cudaError_t e = cudaMemcpyAsync(row_ptr, d->d_row_ptr, (d->n_free + 1) * sizeof(int64_t),
                                  cudaMemcpyDeviceToDevice, st);
  if (e == cudaSuccess && d->hs.nnz)
    e = cudaMemcpyAsync(col_idx, d->d_col, d->hs.nnz * sizeof(int32_t), cudaMemcpyDeviceToDevice, st);
  return e == cudaSuccess ? FE_OK : cuda_fail(e, "fe_dirichlet_csr_pattern");
}

int fe_dirichlet_permutation_host(const fe_dirichlet* d, uint8_t* cnt, int64_t* code_ptr, uint16_t* codes,
                                  int32_t* ncode, uint16_t* pos, int64_t* slot_ptr, int32_t* slots) {
  if (!d || !cnt || !code_ptr || !ncode || !slot_ptr || !slots)
    return feasm::set_error(FE_ERR_INVALID_ARG, "NULL argument");
  if (!d->s->host_only)
    return feasm::set_error(FE_ERR_INVALID_ARG, "the permutation is kept on the host only for host-only spaces");
  const auto& hs = d->hs;
  std::memcpy(cnt, hs.cnt.data(), hs.cnt.size());
  std::memcpy(code_ptr, hs.code_ptr.data(), hs.code_ptr.size() * sizeof(int64_t));
  if (codes) std::memcpy(codes, hs.codes.data(), hs.codes.size() * sizeof(uint16_t));
  std::memcpy(ncode, hs.ncode.data(), hs.ncode.size() * sizeof(int32_t));
  if (pos) std::memcpy(pos, hs.pos.data(), hs.n_codes * sizeof(uint16_t));
  std::memcpy(slot_ptr, hs.slot_ptr.data(), hs.slot_ptr.size() * sizeof(int64_t));
  std::memcpy(slots, hs.slots.data(), hs.slots.size() * sizeof(int32_t));
  return FE_OK;
}

int fe_dirichlet_lift_host(const fe_dirichlet* d, int64_t* n_cells, int64_t* n_entries, int32_t* cells,
                           int32_t* ptr, uint8_t* m, int32_t* fix) {
  if (!d) return feasm::set_error(FE_ERR_INVALID_ARG, "NULL argument");
  if (n_cells) *n_cells = int64_t(d->lift_cell.size());
  if (n_entries) *n_entries = int64_t(d->lift_m.size());
  if (cells) std::memcpy(cells, d->lift_cell.data(), d->lift_cell.size() * sizeof(int32_t));
  if (ptr) std::memcpy(ptr, d->lift_ptr.data(), d->lift_ptr.size() * sizeof(int32_t));
  if (m) std::memcpy(m, d->lift_m.data(), d->lift_m.size());
  if (fix) std::memcpy(fix, d->lift_fix.data(), d->lift_fix.size() * sizeof(int32_t));
  return FE_OK;
}

int fe_assemble_dirichlet(fe_dirichlet* d, const double* coefficients, const double* body_force,
                          const double* u_fixed, double* csr_values, double* rhs, fe_precision prec, void* stream) {
  if (!d) return feasm::set_error(FE_ERR_INVALID_ARG, "NULL argument");
  fe_space* s = d->s;
  if (s->host_only) return feasm::set_error(FE_ERR_INVALID_ARG, "host-only space cannot compute");
  if (prec != FE_PREC_FP64 && prec != FE_PREC_FP32 && prec != FE_PREC_BF16)
    return feasm::set_error(FE_ERR_INVALID_ARG, "unknown precision");
  if ((s->n_cells && !coefficients) || (d->hs.nnz && !csr_values))
    return feasm::set_error(FE_ERR_INVALID_ARG, "NULL coefficients or csr_values");
  if (rhs && !body_force) return feasm::set_error(FE_ERR_INVALID_ARG, "rhs requested without body_force");
  double f[3] = {0.0, 0.0, 0.0};
  if (body_force)
    for (int k = 0; k < s->ncomp; ++k) f[k] = body_force[k];
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (int rc = feasm::cell_stage(s, coefficients, f, prec, st)) return rc;
  if (rhs && u_fixed && !d->lift_cell.empty()) {
    feasm::LiftParams lp;
    lp.n_cells = int64_t(d->lift_cell.size());
    lp.nl = s->nl;
    lp.nlp = s->nlp;
    lp.cell = d->d_lift_cell;
    lp.ptr = d->d_lift_ptr;
    lp.m = d->d_lift_m;
    lp.fix = d->d_lift_fix;
    lp.u_fixed = u_fixed;
    lp.ke = s->d_ke;
    lp.fe = s->d_fe;
    cudaError_t e = feasm::launch_lift(lp, prec, st);
    if (e != cudaSuccess) return cuda_fail(e, "lifting kernel");
  }
  cudaError_t e = feasm::launch_scatter_pattern(s, pattern_of(d), prec, csr_values, rhs, st);
  return e == cudaSuccess ? FE_OK : cuda_fail(e, "scatter kernel");
}

int fe_compliance_work_size(const fe_dirichlet* d, int64_t* n_doubles) {
  if (!d || !n_doubles) return feasm::set_error(FE_ERR_INVALID_ARG, "NULL argument");
  *n_doubles = feasm::compliance_work_doubles(d->n_free, d->hs.nnz);
  return FE_OK;
}

int fe_compliance(fe_dirichlet* d, const double* coefficients, const double* body_force, fe_precision prec,
                  double rtol, int max_iter, double* work, double* u, double* compliance, double* dc_dcoef,
                  int* iterations, double* rel_residual, void* stream) {
  if (!d || !body_force || !work || !compliance || (d->s->hs.n_dofs && !u) || (d->s->n_cells && !coefficients))
    return feasm::set_error(FE_ERR_INVALID_ARG, "NULL argument");
  if (d->s->host_only) return feasm::set_error(FE_ERR_INVALID_ARG, "host-only space cannot compute");
  if (d->s->problem == FE_STOKES)
    return feasm::set_error(FE_ERR_UNSUPPORTED, "the compliance is for Poisson and elasticity (Stokes is indefinite)");
  if (!(rtol > 0.0) || max_iter < 0) return feasm::set_error(FE_ERR_INVALID_ARG, "rtol must be > 0, max_iter >= 0");
  fe_space* s = d->s;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  double* vals = work;
  double* rhs = work + d->hs.nnz;
  if (int rc = fe_assemble_dirichlet(d, coefficients, body_force, nullptr, vals, rhs, prec, stream)) return rc;
  int it_local = 0;
  double rel_local = 0.0;
  feasm::ComplianceArgs a;
  a.n_free = d->n_free;
  a.nnz = d->hs.nnz;
  a.n_dofs = s->hs.n_dofs;
  a.row_ptr = d->d_row_ptr;
  a.col = d->d_col;
  a.label = d->d_label;
  a.work = work;
  a.rtol = rtol;
  a.max_iter = max_iter;
  a.u = u;
  a.compliance = compliance;
  a.iterations = iterations ? iterations : &it_local;
  a.rel_residual = rel_residual ? rel_residual : &rel_local;
  const int rc = feasm::compliance_solve(a, st);
  if (rc) return rc;
  if (dc_dcoef && s->n_cells) {
    const fe_precision pa = prec == FE_PREC_FP64 ? FE_PREC_FP64 : FE_PREC_FP32;
    cudaError_t e = feasm::launch_adjoint(s, u, coefficients, -1.0, dc_dcoef, nullptr, pa, st);
    if (e != cudaSuccess) return cuda_fail(e, "compliance gradient");
  }
  return FE_OK;
}

void fe_dirichlet_destroy(fe_dirichlet* d) {
  if (!d) return;
  if (!d->s->host_only) free_device(d);
  delete d;
}

}  // extern "C"

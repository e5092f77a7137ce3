// C-ABI entry points of libfeasm: space creation (host setup + upload),
// assembly, adjoint, status, and the host-buffer variant.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>

#include "fe_launch.h"

namespace {

thread_local std::string g_last_error;

int fail(int code, const std::string& msg) {
  g_last_error = msg;
  return code;
}

int cuda_fail(cudaError_t e, const char* what) {
  g_last_error = std::string(what) + ": " + cudaGetErrorString(e);
  return e == cudaErrorMemoryAllocation ? FE_ERR_OOM : FE_ERR_CUDA;
}

#define FE_CUDA(call)                                 \
  do {                                                \
    cudaError_t e_ = (call);                          \
    if (e_ != cudaSuccess) return cuda_fail(e_, #call); \
  } while (0)

template <typename T>
cudaError_t upload(T** dst, const T* src, size_t n) {
  *dst = nullptr;
  if (n == 0) return cudaSuccess;
  cudaError_t e = cudaMalloc(reinterpret_cast<void**>(dst), n * sizeof(T));
  if (e != cudaSuccess) return e;
  return cudaMemcpy(*dst, src, n * sizeof(T), cudaMemcpyHostToDevice);
}

void free_device(fe_space* s) {
  void* ptrs[] = {s->d_xv, s->d_w, s->d_xq, s->d_phi, s->d_dphi, s->d_dphi32, s->d_phi2, s->d_cell_dofs, s->d_row_ptr,
                  s->d_col, s->d_cnt, s->d_code_ptr, s->d_codes, s->d_pos, s->d_slot_ptr, s->d_slots, s->d_ke, s->d_fe,
                  s->d_err, s->d_partials, s->d_stage_coef, s->d_stage_vals, s->d_stage_rhs, s->d_sched, s->d_psi};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  for (void* ev : s->range_done)
    if (ev) cudaEventDestroy(static_cast<cudaEvent_t>(ev));
  if (s->copy_stream) cudaStreamDestroy(static_cast<cudaStream_t>(s->copy_stream));
}

// Frees a space under construction unless released (every early return and
// any exception of create_space).
struct SpaceGuard {
  fe_space* s;
  ~SpaceGuard() {
    if (s) {
      free_device(s);
      delete s;
    }
  }
};

int create_space(const fe_mesh_desc* mesh, int order, int quad_points_1d, fe_problem problem, double nu,
                 bool host_only, fe_space** out) {
  if (!out) return fail(FE_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (!mesh || mesh->n_cells < 0 || mesh->n_vertices < 0 || (mesh->n_cells > 0 && !mesh->cell_vertices) ||
      (mesh->n_vertices > 0 && !mesh->coords))
    return fail(FE_ERR_INVALID_ARG, "invalid mesh descriptor");
  if (order < 1 || order > feasm::kMaxOrder) return fail(FE_ERR_INVALID_ARG, "order must be 1..3");
  const int nq1d = quad_points_1d == 0 ? order + 1 : quad_points_1d;
  if (nq1d < 1 || nq1d > feasm::kMaxQ1d) return fail(FE_ERR_INVALID_ARG, "quad_points_1d must be 0 or 1..6");
  if (problem != FE_POISSON && problem != FE_ELASTICITY && problem != FE_STOKES)
    return fail(FE_ERR_INVALID_ARG, "unknown problem");
  if (problem == FE_STOKES && (order < 2 || nq1d != order + 1))
    return fail(FE_ERR_UNSUPPORTED, "Stokes (Taylor-Hood) needs velocity order 2 or 3 and the (p+1)^3 rule");
  if (problem == FE_ELASTICITY && !(nu >= 0.0 && nu < 0.5)) return fail(FE_ERR_INVALID_ARG, "nu must be in [0, 0.5)");
  if (mesh->n_vertices > INT32_MAX) return fail(FE_ERR_UNSUPPORTED, "more than 2^31-1 vertices");
  fe_space* s = new (std::nothrow) fe_space();
  if (!s) return fail(FE_ERR_OOM, "host allocation failed");
  SpaceGuard guard{s};
  s->order = order;
  s->nq1d = nq1d;
  s->problem = problem;
  s->ncomp = problem == FE_POISSON ? 1 : 3;
  s->nu = nu;
  s->n_cells = mesh->n_cells;
  s->n_vertices = mesh->n_vertices;
  s->host_only = host_only;
  feasm::build_ref_tables(order, nq1d, &s->tab);
  s->nb = s->tab.nb;
  s->nq = s->tab.nq;
  s->nbp = problem == FE_STOKES ? order * order * order : 0;
  s->nl = s->ncomp * s->nb + s->nbp;
  s->nlp = (s->nl + 3) & ~3;
  std::string err;
  int rc;
  try {
    rc = feasm::build_host_setup(order, problem, mesh->n_cells, mesh->n_vertices, mesh->cell_vertices, &s->hs, &err);
  } catch (const std::bad_alloc&) {
    rc = FE_ERR_OOM;
    err = "host allocation failed during setup";
  } catch (const std::exception& x) {
    rc = FE_ERR_UNSUPPORTED;
    err = std::string("host setup failed: ") + x.what();
  }
  if (rc) return fail(rc, err);
  if (!host_only) {
    const int cpb = feasm::cells_per_block(s->nb, s->nq);
    if (problem != FE_STOKES && (feasm::cell_smem_bytes(s->nb, s->nq, FE_PREC_FP64, cpb) < 0 ||
                                 feasm::cell_smem_bytes(s->nb, s->nq, FE_PREC_FP32, cpb) < 0))
      return fail(FE_ERR_UNSUPPORTED, "quadrature too large for one block at this order");
    cudaError_t e = cudaGetDevice(&s->device);
    std::vector<double> xv;
    if (e == cudaSuccess) {
      xv.resize(size_t(s->n_cells) * 24);
      for (int64_t c = 0; c < s->n_cells; ++c)
        for (int v = 0; v < 8; ++v)
          for (int k = 0; k < 3; ++k)
            xv[size_t(c) * 24 + v * 3 + k] = mesh->coords[3 * int64_t(mesh->cell_vertices[8 * c + v]) + k];
    }
    std::vector<float> dphi32(s->tab.dphi.begin(), s->tab.dphi.end());
    std::vector<float> phi2(2 * s->tab.phi.size());
    for (size_t i = 0; i < s->tab.phi.size(); ++i) {
      const float hi = float(s->tab.phi[i]);
      phi2[2 * i] = hi;
      phi2[2 * i + 1] = float(s->tab.phi[i] - double(hi));
    }
    const auto& hs = s->hs;
    if (e == cudaSuccess) e = upload(&s->d_xv, xv.data(), xv.size());
    if (e == cudaSuccess) e = upload(&s->d_w, s->tab.w.data(), s->tab.w.size());
    if (e == cudaSuccess) e = upload(&s->d_xq, s->tab.xq.data(), s->tab.xq.size());
    if (e == cudaSuccess) e = upload(&s->d_phi, s->tab.phi.data(), s->tab.phi.size());
    if (e == cudaSuccess) e = upload(&s->d_dphi, s->tab.dphi.data(), s->tab.dphi.size());
    if (e == cudaSuccess) e = upload(&s->d_dphi32, dphi32.data(), dphi32.size());
    if (e == cudaSuccess) e = upload(&s->d_phi2, phi2.data(), phi2.size());
    if (e == cudaSuccess && problem == FE_STOKES) {
      feasm::RefTables tp;  // pressure basis Q_{p-1} at the same quadrature points
      feasm::build_ref_tables(order - 1, nq1d, &tp);
      e = upload(&s->d_psi, tp.phi.data(), tp.phi.size());
    }
    if (e == cudaSuccess) e = upload(&s->d_cell_dofs, hs.cell_dofs.data(), hs.cell_dofs.size());
    if (e == cudaSuccess) e = upload(&s->d_row_ptr, hs.row_ptr.data(), hs.row_ptr.size());
    if (e == cudaSuccess) e = upload(&s->d_col, hs.col.data(), hs.col.size());
    if (e == cudaSuccess) e = upload(&s->d_cnt, hs.cnt.data(), hs.cnt.size());
    if (e == cudaSuccess) e = upload(&s->d_code_ptr, hs.code_ptr.data(), hs.code_ptr.size());
    if (e == cudaSuccess) e = upload(&s->d_codes, hs.codes.data(), hs.codes.size());
    if (e == cudaSuccess) e = upload(&s->d_pos, hs.pos.data(), hs.pos.size());
    if (e == cudaSuccess) e = upload(&s->d_slot_ptr, hs.slot_ptr.data(), hs.slot_ptr.size());
    if (e == cudaSuccess) e = upload(&s->d_slots, hs.slots.data(), hs.slots.size());
    // FP64-sized (the FP32 forms use the first half); 256 bytes of padding for the
    // scatter's whole-chunk reads past the end of the last cell row
    const size_t nke = size_t(s->n_cells) * s->nl * s->nlp;
    if (e == cudaSuccess && nke) e = cudaMalloc(&s->d_ke, nke * sizeof(double) + 256);
    if (e == cudaSuccess && s->n_cells) e = cudaMalloc(&s->d_fe, size_t(s->n_cells) * s->nl * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&s->d_err, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(s->d_err, 0, sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc(&s->d_sched, 2 * sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMemset(s->d_sched, 0, 2 * sizeof(unsigned long long));
    s->n_partials = int((s->n_cells + 127) / 128) + 1;
    if (e == cudaSuccess) e = cudaMalloc(&s->d_partials, size_t(s->n_partials) * sizeof(double));
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return cuda_fail(e, "fe_space_create upload");
    // the large host arrays are no longer needed (cell_dofs, row_ptr and col are kept for inspection)
    std::vector<uint8_t>().swap(s->hs.cnt);
    std::vector<uint16_t>().swap(s->hs.codes);
    std::vector<uint16_t>().swap(s->hs.pos);
    std::vector<int64_t>().swap(s->hs.code_ptr);
    std::vector<int32_t>().swap(s->hs.slots);
  }
  guard.s = nullptr;
  *out = s;
  return FE_OK;
}

int create_common(const fe_mesh_desc* mesh, int order, int quad_points_1d, fe_problem problem, double nu,
                  bool host_only, fe_space** out) {
  return feasm::no_throw("fe_space_create",
                         [&] { return create_space(mesh, order, quad_points_1d, problem, nu, host_only, out); });
}

}  // namespace

namespace feasm {
int set_error(int code, const char* msg) { return fail(code, msg); }

// Poisson on the tensor cores: on request, and by default for the BF16 form of
// Q3 (3x faster there, within its 1e-2 bound). The FP32 form stays on the CUDA
// cores by default: on the tensor cores it is not within 1e-6 on every single
// distorted Q3 cell (their FP32 accumulation truncates), and Q2's 27 x 27 cell
// blocks run faster on the CUDA cores.
static bool tcp_chosen(const fe_space* s, fe_precision prec) {
  return cell_tcp_applicable(s, prec) &&
         (s->cell_kernel == FE_KERNEL_TENSOR_CORE ||
          (s->cell_kernel == FE_KERNEL_AUTO && s->order == 3 && prec == FE_PREC_BF16));
}

// Q3 elasticity on the tensor cores: on request, and by default for BF16.
static bool tce_chosen(const fe_space* s, fe_precision prec) {
  return cell_tce_applicable(s, prec) &&
         (s->cell_kernel == FE_KERNEL_TENSOR_CORE || (s->cell_kernel == FE_KERNEL_AUTO && prec == FE_PREC_BF16));
}

bool cell_on_tensor_cores(const fe_space* s, fe_precision prec) {
  if (s->problem == FE_STOKES || s->cell_kernel == FE_KERNEL_CUDA_CORE) return false;
  return tcp_chosen(s, prec) || tce_chosen(s, prec) || cell_tc_applicable(s, prec);
}

cudaError_t launch_cell_tensor(const fe_space* s, const double* coef, const double force[3], fe_precision prec,
                               cudaStream_t st) {
  if (tcp_chosen(s, prec)) return launch_cell_tcp(s, coef, force, prec, st);
  if (tce_chosen(s, prec)) return launch_cell_tce(s, coef, force, prec, st);
  return launch_cell_tc(s, coef, force, prec, st);
}

int cell_stage(fe_space* s, const double* coef, const double force[3], fe_precision prec, cudaStream_t st) {
  if (s->problem == FE_STOKES) {
    if (prec == FE_PREC_BF16) return fail(FE_ERR_UNSUPPORTED, "Stokes cell integration has FP64 and FP32 forms only");
    if (s->cell_kernel == FE_KERNEL_TENSOR_CORE) return fail(FE_ERR_UNSUPPORTED, "no tensor-core Stokes kernel");
    FE_CUDA(launch_cell_stokes(s, coef, force, prec, st));
    return FE_OK;
  }
  const bool any_tc = cell_tc_applicable(s, prec) || cell_tcp_applicable(s, prec) || cell_tce_applicable(s, prec);
  if (s->cell_kernel == FE_KERNEL_TENSOR_CORE && !any_tc)
    return fail(FE_ERR_UNSUPPORTED, "no tensor-core cell kernel for this order / problem / precision");
  if (cell_on_tensor_cores(s, prec))
    FE_CUDA(launch_cell_tensor(s, coef, force, prec, st));
  else if (q1e_applicable(s, prec))
    FE_CUDA(launch_cell_q1e(s, coef, force, prec, st));
  else
    FE_CUDA(launch_cell_integration(s, coef, force, prec, st));
  return FE_OK;
}
}  // namespace feasm

extern "C" {

const char* fe_last_error(void) { return g_last_error.c_str(); }

int fe_space_create(const fe_mesh_desc* mesh, int order, int quad_points_1d, fe_problem problem, double nu,
                    fe_space** out) {
  return create_common(mesh, order, quad_points_1d, problem, nu, false, out);
}

int fe_space_create_host(const fe_mesh_desc* mesh, int order, int quad_points_1d, fe_problem problem, double nu,
                         fe_space** out) {
  return create_common(mesh, order, quad_points_1d, problem, nu, true, out);
}

int fe_space_block_offset(const fe_space* s, int64_t* n_first) {
  if (!s || !n_first) return fail(FE_ERR_INVALID_ARG, "NULL argument");
  *n_first = s->hs.n_first;
  return FE_OK;
}

int fe_space_sizes(const fe_space* s, int64_t* n_dofs, int64_t* nnz, int64_t* n_cells, int64_t* n_contrib) {
  if (!s) return fail(FE_ERR_INVALID_ARG, "space is NULL");
  if (n_dofs) *n_dofs = s->hs.n_dofs;
  if (nnz) *nnz = s->hs.nnz;
  if (n_cells) *n_cells = s->n_cells;
  if (n_contrib) *n_contrib = s->hs.n_contrib;
  return FE_OK;
}

int fe_space_cell_dofs_host(const fe_space* s, int32_t* cell_dofs) {
  if (!s || !cell_dofs) return fail(FE_ERR_INVALID_ARG, "NULL argument");
  std::memcpy(cell_dofs, s->hs.cell_dofs.data(), s->hs.cell_dofs.size() * sizeof(int32_t));
  return FE_OK;
}

int fe_space_csr_pattern_host(const fe_space* s, int64_t* row_ptr, int32_t* col_idx) {
  if (!s || !row_ptr || (!col_idx && s->hs.nnz)) return fail(FE_ERR_INVALID_ARG, "NULL argument");
  std::memcpy(row_ptr, s->hs.row_ptr.data(), s->hs.row_ptr.size() * sizeof(int64_t));
  if (s->hs.nnz) std::memcpy(col_idx, s->hs.col.data(), s->hs.col.size() * sizeof(int32_t));
  return FE_OK;
}

int fe_space_permutation_host(const fe_space* s, uint8_t* cnt, int64_t* code_ptr, uint16_t* codes,
                              int64_t* slot_ptr, int32_t* slots) {
  if (!s || !cnt || !code_ptr || !slot_ptr || !slots) return fail(FE_ERR_INVALID_ARG, "NULL argument");
  if (!s->host_only) return fail(FE_ERR_INVALID_ARG, "the permutation is kept on the host only for host-only spaces");
  const auto& hs = s->hs;
  std::memcpy(cnt, hs.cnt.data(), hs.cnt.size());
  std::memcpy(code_ptr, hs.code_ptr.data(), hs.code_ptr.size() * sizeof(int64_t));
  if (codes) std::memcpy(codes, hs.codes.data(), hs.codes.size() * sizeof(uint16_t));
  std::memcpy(slot_ptr, hs.slot_ptr.data(), hs.slot_ptr.size() * sizeof(int64_t));
  std::memcpy(slots, hs.slots.data(), hs.slots.size() * sizeof(int32_t));
  return FE_OK;
}

int fe_space_csr_pattern(const fe_space* s, int64_t* row_ptr, int32_t* col_idx, void* stream) {
  if (!s || !row_ptr || (!col_idx && s->hs.nnz)) return fail(FE_ERR_INVALID_ARG, "NULL argument");
  if (s->host_only) return fail(FE_ERR_INVALID_ARG, "host-only space");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  FE_CUDA(cudaMemcpyAsync(row_ptr, s->d_row_ptr, (s->hs.n_dofs + 1) * sizeof(int64_t), cudaMemcpyDeviceToDevice, st));
  if (s->hs.nnz)
    FE_CUDA(cudaMemcpyAsync(col_idx, s->d_col, s->hs.nnz * sizeof(int32_t), cudaMemcpyDeviceToDevice, st));
  return FE_OK;
}

static int check_compute_space(const fe_space* s) {
  if (!s) return fail(FE_ERR_INVALID_ARG, "space is NULL");
  if (s->host_only) return fail(FE_ERR_INVALID_ARG, "host-only space cannot compute");
  return FE_OK;
}

int fe_assemble(fe_space* s, const double* coefficients, const double* body_force, double* csr_values, double* rhs,
                fe_precision prec, void* stream) {
  return fe_assemble_ex(s, coefficients, body_force, csr_values, rhs, prec, stream, nullptr);
}

int fe_assemble_ex(fe_space* s, const double* coefficients, const double* body_force, double* csr_values,
                   double* rhs, fe_precision prec, void* stream, void* event_mid) {
  if (int rc = check_compute_space(s)) return rc;
  if (prec != FE_PREC_FP64 && prec != FE_PREC_FP32 && prec != FE_PREC_BF16)
    return fail(FE_ERR_INVALID_ARG, "unknown precision");
  if ((s->n_cells && !coefficients) || (s->hs.nnz && !csr_values))
    return fail(FE_ERR_INVALID_ARG, "NULL coefficients or csr_values");
  if (rhs && !body_force) return fail(FE_ERR_INVALID_ARG, "rhs requested without body_force");
  double f[3] = {0.0, 0.0, 0.0};
  if (body_force)
    for (int k = 0; k < s->ncomp; ++k) f[k] = body_force[k];
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (int rc = feasm::cell_stage(s, coefficients, f, prec, st)) return rc;
  if (event_mid) FE_CUDA(cudaEventRecord(static_cast<cudaEvent_t>(event_mid), st));
  FE_CUDA(feasm::launch_scatter(s, prec, csr_values, rhs, st));
  return FE_OK;
}

int fe_assemble_host(fe_space* s, const double* coefficients, const double* body_force, double* csr_values,
                     double* rhs, fe_precision prec, void* stream) {
  if (int rc = check_compute_space(s)) return rc;
  if (prec != FE_PREC_FP64 && prec != FE_PREC_FP32 && prec != FE_PREC_BF16)
    return fail(FE_ERR_INVALID_ARG, "unknown precision");
  if ((s->n_cells && !coefficients) || (s->hs.nnz && !csr_values))
    return fail(FE_ERR_INVALID_ARG, "NULL coefficients or csr_values");
  if (rhs && !body_force) return fail(FE_ERR_INVALID_ARG, "rhs requested without body_force");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  constexpr int kRanges = 8;
  if (!s->d_stage_coef) {
    FE_CUDA(cudaMalloc(&s->d_stage_coef, std::max<int64_t>(1, s->n_cells) * sizeof(double)));
    FE_CUDA(cudaMalloc(&s->d_stage_vals, std::max<int64_t>(1, s->hs.nnz) * sizeof(double)));
    FE_CUDA(cudaMalloc(&s->d_stage_rhs, std::max<int64_t>(1, s->hs.n_dofs) * sizeof(double)));
    cudaStream_t cs = nullptr;
    FE_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    s->copy_stream = cs;
    for (int i = 0; i < kRanges; ++i) {
      cudaEvent_t ev = nullptr;
      FE_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
      s->range_done[i] = ev;
    }
  }
  double f[3] = {0.0, 0.0, 0.0};
  if (body_force)
    for (int k = 0; k < s->ncomp; ++k) f[k] = body_force[k];
  double* dr = rhs ? s->d_stage_rhs : nullptr;
  FE_CUDA(cudaMemcpyAsync(s->d_stage_coef, coefficients, s->n_cells * sizeof(double), cudaMemcpyHostToDevice, st));
  if (int rc = feasm::cell_stage(s, s->d_stage_coef, f, prec, st)) return rc;
  // scatter in row ranges (whole items: rows of one node together), each
  // range's results copied out on the copy stream once its launch is done
  cudaStream_t cs = static_cast<cudaStream_t>(s->copy_stream);
  const feasm::ScatterPattern pt = feasm::space_pattern(s);
  const int64_t n = s->hs.n_dofs, unit = s->ncomp;
  const int64_t* rp = s->hs.row_ptr.data();
  for (int c = 0; c < kRanges; ++c) {
    const int64_t r0 = (n * c / kRanges) / unit * unit, r1 = c + 1 == kRanges ? n : (n * (c + 1) / kRanges) / unit * unit;
    if (r1 <= r0) continue;
    FE_CUDA(feasm::launch_scatter_rows(s, pt, prec, s->d_stage_vals, dr, r0, r1, st));
    cudaEvent_t ev = static_cast<cudaEvent_t>(s->range_done[c]);
    FE_CUDA(cudaEventRecord(ev, st));
    FE_CUDA(cudaStreamWaitEvent(cs, ev, 0));
    FE_CUDA(cudaMemcpyAsync(csr_values + rp[r0], s->d_stage_vals + rp[r0], (rp[r1] - rp[r0]) * sizeof(double),
                            cudaMemcpyDeviceToHost, cs));
    if (rhs)
      FE_CUDA(cudaMemcpyAsync(rhs + r0, s->d_stage_rhs + r0, (r1 - r0) * sizeof(double), cudaMemcpyDeviceToHost, cs));
  }
  FE_CUDA(cudaStreamSynchronize(cs));
  FE_CUDA(cudaStreamSynchronize(st));
  return FE_OK;
}

int fe_assemble_adjoint(fe_space* s, const double* u, const double* coefficients, double grad_scale,
                        double* dc_dcoef, double* compliance, fe_precision prec, void* stream) {
  if (int rc = check_compute_space(s)) return rc;
  if (s->problem == FE_STOKES) return fail(FE_ERR_UNSUPPORTED, "the compliance adjoint is for Poisson and elasticity");
  if (s->n_cells && (!u || !dc_dcoef)) return fail(FE_ERR_INVALID_ARG, "NULL u or dc_dcoef");
  if (compliance && !coefficients && s->n_cells) return fail(FE_ERR_INVALID_ARG, "compliance requested without coefficients");
  if (prec != FE_PREC_FP64 && prec != FE_PREC_FP32) return fail(FE_ERR_INVALID_ARG, "adjoint precision must be FP64 or FP32");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (s->n_cells == 0) {
    if (compliance) FE_CUDA(cudaMemsetAsync(compliance, 0, sizeof(double), st));
    return FE_OK;
  }
  FE_CUDA(feasm::launch_adjoint(s, u, coefficients, grad_scale, dc_dcoef, compliance, prec, st));
  return FE_OK;
}

int fe_space_set_kernel(fe_space* s, int cell_kernel) {
  if (!s) return fail(FE_ERR_INVALID_ARG, "space is NULL");
  if (cell_kernel < FE_KERNEL_AUTO || cell_kernel > FE_KERNEL_TENSOR_CORE)
    return fail(FE_ERR_INVALID_ARG, "unknown cell kernel");
  s->cell_kernel = cell_kernel;
  return FE_OK;
}

int fe_status(fe_space* s, void* stream) {
  if (int rc = check_compute_space(s)) return rc;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int h = 0;
  FE_CUDA(cudaMemcpyAsync(&h, s->d_err, sizeof(int), cudaMemcpyDeviceToHost, st));
  FE_CUDA(cudaStreamSynchronize(st));
  FE_CUDA(cudaMemsetAsync(s->d_err, 0, sizeof(int), st));
  FE_CUDA(cudaStreamSynchronize(st));
  if (h & feasm::kErrNegJacobian) return fail(FE_ERR_NEG_JACOBIAN, "non-positive Jacobian determinant at a quadrature point");
  if (h & feasm::kErrTimeout) return fail(FE_ERR_TIMEOUT, "a bounded device wait gave up");
  return FE_OK;
}

void fe_space_destroy(fe_space* s) {
  if (!s) return;
  if (!s->host_only) free_device(s);
  delete s;
}

}  // extern "C"

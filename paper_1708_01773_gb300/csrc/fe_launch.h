// Kernel launchers of libfeasm (defined in fe_kernels.cu).
#pragma once

#include <cuda_runtime.h>

#include "fe_internal.h"

namespace feasm {

// Error bits of the device error word.
constexpr int kErrNegJacobian = 1;
constexpr int kErrTimeout = 2;

// Cell integration: geometry (FP64), physical gradients, cell-matrix
// contraction in the arithmetic of `prec`, cell vectors (FP64). Writes
// s->d_ke (FP64 for FE_PREC_FP64, FP32 otherwise) and s->d_fe.
cudaError_t launch_cell_integration(const fe_space* s, const double* coef, const double force[3],
                                    fe_precision prec, cudaStream_t st);

// Tensor-core (tcgen05) cell integration for Q2 elasticity with the 3^3 rule,
// FP32 (3xTF32) and BF16 forms; same outputs as launch_cell_integration.
bool cell_tc_applicable(const fe_space* s, fe_precision prec);
cudaError_t launch_cell_tc(const fe_space* s, const double* coef, const double force[3], fe_precision prec,
                           cudaStream_t st);

// Whether fe_assemble integrates the cells of `s` on the tensor cores in
// `prec` under the space's kernel selection (FE_KERNEL_AUTO: Q2 elasticity,
// and the BF16 forms of Q3 Poisson and Q3 elasticity; FE_KERNEL_TENSOR_CORE:
// every case a tensor-core kernel covers), and the launch of that kernel.
bool cell_on_tensor_cores(const fe_space* s, fe_precision prec);
cudaError_t launch_cell_tensor(const fe_space* s, const double* coef, const double force[3], fe_precision prec,
                               cudaStream_t st);

// Q1 elasticity (2^3 rule), FP32 and BF16 forms, with the automatic kernel
// choice: the warp-role cell kernel (FP64 geometry on its own warps); same
// outputs as launch_cell_integration.
bool q1e_applicable(const fe_space* s, fe_precision prec);

// Tensor-core (tcgen05) cell integration of the Poisson problem for Q2 and Q3
// with the (p+1)^3 rule, FP32 (3xTF32) and BF16 forms; same outputs as
// launch_cell_integration.
bool cell_tcp_applicable(const fe_space* s, fe_precision prec);
// Tensor-core (tcgen05) cell integration of Q3 elasticity with the 4^3 rule,
// FP32 (3xTF32) and BF16 forms; same outputs as launch_cell_integration.
bool cell_tce_applicable(const fe_space* s, fe_precision prec);
cudaError_t launch_cell_tce(const fe_space* s, const double* coef, const double force[3], fe_precision prec,
                            cudaStream_t st);
cudaError_t launch_cell_tcp(const fe_space* s, const double* coef, const double force[3], fe_precision prec,
                            cudaStream_t st);
cudaError_t launch_cell_q1e(const fe_space* s, const double* coef, const double force[3], fe_precision prec,
                            cudaStream_t st);

// Device arrays and host-side sizes of one assembly permutation: the space's
// own (every DOF a row) or a constrained one (free DOFs only).
struct ScatterPattern {
  int64_t n_rows = 0, nnz = 0, max_row_nnz = 0;
  int max_slots = 0;
  bool node_rows = false, pos_ok = true;
  const int64_t* row_ptr = nullptr;
  const uint8_t* cnt = nullptr;
  const int64_t* code_ptr = nullptr;
  const uint16_t* codes = nullptr;
  const uint16_t* pos = nullptr;
  const int64_t* slot_ptr = nullptr;
  const int32_t* slots = nullptr;
  const int32_t* ncode = nullptr;  // codes per row, or nullptr: slots * n_loc
  unsigned long long* sched = nullptr;  // [2] counters of the dynamic row schedule (zero between launches)
};
ScatterPattern space_pattern(const fe_space* s);

// Stokes (Taylor-Hood) cell integration, FP64 or FP32 form; writes s->d_ke and s->d_fe.
cudaError_t launch_cell_stokes(const fe_space* s, const double* coef, const double force[3], fe_precision prec,
                               cudaStream_t st);

// Deterministic scatter of the cell matrices/vectors into CSR values / RHS.
cudaError_t launch_scatter(const fe_space* s, fe_precision prec, double* values, double* rhs, cudaStream_t st);
cudaError_t launch_scatter_pattern(const fe_space* s, const ScatterPattern& pt, fe_precision prec, double* values,
                                   double* rhs, cudaStream_t st);
// The scatter of rows [r0, r1) only (r0, r1 multiples of the rows per item of
// the pattern: ncomp for node-wise patterns); values are still indexed by the
// CSR positions of the whole pattern, rhs by the row.
cudaError_t launch_scatter_rows(const fe_space* s, const ScatterPattern& pt, fe_precision prec, double* values,
                                double* rhs, int64_t r0, int64_t r1, cudaStream_t st);

// Integrates every cell of `s` into its cell-matrix and cell-vector scratch
// with the kernel chosen by the space's kernel selection. Returns an FE code.
int cell_stage(fe_space* s, const double* coef, const double force[3], fe_precision prec, cudaStream_t st);

// Lifting of strong Dirichlet data into the cell vectors: for the cells
// listed, fe[e][a] -= sum_j A^e[a][m_j] * u_fixed[fix_j] over the cell's fixed
// local columns m_j (every local row a).
struct LiftParams {
  int64_t n_cells = 0;
  int nl = 0, nlp = 0;
  const int32_t* cell = nullptr;  // [n_cells]
  const int32_t* ptr = nullptr;   // [n_cells + 1] into m / fix
  const uint8_t* m = nullptr;     // local column of each fixed DOF of the cell
  const int32_t* fix = nullptr;   // its fixed id
  const double* u_fixed = nullptr;
  const void* ke = nullptr;
  double* fe = nullptr;
};
cudaError_t launch_lift(const LiftParams& lp, fe_precision prec, cudaStream_t st);

// Compliance of a clamped structure: PCG (Jacobi) on the constrained system
// already assembled into work[0 .. nnz) (values) and work[nnz .. nnz + n_free)
// (right-hand side), then u over all DOFs and c = f . u. Synchronises `st`.
struct ComplianceArgs {
  int64_t n_free = 0, nnz = 0, n_dofs = 0;
  const int64_t* row_ptr = nullptr;
  const int32_t* col = nullptr;
  const int32_t* label = nullptr;  // device [n_dofs]
  double* work = nullptr;          // compliance_work_doubles(n_free, nnz)
  double rtol = 1e-10;
  int max_iter = 0;
  double* u = nullptr;             // device [n_dofs]
  double* compliance = nullptr;    // device scalar
  int* iterations = nullptr;       // host
  double* rel_residual = nullptr;  // host
};
int64_t compliance_work_doubles(int64_t n_free, int64_t nnz);
int compliance_solve(const ComplianceArgs& a, cudaStream_t st);

// Threads per block of the adjoint kernel (one cell per thread); its per-block
// partial sums of the compliance are what the reduction scratch holds.
constexpr int kAdjointBlock = 128;

// Records a message for fe_last_error() and returns `code`.
int set_error(int code, const char* msg);

// The adjoint with caller-provided reduction scratch `partials` of capacity
// `max_partials` doubles (one per block of kAdjointBlock cells).
cudaError_t launch_adjoint_with_scratch(const fe_space* s, const double* u, const double* coef, double grad_scale,
                                        double* g, double* compliance, fe_precision prec, double* partials,
                                        int max_partials, cudaStream_t st);

// Compliance sensitivities and (optionally) the compliance.
cudaError_t launch_adjoint(const fe_space* s, const double* u, const double* coef, double grad_scale,
                           double* g, double* compliance, fe_precision prec, cudaStream_t st);

// Dynamic shared memory needed by the cell-integration kernel (bytes), or -1
// if the combination does not fit one block.
long cell_smem_bytes(int nb, int nq, fe_precision prec, int cells_per_block);
int cells_per_block(int nb, int nq);

}  // namespace feasm

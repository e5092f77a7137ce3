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

// Deterministic scatter of the cell matrices/vectors into CSR values / RHS.
cudaError_t launch_scatter(const fe_space* s, fe_precision prec, double* values, double* rhs, cudaStream_t st);

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

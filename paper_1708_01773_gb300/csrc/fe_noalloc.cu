// fe_assemble_adjoint_noalloc: the compliance adjoint with its reduction
// scratch in a fixed, statically allocated device array, so that the call
// allocates no memory at all.
//
// Who needs this: applications that own every byte of device memory through
// their own pool allocator and do not let a library call cudaMalloc behind
// their back, and loops that must not enter the CUDA allocator once running
// (cudaMalloc and cudaFree can synchronise the device). The FE space itself is
// still built once by fe_space_create, outside such a loop.
#include <cuda_runtime.h>

#include "fe_launch.h"

// Partial sums of the compliance, one per block of feasm::kAdjointBlock cells:
// 65,536 doubles (512 KB), i.e. at most 65,536 * 128 = 8,388,608 cells per call
// when the compliance is requested. Every GPU that loads the library holds this
// array until the process exits.
constexpr int kNoAllocPartials = 65536;
static __device__ __align__(256) double g_noalloc_partials[kNoAllocPartials];

namespace {

// Device address of the array in the current context. In host code the name
// g_noalloc_partials is only a host-side stand-in: passing it to a kernel would
// be wrong, so the address comes from cudaGetSymbolAddress with the space's
// device current. It is looked up on every call (the lookup allocates
// nothing): a cached address would dangle once the application resets the
// device (cudaDeviceReset), which tears down the context that held the array.
cudaError_t scratch_address(double** out) {
  void* p = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_partials);
  if (e != cudaSuccess) return e;
  *out = static_cast<double*>(p);
  return cudaSuccess;
}

}  // namespace

extern "C" int fe_assemble_adjoint_noalloc(fe_space* s, const double* u, const double* coefficients,
                                           double grad_scale, double* dc_dcoef, double* compliance,
                                           fe_precision prec, void* stream) {
  if (!s) return feasm::set_error(FE_ERR_INVALID_ARG, "space is NULL");
  if (s->problem == FE_STOKES)
    return feasm::set_error(FE_ERR_UNSUPPORTED, "the compliance adjoint is for Poisson and elasticity");
  if (s->host_only) return feasm::set_error(FE_ERR_INVALID_ARG, "host-only space cannot compute");
  if (s->n_cells && (!u || !dc_dcoef)) return feasm::set_error(FE_ERR_INVALID_ARG, "NULL u or dc_dcoef");
  if (compliance && !coefficients && s->n_cells)
    return feasm::set_error(FE_ERR_INVALID_ARG, "compliance requested without coefficients");
  if (prec != FE_PREC_FP64 && prec != FE_PREC_FP32)
    return feasm::set_error(FE_ERR_INVALID_ARG, "adjoint precision must be FP64 or FP32");
  const int64_t blocks = (s->n_cells + feasm::kAdjointBlock - 1) / feasm::kAdjointBlock;
  if (compliance && blocks > kNoAllocPartials)
    return feasm::set_error(FE_ERR_UNSUPPORTED,
                            "fe_assemble_adjoint_noalloc: more than 8,388,608 cells with the compliance requested "
                            "(limit of its static scratch); use fe_assemble_adjoint");
  int device = 0;
  cudaError_t e = cudaGetDevice(&device);
  if (e != cudaSuccess) return feasm::set_error(FE_ERR_CUDA, cudaGetErrorString(e));
  if (device != s->device)
    return feasm::set_error(FE_ERR_INVALID_ARG, "the current device is not the device of the space");
  double* scratch = nullptr;
  e = scratch_address(&scratch);
  if (e != cudaSuccess) return feasm::set_error(FE_ERR_CUDA, cudaGetErrorString(e));
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (s->n_cells == 0) {
    if (compliance) {
      e = cudaMemsetAsync(compliance, 0, sizeof(double), st);
      if (e != cudaSuccess) return feasm::set_error(FE_ERR_CUDA, cudaGetErrorString(e));
    }
    return FE_OK;
  }
  // No part of the scratch needs to start at zero: every block writes its own
  // partial before the final sum reads it.
  e = feasm::launch_adjoint_with_scratch(s, u, coefficients, grad_scale, dc_dcoef, compliance, prec, scratch,
                                         kNoAllocPartials, st);
  if (e != cudaSuccess) return feasm::set_error(FE_ERR_CUDA, cudaGetErrorString(e));
  return FE_OK;
}

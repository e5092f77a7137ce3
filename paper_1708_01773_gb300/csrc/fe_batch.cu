// Batched assembly of several FE spaces (placeholder until the persistent
// batched driver lands).
#include "fe_launch.h"

extern "C" {

int fe_batch_create(fe_space* const* spaces, int n, int cells_per_item, fe_batch** out) {
  (void)spaces; (void)n; (void)cells_per_item;
  if (out) *out = nullptr;
  return FE_ERR_UNSUPPORTED;
}

int fe_batch_assemble(fe_batch* b, const double* const* coefficients, const double* body_force,
                      double* const* csr_values, double* const* rhs, fe_precision prec, void* stream) {
  (void)b; (void)coefficients; (void)body_force; (void)csr_values; (void)rhs; (void)prec; (void)stream;
  return FE_ERR_UNSUPPORTED;
}

void fe_batch_destroy(fe_batch* b) { (void)b; }

}

// line_newton.cu -- Newton-Krylov method for line contact (method 1).
#include <cuda_runtime.h>

#include "line.h"

namespace ehl {
cudaError_t line_nk_alloc(LineCtx* c) {
  (void)c;
  return cudaSuccess;
}
cudaError_t line_nk_step(LineCtx* c, double* P, double* H0, const double* rough) {
  (void)c;
  (void)P;
  (void)H0;
  (void)rough;
  return cudaErrorNotSupported;
}
}  // namespace ehl

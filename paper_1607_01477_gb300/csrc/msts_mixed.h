// msts_mixed.h -- internal interface of the mixed-precision solve.
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

namespace msts {
size_t mixed_workspace_bytes(int m, int n, int nb, uint32_t flags);
cudaError_t mixed_run(const double2 *U, long long ldu, int m, const double2 *s, int n,
                      const double2 *B, long long ldb, double2 *X, long long ldx, double tol,
                      int max_iter, int nb, uint32_t flags, void *ws, uint32_t *status,
                      int *iters_out, double *eta_out, double *eta0_out, cudaStream_t st);
cudaError_t residual_run(const double2 *U, long long ldu, int m, const double2 *s, int n,
                         const double2 *B, long long ldb, const double2 *X, long long ldx,
                         double2 *R, long long ldr, uint32_t flags, void *oz_ws, uint32_t *status,
                         cudaStream_t st);
}  // namespace msts

// msts_ozaki.h -- internal interface of the tensor-core FP64-accurate residual.
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

namespace msts {
// Workspace for the digit planes of triu(U) and X and their exponents.
size_t ozaki_workspace_bytes(int m, int n);
// Splits triu(U) into BF16 digit planes (once per matrix).
cudaError_t ozaki_prepare(const double2 *U, long long ldu, int m, int n, void *ws, cudaStream_t st);
// R = B - triu(U) X + X diag(s) with the product on the tensor cores; needs a
// prior ozaki_prepare of U into the same workspace.
cudaError_t ozaki_residual(const double2 *U, long long ldu, int m, const double2 *s, int n,
                           const double2 *B, long long ldb, const double2 *X, long long ldx,
                           double2 *R, long long ldr, void *ws, uint32_t *status, cudaStream_t st);
}  // namespace msts

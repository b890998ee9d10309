// msts_eig.h -- internal FP64 complex GEMM shared by the back-transformation
// and the 1-norm pseudospectra.
#pragma once
#include <cuda_runtime.h>

namespace msts {
// C = A B in FP64 (A m x m, B m x n, column-major); B upper triangular when
// triu_b (only k <= j is read).  C must not alias A or B.
cudaError_t zgemm_fp64(const double2 *A, long long lda, const double2 *B, long long ldb, double2 *C, long long ldc,
                       int m, int n, bool triu_b, cudaStream_t st);
}  // namespace msts

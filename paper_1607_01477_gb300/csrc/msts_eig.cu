// msts_eig.cu -- back-transformation of triangular eigenvectors, X = Q Z
// (Alg. 6 second half, Sec. 4: the eigenvectors of A = Q T Q^H are Q times
// those of T), with optional normalisation of every column to unit 2-norm.
//
// The product runs on the tensor cores through the digit-plane splitting of
// msts_ozaki.cu (FP64-accurate; Z upper triangular, so K' chunks past each
// column tile are skipped), or with FP64 FMAs.
#include <algorithm>

#include "../../include/msts.h"
#include "msts_check.h"
#include "msts_common.cuh"
#include "msts_ozaki.h"
#include "msts_eig.h"
#include "msts_trace.h"

namespace msts {
namespace {

constexpr int kT = 32;         // FP64 path: 32 x 32 output tile, 8 x 32 threads, 4 outputs each
constexpr int kKT = 16;        // K step staged in shared memory

// C(i, j) = sum_k A(i, k) B(k, j) in FP64, A m x m, B m x n; with TRIU, B is
// upper triangular (k <= j only: K stops at the tile's last column).
template <bool TRIU>
__global__ void __launch_bounds__(256) k_zgemm(const double2 *A, long long lda, const double2 *B,
                                               long long ldb, double2 *C, long long ldc, int m, int n) {
  __shared__ double2 sA[kKT][kT + 1];
  __shared__ double2 sB[kKT][kT + 1];
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;   // ty in [0, 8)
  const int i0 = blockIdx.y * kT, j0 = blockIdx.x * kT;
  double2 acc[4];
#pragma unroll
  for (int u = 0; u < 4; ++u) acc[u] = make_double2(0.0, 0.0);
  const int kend = TRIU ? min(m, j0 + kT) : m;   // rows of B below the tile's last column are zero
  for (int k0 = 0; k0 < kend; k0 += kKT) {
    for (int idx = threadIdx.x; idx < kKT * kT; idx += 256) {
      const int kk = idx / kT, c = idx % kT;
      const int k = k0 + kk;
      // A(i0 + c, k) and B(k, j0 + c)
      sA[kk][c] = (k < m && i0 + c < m) ? A[(i0 + c) + (long long)k * lda] : make_double2(0.0, 0.0);
      sB[kk][c] = (k < m && j0 + c < n && (!TRIU || k <= j0 + c)) ? B[k + (long long)(j0 + c) * ldb]
                                                                    : make_double2(0.0, 0.0);
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < kKT; ++kk) {
      const double2 q = sA[kk][tx];
#pragma unroll
      for (int u = 0; u < 4; ++u) acc[u] = zfma(acc[u], q, sB[kk][ty + 8 * u]);
    }
    __syncthreads();
  }
  const int i = i0 + tx;
  if (i >= m) return;
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int j = j0 + ty + 8 * u;
    if (j < n) C[i + (long long)j * ldc] = acc[u];
  }
}

// Column j of X scaled to unit 2-norm (a zero column stays zero): the largest
// exponent is taken out first so that the squares neither overflow nor
// underflow; one warp per column.
__global__ void k_normalize_cols(double2 *X, long long ldx, int m, int n) {
  const int lane = threadIdx.x & 31;
  const int j = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (j >= n) return;
  double2 *col = X + (long long)j * ldx;
  int E = -1022;
  for (int r = lane; r < m; r += 32) E = max(E, zexp(col[r]));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) E = max(E, __shfl_xor_sync(0xffffffffu, E, o));
  const double sc = pow2i(-E);
  double s2 = 0.0;
  for (int r = lane; r < m; r += 32) {
    const double a = col[r].x * sc, b = col[r].y * sc;
    s2 = fma(a, a, fma(b, b, s2));
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s2 += __shfl_xor_sync(0xffffffffu, s2, o);
  if (s2 == 0.0) return;
  const double inv = 1.0 / sqrt(s2);              // 1 / ||x 2^-E||_2
  for (int r = lane; r < m; r += 32) {
    const double2 v = col[r];
    col[r] = make_double2(v.x * sc * inv, v.y * sc * inv);
  }
}

}  // namespace

cudaError_t zgemm_fp64(const double2 *A, long long lda, const double2 *B, long long ldb, double2 *C, long long ldc,
                       int m, int n, bool triu_b, cudaStream_t st) {
  if (m == 0 || n == 0) return cudaSuccess;
  const dim3 grid((unsigned)((n + kT - 1) / kT), (unsigned)((m + kT - 1) / kT));
  // Recorded as the FP64 GEMM: 8 FLOPs per complex multiply-add.
  const double macs = triu_b ? 0.5 * (double)m * n * (double)std::min(m, n) : (double)m * m * (double)n;
  void *h = trace_on() ? trace_start(0, 8.0 * macs, 16.0 * ((double)m * m + 2.0 * (double)m * n), st) : nullptr;
  if (triu_b) k_zgemm<true><<<grid, 256, 0, st>>>(A, lda, B, ldb, C, ldc, m, n);
  else k_zgemm<false><<<grid, 256, 0, st>>>(A, lda, B, ldb, C, ldc, m, n);
  trace_stop(h, st);
  count_launches(1);
  return cudaGetLastError();
}

}  // namespace msts

extern "C" {

size_t msts_back_transform_workspace_size(int64_t m, uint32_t flags) {
  if (m < 0 || m > ((int64_t)1 << 30)) return 0;
  if (m == 0 || !(flags & MSTS_TENSOR_GEMM)) return 0;
  return msts::ozaki_workspace_bytes((int)m, (int)m);
}

int msts_back_transform(const msts_z *Q, int64_t ldq, int64_t m, const msts_z *Z, int64_t ldz, msts_z *X,
                        int64_t ldx, void *workspace, size_t workspace_bytes, uint32_t *status, uint32_t flags,
                        void *stream) {
  if (m < 0 || m > ((int64_t)1 << 30)) return -3;
  if (m > 0 && !Q) return -1;
  if (ldq < std::max<int64_t>(1, m)) return -2;
  if (m > 0 && !Z) return -4;
  if (ldz < std::max<int64_t>(1, m)) return -5;
  if (m > 0 && !X) return -6;
  if (ldx < std::max<int64_t>(1, m)) return -7;
  if (flags & ~(uint32_t)(MSTS_TENSOR_GEMM | MSTS_NORMALIZE_COLUMNS)) return -11;
  const size_t need = msts_back_transform_workspace_size(m, flags);
  if (need > 0 && (!workspace || workspace_bytes < need)) return workspace ? -9 : -8;
  if (msts::bad_alignment({Q, Z, X}, workspace)) return MSTS_ERR_ALIGN;
  if (m == 0) return 0;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const double2 *q = reinterpret_cast<const double2 *>(Q);
  const double2 *z = reinterpret_cast<const double2 *>(Z);
  double2 *x = reinterpret_cast<double2 *>(X);
  cudaError_t e;
  if (flags & MSTS_TENSOR_GEMM) {
    e = msts::ozaki_product(q, ldq, (int)m, z, ldz, (int)m, true, x, ldx, workspace, status, st);
  } else {
    e = msts::zgemm_fp64(q, ldq, z, ldz, x, ldx, (int)m, (int)m, true, st);
  }
  if (e != cudaSuccess) return MSTS_ERR_CUDA;
  if (flags & MSTS_NORMALIZE_COLUMNS) {
    msts::k_normalize_cols<<<(unsigned)((m + 7) / 8), 256, 0, st>>>(x, ldx, (int)m, (int)m);
    msts::count_launches(1);
    if (cudaGetLastError() != cudaSuccess) return MSTS_ERR_CUDA;
  }
  return 0;
}

}  // extern "C"

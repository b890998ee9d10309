// msts_mixed.cu -- mixed-precision multi-shift solve with FP64 iterative
// refinement (not in the paper; the paper is FP64 throughout).
//
//   X_0 = solve_lp(B)
//   repeat:  R = B - (U - S) X      (FP64-accurate residual)
//            eta_j = ||R_j||_inf / (||U - s_j I||_inf ||x_j||_inf + ||b_j||_inf)
//            stop when max_j eta_j <= tol (or at the iteration cap)
//            X += solve_lp(R)
//
// solve_lp is the blocked multi-shift solve whose substitution GEMM is a
// low-precision product (the diagonal blocks stay FP64): by default the
// tensor cores' 3-plane split-BF16 product with FP32 accumulation
// (k_oz_update<3>, msts_ozaki.cu), with MSTS_MIXED_FP32_GEMM an FP32 FMA
// product on the CUDA cores.  The residual is computed in FP64 DFMA
// (k_residual) or, with MSTS_RESIDUAL_OZAKI, by the FP64-accurate tensor-core
// product of msts_ozaki.cu.
#include <algorithm>
#include <vector>

#include "msts_check.h"
#include "msts_common.cuh"
#include "msts_engine.h"
#include "msts_mixed.h"
#include "msts_ozaki.h"
#include "msts_trace.h"

namespace msts {

constexpr int kRBM = 64, kRBN = 32, kRKC = 32, kRThreads = 256;

// R = B - triu(U) X + X diag(s), FP64 DFMA.  Tile 64 x 32, K in chunks of 32
// starting at the tile's first row (U is upper triangular).
__global__ void __launch_bounds__(kRThreads)
k_residual(const double2 *U, long long ldu, int m, const double2 *s, int n, const double2 *B,
           long long ldb, const double2 *X, long long ldx, double2 *R, long long ldr) {
  __shared__ double2 sA[kRKC][kRBM + 1];
  __shared__ double2 sX[kRKC][kRBN + 1];
  const int r0 = blockIdx.y * kRBM, c0 = blockIdx.x * kRBN;
  if (r0 >= m || c0 >= n) return;
  const int tid = threadIdx.x, tr = tid & 31, tc = tid >> 5;
  double2 acc[2][4];
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int c = 0; c < 4; ++c) acc[i][c] = make_double2(0.0, 0.0);
  for (int k0 = r0; k0 < m; k0 += kRKC) {
    for (int idx = tid; idx < kRKC * kRBM; idx += kRThreads) {
      const int k = idx / kRBM, r = idx - k * kRBM;
      const int gr = r0 + r, gk = k0 + k;
      sA[k][r] = (gk < m && gr < m && gr <= gk) ? U[gr + (long long)gk * ldu] : make_double2(0.0, 0.0);
    }
    for (int idx = tid; idx < kRKC * kRBN; idx += kRThreads) {
      const int c = idx / kRKC, k = idx - c * kRKC;
      const int gk = k0 + k, gc = c0 + c;
      sX[k][c] = (gk < m && gc < n) ? X[gk + (long long)gc * ldx] : make_double2(0.0, 0.0);
    }
    __syncthreads();
#pragma unroll 4
    for (int k = 0; k < kRKC; ++k) {
      const double2 a0 = sA[k][tr], a1 = sA[k][tr + 32];
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const double2 x = sX[k][tc + 8 * c];
        acc[0][c] = zfma(acc[0][c], a0, x);
        acc[1][c] = zfma(acc[1][c], a1, x);
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    const int col = c0 + tc + 8 * c;
    if (col >= n) continue;
    const double2 sj = s[col];
#pragma unroll
    for (int i = 0; i < 2; ++i) {
      const int row = r0 + tr + 32 * i;
      if (row >= m) continue;
      const double2 x = X[row + (long long)col * ldx];
      const double2 v = zsub(B[row + (long long)col * ldb], acc[i][c]);
      R[row + (long long)col * ldr] = zfma(v, sj, x);
    }
  }
}

// rs[r] = sum_{c > r} |U(r,c)| (off-diagonal row sums), one warp per row.
__global__ void k_offdiag_rowsums(const double2 *U, long long ldu, int m, double *rs) {
  const int lane = threadIdx.x & 31;
  const int r = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (r >= m) return;
  double acc = 0.0;
  for (int c = r + 1 + lane; c < m; c += 32) {
    const double2 u = U[r + (long long)c * ldu];
    acc += sqrt(fma(u.x, u.x, u.y * u.y));
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (lane == 0) rs[r] = acc;
}

// Per column j: eta_j = ||R_j|| / (||U - s_j I||_inf ||x_j|| + ||b_j||), inf-norms
// of moduli; one warp per column.  ||U - s_j I||_inf = max_r rs[r] + |U(r,r) - s_j|.
__global__ void k_eta(const double2 *U, long long ldu, int m, const double2 *s, int n,
                      const double *rs, const double2 *B, long long ldb, const double2 *X,
                      long long ldx, const double2 *R, long long ldr, double *eta) {
  const int lane = threadIdx.x & 31;
  const int j = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (j >= n) return;
  const double2 sj = s[j];
  double an = 0.0, xn = 0.0, bn = 0.0, rn = 0.0;
  for (int r = lane; r < m; r += 32) {
    const double2 d = zsub(U[r + (long long)r * ldu], sj);
    an = fmax(an, rs[r] + hypot(d.x, d.y));
    const double2 x = X[r + (long long)j * ldx], b = B[r + (long long)j * ldb],
                  rr = R[r + (long long)j * ldr];
    xn = fmax(xn, hypot(x.x, x.y));
    bn = fmax(bn, hypot(b.x, b.y));
    rn = fmax(rn, hypot(rr.x, rr.y));
  }
  an = warp_max(an); xn = warp_max(xn); bn = warp_max(bn); rn = warp_max(rn);
  if (lane == 0) {
    const double den = an * xn + bn;
    eta[j] = den > 0.0 ? rn / den : 0.0;
  }
}

// out[0] = max_j eta[j] (single CTA).
__global__ void k_max(const double *v, int n, double *out) {
  __shared__ double red[32];
  double mx = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) mx = fmax(mx, v[i]);
  mx = warp_max(mx);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
  __syncthreads();
  if (threadIdx.x < 32) {
    double w = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
    w = warp_max(w);
    if (threadIdx.x == 0) out[0] = w;
  }
}

// Y = A (copy) or Y += A, column-major m x n.
__global__ void k_copy_or_add(const double2 *A, long long lda, double2 *Y, long long ldy, int m,
                              int n, int add) {
  const long long total = (long long)m * n;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const int r = (int)(i % m), c = (int)(i / m);
    const double2 a = A[r + (long long)c * lda];
    double2 *y = Y + r + (long long)c * ldy;
    *y = add ? zadd(*y, a) : a;
  }
}

static size_t a256(size_t x) { return (x + 255) & ~size_t(255); }

size_t mixed_workspace_bytes(int m, int n, int nb, uint32_t flags) {
  size_t s = a256(sizeof(double2) * (size_t)m * n);   // R
  s += a256(sizeof(double) * (size_t)n);              // eta
  s += a256(sizeof(double) * (size_t)m);              // off-diagonal row sums
  s += a256(sizeof(double) * 2);                      // max eta
  if (flags & MSTS_RESIDUAL_OZAKI) s += ozaki_workspace_bytes(m, n);
  if (!(flags & MSTS_MIXED_FP32_GEMM)) s += a256(ozaki_plan_bytes(m, n, nb));
  return s;
}

cudaError_t residual_run(const double2 *U, long long ldu, int m, const double2 *s, int n,
                         const double2 *B, long long ldb, const double2 *X, long long ldx,
                         double2 *R, long long ldr, uint32_t flags, void *oz_ws, uint32_t *status,
                         cudaStream_t st) {
  if (flags & MSTS_RESIDUAL_OZAKI)
    return ozaki_residual(U, ldu, m, s, n, B, ldb, X, ldx, R, ldr, oz_ws, status, st);
  const double fl = 4.0 * (double)m * m * n;
  void *h = trace_on() ? trace_start(0, fl, 16.0 * ((double)m * m / 2 + 3.0 * m * n), st) : nullptr;
  k_residual<<<dim3((n + kRBN - 1) / kRBN, (m + kRBM - 1) / kRBM), kRThreads, 0, st>>>(
      U, ldu, m, s, n, B, ldb, X, ldx, R, ldr);
  trace_stop(h, st);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t mixed_run(const double2 *U, long long ldu, int m, const double2 *s, int n,
                      const double2 *B, long long ldb, double2 *X, long long ldx, double tol,
                      int max_iter, int nb, uint32_t flags, void *ws, uint32_t *status,
                      int *iters_out, double *eta_out, double *eta0_out, cudaStream_t st) {
  char *cur = static_cast<char *>(ws);
  double2 *R = reinterpret_cast<double2 *>(cur); cur += a256(sizeof(double2) * (size_t)m * n);
  double *eta = reinterpret_cast<double *>(cur); cur += a256(sizeof(double) * (size_t)n);
  double *rs = reinterpret_cast<double *>(cur); cur += a256(sizeof(double) * (size_t)m);
  double *emax = reinterpret_cast<double *>(cur); cur += a256(sizeof(double) * 2);
  void *oz_ws = cur;
  if (flags & MSTS_RESIDUAL_OZAKI) cur += ozaki_workspace_bytes(m, n);
  const bool tensor_lp = !(flags & MSTS_MIXED_FP32_GEMM);
  OzPlan plan{};
  const int cgrid = std::max(1, std::min(8192, (int)(((long long)m * n + 255) / 256)));

  EngineProblem Px{};
  Px.U = U; Px.ldu = ldu; Px.m = m; Px.shifts = s; Px.shift_stride = 1; Px.n = n;
  Px.B = X; Px.ldb = ldx;
  EngineProblem Pr = Px;
  Pr.B = R; Pr.ldb = m;

  cudaError_t e;
  if (flags & MSTS_RESIDUAL_OZAKI) {
    e = ozaki_prepare(U, ldu, m, n, oz_ws, st);
    if (e != cudaSuccess) return e;
  }
  if (tensor_lp) {     // digit planes of U's block panels, for every low-precision solve
    e = ozaki_plan_prepare(&plan, U, ldu, m, n, nb, false, cur, st);
    if (e != cudaSuccess) return e;
    Px.oz = &plan;
    Pr.oz = &plan;
  }
  k_offdiag_rowsums<<<(m + 7) / 8, 256, 0, st>>>(U, ldu, m, rs);
  k_copy_or_add<<<cgrid, 256, 0, st>>>(B, ldb, X, ldx, m, n, 0);
  count_launches(2);
  e = engine_run(&Px, 1, nb, false, false, false, nullptr, status, st, true);   // X_0
  if (e != cudaSuccess) return e;
  double eta_h = 0.0;
  int it = 0;
  for (;; ++it) {
    e = residual_run(U, ldu, m, s, n, B, ldb, X, ldx, R, m, flags, oz_ws, status, st);
    if (e != cudaSuccess) return e;
    k_eta<<<(n + 7) / 8, 256, 0, st>>>(U, ldu, m, s, n, rs, B, ldb, X, ldx, R, m, eta);
    k_max<<<1, 256, 0, st>>>(eta, n, emax);
    count_launches(2);
    e = cudaMemcpyAsync(&eta_h, emax, sizeof(double), cudaMemcpyDeviceToHost, st);
    if (e != cudaSuccess) return e;
    e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return e;
    if (it == 0 && eta0_out) *eta0_out = eta_h;
    if (eta_h <= tol || it >= max_iter) break;
    e = engine_run(&Pr, 1, nb, false, false, false, nullptr, status, st, true);   // D = solve_lp(R)
    if (e != cudaSuccess) return e;
    k_copy_or_add<<<cgrid, 256, 0, st>>>(R, m, X, ldx, m, n, 1);                // X += D
    count_launches(1);
  }
  if (iters_out) *iters_out = it;
  if (eta_out) *eta_out = eta_h;
  if (!(eta_h <= tol) && status) {
    const uint32_t bit = MSTS_STATUS_NOT_CONVERGED;
    uint32_t cur_status = 0;
    e = cudaMemcpyAsync(&cur_status, status, sizeof(uint32_t), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cur_status |= bit;
    if (e == cudaSuccess) e = cudaMemcpyAsync(status, &cur_status, sizeof(uint32_t), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return e;
  }
  return cudaGetLastError();
}

}  // namespace msts

extern "C" {

size_t msts_solve_mixed_workspace_size(int64_t m, int64_t n, int32_t nb, uint32_t flags) {
  if (m < 0 || n < 0 || (nb != 16 && nb != 32 && nb != 64)) return 0;
  return msts::mixed_workspace_bytes((int)m, (int)n, nb, flags);
}

int msts_solve_mixed(const msts_z *U, int64_t ldu, int64_t m, const msts_z *shifts, int64_t n,
                     const msts_z *B, int64_t ldb, msts_z *X, int64_t ldx, double tol,
                     int32_t max_iter, int32_t nb, void *workspace, size_t workspace_bytes,
                     uint32_t *status, uint32_t flags, int32_t *iters, double *eta,
                     double *eta_before, void *stream) {
  const int64_t kMax = (int64_t)1 << 30;
  if (m < 0 || m > kMax) return -3;
  if (m > 0 && !U) return -1;
  if (ldu < (m > 1 ? m : 1)) return -2;
  if (n < 0 || n > kMax) return -5;
  if (n > 0 && !shifts) return -4;
  if (m > 0 && n > 0 && (!B || !X)) return !B ? -6 : -8;
  if (ldb < (m > 1 ? m : 1)) return -7;
  if (ldx < (m > 1 ? m : 1)) return -9;
  if (!(tol >= 0.0)) return -10;
  if (max_iter < 0) return -11;
  if (nb != 16 && nb != 32 && nb != 64) return -12;
  if ((flags & ~(uint32_t)(MSTS_RESIDUAL_OZAKI | MSTS_MIXED_FP32_GEMM)) != 0) return -16;
  if (msts::bad_alignment({U, shifts, B, X}, workspace)) return MSTS_ERR_ALIGN;
  if (m == 0 || n == 0) {
    if (iters) *iters = 0;
    if (eta) *eta = 0.0;
    if (eta_before) *eta_before = 0.0;
    return 0;
  }
  const size_t need = msts_solve_mixed_workspace_size(m, n, nb, flags);
  if (!workspace || workspace_bytes < need) return workspace ? -14 : -13;
  int it = 0;
  double e_final = 0.0, e0 = 0.0;
  const cudaError_t e = msts::mixed_run(
      reinterpret_cast<const double2 *>(U), ldu, (int)m, reinterpret_cast<const double2 *>(shifts),
      (int)n, reinterpret_cast<const double2 *>(B), ldb, reinterpret_cast<double2 *>(X), ldx, tol,
      max_iter, nb, flags, workspace, status, &it, &e_final, &e0, static_cast<cudaStream_t>(stream));
  if (iters) *iters = it;
  if (eta) *eta = e_final;
  if (eta_before) *eta_before = e0;
  return e == cudaSuccess ? 0 : MSTS_ERR_CUDA;
}

size_t msts_residual_workspace_size(int64_t m, int64_t n, uint32_t flags) {
  if (m < 0 || n < 0) return 0;
  return (flags & MSTS_RESIDUAL_OZAKI) ? msts::ozaki_workspace_bytes((int)m, (int)n) : 0;
}

int msts_residual(const msts_z *U, int64_t ldu, int64_t m, const msts_z *shifts, int64_t n,
                  const msts_z *B, int64_t ldb, const msts_z *X, int64_t ldx, msts_z *R, int64_t ldr,
                  void *workspace, size_t workspace_bytes, uint32_t *status, uint32_t flags,
                  void *stream) {
  const int64_t kMax = (int64_t)1 << 30;
  if (m < 0 || m > kMax) return -3;
  if (m > 0 && !U) return -1;
  if (ldu < (m > 1 ? m : 1)) return -2;
  if (n < 0 || n > kMax) return -5;
  if (n > 0 && !shifts) return -4;
  if (m > 0 && n > 0 && (!B || !X || !R)) return !B ? -6 : (!X ? -8 : -10);
  if (ldb < (m > 1 ? m : 1)) return -7;
  if (ldx < (m > 1 ? m : 1)) return -9;
  if (ldr < (m > 1 ? m : 1)) return -11;
  if ((flags & ~(uint32_t)MSTS_RESIDUAL_OZAKI) != 0) return -15;
  if (msts::bad_alignment({U, shifts, B, X, R}, workspace)) return MSTS_ERR_ALIGN;
  if (m == 0 || n == 0) return 0;
  const size_t need = msts_residual_workspace_size(m, n, flags);
  if (need > 0 && (!workspace || workspace_bytes < need)) return workspace ? -13 : -12;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const double2 *Ud = reinterpret_cast<const double2 *>(U);
  if (flags & MSTS_RESIDUAL_OZAKI) {
    if (msts::ozaki_prepare(Ud, ldu, (int)m, (int)n, workspace, st) != cudaSuccess) return MSTS_ERR_CUDA;
  }
  const cudaError_t e = msts::residual_run(
      Ud, ldu, (int)m, reinterpret_cast<const double2 *>(shifts), (int)n,
      reinterpret_cast<const double2 *>(B), ldb, reinterpret_cast<const double2 *>(X), ldx,
      reinterpret_cast<double2 *>(R), ldr, flags, workspace, status, st);
  return e == cudaSuccess ? 0 : MSTS_ERR_CUDA;
}

}  // extern "C"

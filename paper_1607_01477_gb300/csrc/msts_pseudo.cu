// msts_pseudo.cu -- pseudospectra by the Van Loan / Lui method (Sec. 5,
// Alg. 7): sigma_min(T - z I) for every grid point z from the largest
// eigenvalue of (T - zI)^{-H} (T - zI)^{-1}, estimated by Lanczos.
//
// The grid points are the shifts of one multi-shift solve (Sec. 5, last
// paragraph): every Lanczos step applies the operator to all N points with
// two engine solves (upper T - zI, then the conjugate-transposed lower solve),
// followed by one fused per-point kernel for the Lanczos recurrence (alpha,
// the three-term update, full reorthogonalisation by classical Gram-Schmidt
// with a second pass when the first removed more than half of ||w||^2, beta and
// the next Lanczos vector).  The tridiagonal's largest
// eigenvalue is then found per point by Sturm-count bisection.
#include <math_constants.h>

#include <algorithm>

#include "msts_check.h"
#include "msts_common.cuh"
#include "msts_engine.h"
#include "msts_ozaki.h"
#include "msts_trace.h"

namespace msts {

constexpr int kLzThreads = 256;
constexpr int kLzWarps = kLzThreads / 32;
constexpr int kMaxIters = 64;
constexpr int kLzGroup = 2;              // Lanczos vectors per warp reduction (a power of two <= 16)

struct LanczosState {
  double2 *V;        // (K+1) Lanczos vectors, vector k of point p at V + k*vstride + p*m
  long long vstride; // m * N
  double2 *W;        // m x N work block (leading dimension m)
  double *alpha;     // N x iters
  double *beta;      // N x iters
  int *steps;        // N
  double *amax;      // N: max |alpha_i| so far
  int *active;       // N
  int m, N, iters, K;
};

__device__ __forceinline__ double block_sum(double v, double *red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double s = 0.0;
#pragma unroll
  for (int w = 0; w < kLzWarps; ++w) s += red[w];
  return s;
}

// v_0 = V0(:,p) / ||V0(:,p)||_2; clears the per-point state.
__global__ void __launch_bounds__(kLzThreads)
k_lanczos_init(LanczosState S, const double2 *V0, long long ldv) {
  __shared__ double red[kLzWarps];
  const int p = blockIdx.x;
  const double2 *src = V0 + (long long)p * ldv;
  double ss = 0.0;
  for (int r = threadIdx.x; r < S.m; r += kLzThreads) ss += src[r].x * src[r].x + src[r].y * src[r].y;
  const double inv = 1.0 / sqrt(block_sum(ss, red));
  double2 *v0 = S.V + (long long)p * S.m;
  for (int r = threadIdx.x; r < S.m; r += kLzThreads) v0[r] = zscale(src[r], inv);
  for (int k = threadIdx.x; k < S.iters; k += kLzThreads) {
    S.alpha[(long long)p * S.iters + k] = 0.0;
    S.beta[(long long)p * S.iters + k] = 0.0;
  }
  if (threadIdx.x == 0) { S.steps[p] = 0; S.amax[p] = 0.0; S.active[p] = 1; }
}

// W(:,p) = v_k(:,p) (the right-hand side of this step's two solves).
__global__ void k_lanczos_load(LanczosState S, int k) {
  const long long total = (long long)S.m * S.N;
  const double2 *vk = S.V + (long long)k * S.vstride;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x)
    S.W[i] = vk[i];
}

// One CTA per grid point: the Lanczos recurrence after w = A v_k.
__global__ void __launch_bounds__(kLzThreads) k_lanczos_step(LanczosState S, int k) {
  __shared__ double red[kLzWarps];
  __shared__ double2 part[kMaxIters + 1][kLzWarps];
  __shared__ double2 h[kMaxIters + 1];
  const int p = blockIdx.x;
  if (!S.active[p]) return;
  const int m = S.m;
  double2 *w = S.W + (long long)p * m;
  const double2 *vk = S.V + (long long)k * S.vstride + (long long)p * m;

  // alpha_k = Re(v_k^H w)
  double a = 0.0;
  for (int r = threadIdx.x; r < m; r += kLzThreads) a += vk[r].x * w[r].x + vk[r].y * w[r].y;
  a = block_sum(a, red);
  const double bprev = k > 0 ? S.beta[(long long)p * S.iters + k - 1] : 0.0;
  const double2 *vp = k > 0 ? S.V + (long long)(k - 1) * S.vstride + (long long)p * m : nullptr;
  for (int r = threadIdx.x; r < m; r += kLzThreads) {
    double2 x = zsub(w[r], zscale(vk[r], a));
    if (k > 0) x = zsub(x, zscale(vp[r], bprev));
    w[r] = x;
  }
  __syncthreads();
  // Full reorthogonalisation against v_0..v_k by classical Gram-Schmidt, run
  // a second time only when the first pass removed more than half of ||w||^2.
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  double n0 = 0.0;
  for (int r = threadIdx.x; r < m; r += kLzThreads) n0 += w[r].x * w[r].x + w[r].y * w[r].y;
  n0 = block_sum(n0, red);
  for (int pass = 0; pass < 2; ++pass) {
    for (int i = 0; i <= k; ++i) {
      const double2 *vi = S.V + (long long)i * S.vstride + (long long)p * m;
      double2 s = make_double2(0.0, 0.0);
      for (int r = threadIdx.x; r < m; r += kLzThreads) s = zfma_cj(s, vi[r], w[r]);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        s.x += __shfl_xor_sync(0xffffffffu, s.x, o);
        s.y += __shfl_xor_sync(0xffffffffu, s.y, o);
      }
      if (lane == 0) part[i][warp] = s;
    }
    __syncthreads();
    for (int i = threadIdx.x; i <= k; i += kLzThreads) {
      double2 s = make_double2(0.0, 0.0);
#pragma unroll
      for (int ww = 0; ww < kLzWarps; ++ww) s = zadd(s, part[i][ww]);
      h[i] = s;
    }
    __syncthreads();
    double n1 = 0.0;
    for (int r = threadIdx.x; r < m; r += kLzThreads) {
      double2 x = w[r];
      for (int i = 0; i <= k; ++i)
        x = zfms(x, S.V[(long long)i * S.vstride + (long long)p * m + r], h[i]);
      w[r] = x;
      n1 += x.x * x.x + x.y * x.y;
    }
    __syncthreads();
    if (pass == 0 && !(block_sum(n1, red) < 0.5 * n0)) break;   // CTA-uniform
  }
  double bb = 0.0;
  for (int r = threadIdx.x; r < m; r += kLzThreads) bb += w[r].x * w[r].x + w[r].y * w[r].y;
  const double beta = sqrt(block_sum(bb, red));
  const double amax = fmax(S.amax[p], fabs(a));
  const bool stop = (k == S.K - 1) || (beta <= 1e-14 * amax);
  {  // v_{k+1} = w / beta_k (zero once the recurrence has stopped)
    double2 *vn = S.V + (long long)(k + 1) * S.vstride + (long long)p * m;
    const double inv = stop ? 0.0 : 1.0 / beta;
    for (int r = threadIdx.x; r < m; r += kLzThreads)
      vn[r] = stop ? make_double2(0.0, 0.0) : zscale(w[r], inv);
  }
  if (threadIdx.x == 0) {
    S.alpha[(long long)p * S.iters + k] = a;
    S.beta[(long long)p * S.iters + k] = beta;
    S.amax[p] = amax;
    S.steps[p] = k + 1;
    if (stop) S.active[p] = 0;
  }
}

// The same step with w held in registers (element r = threadIdx.x + 256 q of
// this point, q < RW): the reorthogonalisation then reads only the Lanczos
// vectors from memory, not w again for every dot product and update.  The
// sums run over the same elements in the same order as k_lanczos_step.
template <int RW>
__global__ void __launch_bounds__(kLzThreads) k_lanczos_step_r(LanczosState S, int k) {
  __shared__ double red[kLzWarps];
  __shared__ double2 part[kMaxIters + 1][kLzWarps];
  __shared__ double2 h[kMaxIters + 1];
  const int p = blockIdx.x;
  if (!S.active[p]) return;
  const int m = S.m;
  const double2 *wsrc = S.W + (long long)p * m;
  const double2 *vk = S.V + (long long)k * S.vstride + (long long)p * m;
  double2 w[RW];
#pragma unroll
  for (int q = 0; q < RW; ++q) {
    const int r = threadIdx.x + kLzThreads * q;
    w[q] = r < m ? wsrc[r] : make_double2(0.0, 0.0);
  }
  // alpha_k = Re(v_k^H w)
  double a = 0.0;
#pragma unroll
  for (int q = 0; q < RW; ++q) {
    const int r = threadIdx.x + kLzThreads * q;
    if (r < m) a += vk[r].x * w[q].x + vk[r].y * w[q].y;
  }
  a = block_sum(a, red);
  const double bprev = k > 0 ? S.beta[(long long)p * S.iters + k - 1] : 0.0;
  const double2 *vp = k > 0 ? S.V + (long long)(k - 1) * S.vstride + (long long)p * m : nullptr;
#pragma unroll
  for (int q = 0; q < RW; ++q) {
    const int r = threadIdx.x + kLzThreads * q;
    if (r < m) {
      double2 x = zsub(w[q], zscale(vk[r], a));
      if (k > 0) x = zsub(x, zscale(vp[r], bprev));
      w[q] = x;
    }
  }
  // Full reorthogonalisation against v_0..v_k by classical Gram-Schmidt, run
  // a second time only when the first pass removed more than half of ||w||^2.
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  double n0 = 0.0;
#pragma unroll
  for (int q = 0; q < RW; ++q) n0 += w[q].x * w[q].x + w[q].y * w[q].y;
  n0 = block_sum(n0, red);
  for (int pass = 0; pass < 2; ++pass) {
    // v_i^H w for kLzGroup vectors at a time: each thread's partial sums (over
    // its elements in increasing order), then one reduce-scatter butterfly
    // over the warp for all of them (lanes l and l ^ o add at offsets 16, 8,
    // 4, 2, 1 as in a per-value tree, so every sum is the same; with two
    // vectors per group, 3 FP64 additions per vector instead of 10).
    for (int i0 = 0; i0 <= k; i0 += kLzGroup) {
      double v[2 * kLzGroup];            // Re, Im of the group's partial sums
#pragma unroll
      for (int g = 0; g < 2 * kLzGroup; ++g) v[g] = 0.0;
#pragma unroll
      for (int q = 0; q < RW; ++q) {
        const int r = threadIdx.x + kLzThreads * q;
#pragma unroll
        for (int g = 0; g < kLzGroup; ++g)
          if (r < m && i0 + g <= k) {
            const double2 t = zfma_cj(make_double2(v[2 * g], v[2 * g + 1]),
                                      S.V[(long long)(i0 + g) * S.vstride + (long long)p * m + r], w[q]);
            v[2 * g] = t.x;
            v[2 * g + 1] = t.y;
          }
      }
#pragma unroll
      for (int o = 16, n = 2 * kLzGroup; o > 0; o >>= 1) {
        if (n > 1) {                     // keep the half named by this lane's bit o, add the partner's
          const bool up = (lane & o) != 0;
          n >>= 1;
#pragma unroll
          for (int g = 0; g < n; ++g) {
            const double send = up ? v[g] : v[g + n], keep = up ? v[g + n] : v[g];
            v[g] = keep + __shfl_xor_sync(0xffffffffu, send, o);
          }
        } else {
          v[0] += __shfl_xor_sync(0xffffffffu, v[0], o);
        }
      }
      // lane l now holds value (l / (32 / (2 kLzGroup))) of the group
      constexpr int kSpan = 32 / (2 * kLzGroup);
      const int vi = lane / kSpan;
      if (lane % kSpan == 0 && i0 + (vi >> 1) <= k)
        reinterpret_cast<double *>(&part[i0 + (vi >> 1)][warp])[vi & 1] = v[0];
    }
    __syncthreads();
    for (int i = threadIdx.x; i <= k; i += kLzThreads) {
      double2 t = make_double2(0.0, 0.0);
#pragma unroll
      for (int ww = 0; ww < kLzWarps; ++ww) t = zadd(t, part[i][ww]);
      h[i] = t;
    }
    __syncthreads();
    // w -= V h, vector by vector (every element still takes v_0 .. v_k in
    // order; the loads of one vector are independent of each other)
    for (int i = 0; i <= k; ++i) {
      const double2 hi = h[i];
      const double2 *vi = S.V + (long long)i * S.vstride + (long long)p * m;
#pragma unroll
      for (int q = 0; q < RW; ++q) {
        const int r = threadIdx.x + kLzThreads * q;
        if (r < m) w[q] = zfms(w[q], vi[r], hi);
      }
    }
    double n1 = 0.0;
#pragma unroll
    for (int q = 0; q < RW; ++q) {
      const int r = threadIdx.x + kLzThreads * q;
      if (r < m) n1 += w[q].x * w[q].x + w[q].y * w[q].y;
    }
    __syncthreads();
    if (pass == 0 && !(block_sum(n1, red) < 0.5 * n0)) break;   // CTA-uniform
  }
  double bb = 0.0;
#pragma unroll
  for (int q = 0; q < RW; ++q) bb += w[q].x * w[q].x + w[q].y * w[q].y;
  const double beta = sqrt(block_sum(bb, red));
  const double amax = fmax(S.amax[p], fabs(a));
  const bool stop = (k == S.K - 1) || (beta <= 1e-14 * amax);
  {  // v_{k+1} = w / beta_k (zero once the recurrence has stopped)
    double2 *vn = S.V + (long long)(k + 1) * S.vstride + (long long)p * m;
    const double inv = stop ? 0.0 : 1.0 / beta;
#pragma unroll
    for (int q = 0; q < RW; ++q) {
      const int r = threadIdx.x + kLzThreads * q;
      if (r < m) vn[r] = stop ? make_double2(0.0, 0.0) : zscale(w[q], inv);
    }
  }
  if (threadIdx.x == 0) {
    S.alpha[(long long)p * S.iters + k] = a;
    S.beta[(long long)p * S.iters + k] = beta;
    S.amax[p] = amax;
    S.steps[p] = k + 1;
    if (stop) S.active[p] = 0;
  }
}

static void launch_lanczos_step(const LanczosState &S, int k, cudaStream_t st) {
  const int m = S.m;
  if (m <= kLzThreads) k_lanczos_step_r<1><<<S.N, kLzThreads, 0, st>>>(S, k);
  else if (m <= 2 * kLzThreads) k_lanczos_step_r<2><<<S.N, kLzThreads, 0, st>>>(S, k);
  else if (m <= 4 * kLzThreads) k_lanczos_step_r<4><<<S.N, kLzThreads, 0, st>>>(S, k);
  else if (m <= 8 * kLzThreads) k_lanczos_step_r<8><<<S.N, kLzThreads, 0, st>>>(S, k);
  else if (m <= 16 * kLzThreads) k_lanczos_step_r<16><<<S.N, kLzThreads, 0, st>>>(S, k);
  else k_lanczos_step<<<S.N, kLzThreads, 0, st>>>(S, k);
}

// Number of eigenvalues of tridiag(b, a, b) below x (negative LDL^T pivots).
__device__ int sturm_below(const double *a, const double *b, int k, double x, double pivmin) {
  int c = 0;
  double d = a[0] - x;
  if (d < 0.0) ++c;
  for (int i = 1; i < k; ++i) {
    if (fabs(d) < pivmin) d = -pivmin;
    d = (a[i] - x) - b[i - 1] * b[i - 1] / d;
    if (d < 0.0) ++c;
  }
  return c;
}

// One thread per point: theta_max of the Lanczos tridiagonal by bisection on
// the Gershgorin interval, sigma_min = 1 / sqrt(theta_max).
__global__ void k_ritz(LanczosState S, double *sigma_min) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= S.N) return;
  const double *a = S.alpha + (long long)p * S.iters;
  const double *b = S.beta + (long long)p * S.iters;
  const int k = S.steps[p];
  if (k <= 0) { sigma_min[p] = CUDART_INF; return; }
  double lo = a[0], hi = a[0], b2 = 0.0;
  for (int i = 0; i < k; ++i) {
    const double rad = (i > 0 ? fabs(b[i - 1]) : 0.0) + (i + 1 < k ? fabs(b[i]) : 0.0);
    lo = fmin(lo, a[i] - rad);
    hi = fmax(hi, a[i] + rad);
    if (i + 1 < k) b2 = fmax(b2, b[i] * b[i]);
  }
  const double pivmin = kDblMin * fmax(b2, 1.0);
  const double wdt = fmax(fabs(lo), fabs(hi));
  lo -= 4.0 * kEps * wdt + pivmin;
  hi += 4.0 * kEps * wdt + pivmin;
  for (int it = 0; it < 4096; ++it) {
    const double mid = 0.5 * (lo + hi);
    if (mid <= lo || mid >= hi) break;
    if (sturm_below(a, b, k, mid, pivmin) >= k) hi = mid; else lo = mid;
  }
  sigma_min[p] = 1.0 / sqrt(0.5 * (lo + hi));
}

static size_t a256(size_t x) { return (x + 255) & ~size_t(255); }

size_t pseudo_workspace_bytes(int m, int N, int iters, int nb, uint32_t flags) {
  const int K = std::min(iters, m);
  size_t s = 0;
  s += a256(sizeof(double2) * (size_t)(K + 1) * m * N);  // V
  s += a256(sizeof(double2) * (size_t)m * N);            // W
  s += a256(sizeof(double) * (size_t)N * iters) * 2;     // alpha, beta
  s += a256(sizeof(int) * (size_t)N) * 2;                 // steps, active
  s += a256(sizeof(double) * (size_t)N);                 // amax
  EngineProblem p{};
  p.m = m; p.n = N;
  s += a256(engine_workspace_bytes(&p, 1, nb, false));
  if (flags & MSTS_TENSOR_GEMM) s += 2 * a256(ozaki_plan_bytes(m, N, nb));   // upper and conj plans
  return s;
}

cudaError_t pseudo_run(const double2 *T, long long ldt, int m, const double2 *z, int N,
                       const double2 *V0, long long ldv, int iters, double *sigma_min,
                       double *alpha, double *beta, int *steps, int nb, uint32_t flags, void *ws,
                       uint32_t *status, cudaStream_t st) {
  const int K = std::min(iters, m);
  char *cur = static_cast<char *>(ws);
  LanczosState S;
  S.m = m; S.N = N; S.iters = iters; S.K = K;
  S.vstride = (long long)m * N;
  S.V = reinterpret_cast<double2 *>(cur); cur += a256(sizeof(double2) * (size_t)(K + 1) * m * N);
  S.W = reinterpret_cast<double2 *>(cur); cur += a256(sizeof(double2) * (size_t)m * N);
  double *al = reinterpret_cast<double *>(cur); cur += a256(sizeof(double) * (size_t)N * iters);
  double *be = reinterpret_cast<double *>(cur); cur += a256(sizeof(double) * (size_t)N * iters);
  int *stp = reinterpret_cast<int *>(cur); cur += a256(sizeof(int) * (size_t)N);
  S.active = reinterpret_cast<int *>(cur); cur += a256(sizeof(int) * (size_t)N);
  S.amax = reinterpret_cast<double *>(cur); cur += a256(sizeof(double) * (size_t)N);
  S.alpha = alpha ? alpha : al;
  S.beta = beta ? beta : be;
  S.steps = steps ? steps : stp;
  void *engine_ws = cur;

  EngineProblem P{};
  P.U = T; P.ldu = ldt; P.m = m; P.shifts = z; P.shift_stride = 1; P.n = N;
  P.B = S.W; P.ldb = m;
  EngineProblem Pc = P;
  OzPlan up, lo;
  if (flags & MSTS_TENSOR_GEMM) {
    // Digit planes of T for both solves, made once for all Lanczos steps.
    cur += a256(engine_workspace_bytes(&P, 1, nb, false));
    cudaError_t e = ozaki_plan_prepare(&up, T, ldt, m, N, nb, false, cur, st);
    if (e != cudaSuccess) return e;
    cur += a256(ozaki_plan_bytes(m, N, nb));
    e = ozaki_plan_prepare(&lo, T, ldt, m, N, nb, true, cur, st);
    if (e != cudaSuccess) return e;
    P.oz = &up;
    Pc.oz = &lo;
  }

  k_lanczos_init<<<N, kLzThreads, 0, st>>>(S, V0, ldv);
  count_launches(1);
  for (int k = 0; k < K; ++k) {
    k_lanczos_load<<<std::max(1, std::min(4096, (int)(((long long)m * N + 255) / 256))), 256, 0, st>>>(S, k);
    cudaError_t e = engine_run(&P, 1, nb, false, false, false, engine_ws, status, st);  // (T - zI)^{-1}
    if (e != cudaSuccess) return e;
    e = engine_run(&Pc, 1, nb, false, true, false, engine_ws, status, st);              // (T - zI)^{-H}
    if (e != cudaSuccess) return e;
    // algorithmic bytes of the step: w read and written, v_0..v_k read twice
    // (projections and their removal), v_{k+1} written; FLOPs of the same passes
    void *h = trace_on() ? trace_start(4, 8.0 * (2.0 * (k + 1) + 2.0) * m * (double)N,
                                       16.0 * (2.0 * (k + 1) + 3.0) * m * (double)N, st)
                         : nullptr;
    launch_lanczos_step(S, k, st);
    trace_stop(h, st);
    count_launches(2);
  }
  k_ritz<<<(N + 127) / 128, 128, 0, st>>>(S, sigma_min);
  count_launches(1);
  return cudaGetLastError();
}

}  // namespace msts

extern "C" {

size_t msts_pseudospectra_workspace_size(int64_t m, int64_t N, int32_t iters, int32_t nb,
                                         uint32_t flags) {
  if (m < 0 || N < 0 || iters < 1 || iters > msts::kMaxIters) return 0;
  if (nb != 16 && nb != 32 && nb != 64) return 0;
  return msts::pseudo_workspace_bytes((int)m, (int)N, iters, nb, flags);
}

int msts_pseudospectra(const msts_z *T, int64_t ldt, int64_t m, const msts_z *z, int64_t N,
                       const msts_z *V0, int64_t ldv, int32_t iters, double *sigma_min,
                       double *alpha, double *beta, int32_t *steps, int32_t nb, void *workspace,
                       size_t workspace_bytes, uint32_t *status, uint32_t flags, void *stream) {
  const int64_t kMax = (int64_t)1 << 30;
  if (m < 0 || m > kMax) return -3;
  if (m > 0 && !T) return -1;
  if (ldt < (m > 1 ? m : 1)) return -2;
  if (N < 0 || N > kMax) return -5;
  if (N > 0 && !z) return -4;
  if (N > 0 && m > 0 && !V0) return -6;
  if (ldv < (m > 1 ? m : 1)) return -7;
  if (iters < 1 || iters > msts::kMaxIters) return -8;
  if (N > 0 && !sigma_min) return -9;
  if (nb != 16 && nb != 32 && nb != 64) return -13;
  if ((flags & ~(uint32_t)MSTS_TENSOR_GEMM) != 0) return -17;
  if (msts::bad_alignment({T, z, V0}, workspace)) return MSTS_ERR_ALIGN;
  if (m == 0 || N == 0) return 0;
  const size_t need = msts_pseudospectra_workspace_size(m, N, iters, nb, flags);
  if (!workspace || workspace_bytes < need) return workspace ? -15 : -14;
  const cudaError_t e = msts::pseudo_run(
      reinterpret_cast<const double2 *>(T), ldt, (int)m, reinterpret_cast<const double2 *>(z),
      (int)N, reinterpret_cast<const double2 *>(V0), ldv, iters, sigma_min, alpha, beta, steps,
      nb, flags, workspace, status, static_cast<cudaStream_t>(stream));
  return e == cudaSuccess ? 0 : MSTS_ERR_CUDA;
}

}  // extern "C"

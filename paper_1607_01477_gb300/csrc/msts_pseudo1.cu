// msts_pseudo1.cu -- 1-norm pseudospectra and the automatic portrait grid.
//
// 1-norm pseudospectra (footnote to Sec. 5): for every grid point z_p an
// estimate of ||R_p||_1, R_p = Q (T - z_p I)^{-1} Q^H (the resolvent of
// A = Q T Q^H up to sign; Q = I when absent), by Hager's estimator with
// Higham's refinements (one column, at most five gradient steps, the
// alternative vector at the end).  Every application of R_p or R_p^H to the
// current vectors of all live grid points is ONE multi-shift solve with the
// grid points as shifts (plain, or conjugate-transposed for R^H), between two
// products with Q^H and Q when Q is given.  Points whose estimate has
// converged drop out: the live columns are compacted after every step, so a
// step costs in proportion to the points still iterating.
//
// Per step, on column c of the compacted block (grid point p = map[c]):
//   after R   (y = R x):    s = ||y||_1; start: est = g = s, kind = -1;
//                           later: stop if s <= est, else est = g = s,
//                           kind = the column index that produced x;
//                           survivors continue with sign(y) = y/|y| (1 at 0);
//   after R^H (w = R^H sign y): steps += 1; j = first argmax |w_i|;
//                           stop if |w_j| <= g, else continue with x = e_j;
//   alternative: s = ||R x_alt||_1, x_alt(i) = (-1)^i (1 + i/(m-1));
//                           est = max(est, 2 s / (3m)) (kind = -2 if it wins).
//
// Portrait grid (the SpectralPortrait driver listed in Sec. 6; the paper leaves the
// grid to the software): the bounding box of diag(T) widened on every side by
// h = max(box side / 4, 2^-20 max(1, max |Re|, |Im| of the diagonal)), nx x ny
// equispaced points, every value a fixed sequence of single roundings.
#include <algorithm>

#include "../../include/msts.h"
#include "msts_check.h"
#include "msts_eig.h"
#include "msts_ozaki.h"
#include "msts_remap.h"
#include "msts_trace.h"

namespace msts {
namespace {

constexpr int kP1Threads = 256;
constexpr int kScanThreads = 1024;
constexpr int kMaxSteps = 5;

enum P1Mode { kStart = 0, kAfterRH = 1, kAfterR = 2, kAlt = 3 };

__device__ __forceinline__ double zmod(double2 v) { return hypot(v.x, v.y); }

// Column fill (one CTA per column): 1/m everywhere, or the alternative vector.
__global__ void k_p1_fill(double2 *X, long long ldx, int m, int ncols, int alt) {
  const int c = blockIdx.x;
  if (c >= ncols) return;
  for (int i = threadIdx.x; i < m; i += blockDim.x) {
    double v;
    if (alt) {
      v = 1.0 + (double)i / (double)(m - 1);
      if (i & 1) v = -v;
    } else {
      v = 1.0 / (double)m;
    }
    X[i + (long long)c * ldx] = make_double2(v, 0.0);
  }
}

__global__ void k_iota(int *map, const double2 *z, double2 *zc, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) {
    map[i] = i;
    zc[i] = z[i];
  }
}

// One CTA per compacted column: ||x||_1 and the first argmax of |x_i|, then
// the estimator's decision for that grid point (see the file comment).
__global__ void __launch_bounds__(kP1Threads) k_p1_decide(const double2 *X, long long ldx, int m, int nc,
                                                         const int *map, int mode, double *g, double *est,
                                                         int *kind, int *jcand, int *steps, int *keep) {
  __shared__ double s_sum[kP1Threads / 32];
  __shared__ double s_vmax[kP1Threads / 32];
  __shared__ int s_jmax[kP1Threads / 32];
  const int c = blockIdx.x;
  if (c >= nc) return;
  const double2 *col = X + (long long)c * ldx;
  double sum = 0.0, vmax = -1.0;
  int jmax = 0;
  for (int i = threadIdx.x; i < m; i += kP1Threads) {
    const double a = zmod(col[i]);
    sum += a;
    if (a > vmax) { vmax = a; jmax = i; }          // increasing i within a thread: the first maximum
  }
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    sum += __shfl_xor_sync(0xffffffffu, sum, o);
    const double v2 = __shfl_xor_sync(0xffffffffu, vmax, o);
    const int j2 = __shfl_xor_sync(0xffffffffu, jmax, o);
    if (v2 > vmax || (v2 == vmax && j2 < jmax)) { vmax = v2; jmax = j2; }
  }
  if (lane == 0) { s_sum[w] = sum; s_vmax[w] = vmax; s_jmax[w] = jmax; }
  __syncthreads();
  if (threadIdx.x != 0) return;
  sum = s_sum[0]; vmax = s_vmax[0]; jmax = s_jmax[0];
  for (int k = 1; k < kP1Threads / 32; ++k) {
    sum += s_sum[k];
    if (s_vmax[k] > vmax || (s_vmax[k] == vmax && s_jmax[k] < jmax)) { vmax = s_vmax[k]; jmax = s_jmax[k]; }
  }
  const int p = map ? map[c] : c;
  switch (mode) {
    case kStart:
      g[p] = sum; est[p] = sum; kind[p] = -1; steps[p] = 0;
      keep[c] = m > 1;
      break;
    case kAfterRH:
      steps[p] += 1;
      if (vmax <= g[p]) keep[c] = 0;
      else { keep[c] = 1; jcand[p] = jmax; }
      break;
    case kAfterR:
      if (sum <= est[p]) keep[c] = 0;
      else { keep[c] = 1; est[p] = sum; g[p] = sum; kind[p] = jcand[p]; }
      break;
    default: {   // kAlt
      const double alt = 2.0 * sum / (3.0 * (double)m);
      if (alt > est[p]) { est[p] = alt; kind[p] = -2; }
    }
  }
}

// Order-preserving compaction of the kept columns (one CTA): newpos[c], the
// new map and shifts, and the new count.
__global__ void __launch_bounds__(kScanThreads) k_p1_scan(const int *keep, int nc, const int *map_in,
                                                         const double2 *z_in, int *map_out, double2 *z_out,
                                                         int *newpos, int *n_out) {
  __shared__ int s_warp[kScanThreads / 32];
  __shared__ int s_base;
  if (threadIdx.x == 0) s_base = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int c0 = 0; c0 < nc; c0 += kScanThreads) {
    const int c = c0 + threadIdx.x;
    const int k = c < nc ? keep[c] : 0;
    int incl = k;                                  // inclusive scan within the warp
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int t = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += t;
    }
    if (lane == 31) s_warp[w] = incl;
    __syncthreads();
    if (w == 0) {
      int v = s_warp[lane];
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += t;
      }
      s_warp[lane] = v;                            // inclusive prefix of the warp totals
    }
    __syncthreads();
    const int pos = s_base + (w > 0 ? s_warp[w - 1] : 0) + incl - k;
    if (c < nc) {
      newpos[c] = k ? pos : -1;
      if (k) {
        map_out[pos] = map_in[c];
        z_out[pos] = z_in[c];
      }
    }
    __syncthreads();
    if (threadIdx.x == kScanThreads - 1) s_base = pos + k;
    __syncthreads();
  }
  if (threadIdx.x == 0) *n_out = s_base;
}

// The next vectors of the kept columns, at their compacted positions:
// sign(y) of the old column (unit == 0) or e_{jcand} (unit == 1).
__global__ void __launch_bounds__(kP1Threads) k_p1_emit(const double2 *Xin, double2 *Xout, long long ldx, int m,
                                                       int nc, const int *newpos, const int *map_in,
                                                       const int *jcand, int unit) {
  const int c = blockIdx.x;
  if (c >= nc) return;
  const int q = newpos[c];
  if (q < 0) return;
  double2 *out = Xout + (long long)q * ldx;
  if (unit) {
    const int j = jcand[map_in[c]];
    for (int i = threadIdx.x; i < m; i += kP1Threads) out[i] = make_double2(i == j ? 1.0 : 0.0, 0.0);
  } else {
    const double2 *in = Xin + (long long)c * ldx;
    for (int i = threadIdx.x; i < m; i += kP1Threads) {
      const double2 v = in[i];
      const double a = zmod(v);
      out[i] = a == 0.0 ? make_double2(1.0, 0.0) : make_double2(v.x / a, v.y / a);
    }
  }
}

// Bounding box of diag(T) and the margin (one CTA): box = (x0, x1, y0, y1).
__global__ void __launch_bounds__(256) k_grid_box(const double2 *T, long long ldt, int m, double *box) {
  __shared__ double s[4][8];
  __shared__ double s_big[8];
  double a = INFINITY, b = -INFINITY, c = INFINITY, d = -INFINITY, big = 1.0;
  for (int i = threadIdx.x; i < m; i += 256) {
    const double2 t = T[i + (long long)i * ldt];
    a = fmin(a, t.x); b = fmax(b, t.x); c = fmin(c, t.y); d = fmax(d, t.y);
    big = fmax(big, fmax(fabs(t.x), fabs(t.y)));
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    a = fmin(a, __shfl_xor_sync(0xffffffffu, a, o));
    b = fmax(b, __shfl_xor_sync(0xffffffffu, b, o));
    c = fmin(c, __shfl_xor_sync(0xffffffffu, c, o));
    d = fmax(d, __shfl_xor_sync(0xffffffffu, d, o));
    big = fmax(big, __shfl_xor_sync(0xffffffffu, big, o));
  }
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) { s[0][w] = a; s[1][w] = b; s[2][w] = c; s[3][w] = d; s_big[w] = big; }
  __syncthreads();
  if (threadIdx.x != 0) return;
  for (int k = 1; k < 8; ++k) {
    a = fmin(a, s[0][k]); b = fmax(b, s[1][k]); c = fmin(c, s[2][k]); d = fmax(d, s[3][k]);
    big = fmax(big, s_big[k]);
  }
  a = fmin(a, s[0][0]); b = fmax(b, s[1][0]); c = fmin(c, s[2][0]); d = fmax(d, s[3][0]);
  big = fmax(big, s_big[0]);
  const double wid = __dsub_rn(b, a), hgt = __dsub_rn(d, c);
  double h = __dmul_rn(0.25, fmax(wid, hgt));
  const double hmin = ldexp(big, -20);
  if (h < hmin) h = hmin;
  box[0] = __dsub_rn(a, h);
  box[1] = __dadd_rn(b, h);
  box[2] = __dsub_rn(c, h);
  box[3] = __dadd_rn(d, h);
}

__global__ void k_grid_points(const double *box, int nx, int ny, double2 *z) {
  const long long n = (long long)nx * ny;
  const double x0 = box[0], y0 = box[2];
  const double dx = nx > 1 ? __ddiv_rn(__dsub_rn(box[1], x0), (double)(nx - 1)) : 0.0;
  const double dy = ny > 1 ? __ddiv_rn(__dsub_rn(box[3], y0), (double)(ny - 1)) : 0.0;
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x) {
    const int k = (int)(q % nx), l = (int)(q / nx);
    z[q] = make_double2(__dadd_rn(x0, __dmul_rn((double)k, dx)), __dadd_rn(y0, __dmul_rn((double)l, dy)));
  }
}

size_t a256(size_t x) { return (x + 255) & ~size_t(255); }

struct P1Layout {
  size_t xa, xb, qh, oz, eng, st;   // byte offsets
  size_t total, eng_bytes;
};

P1Layout p1_layout(int64_t m, int64_t N, int32_t nb, bool with_q, uint32_t flags) {
  P1Layout L{};
  const size_t blk = a256((size_t)m * (size_t)N * sizeof(double2));
  size_t off = 0;
  L.xa = off; off += blk;
  L.xb = off; off += blk;
  L.qh = off; off += with_q ? a256((size_t)m * (size_t)m * sizeof(double2)) : 0;
  L.oz = off; off += (with_q && (flags & MSTS_TENSOR_GEMM)) ? a256(ozaki_workspace_bytes((int)m, (int)N)) : 0;
  const uint32_t ef = flags & MSTS_TENSOR_GEMM;
  L.eng_bytes = std::max(msts_solve_workspace_size(m, N, nb, ef), msts_solve_workspace_size(m, N, nb, ef | MSTS_CONJ_TRANS));
  L.eng = off; off += a256(L.eng_bytes);
  L.st = off;
  // g (N doubles), jcand, keep, newpos, map_a, map_b (N ints each), z_a, z_b (N complex), n_act (1 int)
  off += a256(8 * (size_t)N) + 5 * a256(4 * (size_t)N) + 2 * a256(16 * (size_t)N) + 256;
  L.total = off;
  return L;
}

constexpr int64_t kMaxDim = (int64_t)1 << 30;

}  // namespace
}  // namespace msts

extern "C" {

size_t msts_pseudospectra_1norm_workspace_size(int64_t m, int64_t N, int32_t nb, int32_t with_q, uint32_t flags) {
  if (m < 0 || N < 0 || m > msts::kMaxDim || N > msts::kMaxDim) return 0;
  if ((flags & ~(uint32_t)MSTS_TENSOR_GEMM) != 0 || (nb != 16 && nb != 32 && nb != 64)) return 0;
  if (m == 0 || N == 0) return 0;
  return msts::p1_layout(m, N, nb, with_q != 0, flags).total;
}

int msts_pseudospectra_1norm(const msts_z *T, int64_t ldt, int64_t m, const msts_z *Q, int64_t ldq,
                             const msts_z *z, int64_t N, double *est, int32_t *kind, int32_t *steps, int32_t nb,
                             void *workspace, size_t workspace_bytes, uint32_t *status, uint32_t flags,
                             void *stream) {
  if (m < 0 || m > msts::kMaxDim) return -3;
  if (m > 0 && !T) return -1;
  if (ldt < std::max<int64_t>(1, m)) return -2;
  if (Q && ldq < std::max<int64_t>(1, m)) return -4;
  if (N < 0 || N > msts::kMaxDim) return -6;
  if (N > 0 && !z) return -5;
  if (N > 0 && (!est || !kind || !steps)) return -7;
  if (nb != 16 && nb != 32 && nb != 64) return -8;
  if ((flags & ~(uint32_t)MSTS_TENSOR_GEMM) != 0) return -11;
  const size_t need = msts_pseudospectra_1norm_workspace_size(m, N, nb, Q != nullptr, flags);
  if (need > 0 && (!workspace || workspace_bytes < need)) return workspace ? -10 : -9;
  if (msts::bad_alignment({T, Q, z}, workspace)) return MSTS_ERR_ALIGN;
  if (m == 0 || N == 0) return 0;
  using namespace msts;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const bool tensor = (flags & MSTS_TENSOR_GEMM) != 0;
  const P1Layout L = p1_layout(m, N, nb, Q != nullptr, flags);
  char *ws = static_cast<char *>(workspace);
  double2 *XA = reinterpret_cast<double2 *>(ws + L.xa);
  double2 *XB = reinterpret_cast<double2 *>(ws + L.xb);
  double2 *QH = reinterpret_cast<double2 *>(ws + L.qh);
  void *ozws = ws + L.oz;
  void *eng = ws + L.eng;
  char *sp = ws + L.st;
  double *g = reinterpret_cast<double *>(sp); sp += a256(8 * (size_t)N);
  int *jcand = reinterpret_cast<int *>(sp); sp += a256(4 * (size_t)N);
  int *keep = reinterpret_cast<int *>(sp); sp += a256(4 * (size_t)N);
  int *newpos = reinterpret_cast<int *>(sp); sp += a256(4 * (size_t)N);
  int *map_a = reinterpret_cast<int *>(sp); sp += a256(4 * (size_t)N);
  int *map_b = reinterpret_cast<int *>(sp); sp += a256(4 * (size_t)N);
  double2 *z_a = reinterpret_cast<double2 *>(sp); sp += a256(16 * (size_t)N);
  double2 *z_b = reinterpret_cast<double2 *>(sp); sp += a256(16 * (size_t)N);
  int *n_act = reinterpret_cast<int *>(sp);
  const double2 *q = reinterpret_cast<const double2 *>(Q);
  const int mi = (int)m, Ni = (int)N;
  const uint32_t ef = tensor ? MSTS_TENSOR_GEMM : 0u;
  auto ok = [](cudaError_t e) { return e == cudaSuccess; };

  if (q && !ok(remap(q, ldq, QH, m, mi, mi, true, false, false, true, false, st))) return MSTS_ERR_CUDA;
  // X <- R X (adj = false) or R^H X (adj = true) on the first nc columns of X,
  // shifts zc; Y is scratch (the Q products need an out-of-place target).
  auto apply = [&](double2 *X, double2 *Y, int nc, const double2 *zc, bool adj) -> int {
    double2 *S = X;
    if (q) {
      const cudaError_t e = tensor ? ozaki_product(QH, m, mi, X, m, nc, false, Y, m, ozws, status, st)
                                   : zgemm_fp64(QH, m, X, m, Y, m, mi, nc, false, st);
      if (!ok(e)) return MSTS_ERR_CUDA;
      S = Y;
    }
    const int rc = msts_solve(T, ldt, m, reinterpret_cast<const msts_z *>(zc), nc, reinterpret_cast<msts_z *>(S),
                              m, nullptr, nullptr, nb, eng, L.eng_bytes, status, ef | (adj ? MSTS_CONJ_TRANS : 0u),
                              stream);
    if (rc != 0) return rc;
    if (q) {
      const cudaError_t e = tensor ? ozaki_product(q, ldq, mi, Y, m, nc, false, X, m, ozws, status, st)
                                   : zgemm_fp64(q, ldq, Y, m, X, m, mi, nc, false, st);
      if (!ok(e)) return MSTS_ERR_CUDA;
    }
    return 0;
  };
  auto decide = [&](const double2 *X, int nc, const int *map, int mode) -> bool {
    k_p1_decide<<<(unsigned)nc, kP1Threads, 0, st>>>(X, m, mi, nc, map, mode, g, est, kind, jcand, steps, keep);
    count_launches(1);
    return ok(cudaGetLastError());
  };
  // compaction: kept columns of the current block move to the other buffer
  auto compact = [&](int nc, bool unit, int &n_new) -> bool {
    k_p1_scan<<<1, kScanThreads, 0, st>>>(keep, nc, map_a, z_a, map_b, z_b, newpos, n_act);
    k_p1_emit<<<(unsigned)nc, kP1Threads, 0, st>>>(XA, XB, m, mi, nc, newpos, map_a, jcand, unit ? 1 : 0);
    count_launches(2);
    if (!ok(cudaGetLastError())) return false;
    if (!ok(cudaMemcpyAsync(&n_new, n_act, sizeof(int), cudaMemcpyDeviceToHost, st))) return false;
    if (!ok(cudaStreamSynchronize(st))) return false;
    std::swap(XA, XB);
    std::swap(map_a, map_b);
    std::swap(z_a, z_b);
    return true;
  };
  // start: x = e/m for every point
  k_iota<<<(unsigned)((N + 255) / 256), 256, 0, st>>>(map_a, reinterpret_cast<const double2 *>(z), z_a, Ni);
  k_p1_fill<<<(unsigned)N, 256, 0, st>>>(XA, m, mi, Ni, 0);
  count_launches(2);
  if (!ok(cudaGetLastError())) return MSTS_ERR_CUDA;
  int rc = apply(XA, XB, Ni, z_a, false);
  if (rc != 0) return rc;
  if (!decide(XA, Ni, map_a, kStart)) return MSTS_ERR_CUDA;
  int nc = 0;
  if (!compact(Ni, false, nc)) return MSTS_ERR_CUDA;
  for (int it = 0; it < kMaxSteps && nc > 0; ++it) {
    if ((rc = apply(XA, XB, nc, z_a, true)) != 0) return rc;       // w = R^H sign(y)
    if (!decide(XA, nc, map_a, kAfterRH)) return MSTS_ERR_CUDA;
    if (!compact(nc, true, nc)) return MSTS_ERR_CUDA;
    if (nc == 0) break;
    if ((rc = apply(XA, XB, nc, z_a, false)) != 0) return rc;      // y = R e_j
    if (!decide(XA, nc, map_a, kAfterR)) return MSTS_ERR_CUDA;
    if (!compact(nc, false, nc)) return MSTS_ERR_CUDA;
  }
  if (m > 1) {                                                     // the alternative vector, every point
    k_iota<<<(unsigned)((N + 255) / 256), 256, 0, st>>>(map_a, reinterpret_cast<const double2 *>(z), z_a, Ni);
    k_p1_fill<<<(unsigned)N, 256, 0, st>>>(XA, m, mi, Ni, 1);
    count_launches(2);
    if (!ok(cudaGetLastError())) return MSTS_ERR_CUDA;
    if ((rc = apply(XA, XB, Ni, z_a, false)) != 0) return rc;
    if (!decide(XA, Ni, map_a, kAlt)) return MSTS_ERR_CUDA;
  }
  return 0;
}

int msts_portrait_grid(const msts_z *T, int64_t ldt, int64_t m, int64_t nx, int64_t ny, msts_z *z, double *box,
                       void *stream) {
  if (m < 1 || m > msts::kMaxDim) return -3;
  if (!T) return -1;
  if (ldt < m) return -2;
  if (nx < 1 || ny < 1 || nx > msts::kMaxDim || ny > msts::kMaxDim || nx * ny > ((int64_t)1 << 40)) return -4;
  if (!z) return -5;
  if (!box) return -6;
  if (msts::bad_alignment({T, z}, nullptr)) return MSTS_ERR_ALIGN;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  msts::k_grid_box<<<1, 256, 0, st>>>(reinterpret_cast<const double2 *>(T), ldt, (int)m, box);
  const long long n = nx * ny;
  const unsigned blocks = (unsigned)std::min<long long>((n + 255) / 256, 152 * 16);
  msts::k_grid_points<<<blocks, 256, 0, st>>>(box, (int)nx, (int)ny, reinterpret_cast<double2 *>(z));
  msts::count_launches(2);
  return cudaGetLastError() == cudaSuccess ? 0 : MSTS_ERR_CUDA;
}

}  // extern "C"

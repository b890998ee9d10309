// msts_variant.cu -- the other triangular variants of the multi-shift solve
// (footnote to Sec. 2: lower-triangular and right-hand cases).
//
// The operator is M_j = op(A) - s_j I with op(A) in {A, A^T, A^H} and A upper
// or lower triangular; left side M_j x_j = b_j (columns of B), right side
// x_j^T M_j = b_j^T (rows of B).  A right-side system is the left-side system
// with the transposed operator, op'(A) - s_j I (A -> A^T, A^T -> A,
// A^H -> conj(A)).  The effective left operator E = op'(A) is mapped onto the
// upper-triangular engine of msts_solve:
//   - E = A, A upper                     : A used in place;
//   - E = A^H, A upper, plain solve      : the engine's conjugate-transposed
//                                          form with the shifts conjugated;
//   - otherwise                          : E written out as an upper-triangular
//     U' in the solve's own order -- U' = E when E is upper triangular, else
//     the reversal U'(r,c) = E(m-1-r, m-1-c) with the right-hand sides
//     reversed alike -- so that Alg. 3 / Alg. 5 run in the variant's
//     substitution order, the blocks cut from the end where it starts.
// Right-hand sides that are rows of B, or reversed, are gathered into a
// column-major m x n copy and scattered back after the solve.  Every remap is
// an exact permutation (and conjugation) of values: one pass over A and two
// over B, all HBM-bound.
#include <algorithm>

#include "../../include/msts.h"
#include "msts_check.h"
#include "msts_remap.h"
#include "msts_trace.h"

namespace msts {
namespace {

constexpr int kRT = 32;   // remap tile: 32 x 32 elements, 32 x 8 threads

__device__ __forceinline__ double2 maybe_conj(double2 v, int conj) {
  return conj ? make_double2(v.x, -v.y) : v;
}

// dst(r, c) = [conj] src(p, q) for r < rows, c < cols, where
//   r' = rev_r ? rows-1-r : r,   c' = rev_c ? cols-1-c : c,
//   (p, q) = TR ? (c', r') : (r', c');
// with `upper`, only r <= c is written.  Without TR consecutive threads read
// and write consecutive rows directly; with TR the tile passes through shared
// memory so that both the reads and the writes are along columns.
template <bool TR>
__device__ __forceinline__ void remap_tile(const double2 *__restrict__ src, long long lds,
                                           double2 *__restrict__ dst, long long ldd, int rows, int cols,
                                           int rev_r, int rev_c, int conj, int upper, int r0, int c0,
                                           double2 (*tile)[kRT + 1]) {
  if (upper && r0 > c0 + kRT - 1) return;                  // tile wholly below the diagonal (block-uniform)
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // ty in [0, 8)
  if constexpr (!TR) {
    const int r = r0 + tx;
    if (r >= rows) return;
    const int rp = rev_r ? rows - 1 - r : r;
#pragma unroll
    for (int u = 0; u < kRT / 8; ++u) {
      const int c = c0 + ty + 8 * u;
      if (c >= cols || (upper && r > c)) continue;
      const int cp = rev_c ? cols - 1 - c : c;
      dst[r + (long long)c * ldd] = maybe_conj(src[rp + (long long)cp * lds], conj);
    }
  } else {
    // load: lane tx walks the source rows p = c'(c0 + tx), which are contiguous
#pragma unroll
    for (int u = 0; u < kRT / 8; ++u) {
      const int lr = ty + 8 * u, lc = tx;
      const int r = r0 + lr, c = c0 + lc;
      if (r < rows && c < cols) {
        const int rp = rev_r ? rows - 1 - r : r, cp = rev_c ? cols - 1 - c : c;
        tile[lr][lc] = src[cp + (long long)rp * lds];
      }
    }
    __syncthreads();
    const int r = r0 + tx;
    if (r >= rows) return;
#pragma unroll
    for (int u = 0; u < kRT / 8; ++u) {
      const int lc = ty + 8 * u, c = c0 + lc;
      if (c >= cols || (upper && r > c)) continue;
      dst[r + (long long)c * ldd] = maybe_conj(tile[tx][lc], conj);
    }
  }
}

// One CTA per 32 x 32 tile of dst; tile columns beyond the grid's y extent
// are walked in a loop (the barrier between tiles keeps `tile` private).
template <bool TR>
__global__ void __launch_bounds__(256) k_remap(const double2 *__restrict__ src, long long lds,
                                              double2 *__restrict__ dst, long long ldd, int rows, int cols,
                                              int rev_r, int rev_c, int conj, int upper) {
  __shared__ double2 tile[kRT][kRT + 1];
  const int r0 = blockIdx.x * kRT;
  const int ct = (cols + kRT - 1) / kRT;
  for (int cy = blockIdx.y; cy < ct; cy += gridDim.y) {
    remap_tile<TR>(src, lds, dst, ldd, rows, cols, rev_r, rev_c, conj, upper, r0, cy * kRT, tile);
    if (TR) __syncthreads();
  }
}

__global__ void k_conj_vec(const double2 *__restrict__ s, double2 *__restrict__ t, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) t[i] = make_double2(s[i].x, -s[i].y);
}

// Code of op' for the effective left operator: 0 = A, 1 = A^T, 2 = A^H,
// 3 = conj(A).
int effective_op(int32_t side, int32_t trans) {
  if (side == MSTS_SIDE_LEFT) return trans;
  return trans == MSTS_OP_N ? 1 : (trans == MSTS_OP_T ? 0 : 3);
}

enum Route { kDirect = 0, kConjEngine = 1, kRemap = 2 };

struct Plan {
  Route route;
  bool rev;          // E lower triangular: the solve runs on the reversal
  bool tr;           // E reads A transposed
  bool conj;         // E conjugates A
  bool gather_b;     // right-hand sides copied into an m x n column-major array
  size_t u_bytes, b_bytes, s_bytes, eng_bytes;
  uint32_t eng_flags;
};

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

Plan make_plan(int32_t side, int32_t uplo, int32_t trans, int64_t m, int64_t n, int32_t nb, uint32_t flags) {
  Plan P{};
  const int op = effective_op(side, trans);
  const bool e_upper = (uplo == MSTS_UPLO_UPPER) == (op == 0 || op == 3);
  const bool safe = (flags & MSTS_SAFE) != 0;
  P.rev = !e_upper;
  P.tr = op == 1 || op == 2;
  P.conj = op == 2 || op == 3;
  if (op == 0 && uplo == MSTS_UPLO_UPPER) P.route = kDirect;
  else if (op == 2 && uplo == MSTS_UPLO_UPPER && !safe) P.route = kConjEngine;
  else P.route = kRemap;
  if (P.route == kConjEngine) P.rev = false;               // the engine's forward substitution
  P.gather_b = side == MSTS_SIDE_RIGHT || P.rev;
  P.eng_flags = flags | (P.route == kConjEngine ? MSTS_CONJ_TRANS : 0u);
  P.u_bytes = P.route == kRemap ? align256((size_t)m * (size_t)m * sizeof(double2)) : 0;
  P.b_bytes = P.gather_b ? align256((size_t)m * (size_t)n * sizeof(double2)) : 0;
  P.s_bytes = P.route == kConjEngine ? align256((size_t)n * sizeof(double2)) : 0;
  P.eng_bytes = msts_solve_workspace_size(m, n, nb, P.eng_flags);
  return P;
}

bool args_ok(int32_t side, int32_t uplo, int32_t trans) {
  return (side == MSTS_SIDE_LEFT || side == MSTS_SIDE_RIGHT) &&
         (uplo == MSTS_UPLO_UPPER || uplo == MSTS_UPLO_LOWER) &&
         (trans == MSTS_OP_N || trans == MSTS_OP_T || trans == MSTS_OP_C);
}

constexpr int64_t kMaxDim = (int64_t)1 << 30;

}  // namespace

cudaError_t remap(const double2 *src, long long lds, double2 *dst, long long ldd, int rows, int cols,
                  bool tr, bool rev_r, bool rev_c, bool conj, bool upper, cudaStream_t st) {
  if (rows == 0 || cols == 0) return cudaSuccess;
  const dim3 grid((unsigned)((rows + kRT - 1) / kRT), (unsigned)std::min((cols + kRT - 1) / kRT, 65535));
  if (tr)
    k_remap<true><<<grid, 256, 0, st>>>(src, lds, dst, ldd, rows, cols, rev_r, rev_c, conj, upper);
  else
    k_remap<false><<<grid, 256, 0, st>>>(src, lds, dst, ldd, rows, cols, rev_r, rev_c, conj, upper);
  count_launches(1);
  return cudaGetLastError();
}

}  // namespace msts

extern "C" {

size_t msts_solve_variant_workspace_size(int32_t side, int32_t uplo, int32_t trans, int64_t m, int64_t n,
                                         int32_t nb, uint32_t flags) {
  if (!msts::args_ok(side, uplo, trans) || m < 0 || n < 0 || m > msts::kMaxDim || n > msts::kMaxDim) return 0;
  if ((flags & ~(uint32_t)(MSTS_SAFE | MSTS_TENSOR_GEMM)) != 0) return 0;
  if (nb != 16 && nb != 32 && nb != 64) return 0;
  const msts::Plan P = msts::make_plan(side, uplo, trans, m, n, nb, flags);
  return P.u_bytes + P.b_bytes + P.s_bytes + P.eng_bytes;
}

int msts_solve_variant(int32_t side, int32_t uplo, int32_t trans, const msts_z *A, int64_t lda, int64_t m,
                       const msts_z *shifts, int64_t n, msts_z *B, int64_t ldb, double *scales,
                       int32_t *scale_exp, int32_t nb, void *workspace, size_t workspace_bytes,
                       uint32_t *status, uint32_t flags, void *stream) {
  const bool safe = (flags & MSTS_SAFE) != 0;
  if (!msts::args_ok(side, uplo, trans)) return -15;
  if (m < 0 || m > msts::kMaxDim) return -3;
  if (m > 0 && !A) return -1;
  if (lda < std::max<int64_t>(1, m)) return -2;
  if (n < 0 || n > msts::kMaxDim) return -5;
  if (n > 0 && !shifts) return -4;
  if (m > 0 && n > 0 && !B) return -6;
  if (ldb < std::max<int64_t>(1, side == MSTS_SIDE_LEFT ? m : n)) return -7;
  if (safe && n > 0 && (!scales || !scale_exp)) return scales ? -9 : -8;
  if (nb != 16 && nb != 32 && nb != 64) return -10;
  if ((flags & ~(uint32_t)(MSTS_SAFE | MSTS_TENSOR_GEMM)) != 0) return -14;
  const size_t need = msts_solve_variant_workspace_size(side, uplo, trans, m, n, nb, flags);
  if (need > 0 && (!workspace || workspace_bytes < need)) return workspace ? -12 : -11;
  if (msts::bad_alignment({A, shifts, B}, workspace)) return MSTS_ERR_ALIGN;
  if (m == 0 || n == 0) return 0;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const msts::Plan P = msts::make_plan(side, uplo, trans, m, n, nb, flags);
  char *ws = static_cast<char *>(workspace);
  double2 *Up = reinterpret_cast<double2 *>(ws);
  double2 *Bp = reinterpret_cast<double2 *>(ws + P.u_bytes);
  double2 *sp = reinterpret_cast<double2 *>(ws + P.u_bytes + P.b_bytes);
  char *eng = ws + P.u_bytes + P.b_bytes + P.s_bytes;
  double2 *b = reinterpret_cast<double2 *>(B);
  const double2 *a = reinterpret_cast<const double2 *>(A);
  const int mi = (int)m, ni = (int)n;
  const bool right = side == MSTS_SIDE_RIGHT;

  const msts_z *U = A;
  int64_t ldu = lda;
  if (P.route == msts::kRemap) {
    if (msts::remap(a, lda, Up, m, mi, mi, P.tr, P.rev, P.rev, P.conj, true, st) != cudaSuccess)
      return MSTS_ERR_CUDA;
    U = reinterpret_cast<const msts_z *>(Up);
    ldu = m;
  }
  const msts_z *s = shifts;
  if (P.route == msts::kConjEngine) {
    msts::k_conj_vec<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(reinterpret_cast<const double2 *>(shifts), sp,
                                                                    ni);
    msts::count_launches(1);
    if (cudaGetLastError() != cudaSuccess) return MSTS_ERR_CUDA;
    s = reinterpret_cast<const msts_z *>(sp);
  }
  msts_z *X = B;
  int64_t ldx = ldb;
  if (P.gather_b) {
    // Bp(r, j) = B(R(r), j) (left) or B(j, R(r)) (right), R the reversal when rev
    if (msts::remap(b, ldb, Bp, m, mi, ni, right, P.rev, false, false, false, st) != cudaSuccess)
      return MSTS_ERR_CUDA;
    X = reinterpret_cast<msts_z *>(Bp);
    ldx = m;
  }
  int rc = msts_solve(U, ldu, m, s, n, X, ldx, scales, scale_exp, nb, eng, P.eng_bytes, status, P.eng_flags,
                      stream);
  if (rc != 0) return rc;
  if (P.gather_b) {
    // left: B(i, j) = Bp(R(i), j); right: B(j, i) = Bp(R(i), j)
    const cudaError_t e = right ? msts::remap(Bp, m, b, ldb, ni, mi, true, false, P.rev, false, false, st)
                                : msts::remap(Bp, m, b, ldb, mi, ni, false, P.rev, false, false, false, st);
    if (e != cudaSuccess) return MSTS_ERR_CUDA;
  }
  return 0;
}

}  // extern "C"

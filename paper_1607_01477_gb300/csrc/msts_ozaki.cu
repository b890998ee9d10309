// msts_ozaki.cu -- FP64-accurate complex product P = triu(U) X on the BF16
// tensor cores (tcgen05), used for the refinement residual
// R = B - (U - S) X = B - P + X diag(s) of the mixed-precision solve.
//
// Method: error-free splitting of both operands into integer digit planes
// (the splitting of Ozaki, Ogita, Oishi & Rump, Numer. Algorithms 59, 2012),
// written here for the tcgen05 pipeline:
//  * real embedding: with A'(2r, 2k..2k+1) = (Re U, -Im U),
//    A'(2r+1, 2k..2k+1) = (Im U, Re U) and B' = X read as real numbers
//    (its interleaved storage already is [Re X(k); Im X(k)]), the real
//    product A' B' holds Re P in its even rows and Im P in its odd rows;
//  * every row r of U gets an exponent e_r with |Re U(r,k)|, |Im U(r,k)| <
//    2^e_r, every column j of X an exponent f_j likewise; each entry then is
//    2^e sum_{s=1..8} d_s 2^{-7s} + (remainder < 2^{e-56}) with signed integer
//    digits |d_s| <= 127, exactly representable in BF16;
//  * A' B' = 2^{e_r + f_j} sum_{d=2..9} 2^{-7d} D_d with D_d = sum_{s+t=d}
//    (digit plane s of A') (digit plane t of B'); products with s + t > 9 are
//    dropped (each below 2^{-49} of the leading term's scale);
//  * K' is processed in chunks of 64: within a chunk every |D_d| <= 8 * 64 *
//    127^2 < 2^24, so the FP32 accumulation in tensor memory is exact; the
//    epilogue warps turn each chunk's D_d into integers and add them into two
//    int64 accumulators per output (HI for d <= 4, LO for d >= 5), so nothing
//    is rounded until the final conversion to FP64.
// The result is accurate to about 2^-50 relative to K' max|U(r,:)| max|X(:,j)|.
//
// Kernel layout (one CTA per 128 x 32 output tile of A' B'; 10 warps):
//  warp 8  : TMA producer (B digit planes per chunk, A planes through a ring);
//  warp 9  : one thread issues the MMAs of each chunk: for every A plane one
//            MMA per 16-wide K step against all the B planes it pairs with
//            (N = 32 x (9 - s)), into 8 TMEM accumulators laid out by diagonal
//            (double-buffered: 2 x 8 x 32 = 512 columns);
//  warps 0-7: epilogue, one thread per TMEM lane (= output row) and half
//            of the tile's columns.
// Every mbarrier wait is bounded; a timeout raises MSTS_STATUS_TIMEOUT in the
// status word (which also makes the waits of all other CTAs give up) and the
// kernel drains without hanging.
#include <cuda.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <memory>
#include <mutex>

#include "msts_common.cuh"
#include "msts_digits.cuh"
#include "msts_ozaki.h"
#include "msts_tc.cuh"
#include "msts_trace.h"

namespace msts {

constexpr int kNumSMsOz = 152;   // SMs of the part (grid sizing)
constexpr int kOzKC = 64;        // K' per chunk: one 128-byte swizzle row of BF16
constexpr int kOzBM = 128;       // real rows per tile (= TMEM lanes)
constexpr int kOzBN = 32;        // columns per tile
constexpr int kOzRing = 6;       // A-plane ring depth
constexpr int kOzEpi = 8;         // epilogue warps: two per TMEM lane quarter, 16 columns each
constexpr int kOzThreads = 32 * kOzEpi + 64;  // + producer + MMA
constexpr int kOzAccCols = kOzS * kOzBN;   // 8 diagonals x 32 columns per buffer
constexpr uint32_t kOzABytes = kOzBM * kOzKC * 2;          // 16 KB per A plane
constexpr uint32_t kOzBBytes = kOzS * kOzBN * kOzKC * 2;   // 32 KB for all B planes
constexpr size_t kOzSmem = 2 * kOzBBytes + kOzRing * kOzABytes + 1024;

static size_t a256(size_t x) { return (x + 255) & ~size_t(255); }
static int kpad(int m) { return ((2 * m + kOzKC - 1) / kOzKC) * kOzKC; }

size_t ozaki_workspace_bytes(int m, int n) {
  const size_t K = (size_t)kpad(m);
  return a256((size_t)kOzS * 2 * m * K * 2) + a256((size_t)kOzS * n * K * 2) + a256(4 * (size_t)m) +
         a256(4 * (size_t)n);
}

struct OzakiBufs {
  __nv_bfloat16 *Ap, *Bp;
  int *rexp, *cexp;
  int K;
};
static OzakiBufs carve(void *ws, int m, int n) {
  OzakiBufs o;
  o.K = kpad(m);
  char *c = static_cast<char *>(ws);
  o.Ap = reinterpret_cast<__nv_bfloat16 *>(c); c += a256((size_t)kOzS * 2 * m * o.K * 2);
  o.Bp = reinterpret_cast<__nv_bfloat16 *>(c); c += a256((size_t)kOzS * n * o.K * 2);
  o.rexp = reinterpret_cast<int *>(c); c += a256(4 * (size_t)m);
  o.cexp = reinterpret_cast<int *>(c);
  return o;
}

// e_r for every row of triu(U) (or of the whole m x kc matrix with full): one
// warp per row.
__global__ void k_oz_rowexp(const double2 *U, long long ldu, int m, int kc, int *rexp, int full) {
  const int lane = threadIdx.x & 31;
  const int r = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (r >= m) return;
  int e = -(1 << 29);
  for (int k = (full ? 0 : r) + lane; k < kc; k += 32) e = max(e, bound_exp(U[r + (long long)k * ldu]));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) e = max(e, __shfl_xor_sync(0xffffffffu, e, o));
  if (lane == 0) rexp[r] = e < -(1 << 28) ? 0 : e;
}

// Digit planes of A': plane s, row i, column k' at Ap[(s * 2m + i) * K + k'].
// Thread (k, r) writes rows 2r, 2r+1 at columns 2k, 2k+1 of every plane
// (zero outside the upper triangle unless full, and in the padding).
__global__ void k_oz_slice_A(const double2 *U, long long ldu, int m, int kc, const int *rexp,
                             __nv_bfloat16 *Ap, int K, int full) {
  const int r = blockIdx.y;
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (2 * k >= K) return;
  float dr[kOzS], di[kOzS];
  if ((full || k >= r) && k < kc) {
    const double2 u = U[r + (long long)k * ldu];
    digits8(u.x, rexp[r], dr);
    digits8(u.y, rexp[r], di);
  } else {
#pragma unroll
    for (int s = 0; s < kOzS; ++s) dr[s] = di[s] = 0.f;
  }
  const size_t rows = 2 * (size_t)m;
#pragma unroll
  for (int s = 0; s < kOzS; ++s) {
    __nv_bfloat162 *p0 = reinterpret_cast<__nv_bfloat162 *>(Ap + (s * rows + 2 * (size_t)r) * K + 2 * k);
    __nv_bfloat162 *p1 = reinterpret_cast<__nv_bfloat162 *>(Ap + (s * rows + 2 * (size_t)r + 1) * K + 2 * k);
    *p0 = __floats2bfloat162_rn(dr[s], -di[s]);   // row 2r:   (Re U, -Im U)
    *p1 = __floats2bfloat162_rn(di[s], dr[s]);    // row 2r+1: (Im U,  Re U)
  }
}

// Digit planes of B' = X (as real): plane t, column j, k' at Bp[(t * n + j) * K + k'],
// with the column exponent f_j (triu: X upper triangular, rows k > j read as
// zero); one CTA per column.
__global__ void k_oz_slice_B(const double2 *X, long long ldx, int m, int n, int *cexp,
                             __nv_bfloat16 *Bp, int K, int triu) {
  __shared__ int red[32];
  const int j = blockIdx.x;
  const double2 *col = X + (long long)j * ldx;
  const int mend = triu ? min(m, j + 1) : m;         // rows read (upper triangle only with triu)
  int e = -(1 << 29);
  for (int k = threadIdx.x; k < mend; k += blockDim.x) e = max(e, bound_exp(col[k]));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) e = max(e, __shfl_xor_sync(0xffffffffu, e, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = e;
  __syncthreads();
  e = red[0];
  for (int w = 1; w < (int)(blockDim.x >> 5); ++w) e = max(e, red[w]);
  if (e < -(1 << 28)) e = 0;
  if (threadIdx.x == 0) cexp[j] = e;
  for (int k = threadIdx.x; 2 * k < K; k += blockDim.x) {
    float dr[kOzS], di[kOzS];
    if (k < mend) {
      const double2 x = col[k];
      digits8(x.x, e, dr);
      digits8(x.y, e, di);
    } else {
#pragma unroll
      for (int s = 0; s < kOzS; ++s) dr[s] = di[s] = 0.f;
    }
#pragma unroll
    for (int t = 0; t < kOzS; ++t)
      *reinterpret_cast<__nv_bfloat162 *>(Bp + ((size_t)t * n + j) * K + 2 * k) =
          __floats2bfloat162_rn(dr[t], di[t]);
  }
}

// Arguments of the digit-plane product kernel.  Two epilogues share it:
//  kResidual: R = B - P + s_j X over rows [0, 2m) of A' (K' from the tile's
//             diagonal to the end: U is upper triangular);
//  kUpdate:   the substitution step of the blocked solve,
//             B(r, col) = 2^-pend(col) B(r, col) - P(r, col) over real rows
//             [row_lo, row_hi) of A' and `ncols` columns starting at col_base,
//             K' = the chunks of this block (a_x0 = its first column in the
//             block-layout planes);
//  kProduct:  R = P over rows [0, 2m) (A dense; with triu_b the K' chunks
//             below the column tile's last diagonal entry are skipped, B being
//             upper triangular).
struct OzArgs {
  const double2 *B; long long ldb;    // residual: right-hand side; update: matrix updated in place
  const double2 *X; long long ldx;    // residual only
  const double2 *s;                   // residual only
  double2 *R; long long ldr;          // residual: output; update: = B
  const int *rexp;                    // exponent of complex row r (update: of this block's panel)
  const int *cexp;                    // exponent of local column c
  const int *pend;                    // update: pending rescale per global column (safe), or null
  int m, n, K;                        // residual: order, columns, K'; update: K = chunks * 64
  int a_x0;                           // update: first K' column of this block in the A planes
  int row_lo, row_hi;                 // update: real rows of A' updated
  int col_base, ncols;                // update: global column of local column 0, local columns
  int triu_b;                         // product: B upper triangular
  uint32_t *status;
};

// Digit planes of B' = X^H (as real): column c of B' is conj(X(c, 0:kc)), at
// Bp[(t * mc + c) * K + k'], exponent f_c over that row of X; one CTA per column.
__global__ void k_oz_slice_BH(const double2 *X, long long ldx, int mc, int kc, int *cexp, __nv_bfloat16 *Bp,
                              int K) {
  __shared__ int red[32];
  const int c = blockIdx.x;
  int e = -(1 << 29);
  for (int k = threadIdx.x; k < kc; k += blockDim.x) e = max(e, bound_exp(X[c + (long long)k * ldx]));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) e = max(e, __shfl_xor_sync(0xffffffffu, e, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = e;
  __syncthreads();
  e = red[0];
  for (int w = 1; w < (int)(blockDim.x >> 5); ++w) e = max(e, red[w]);
  if (e < -(1 << 28)) e = 0;
  if (threadIdx.x == 0) cexp[c] = e;
  for (int k = threadIdx.x; 2 * k < K; k += blockDim.x) {
    float dr[kOzS], di[kOzS];
    if (k < kc) {
      const double2 x = X[c + (long long)k * ldx];
      digits8(x.x, e, dr);
      digits8(-x.y, e, di);
    } else {
#pragma unroll
      for (int t = 0; t < kOzS; ++t) dr[t] = di[t] = 0.f;
    }
#pragma unroll
    for (int t = 0; t < kOzS; ++t)
      *reinterpret_cast<__nv_bfloat162 *>(Bp + ((size_t)t * mc + c) * K + 2 * k) = __floats2bfloat162_rn(dr[t], di[t]);
  }
}

enum { kResidual = 0, kUpdate = 1, kProduct = 2, kNegTriu = 3 };

// One output tile (bx, by) of the product; pA, pB and args point into the
// kernel's parameter space (a plain launch, or one problem of a batch).
template <int MODE>
__device__ __forceinline__ void oz_gemm_tile(const CUtensorMap *pA, const CUtensorMap *pB, const OzArgs &args,
                                             int bx, int by) {
  using namespace tc;
  extern __shared__ uint8_t smem_raw[];
  uint8_t *base = smem_raw + ((1024 - (smem_u32(smem_raw) & 1023)) & 1023);
  uint8_t *sB = base;                         // 2 buffers x 32 KB
  uint8_t *sA = base + 2 * kOzBBytes;         // ring of kOzRing x 16 KB
  __shared__ uint64_t bfull[2], bempty[2], afull[kOzRing], aempty[kOzRing], accfull[2], accempty[2];
  __shared__ uint64_t mma_done;
  __shared__ uint32_t tmem_base;
  __shared__ int fail;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int i0 = (MODE == kUpdate ? args.row_lo : 0) + by * kOzBM;   // first real row
  const int j0 = bx * kOzBN;                                         // first local column
  // Residual: U is upper, so K' columns below the tile's first row vanish;
  // product with an upper-triangular B: K' rows past the tile's last column do.
  const int c_begin = MODE == kResidual ? i0 / kOzKC : 0;
  const int nch = MODE == kProduct && args.triu_b
                      ? min(args.K / kOzKC, (2 * (j0 + kOzBN) + kOzKC - 1) / kOzKC)
                      : args.K / kOzKC - c_begin;
  const int ax0 = MODE == kUpdate ? args.a_x0 : 0;

  if (warp == 0) tmem_alloc(&tmem_base, 512);
  if (threadIdx.x == 0) {
    for (int i = 0; i < 2; ++i) {
      mbar_init(&bfull[i], 1); mbar_init(&bempty[i], 1);
      mbar_init(&accfull[i], 1); mbar_init(&accempty[i], 32 * kOzEpi);
    }
    for (int i = 0; i < kOzRing; ++i) { mbar_init(&afull[i], 1); mbar_init(&aempty[i], 1); }
    mbar_init(&mma_done, 1);
    fail = 0;
    fence_barrier_init();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_base;
  auto wait = [&](uint64_t *bar, uint32_t parity) {
    const bool ok = mbar_wait(bar, parity, args.status, MSTS_STATUS_TIMEOUT);
    if (!ok) raise_status(args.status, MSTS_STATUS_TIMEOUT);   // tell the other CTAs at once
    return ok;
  };
  int a_issued = 0, b_issued = 0;             // TMA loads the producer issued

  if (warp == kOzEpi) {
    // ---------------- TMA producer ----------------
    if (lane == 0) {
      prefetch_tmap(pA);
      prefetch_tmap(pB);
      int ia = 0;
      for (int c = 0; c < nch; ++c) {
        const int kk = (c_begin + c) * kOzKC;
        const int bb = c & 1;
        if (c >= 2 && !wait(&bempty[bb], ((c >> 1) - 1) & 1)) { fail = 1; break; }
        mbar_arrive_expect_tx(&bfull[bb], kOzBBytes);
        tma_load_3d(sB + bb * kOzBBytes, pB, &bfull[bb], kk, j0, 0);
        ++b_issued;
        for (int s = 0; s < kOzS; ++s, ++ia) {
          const int slot = ia % kOzRing;
          if (ia >= kOzRing && !wait(&aempty[slot], ((ia / kOzRing) - 1) & 1)) { fail = 1; break; }
          mbar_arrive_expect_tx(&afull[slot], kOzABytes);
          tma_load_3d(sA + slot * kOzABytes, pA, &afull[slot], ax0 + kk, i0, s);
        }
        if (fail) break;
      }
      a_issued = ia;
    }
  } else if (warp == kOzEpi + 1) {
    // ---------------- MMA issuer ----------------
    if (lane == 0) {
      int ia = 0;
      for (int c = 0; c < nch && !fail; ++c) {
        const int bb = c & 1, ab = c & 1;
        if (c >= 2 && !wait(&accempty[ab], ((c >> 1) - 1) & 1)) { fail = 1; break; }
        if (!wait(&bfull[bb], (c >> 1) & 1)) { fail = 1; break; }
        tc_fence_after();
        const uint32_t bbase = smem_u32(sB + bb * kOzBBytes);
        const uint32_t dbase = tmem + ab * kOzAccCols;
        for (int s = 0; s < kOzS; ++s, ++ia) {
          const int slot = ia % kOzRing;
          if (!wait(&afull[slot], (ia / kOzRing) & 1)) { fail = 1; break; }
          tc_fence_after();
          const uint32_t abase = smem_u32(sA + slot * kOzABytes);
          // A plane s+1 against B planes 1..8-s at once: the B planes sit one
          // after another in shared memory and the diagonal accumulators one
          // after another in TMEM, so the N = 32 (8 - s) wide product written at
          // column 32 s puts (A_{s+1} B_{t+1}) into accumulator s + t.
          const uint32_t idesc_s = idesc_bf16(kOzBM, kOzBN * (kOzS - s));
          const uint32_t d = dbase + (uint32_t)(s * kOzBN);
#pragma unroll
          for (int k = 0; k < kOzKC / 16; ++k)
            mma_bf16(d, sdesc_k128(abase + 32 * k), sdesc_k128(bbase + 32 * k), idesc_s,
                     (s > 0 || k > 0) ? 1u : 0u);
          mma_commit(&aempty[slot]);                         // A plane consumed
        }
        if (fail) break;
        mma_commit(&bempty[bb]);                             // B planes consumed
        mma_commit(&accfull[ab]);                            // accumulators ready
      }
      // Drain: every MMA this thread issued has finished before TMEM is freed.
      mma_commit(&mma_done);
      if (!wait(&mma_done, 0)) fail = 1;
    }
  } else {
    // ---------------- epilogue: warp w reads TMEM lanes 32 (w mod 4).. (its
    // rows) and the kEC columns starting at kEC (w / 4) -------------------
    constexpr int kEC = kOzBN * 4 / kOzEpi;
    const int quarter = warp & 3, cg = warp >> 2;
    long long hi[kEC], lo[kEC];
#pragma unroll
    for (int j = 0; j < kEC; ++j) hi[j] = lo[j] = 0;
    const uint32_t lane_addr = (uint32_t)(32 * quarter) << 16;
    bool ok = true;
    for (int c = 0; c < nch; ++c) {
      const int ab = c & 1;
      // one decision per warp: the reads below are warp-wide (.sync.aligned)
      if (!__all_sync(0xffffffffu, wait(&accfull[ab], (c >> 1) & 1))) { ok = false; break; }
      tc_fence_after();
#pragma unroll
      for (int d = 0; d < kOzS; ++d) {                       // diagonal s + t = d + 2
        uint32_t v[kEC];
        tmem_ld16(tmem + lane_addr + ab * kOzAccCols + d * kOzBN + kEC * cg, v);
        tmem_ld_wait();
#pragma unroll
        for (int j = 0; j < kEC; ++j) {
          const long long q = (long long)__float2int_rn(__uint_as_float(v[j]));   // exact integer
          if (d <= 2) hi[j] += q << (kOzBits * (2 - d));
          else lo[j] += q << (kOzBits * (7 - d));
        }
      }
      tc_fence_before();
      mbar_arrive(&accempty[ab]);
    }
    if (!ok) fail = 1;
    // P = 2^(e_r + f_j) (hi 2^-28 + lo 2^-63)
    const int i = i0 + 32 * quarter + lane;                  // real row of A'
    const bool row_ok = MODE != kUpdate ? i < 2 * args.m : i < args.row_hi;
    if (ok && row_ok) {
      const int r = i >> 1, part = i & 1;
      const int er = args.rexp[r];
#pragma unroll
      for (int j = 0; j < kEC; ++j) {
        const int lc = j0 + kEC * cg + j;
        if (lc >= (MODE != kUpdate ? args.n : args.ncols)) continue;
        const double p = scalbn(fma((double)hi[j], 0x1p-28, (double)lo[j] * 0x1p-63), er + args.cexp[lc]);
        if (MODE == kProduct) {
          reinterpret_cast<double *>(args.R + r + (long long)lc * args.ldr)[part] = p;
        } else if (MODE == kNegTriu) {             // -triu(P): zero below the diagonal
          reinterpret_cast<double *>(args.R + r + (long long)lc * args.ldr)[part] = r <= lc ? -p : 0.0;
        } else if (MODE == kResidual) {
          const double2 x = args.X[r + (long long)lc * args.ldx];
          const double2 sj = args.s[lc];
          const double2 b = args.B[r + (long long)lc * args.ldb];
          const double sx = part ? fma(sj.x, x.y, sj.y * x.x) : fma(sj.x, x.x, -sj.y * x.y);
          double *out = reinterpret_cast<double *>(args.R + r + (long long)lc * args.ldr) + part;
          *out = ((part ? b.y : b.x) - p) + sx;
        } else {
          const int col = args.col_base + lc;
          double *out = reinterpret_cast<double *>(args.R + r + (long long)col * args.ldr) + part;
          double v = *out;
          if (args.pend) { const int pe = args.pend[col]; if (pe) v = dshift(v, pe); }
          *out = v - p;
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (fail) {
    // A wait gave up.  Before TMEM is freed and the CTA exits, the bulk copies
    // and MMAs it issued must have landed: wait for the last load into every
    // buffer and for the MMA drain, each with the time limit only (the abort
    // bit that the give-up set would end these waits at once).
    if (warp == kOzEpi && lane == 0) {
      for (int i = max(0, a_issued - kOzRing); i < a_issued; ++i)
        mbar_wait(&afull[i % kOzRing], (i / kOzRing) & 1);
      for (int i = max(0, b_issued - 2); i < b_issued; ++i) mbar_wait(&bfull[i & 1], (i >> 1) & 1);
    } else if (warp == kOzEpi + 1 && lane == 0) {
      mbar_wait(&mma_done, 0);
    }
    tc_fence_before();
    __syncthreads();
  }
  if (fail && threadIdx.x == 0) raise_status(args.status, MSTS_STATUS_TIMEOUT);
  if (warp == 0) tmem_dealloc(tmem, 512);
}

template <int MODE>
__global__ void __launch_bounds__(kOzThreads, 1)
k_oz_gemm(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
          const __grid_constant__ OzArgs args) {
  oz_gemm_tile<MODE>(&tmA, &tmB, args, blockIdx.x, blockIdx.y);
}

// The substitution step of a batch of problems in one launch: problem z =
// blockIdx.z with its own tensor maps and arguments; CTAs past a problem's
// tiles leave before any set-up.
struct OzBatch {
  CUtensorMap tmA[kMaxProbs];
  CUtensorMap tmB[kMaxProbs];
  OzArgs args[kMaxProbs];
  int tiles_n[kMaxProbs], tiles_m[kMaxProbs];
};

template <int MODE>
__global__ void __launch_bounds__(kOzThreads, 1) k_oz_batched(const __grid_constant__ OzBatch b) {
  const int z = blockIdx.z;
  if ((int)blockIdx.x >= b.tiles_n[z] || (int)blockIdx.y >= b.tiles_m[z]) return;
  if (MODE == kNegTriu) {                 // a tile wholly below the diagonal is zero: no product
    const OzArgs &a = b.args[z];
    const int r0 = blockIdx.y * (kOzBM / 2), c0 = blockIdx.x * kOzBN;
    if (r0 > c0 + kOzBN - 1) {
      for (int idx = threadIdx.x; idx < (kOzBM / 2) * kOzBN; idx += blockDim.x) {
        const int r = r0 + idx % (kOzBM / 2), c = c0 + idx / (kOzBM / 2);
        if (r < a.m && c < a.n) a.R[r + (long long)c * a.ldr] = make_double2(0.0, 0.0);
      }
      return;
    }
  }
  oz_gemm_tile<MODE>(&b.tmA[z], &b.tmB[z], b.args[z], blockIdx.x, blockIdx.y);
}

// ----- host side -------------------------------------------------------------
// A status word of the library's own for calls made without one (the bounded
// waits still need somewhere to publish a timeout to the other CTAs).  It is
// cleared on the call's stream before every such call, so a timeout of one
// call never makes a later one give up; its address is looked up once per
// device, with that device current.  Calls without a status word that overlap
// on the GPU (different streams) share it: a timeout in one may end the waits
// of the other early, which that call cannot report either.
__device__ uint32_t g_oz_abort_word;
constexpr int kAbortDevices = 64;
static std::mutex g_abort_mu;
static uint32_t *g_abort_addr[kAbortDevices] = {};
uint32_t *ozaki_call_status(uint32_t *status, cudaStream_t st) {
  if (status) return status;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kAbortDevices) return nullptr;
  uint32_t *p = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_abort_mu);
    if (!g_abort_addr[dev]) {
      void *a = nullptr;
      if (cudaGetSymbolAddress(&a, g_oz_abort_word) == cudaSuccess) g_abort_addr[dev] = static_cast<uint32_t *>(a);
    }
    p = g_abort_addr[dev];
  }
  if (p && cudaMemsetAsync(p, 0, sizeof(uint32_t), st) != cudaSuccess) return nullptr;
  return p;
}
// Host-side fault injection for the tests: ORs `bits` into the library's
// status word for calls made without one, on the current device, ordered on
// `stream` (the bits stay until the next call without a status word clears
// the word).  Returns 0 or MSTS_ERR_CUDA.
extern "C" int msts_inject_fallback_status(uint32_t bits, void *stream) {
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kAbortDevices) return MSTS_ERR_CUDA;
  uint32_t *p = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_abort_mu);
    if (!g_abort_addr[dev]) {
      void *a = nullptr;
      if (cudaGetSymbolAddress(&a, g_oz_abort_word) == cudaSuccess) g_abort_addr[dev] = static_cast<uint32_t *>(a);
    }
    p = g_abort_addr[dev];
  }
  if (!p) return MSTS_ERR_CUDA;
  uint32_t cur = 0;
  if (cudaMemcpyAsync(&cur, p, sizeof(uint32_t), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return MSTS_ERR_CUDA;
  cur |= bits;
  if (cudaMemcpyAsync(p, &cur, sizeof(uint32_t), cudaMemcpyHostToDevice, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return MSTS_ERR_CUDA;
  return 0;
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *,
                                  const cuuint64_t *, const cuuint64_t *, const cuuint32_t *,
                                  const cuuint32_t *, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess && q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
  });
  return fn;
}

// 3-D map over digit planes: dims (K, rows, kOzS), box (64, box_rows, box_planes).
static bool make_map(CUtensorMap *map, void *ptr, int K, int rows, int box_rows, int box_planes) {
  EncodeTiledFn enc = encode_fn();
  if (!enc) return false;
  const cuuint64_t dims[3] = {(cuuint64_t)K, (cuuint64_t)rows, (cuuint64_t)kOzS};
  const cuuint64_t strides[2] = {(cuuint64_t)K * 2, (cuuint64_t)K * 2 * (cuuint64_t)rows};
  const cuuint32_t box[3] = {(cuuint32_t)kOzKC, (cuuint32_t)box_rows, (cuuint32_t)box_planes};
  const cuuint32_t es[3] = {1, 1, 1};
  return enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, ptr, dims, strides, box, es,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

cudaError_t ozaki_prepare(const double2 *U, long long ldu, int m, int n, void *ws, cudaStream_t st) {
  OzakiBufs o = carve(ws, m, n);
  k_oz_rowexp<<<(m + 7) / 8, 256, 0, st>>>(U, ldu, m, m, o.rexp, 0);
  k_oz_slice_A<<<dim3((o.K / 2 + 255) / 256, m), 256, 0, st>>>(U, ldu, m, m, o.rexp, o.Ap, o.K, 0);
  count_launches(2);
  return cudaGetLastError();
}

cudaError_t ozaki_residual(const double2 *U, long long ldu, int m, const double2 *s, int n,
                           const double2 *B, long long ldb, const double2 *X, long long ldx,
                           double2 *R, long long ldr, void *ws, uint32_t *status, cudaStream_t st) {
  (void)U; (void)ldu;
  OzakiBufs o = carve(ws, m, n);
  k_oz_slice_B<<<n, 256, 0, st>>>(X, ldx, m, n, o.cexp, o.Bp, o.K, 0);
  count_launches(1);
  CUtensorMap tmA, tmB;
  if (!make_map(&tmA, o.Ap, o.K, 2 * m, kOzBM, 1) || !make_map(&tmB, o.Bp, o.K, n, kOzBN, kOzS))
    return cudaErrorNotSupported;
  OzArgs a{};
  a.B = B; a.ldb = ldb; a.X = X; a.ldx = ldx; a.s = s; a.R = R; a.ldr = ldr;
  a.rexp = o.rexp; a.cexp = o.cexp; a.m = m; a.n = n; a.K = o.K; a.status = ozaki_call_status(status, st);
  if (!status && a.status) {
    const cudaError_t ce = cudaMemsetAsync(a.status, 0, sizeof(uint32_t), st);
    if (ce != cudaSuccess) return ce;
  }
  cudaError_t e = cudaFuncSetAttribute(k_oz_gemm<kResidual>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kOzSmem);
  if (e != cudaSuccess) return e;
  // BF16 MMA FLOPs issued: per tile, (K/64 - first chunk) chunks of 36 digit
  // pairs x 4 K-steps of 128 x 32 x 16.
  double mma_flops = 0.0;
  const int tiles_n = (n + kOzBN - 1) / kOzBN, tiles_m = (2 * m + kOzBM - 1) / kOzBM;
  for (int y = 0; y < tiles_m; ++y)
    mma_flops += (double)(o.K / kOzKC - (y * kOzBM) / kOzKC) * tiles_n;
  mma_flops *= 36.0 * (kOzKC / 16) * 2.0 * kOzBM * kOzBN * 16;
  void *h = trace_on() ? trace_start(3, mma_flops, (double)kOzS * (2.0 * m * o.K + (double)n * o.K), st)
                       : nullptr;
  k_oz_gemm<kResidual><<<dim3((n + kOzBN - 1) / kOzBN, (2 * m + kOzBM - 1) / kOzBM), kOzThreads, kOzSmem, st>>>(tmA, tmB, a);
  trace_stop(h, st);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t ozaki_product(const double2 *A, long long lda, int m, const double2 *Bm, long long ldbm, int n,
                          bool triu_b, double2 *C, long long ldc, void *ws, uint32_t *status, cudaStream_t st) {
  if (m == 0 || n == 0) return cudaSuccess;
  OzakiBufs o = carve(ws, m, n);
  k_oz_rowexp<<<(m + 7) / 8, 256, 0, st>>>(A, lda, m, m, o.rexp, 1);
  k_oz_slice_A<<<dim3((o.K / 2 + 255) / 256, m), 256, 0, st>>>(A, lda, m, m, o.rexp, o.Ap, o.K, 1);
  k_oz_slice_B<<<n, 256, 0, st>>>(Bm, ldbm, m, n, o.cexp, o.Bp, o.K, triu_b ? 1 : 0);
  count_launches(3);
  CUtensorMap tmA, tmB;
  if (!make_map(&tmA, o.Ap, o.K, 2 * m, kOzBM, 1) || !make_map(&tmB, o.Bp, o.K, n, kOzBN, kOzS))
    return cudaErrorNotSupported;
  OzArgs a{};
  a.R = C; a.ldr = ldc;
  a.rexp = o.rexp; a.cexp = o.cexp; a.m = m; a.n = n; a.K = o.K; a.triu_b = triu_b ? 1 : 0;
  a.status = ozaki_call_status(status, st);
  cudaError_t e = cudaFuncSetAttribute(k_oz_gemm<kProduct>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kOzSmem);
  if (e != cudaSuccess) return e;
  // BF16 MMA FLOPs issued: per tile, its K' chunks of 36 digit pairs x 4
  // K-steps of 128 x 32 x 16.
  double chunks = 0.0;
  const int tiles_n = (n + kOzBN - 1) / kOzBN, tiles_m = (2 * m + kOzBM - 1) / kOzBM;
  for (int x = 0; x < tiles_n; ++x)
    chunks += triu_b ? std::min(o.K / kOzKC, (2 * (x * kOzBN + kOzBN) + kOzKC - 1) / kOzKC) : o.K / kOzKC;
  const double mma_flops = chunks * tiles_m * 36.0 * (kOzKC / 16) * 2.0 * kOzBM * kOzBN * 16;
  void *h = trace_on() ? trace_start(2, mma_flops, (double)kOzS * (2.0 * m * o.K + (double)n * o.K), st)
                       : nullptr;
  k_oz_gemm<kProduct><<<dim3(tiles_n, tiles_m), kOzThreads, kOzSmem, st>>>(tmA, tmB, a);
  trace_stop(h, st);
  count_launches(1);
  return cudaGetLastError();
}

// ===========================================================================
// Substitution step of the blocked solve on the tensor cores.
//
// Block layout of the A digit planes: block b (rows [lo_b, hi_b) of U) owns
// K' columns [b KB, b KB + 2 (hi_b - lo_b)) of every plane (zero-padded to KB,
// a multiple of 64), so each block's panel starts on a 128-byte TMA boundary.
//  upper (Alg. 3/5): A'(2r.., b KB + 2(k - lo_b)) from U(r, k), r < lo_b;
//  conj (forward substitution with U^H): from conj(U(k, r)), r >= hi_b.
// Row exponents are per (block, row): rexp[b m + r] over the block's columns,
// which keeps the digits of each panel as fine as the panel itself allows.
// ===========================================================================
// Panel width in K' of one block: 2 real columns per complex column, twice as
// many for a generalized problem ([U | V] against [X; -lambda X]).
static int kb_of(int nb, bool gen) { return (((gen ? 4 : 2) * nb + kOzKC - 1) / kOzKC) * kOzKC; }

size_t ozaki_plan_bytes(int m, int n, int nb, bool gen) {
  const int nblk = (m + nb - 1) / nb, KB = kb_of(nb, gen);
  return a256((size_t)kOzS * 2 * m * (size_t)nblk * KB * 2) + a256(4 * (size_t)nblk * m) +
         a256((size_t)kOzS * n * KB * 2) + a256(4 * (size_t)n);
}

// With V (generalized problem, upper only) the panel row is
// [U(r, lo:hi) | V(r, lo:hi)], one exponent for both halves.
// Row r of block b's panel: its exponent and its 8 digit planes (one warp).
template <bool CONJ>
__device__ __forceinline__ void ozs_prepare_row(const double2 *U, long long ldu, const double2 *V, long long ldv,
                                                int m, int nb, int KB, int nblk, __nv_bfloat16 *planes, int *rexp,
                                                int b, int r) {
  const int lane = threadIdx.x & 31;
  const int hi = m - b * nb, lo = hi - nb < 0 ? 0 : hi - nb, w = hi - lo;
  const bool used = CONJ ? r >= hi : r < lo;
  // Rows that the substitution of this block never updates are left unwritten:
  // the update reads only used rows (others at most fill a tile whose outputs
  // are masked, and an MMA row depends on its own A row only).
  if (!used) return;                                   // warp-uniform (one warp per row)
  const int wt = V ? 2 * w : w;                        // complex columns of the panel
  auto entry = [&](int k) {   // the complex entry of A' row r at column k of the block
    if (k >= wt) return make_double2(0.0, 0.0);
    if (k >= w) return V[r + (long long)(lo + k - w) * ldv];
    return CONJ ? zconj(U[(lo + k) + (long long)r * ldu]) : U[r + (long long)(lo + k) * ldu];
  };
  int e = -(1 << 29);
  for (int k = lane; k < wt; k += 32) e = max(e, bound_exp(entry(k)));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) e = max(e, __shfl_xor_sync(0xffffffffu, e, o));
  if (e < -(1 << 28)) e = 0;
  if (lane == 0) rexp[(size_t)b * m + r] = e;
  const size_t rows = 2 * (size_t)m, width = (size_t)nblk * KB;
  for (int k = lane; 2 * k < KB; k += 32) {
    float dr[kOzS], di[kOzS];
    const double2 u = entry(k);
    digits8(u.x, e, dr);
    digits8(u.y, e, di);
#pragma unroll
    for (int q = 0; q < kOzS; ++q) {
      const size_t col = (size_t)b * KB + 2 * k;
      *reinterpret_cast<__nv_bfloat162 *>(planes + (q * rows + 2 * (size_t)r) * width + col) =
          __floats2bfloat162_rn(dr[q], -di[q]);
      *reinterpret_cast<__nv_bfloat162 *>(planes + (q * rows + 2 * (size_t)r + 1) * width + col) =
          __floats2bfloat162_rn(di[q], dr[q]);
    }
  }
}

template <bool CONJ>
__global__ void k_ozs_prepare(const double2 *U, long long ldu, const double2 *V, long long ldv, int m, int nb,
                              int KB, __nv_bfloat16 *planes, int *rexp) {
  const int r = blockIdx.y * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (r >= m) return;
  ozs_prepare_row<CONJ>(U, ldu, V, ldv, m, nb, KB, gridDim.x, planes, rexp, blockIdx.x, r);
}
// The planes of every problem of a batch in one launch (problem in grid.z).
struct OzPrepItem {
  const double2 *U;
  long long ldu;
  int m, nb, KB, nblk;
  __nv_bfloat16 *planes;
  int *rexp;
};
struct OzPrepTable {
  OzPrepItem p[kMaxProbs];
};
// Each CTA walks (block, 8-row group) pairs of its problem with a grid stride,
// so that the grid is sized by the work rather than by the largest problem.
template <bool CONJ>
__global__ void k_ozs_prepare_batched(const __grid_constant__ OzPrepTable t) {
  const OzPrepItem &q = t.p[blockIdx.z];
  const int groups = (q.m + 7) / 8, items = groups * q.nblk, warp = threadIdx.x >> 5;
  for (int w = blockIdx.x; w < items; w += gridDim.x) {
    const int b = w % q.nblk, r = (w / q.nblk) * 8 + warp;
    if (r < q.m) ozs_prepare_row<CONJ>(q.U, q.ldu, nullptr, 0, q.m, q.nb, q.KB, q.nblk, q.planes, q.rexp, b, r);
  }
}

// Digit planes of X(lo:hi, jstart + c) for this block step: plane t, local
// column c, K' = 2 (k - lo) + {0,1}; one warp per column.  With lam
// (generalized problem) the column is [X(lo:hi, j); -lam_j X(lo:hi, j)],
// lam_j = lam[j lam_stride], the products rounded once in FP64.
__global__ void k_ozs_slice_X(const double2 *B, long long ldb, int lo, int w, int jstart, int ncols,
                              int KB, __nv_bfloat16 *bp, int *cexp, const double2 *lam, long long lam_stride) {
  const int lane = threadIdx.x & 31;
  const int c = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (c >= ncols) return;
  const double2 *col = B + (long long)(jstart + c) * ldb + lo;
  const double2 nl = lam ? lam[(long long)(jstart + c) * lam_stride] : make_double2(0.0, 0.0);
  const double2 mlam = make_double2(-nl.x, -nl.y);
  const int wt = lam ? 2 * w : w;
  auto entry = [&](int k) {
    if (k >= wt) return make_double2(0.0, 0.0);
    return k < w ? col[k] : zmul_rn(mlam, col[k - w]);
  };
  int e = -(1 << 29);
  for (int k = lane; k < wt; k += 32) e = max(e, bound_exp(entry(k)));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) e = max(e, __shfl_xor_sync(0xffffffffu, e, o));
  if (e < -(1 << 28)) e = 0;
  if (lane == 0) cexp[c] = e;
  for (int k = lane; 2 * k < KB; k += 32) {
    float dr[kOzS], di[kOzS];
    const double2 x = entry(k);
    digits8(x.x, e, dr);
    digits8(x.y, e, di);
#pragma unroll
    for (int t = 0; t < kOzS; ++t)
      *reinterpret_cast<__nv_bfloat162 *>(bp + ((size_t)t * ncols + c) * KB + 2 * k) =
          __floats2bfloat162_rn(dr[t], di[t]);
  }
}

cudaError_t ozaki_plan_init(OzPlan *plan, int m, int n, int nb, bool conj, void *ws, bool gen) {
  if (gen && conj) return cudaErrorInvalidValue;
  const int nblk = (m + nb - 1) / nb, KB = kb_of(nb, gen);
  char *c = static_cast<char *>(ws);
  plan->planes = reinterpret_cast<__nv_bfloat16 *>(c); c += a256((size_t)kOzS * 2 * m * (size_t)nblk * KB * 2);
  plan->rexp = reinterpret_cast<int *>(c); c += a256(4 * (size_t)nblk * m);
  plan->bp = reinterpret_cast<__nv_bfloat16 *>(c); c += a256((size_t)kOzS * n * KB * 2);
  plan->cexp = reinterpret_cast<int *>(c);
  plan->m = m; plan->nb = nb; plan->nblk = nblk; plan->KB = KB; plan->nmax = n; plan->conj = conj;
  if (!make_map(&plan->tmA, plan->planes, nblk * KB, 2 * m, kOzBM, 1)) return cudaErrorNotSupported;
  if (n > 0 && !make_map(&plan->tmB, plan->bp, KB, n, kOzBN, kOzS)) return cudaErrorNotSupported;
  return cudaSuccess;
}

cudaError_t ozaki_plan_prepare(OzPlan *plan, const double2 *U, long long ldu, int m, int n, int nb,
                               bool conj, void *ws, cudaStream_t st, const double2 *V, long long ldv) {
  cudaError_t e = ozaki_plan_init(plan, m, n, nb, conj, ws, V != nullptr);
  if (e != cudaSuccess) return e;
  const dim3 grid(plan->nblk, (m + 7) / 8);
  if (conj) k_ozs_prepare<true><<<grid, 256, 0, st>>>(U, ldu, nullptr, 0, m, nb, plan->KB, plan->planes, plan->rexp);
  else k_ozs_prepare<false><<<grid, 256, 0, st>>>(U, ldu, V, ldv, m, nb, plan->KB, plan->planes, plan->rexp);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t ozaki_plans_prepare(const OzPlanSrc *src, int count, cudaStream_t st) {
  for (int base = 0; base < count; base += kMaxProbs) {
    const int cnt = std::min(kMaxProbs, count - base);
    for (int conj = 0; conj < 2; ++conj) {
      OzPrepTable t;
      int k = 0, maxm = 0, maxb = 0;
      for (int i = 0; i < cnt; ++i) {
        const OzPlanSrc &q = src[base + i];
        if (q.plan->conj != (conj != 0) || q.plan->m == 0) continue;
        t.p[k++] = OzPrepItem{q.U, q.ldu, q.plan->m, q.plan->nb, q.plan->KB, q.plan->nblk, q.plan->planes,
                              q.plan->rexp};
        maxm = std::max(maxm, q.plan->m);
        maxb = std::max(maxb, q.plan->nblk);
      }
      if (k == 0) continue;
      const int items = maxb * ((maxm + 7) / 8);
      const dim3 grid(std::min(items, 4 * kNumSMsOz), 1, k);
      if (conj) k_ozs_prepare_batched<true><<<grid, 256, 0, st>>>(t);
      else k_ozs_prepare_batched<false><<<grid, 256, 0, st>>>(t);
      count_launches(1);
      const cudaError_t e = cudaGetLastError();
      if (e != cudaSuccess) return e;
    }
  }
  return cudaSuccess;
}

// W 2^ex rounded to the nearest double, assembled with integer operations
// (exponent field and rounded 53-bit significand) so that the conversion and
// the scaling cost no FP64 instruction; |W| < 2^62.  Outside the normal range
// it falls back to FP64 scalbn.
__device__ __forceinline__ double i64_ldexp_slow(long long W, int ex) { return scalbn((double)W, ex); }
__device__ __forceinline__ double i64_ldexp(long long W, int ex) {
  const unsigned long long a = W < 0 ? 0ull - (unsigned long long)W : (unsigned long long)W;
  const int lz = __clzll((long long)a);                // 64 when W == 0
  const int E = 1023 + 63 - lz + ex;                   // biased exponent of the result
  if (a != 0 && (E <= 0 || E >= 2046)) return i64_ldexp_slow(W, ex);
  const unsigned long long nrm = a << (lz & 63);       // leading one at bit 63
  unsigned long long sig = nrm >> 11;                  // 53 bits, leading one at bit 52
  const unsigned long long rest = nrm & 0x7ffull;      // the 11 bits rounded away
  sig += (rest > 0x400ull || (rest == 0x400ull && (sig & 1ull))) ? 1ull : 0ull;   // nearest, ties to even
  // (E - 1) << 52 plus the significand with its leading one adds that one into
  // the exponent field; a rounding carry to 2^53 moves it up one more.
  const unsigned long long bits = ((unsigned long long)(E - 1) << 52) + sig;
  return a == 0 ? 0.0 : __longlong_as_double((long long)(bits | (W < 0 ? 0x8000000000000000ull : 0ull)));
}

// Exact integer value of an FP32 accumulator holding an integer of magnitude
// below 2^22, without a conversion instruction: adding 1.5 2^23 puts it in the
// low mantissa bits.
__device__ __forceinline__ int f32_small_int(uint32_t f) {
  return __float_as_int(__uint_as_float(f) + 12582912.0f) - 0x4B400000;
}

// a 2^7 + b for two such accumulators, the two offsets folded into one.
__device__ __forceinline__ int f32_small_pair(uint32_t a, uint32_t b) {
  const int ia = __float_as_int(__uint_as_float(a) + 12582912.0f);
  const int ib = __float_as_int(__uint_as_float(b) + 12582912.0f);
  // modulo 2^32 (the result fits an int32)
  return (int)((uint32_t)ia * (1u << kOzBits) + (uint32_t)ib - 0x4B400000u * ((1u << kOzBits) + 1u));
}

// W = P01 2^35 + P23 2^21 + P45 2^7 + floor(P67 / 2^7) as two 32-bit words
// (h signed high word, l low word): two wide multiply-adds (the multiply-add
// pipe, which the epilogue leaves mostly idle) and one add of the top term.
__device__ __forceinline__ void fold_w(int P01, int P23, int P45, int P67, int &h, uint32_t &l) {
  long long t;
  asm("mad.wide.s32 %0, %1, %2, %3;" : "=l"(t) : "r"(P45), "r"(1 << 7), "l"((long long)(P67 >> 7)));
  asm("mad.wide.s32 %0, %1, %2, %3;" : "=l"(t) : "r"(P23), "r"(1 << 21), "l"(t));
  h = (int)(t >> 32) + (P01 << 3);                     // |P01| < 2^28: no overflow
  l = (uint32_t)t;
}

// (h, l) 2^ex rounded to the nearest double (ties to even), from 32-bit
// integer operations only; |W| < 2^62.  Sets slow when the result leaves the
// normal range, and for 0 < |W| < 2^32 (rare: a product 2^-24 below its
// digit scale), so that the normalisation needs one leading-zero count: the
// caller then uses i64_ldexp, which gives the same value.
__device__ __forceinline__ double w_ldexp_fast(int h, uint32_t l, int ex, bool &slow) {
  const uint32_t sg = (uint32_t)(h >> 31);              // 0 or all ones
  uint32_t al, ah;                                      // |W| = (W ^ sg) - sg
  asm("{\n\t"
      "sub.cc.u32 %0, %2, %4;\n\t"
      "subc.u32 %1, %3, %4;\n\t"
      "}"
      : "=r"(al), "=r"(ah)
      : "r"(l ^ sg), "r"((uint32_t)h ^ sg), "r"(sg));
  const bool zero = (ah | al) == 0u;
  const int lz = __clz((int)ah) & 31;                   // ah != 0 on the fast path
  const int E = 1023 + 63 - lz + ex;                    // biased exponent
  slow |= !zero && (ah == 0u || (unsigned)(E - 1) >= 2045u);
  const uint32_t th = __funnelshift_l(al, ah, lz), tl = al << lz;   // normalised: bit 63 set
  const uint32_t sh = th >> 11, sl0 = __funnelshift_r(tl, th, 11);  // 53-bit significand
  const uint32_t inc = ((tl & 0x7ffu) + 0x3ffu + (sl0 & 1u)) >> 11;  // nearest, ties to even
  uint32_t sl, rh = sh;
  asm("{\n\t"
      "add.cc.u32 %0, %2, %3;\n\t"
      "addc.u32 %1, %1, 0;\n\t"
      "}"
      : "=r"(sl), "+r"(rh)
      : "r"(sl0), "r"(inc));
  // (E - 1) << 20 plus the significand with its leading one adds that one into
  // the exponent field; a rounding carry to 2^53 moves it up one more.
  rh = (((uint32_t)(E - 1) << 20) + rh) | ((uint32_t)h & 0x80000000u);
  return __hiloint2double(zero ? 0 : (int)rh, zero ? 0 : (int)sl);
}

// One output of the update through the FP64 routines (the rare cases that
// leave the normal range); kept out of line so that the common path carries
// none of its instructions.
__device__ __noinline__ double update_out_slow(double v, int pe, int h, uint32_t l, int ex) {
  const long long W = (long long)(((unsigned long long)(uint32_t)h << 32) | l);
  return (pe ? dshift(v, pe) : v) - i64_ldexp(W, ex);
}

// Persistent form of the substitution step for one 64-wide K chunk per block
// (n_b <= 32): each CTA walks a contiguous run of output tiles in row-major
// order, keeping the 8 A digit planes of its current row tile resident in
// shared memory (reloaded only when the row tile changes) while the B planes of
// successive column tiles stream through two buffers; TMEM accumulators are
// double-buffered so the epilogue of one tile overlaps the MMAs of the next.
// The epilogue folds the 8 diagonal sums into one int64
// W = sum_d D_d 2^(42 - 7d) (exact for d <= 6, the last diagonal truncated
// below 2^-56; |W| < 2^62 because every digit expansion is below 1) and applies
// B = 2^-pend B - W 2^(e_r + f_j - 56) with a single FP64 subtraction.
//
// The same kernel with NP = 3 planes (kOzLpPlanes) is the low-precision
// substitution product of the mixed-precision solve: each operand keeps its 3
// leading 7-bit digit planes (a split of every entry into 3 BF16 pieces, 21
// bits below the row's or column's power of two), the 6 plane pairs with
// s + t <= 4 are multiplied with FP32 accumulation in TMEM, and the epilogue
// sums the 3 diagonals in FP32 and subtracts the product from B in FP64:
// accurate to about 2^-20 relative to K' max|U(r,:)| max|X(:,j)|, the
// accuracy class of an FP32 product, which the FP64 refinement then corrects.
constexpr int kOzLpPlanes = 3;
template <int NP>
constexpr size_t ozu_smem() {
  return (size_t)NP * kOzABytes + 2 * (size_t)NP * kOzBN * kOzKC * 2 + 1024;
}
constexpr int kOzPersistentCtas = 152;             // one CTA per SM
constexpr int kOzuEpiWarps = 16;                   // epilogue warps (4 per sub-partition)
constexpr int kOzuThreads = 32 * kOzuEpiWarps + 64; // + producer + MMA

// float f times 2^ex as a double from the IEEE fields (exact: every float is a
// double); `slow` is set when f is subnormal or the result leaves the normal range.
__device__ __forceinline__ double f32_ldexp(float f, int ex, bool &slow) {
  const uint32_t u = __float_as_uint(f);
  const int e8 = (int)((u >> 23) & 0xffu);
  const uint32_t man = u & 0x7fffffu;
  const int E = e8 - 127 + 1023 + ex;
  slow |= (e8 == 0 && man != 0u) || (e8 != 0 && (E <= 0 || E >= 2047));
  if (e8 == 0) return __hiloint2double((int)(u & 0x80000000u), 0);   // +-0
  return __hiloint2double((int)((u & 0x80000000u) | ((uint32_t)E << 20) | (man >> 3)), (int)(man << 29));
}
__device__ __noinline__ double update_out_slow_lp(double v, int pe, float W, int ex) {
  return (pe ? dshift(v, pe) : v) - scalbn((double)W, ex);
}

// The tiles of one launch: MAXP problems' output tiles (each row-major over its
// row and column tiles), concatenated; tile t belongs to the problem p with
// tile_base[p] <= t < tile_base[p + 1].  One problem for the substitution
// step of a single solve, every problem of a batch for a batched one.
template <int MAXP>
struct OzUpdTab {
  CUtensorMap tmA[MAXP];
  CUtensorMap tmB[MAXP];
  OzArgs args[MAXP];
  int tiles_n[MAXP], tile_base[MAXP + 1];
  int tiles_total;
};

// Position of tile t in its problem, for tiles visited in increasing order:
// row-major over the rectangle of row and column tiles, or (TRI) over the
// tiles that meet the upper triangle of an m x m output, row tile rt holding
// the column tiles 2 rt .. tiles_n - 1 (a row tile spans 64 complex rows).
template <int MAXP, bool TRI>
struct TileCursor {
  int p = 0, rt = 0, rs = 0, cnt = -1;
  __device__ __forceinline__ void at(const OzUpdTab<MAXP> &T, int t, int &prob, int &row_t, int &col_t) {
    const int p0 = p;
    if constexpr (MAXP > 1)
      while (t >= T.tile_base[p + 1]) ++p;
    const int lt = t - T.tile_base[p], tn = T.tiles_n[p];
    if constexpr (!TRI) {
      row_t = lt / tn;
      col_t = lt - row_t * tn;
    } else {
      if (p != p0 || cnt < 0) { rt = 0; rs = 0; cnt = tn; }
      while (lt >= rs + cnt) { rs += cnt; ++rt; cnt = max(0, tn - 2 * rt); }
      row_t = rt;
      col_t = 2 * rt + (lt - rs);
    }
    prob = p;
  }
};

// TRI: the adjoint's dU = -triu(P) (P = L X^H, nothing read from the output):
// the tiles meeting the upper triangle, each output -P, strictly lower
// entries 0 (the tiles wholly below the diagonal are zeroed apart).
template <int NP, int MAXP, bool TRI = false>
__global__ void __launch_bounds__(kOzuThreads, 1) k_oz_update(const __grid_constant__ OzUpdTab<MAXP> T) {
  using namespace tc;
  static_assert(NP == kOzS || NP == kOzLpPlanes, "8 planes (FP64-accurate) or 3 (low precision)");
  constexpr uint32_t kBBytes = (uint32_t)NP * kOzBN * kOzKC * 2;   // B planes of one tile
  constexpr int kAcc = NP * kOzBN;                                  // TMEM columns per buffer
  constexpr uint32_t kTmemCols = 2 * kAcc > 256 ? 512 : 256;
  extern __shared__ uint8_t smem_raw[];
  uint8_t *base = smem_raw + ((1024 - (smem_u32(smem_raw) & 1023)) & 1023);
  uint8_t *sA = base;                               // NP resident A planes x 16 KB
  uint8_t *sB = base + NP * kOzABytes;              // 2 buffers of NP B planes
  __shared__ uint64_t afull, aempty, bfull[2], bempty[2], accfull[2], accempty[2], mma_done;
  __shared__ uint32_t tmem_base;
  __shared__ int fail;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int per = (T.tiles_total + gridDim.x - 1) / gridDim.x;
  const int t0 = blockIdx.x * per, t1 = min(T.tiles_total, t0 + per);
  uint32_t *const status = T.args[0].status;       // one status word for the launch

  if (warp == 0) tmem_alloc(&tmem_base, kTmemCols);
  if (threadIdx.x == 0) {
    mbar_init(&afull, 1);
    mbar_init(&aempty, 1);
    mbar_init(&mma_done, 1);
    for (int i = 0; i < 2; ++i) {
      mbar_init(&bfull[i], 1);
      mbar_init(&bempty[i], 1);
      mbar_init(&accfull[i], 1);
      mbar_init(&accempty[i], 32 * kOzuEpiWarps);
    }
    fail = 0;
    fence_barrier_init();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_base;
  auto wait = [&](uint64_t *bar, uint32_t parity) {
    const bool ok = mbar_wait(bar, parity, status, MSTS_STATUS_TIMEOUT);
    if (!ok) raise_status(status, MSTS_STATUS_TIMEOUT);
    return ok;
  };
  int a_issued = 0, b_issued = 0;                   // A reloads and B loads the producer issued

  if (warp == kOzuEpiWarps) {
    if (lane == 0) {                                // ---------------- TMA producer
      if (MAXP == 1) {
        prefetch_tmap(&T.tmA[0]);
        prefetch_tmap(&T.tmB[0]);
      }
      pdl_wait();                                   // the X planes come from the diagonal step
      int prev_rt = -1, prev_p = -1, na = 0;
      TileCursor<MAXP, TRI> cur;
      for (int t = t0, k = 0; t < t1; ++t, ++k) {
        int p, rt, ct;
        cur.at(T, t, p, rt, ct);
        if (rt != prev_rt || p != prev_p) {         // new row tile: reload the A planes
          if (na > 0 && !wait(&aempty, (na - 1) & 1)) { fail = 1; break; }
          mbar_arrive_expect_tx(&afull, NP * kOzABytes);
          for (int q = 0; q < NP; ++q)
            tma_load_3d(sA + q * kOzABytes, &T.tmA[p], &afull, T.args[p].a_x0, T.args[p].row_lo + rt * kOzBM, q);
          ++na;
          prev_rt = rt;
          prev_p = p;
        }
        const int bb = k & 1;
        if (k >= 2 && !wait(&bempty[bb], ((k >> 1) - 1) & 1)) { fail = 1; break; }
        mbar_arrive_expect_tx(&bfull[bb], kBBytes);
        tma_load_3d(sB + bb * kBBytes, &T.tmB[p], &bfull[bb], 0, ct * kOzBN, 0);
        ++b_issued;
      }
      a_issued = na;
    }
  } else if (warp == kOzuEpiWarps + 1) {
    if (lane == 0) {                                // ---------------- MMA issuer
      // wait in hardware for the diagonal step rather than spinning on the
      // first barrier beside its CTAs
      pdl_wait();
      int prev_rt = -1, prev_p = -1, na = 0;
      TileCursor<MAXP, TRI> cur;
      for (int t = t0, k = 0; t < t1 && !fail; ++t, ++k) {
        int p, rt, ct;
        cur.at(T, t, p, rt, ct);
        if (rt != prev_rt || p != prev_p) {
          if (na > 0) mma_commit(&aempty);          // old planes free once their MMAs finish
          if (!wait(&afull, na & 1)) { fail = 1; break; }
          ++na;
          prev_rt = rt;
          prev_p = p;
        }
        const int bb = k & 1, ab = k & 1;
        if (k >= 2 && !wait(&accempty[ab], ((k >> 1) - 1) & 1)) { fail = 1; break; }
        if (!wait(&bfull[bb], (k >> 1) & 1)) { fail = 1; break; }
        tc_fence_after();
        const uint32_t bbase = smem_u32(sB + bb * kBBytes);
        const uint32_t dbase = tmem + ab * kAcc;
        for (int q = 0; q < NP; ++q) {
          // A plane q+1 against B planes 1..NP-q at once (N = 32 (NP - q)
          // written at column 32 q), as in the chunked kernel above.
          const uint32_t abase = smem_u32(sA + q * kOzABytes);
          const uint32_t idesc_q = idesc_bf16(kOzBM, kOzBN * (NP - q));
#pragma unroll
          for (int kk = 0; kk < kOzKC / 16; ++kk)
            mma_bf16(dbase + (uint32_t)(q * kOzBN), sdesc_k128(abase + 32 * kk), sdesc_k128(bbase + 32 * kk),
                     idesc_q, (q > 0 || kk > 0) ? 1u : 0u);
        }
        mma_commit(&bempty[bb]);
        mma_commit(&accfull[ab]);
      }
      mma_commit(&mma_done);                        // drain before TMEM is freed
      if (!wait(&mma_done, 0)) fail = 1;
    }
  } else {                                          // ---------------- epilogue warps
    // Warp w reads TMEM lanes 32 (w mod 4) .. + 31 (its rows) and kCW columns
    // of every tile starting at kCW (w / 4).  Everything a tile reads from
    // memory (its B values, column and row exponents) is fetched while the
    // previous tile is processed, so no memory latency sits between tiles.
    const int quarter = warp & 3, cgroup = warp >> 2;
    const uint32_t lane_addr = (uint32_t)(32 * quarter) << 16;
    constexpr int kCW = kOzBN * 4 / kOzuEpiWarps, kQ = 4, kPasses = kCW / kQ;
    struct TileIn {
      double b[kCW];                                // B(row, columns of this warp)
      double *base;                                 // &B(row, first column of this warp)
      long long ldr2;                               // column stride of B in doubles
      int cx, pe;                                   // lane j: f_j - 56 and pend of column j
      int er, nval;
      bool row_ok, any_pe;                          // any_pe: some column of the tile has a pending scaling
      int rc, cc;                                   // TRI: this thread's complex row, the warp's first column
    };
    TileCursor<MAXP, TRI> fc;                       // the tile being fetched
    auto fetch = [&](int t, TileIn &in) {
      int pf, rt, ct;
      fc.at(T, t, pf, rt, ct);
      const OzArgs &args = T.args[pf];
      const int i = args.row_lo + rt * kOzBM + 32 * quarter + lane;   // real row of A'
      const int r = i >> 1, part = i & 1;
      const long long ldr2 = 2 * args.ldr;
      in.ldr2 = ldr2;
      in.row_ok = i < args.row_hi;
      in.nval = min(kOzBN, args.ncols - ct * kOzBN);
      in.cx = lane < in.nval ? args.cexp[ct * kOzBN + lane] - (NP == kOzS ? 56 : 14) : 0;
      in.pe = (lane < in.nval && args.pend) ? args.pend[args.col_base + ct * kOzBN + lane] : 0;
      in.any_pe = __any_sync(0xffffffffu, in.pe != 0);
      in.er = in.row_ok ? args.rexp[r] : 0;
      const int c0 = kCW * cgroup;
      in.base = reinterpret_cast<double *>(args.R + r + (long long)(args.col_base + ct * kOzBN + c0) * args.ldr) + part;
      in.rc = r;
      in.cc = args.col_base + ct * kOzBN + c0;
      const double *pj = in.base;
#pragma unroll
      for (int j = 0; j < kCW; ++j, pj += ldr2) in.b[j] = (!TRI && in.row_ok && c0 + j < in.nval) ? *pj : 0.0;
    };
    TileIn cur, nxt;
    pdl_wait();                                     // B, exponents and pending scalings of the diagonal step
    if (t0 < t1) fetch(t0, cur);
    for (int t = t0, k = 0; t < t1; ++t, ++k) {
      const int ab = k & 1;
      // one decision per warp: the TMEM reads and shuffles below are warp-wide
      if (!__all_sync(0xffffffffu, wait(&accfull[ab], (k >> 1) & 1))) { fail = 1; break; }
      tc_fence_after();
      if (t + 1 < t1) fetch(t + 1, nxt);            // in flight during this tile
      const int c0 = kCW * cgroup;
#pragma unroll
      for (int h = 0; h < kPasses; ++h) {
        const int cp = c0 + kQ * h;                 // first column of this pass
        double out[kQ];
        if constexpr (NP == kOzLpPlanes) {
          // FP32 accumulation: W = D_0 + 2^-7 (D_1 + 2^-7 D_2), the product
          // W 2^(e_r + f_j - 14) subtracted from B in FP64.
          uint32_t v[NP][kQ];
#pragma unroll
          for (int d = 0; d < NP; ++d) tmem_ld4(tmem + lane_addr + ab * kAcc + d * kOzBN + cp, v[d]);
          tmem_ld_wait();
          if (h == kPasses - 1) {
            tc_fence_before();
            mbar_arrive(&accempty[ab]);
          }
          float Wf[kQ];
          bool slow = false;
#pragma unroll
          for (int j = 0; j < kQ; ++j) {
            Wf[j] = fmaf(fmaf(__uint_as_float(v[2][j]), 0x1p-7f, __uint_as_float(v[1][j])), 0x1p-7f,
                         __uint_as_float(v[0][j]));
            const int ex = cur.er + __shfl_sync(0xffffffffu, cur.cx, cp + j);
            const int pe = __shfl_sync(0xffffffffu, cur.pe, cp + j);
            const double bv = cur.b[kQ * h + j];
            const int vh = __double2hiint(bv), vl = __double2loint(bv);
            const int ev = (vh >> 20) & 0x7ff;
            const bool nz = ((vh & 0x7fffffff) | vl) != 0;
            slow |= pe != 0 && nz && (ev <= pe || ev == 0x7ff);
            const int vh2 = (pe != 0 && nz) ? vh - (pe << 20) : vh;
            out[j] = __hiloint2double(vh2, vl) - f32_ldexp(Wf[j], ex, slow);
          }
          slow = slow && cur.row_ok;
          if (__any_sync(0xffffffffu, slow)) {
#pragma unroll
            for (int j = 0; j < kQ; ++j) {
              const int ex = cur.er + __shfl_sync(0xffffffffu, cur.cx, cp + j);
              const int pe = __shfl_sync(0xffffffffu, cur.pe, cp + j);
              out[j] = update_out_slow_lp(cur.b[kQ * h + j], pe, Wf[j], ex);
            }
          }
        } else {
          // W = sum_d D_d 2^(42 - 7d), the diagonals paired first in int32:
          // |D_d| <= (d + 1) 64 127^2, so D_{2c} 2^7 + D_{2c+1} < 2^30 for d <= 7.
          // (D_0..D_3 are below 2^22 and are read without a conversion.)
          uint32_t v[kOzS][kQ];                       // all diagonals of the pass, one wait
  #pragma unroll
          for (int d = 0; d < kOzS; ++d) tmem_ld4(tmem + lane_addr + ab * kAcc + d * kOzBN + cp, v[d]);
          tmem_ld_wait();
          int P[kOzS / 2][kQ];
  #pragma unroll
          for (int c = 0; c < kOzS / 2; ++c)
  #pragma unroll
            for (int j = 0; j < kQ; ++j)
              P[c][j] = c < 2 ? f32_small_pair(v[2 * c][j], v[2 * c + 1][j])
                              : __float2int_rn(__uint_as_float(v[2 * c][j])) * (1 << kOzBits) +
                                    __float2int_rn(__uint_as_float(v[2 * c + 1][j]));   // exact integers
          if (h == kPasses - 1) {
            tc_fence_before();
            mbar_arrive(&accempty[ab]);
          }
          int Wh[kQ];
          uint32_t Wl[kQ];
  #pragma unroll
          for (int j = 0; j < kQ; ++j) fold_w(P[0][j], P[1][j], P[2][j], P[3][j], Wh[j], Wl[j]);
          // Branch-free outputs: the pending scaling on the exponent field and
          // the product by w_ldexp_fast; a pass where either leaves the normal
          // range is redone with the FP64 routines.  Tiles with no pending
          // scaling (the common case) skip its tests.
          bool slow = false;
          if (!cur.any_pe) {
  #pragma unroll
            for (int j = 0; j < kQ; ++j) {
              const int ex = cur.er + __shfl_sync(0xffffffffu, cur.cx, cp + j);
              out[j] = cur.b[kQ * h + j] - w_ldexp_fast(Wh[j], Wl[j], ex, slow);
            }
          } else {
  #pragma unroll
          for (int j = 0; j < kQ; ++j) {
            const int ex = cur.er + __shfl_sync(0xffffffffu, cur.cx, cp + j);
            const int pe = __shfl_sync(0xffffffffu, cur.pe, cp + j);
            const double v = cur.b[kQ * h + j];
            const int vh = __double2hiint(v), vl = __double2loint(v);
            const int ev = (vh >> 20) & 0x7ff;
            const bool nz = ((vh & 0x7fffffff) | vl) != 0;
            // Only normal values are scaled on the exponent field (zero stays
            // zero); subnormals, values that would become subnormal, inf and
            // NaN go the slow way.  (Word-wise tests: a test of all bits but
            // the sign against zero may be compiled into an FP64 comparison.)
            slow |= pe != 0 && nz && (ev <= pe || ev == 0x7ff);
            const int vh2 = (pe != 0 && nz) ? vh - (pe << 20) : vh;
            out[j] = __hiloint2double(vh2, vl) - w_ldexp_fast(Wh[j], Wl[j], ex, slow);
          }
          }
          slow = slow && cur.row_ok;                  // rows past the range hold no planes
          if (__any_sync(0xffffffffu, slow)) {        // rare; same values where both apply
  #pragma unroll
            for (int j = 0; j < kQ; ++j) {
              const int ex = cur.er + __shfl_sync(0xffffffffu, cur.cx, cp + j);
              const int pe = __shfl_sync(0xffffffffu, cur.pe, cp + j);
              out[j] = update_out_slow(cur.b[kQ * h + j], pe, Wh[j], Wl[j], ex);
            }
          }
        }
        if constexpr (TRI) {                        // strictly below the diagonal: zero
#pragma unroll
          for (int j = 0; j < kQ; ++j)
            if (cur.rc > cur.cc + kQ * h + j) out[j] = 0.0;
        }
        const long long ldr2 = cur.ldr2;
        double *pj = cur.base + kQ * h * ldr2;
#pragma unroll
        for (int j = 0; j < kQ; ++j, pj += ldr2)
          if (cur.row_ok && cp + j < cur.nval) *pj = out[j];
      }
      cur = nxt;
    }
  }
  tc_fence_before();
  __syncthreads();
  if (fail) {
    // A wait gave up: the copies and MMAs this CTA issued land before TMEM is
    // freed (time-limited waits that ignore the abort bit, as in oz_gemm_tile).
    if (warp == kOzuEpiWarps && lane == 0) {
      if (a_issued > 0) mbar_wait(&afull, (a_issued - 1) & 1);
      for (int i = max(0, b_issued - 2); i < b_issued; ++i) mbar_wait(&bfull[i & 1], (i >> 1) & 1);
    } else if (warp == kOzuEpiWarps + 1 && lane == 0) {
      mbar_wait(&mma_done, 0);
    }
    tc_fence_before();
    __syncthreads();
  }
  if (fail && threadIdx.x == 0) raise_status(status, MSTS_STATUS_TIMEOUT);
  if (warp == 0) tmem_dealloc(tmem, kTmemCols);
}

cudaError_t ozaki_update(const OzPlan &plan, int b, int lo, int hi, double2 *B, long long ldb,
                         int jstart, int ncols, const int *pend, uint32_t *status, double flops,
                         cudaStream_t st, bool planes_ready, const double2 *lam, long long lam_stride, bool lp) {
  const int row_lo = plan.conj ? 2 * hi : 0, row_hi = plan.conj ? 2 * plan.m : 2 * lo;
  if (ncols <= 0 || row_hi <= row_lo) return cudaSuccess;
  if (!planes_ready) {
    k_ozs_slice_X<<<(ncols + 7) / 8, 256, 0, st>>>(B, ldb, lo, hi - lo, jstart, ncols, plan.KB, plan.bp,
                                                  plan.cexp, lam, lam_stride);
    count_launches(1);
  }
  lp = lp && plan.KB == kOzKC;          // the 3-plane product exists in the persistent form only
  CUtensorMap tmB;
  if (!make_map(&tmB, plan.bp, plan.KB, ncols, kOzBN, lp ? kOzLpPlanes : kOzS)) return cudaErrorNotSupported;
  OzArgs a{};
  a.B = B; a.ldb = ldb; a.R = B; a.ldr = ldb;
  a.rexp = plan.rexp + (size_t)b * plan.m;
  a.cexp = plan.cexp;
  a.pend = pend;
  a.m = plan.m; a.n = ncols; a.K = plan.KB;
  a.a_x0 = b * plan.KB;
  a.row_lo = row_lo; a.row_hi = row_hi;
  a.col_base = jstart; a.ncols = ncols;
  a.status = ozaki_call_status(status, st);
  if (plan.KB == kOzKC) {
    const int tiles_n = (ncols + kOzBN - 1) / kOzBN, tiles_m = (row_hi - row_lo + kOzBM - 1) / kOzBM;
    const int total = tiles_n * tiles_m;
    // BF16 MMA FLOPs issued: NP (NP + 1) / 2 digit pairs x 4 K-steps of 128 x 32 x 16 per tile
    const int np = lp ? kOzLpPlanes : kOzS;
    const double mma_flops = (double)total * (np * (np + 1) / 2) * (kOzKC / 16) * 2.0 * kOzBM * kOzBN * 16;
    void *h = trace_on() ? trace_start(2, mma_flops, (double)total * np * kOzBN * kOzKC * 2, st) : nullptr;
    OzUpdTab<1> tab;
    tab.tmA[0] = plan.tmA;
    tab.tmB[0] = tmB;
    tab.args[0] = a;
    tab.tiles_n[0] = tiles_n;
    tab.tile_base[0] = 0;
    tab.tile_base[1] = total;
    tab.tiles_total = total;
    cudaError_t e;
    if (lp) {
      e = cudaFuncSetAttribute(k_oz_update<kOzLpPlanes, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)ozu_smem<kOzLpPlanes>());
      if (e == cudaSuccess)
        e = launch_pdl(k_oz_update<kOzLpPlanes, 1>, dim3(std::min(total, kOzPersistentCtas)), dim3(kOzuThreads),
                       ozu_smem<kOzLpPlanes>(), st, tab);
    } else {
      e = cudaFuncSetAttribute(k_oz_update<kOzS, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)ozu_smem<kOzS>());
      if (e == cudaSuccess)
        e = launch_pdl(k_oz_update<kOzS, 1>, dim3(std::min(total, kOzPersistentCtas)), dim3(kOzuThreads),
                       ozu_smem<kOzS>(), st, tab);
    }
    trace_stop(h, st);
    count_launches(1);
    return e != cudaSuccess ? e : cudaGetLastError();
  }
  cudaError_t e = cudaFuncSetAttribute(k_oz_gemm<kUpdate>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kOzSmem);
  if (e != cudaSuccess) return e;
  // Recorded as the tensor-core kernel: BF16 MMA FLOPs issued (36 digit pairs x
  // 4 K-steps of 128 x 32 x 16 per tile and chunk) and the plane bytes it loads.
  const double tiles = (double)((ncols + kOzBN - 1) / kOzBN) * ((row_hi - row_lo + kOzBM - 1) / kOzBM);
  const double chunks = plan.KB / kOzKC;
  const double mma_flops = tiles * chunks * 36.0 * (kOzKC / 16) * 2.0 * kOzBM * kOzBN * 16;
  (void)flops;
  void *h = trace_on() ? trace_start(2, mma_flops, tiles * chunks * (kOzS * kOzABytes + kOzBBytes), st)
                       : nullptr;
  k_oz_gemm<kUpdate><<<dim3((ncols + kOzBN - 1) / kOzBN, (row_hi - row_lo + kOzBM - 1) / kOzBM), kOzThreads,
                       kOzSmem, st>>>(plan.tmA, tmB, a);
  trace_stop(h, st);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t ozaki_update_batched(const OzBatchStep *steps, int count, uint32_t *status, cudaStream_t st) {
  if (count <= 0) return cudaSuccess;
  if (count > kMaxProbs) return cudaErrorInvalidValue;
  std::unique_ptr<OzBatch> hb(new OzBatch());
  int max_tn = 0, max_tm = 0;
  double tiles = 0.0, chunk_tiles = 0.0;
  for (int i = 0; i < count; ++i) {
    const OzBatchStep &q = steps[i];
    hb->tiles_n[i] = hb->tiles_m[i] = 0;
    if (!q.plan) continue;
    const OzPlan &plan = *q.plan;
    const int row_lo = plan.conj ? 2 * q.hi : 0, row_hi = plan.conj ? 2 * plan.m : 2 * q.lo;
    if (q.ncols <= 0 || row_hi <= row_lo) continue;
    hb->tmA[i] = plan.tmA;
    if (q.ncols == plan.nmax) hb->tmB[i] = plan.tmB;
    else if (!make_map(&hb->tmB[i], plan.bp, plan.KB, q.ncols, kOzBN, kOzS)) return cudaErrorNotSupported;
    OzArgs a{};
    a.B = q.B; a.ldb = q.ldb; a.R = q.B; a.ldr = q.ldb;
    a.rexp = plan.rexp + (size_t)q.b * plan.m;
    a.cexp = plan.cexp;
    a.pend = q.pend;
    a.m = plan.m; a.n = q.ncols; a.K = plan.KB;
    a.a_x0 = q.b * plan.KB;
    a.row_lo = row_lo; a.row_hi = row_hi;
    a.col_base = q.jstart; a.ncols = q.ncols;
    a.status = ozaki_call_status(status, st);
    hb->args[i] = a;
    hb->tiles_n[i] = (q.ncols + kOzBN - 1) / kOzBN;
    hb->tiles_m[i] = (row_hi - row_lo + kOzBM - 1) / kOzBM;
    max_tn = std::max(max_tn, hb->tiles_n[i]);
    max_tm = std::max(max_tm, hb->tiles_m[i]);
    tiles += (double)hb->tiles_n[i] * hb->tiles_m[i];
    chunk_tiles += (double)hb->tiles_n[i] * hb->tiles_m[i] * (plan.KB / kOzKC);
  }
  if (max_tn == 0) return cudaSuccess;
  if (chunk_tiles == tiles) {
    // one K chunk per block (n_b <= 32): the persistent kernel over every
    // problem's tiles, a row tile's U planes resident across its column tiles
    std::unique_ptr<OzUpdTab<kMaxProbs>> tb(new OzUpdTab<kMaxProbs>());
    int k = 0, total = 0;
    for (int i = 0; i < count; ++i) {
      const int nt = hb->tiles_n[i] * hb->tiles_m[i];
      if (nt == 0) continue;
      tb->tmA[k] = hb->tmA[i];
      tb->tmB[k] = hb->tmB[i];
      tb->args[k] = hb->args[i];
      tb->tiles_n[k] = hb->tiles_n[i];
      tb->tile_base[k] = total;
      total += nt;
      ++k;
    }
    for (int i = k; i <= kMaxProbs; ++i) tb->tile_base[i] = total;   // past the last problem
    tb->tiles_total = total;
    cudaError_t e = cudaFuncSetAttribute(k_oz_update<kOzS, kMaxProbs>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)ozu_smem<kOzS>());
    if (e != cudaSuccess) return e;
    const double mma_flops = tiles * 36.0 * (kOzKC / 16) * 2.0 * kOzBM * kOzBN * 16;
    void *h = trace_on() ? trace_start(2, mma_flops, tiles * kOzS * kOzBN * kOzKC * 2, st) : nullptr;
    e = launch_pdl(k_oz_update<kOzS, kMaxProbs>, dim3(std::min(total, kOzPersistentCtas)), dim3(kOzuThreads),
                   ozu_smem<kOzS>(), st, *tb);
    trace_stop(h, st);
    count_launches(1);
    return e != cudaSuccess ? e : cudaGetLastError();
  }
  cudaError_t e = cudaFuncSetAttribute(k_oz_batched<kUpdate>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kOzSmem);
  if (e != cudaSuccess) return e;
  const double mma_flops = chunk_tiles * 36.0 * (kOzKC / 16) * 2.0 * kOzBM * kOzBN * 16;
  void *h = trace_on() ? trace_start(2, mma_flops, chunk_tiles * (kOzS * kOzABytes + kOzBBytes), st) : nullptr;
  k_oz_batched<kUpdate><<<dim3(max_tn, max_tm, count), kOzThreads, kOzSmem, st>>>(*hb);
  trace_stop(h, st);
  count_launches(1);
  (void)tiles;
  return cudaGetLastError();
}

// dU = -triu(L X^H) for a batch (the adjoint's product, K = n): per problem
// the digit planes of L (rows) and of X^H (columns of B' = conjugated rows of
// X) in its own workspace slice, then every problem's tiles in one launch.
size_t ozaki_neg_triu_bytes(int m, int n) {
  const size_t K = (size_t)kpad(n);
  return a256((size_t)kOzS * 2 * m * K * 2) + a256((size_t)kOzS * m * K * 2) + a256(4 * (size_t)m) * 2;
}

// The chunked form (more than 64 shifts: several K chunks per tile).
static cudaError_t ozaki_neg_triu_chunked(const OzNegTriuItem *items, int count, void *ws, uint32_t *status,
                                          cudaStream_t st) {
  if (count <= 0) return cudaSuccess;
  if (count > kMaxProbs) return cudaErrorInvalidValue;
  std::unique_ptr<OzBatch> hb(new OzBatch());
  char *cur = static_cast<char *>(ws);
  int max_tn = 0, max_tm = 0;
  double chunk_tiles = 0.0;
  for (int i = 0; i < count; ++i) {
    const OzNegTriuItem &q = items[i];
    hb->tiles_n[i] = hb->tiles_m[i] = 0;
    if (q.m <= 0) continue;
    const int m = q.m, n = q.n, K = kpad(n > 0 ? n : 1);
    __nv_bfloat16 *Ap = reinterpret_cast<__nv_bfloat16 *>(cur); cur += a256((size_t)kOzS * 2 * m * K * 2);
    __nv_bfloat16 *Bp = reinterpret_cast<__nv_bfloat16 *>(cur); cur += a256((size_t)kOzS * m * K * 2);
    int *rexp = reinterpret_cast<int *>(cur); cur += a256(4 * (size_t)m);
    int *cexp = reinterpret_cast<int *>(cur); cur += a256(4 * (size_t)m);
    k_oz_rowexp<<<(m + 7) / 8, 256, 0, st>>>(q.L, q.ldl, m, n, rexp, 1);
    k_oz_slice_A<<<dim3((K / 2 + 255) / 256, m), 256, 0, st>>>(q.L, q.ldl, m, n, rexp, Ap, K, 1);
    k_oz_slice_BH<<<m, 256, 0, st>>>(q.X, q.ldx, m, n, cexp, Bp, K);
    count_launches(3);
    if (!make_map(&hb->tmA[i], Ap, K, 2 * m, kOzBM, 1) || !make_map(&hb->tmB[i], Bp, K, m, kOzBN, kOzS))
      return cudaErrorNotSupported;
    OzArgs a{};
    a.R = q.dU; a.ldr = q.lddu;
    a.rexp = rexp; a.cexp = cexp;
    a.m = m; a.n = m; a.K = K;
    a.status = ozaki_call_status(status, st);
    hb->args[i] = a;
    hb->tiles_n[i] = (m + kOzBN - 1) / kOzBN;
    hb->tiles_m[i] = (2 * m + kOzBM - 1) / kOzBM;
    max_tn = std::max(max_tn, hb->tiles_n[i]);
    max_tm = std::max(max_tm, hb->tiles_m[i]);
    chunk_tiles += 0.5 * hb->tiles_n[i] * hb->tiles_m[i] * (K / kOzKC);
  }
  if (max_tn == 0) return cudaGetLastError();
  cudaError_t e = cudaFuncSetAttribute(k_oz_batched<kNegTriu>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kOzSmem);
  if (e != cudaSuccess) return e;
  const double mma_flops = chunk_tiles * 36.0 * (kOzKC / 16) * 2.0 * kOzBM * kOzBN * 16;
  void *h = trace_on() ? trace_start(2, mma_flops, chunk_tiles * (kOzS * kOzABytes + kOzBBytes), st) : nullptr;
  k_oz_batched<kNegTriu><<<dim3(max_tn, max_tm, count), kOzThreads, kOzSmem, st>>>(*hb);
  trace_stop(h, st);
  count_launches(1);
  return cudaGetLastError();
}

// The operands of dU = -triu(L X^H) for every problem of a batch (one K chunk:
// n <= 32): blockIdx.y = 0, one warp per row r of L, its exponent e_r and the
// A planes of row r (the layout of k_oz_slice_A); blockIdx.y = 1, one warp per
// row c of X, the exponent f_c of conj(X(c, :)) and its B planes (the layout
// of k_oz_slice_BH).  Problem in grid.z.
struct OzAdjSliceItem {
  const double2 *L; long long ldl;
  const double2 *X; long long ldx;
  int m, n;
  __nv_bfloat16 *Ap, *Bp;
  int *rexp, *cexp;
};
struct OzAdjSliceTable {
  OzAdjSliceItem p[kMaxProbs];
};
__global__ void k_oz_slice_adj(const __grid_constant__ OzAdjSliceTable t) {
  const OzAdjSliceItem &q = t.p[blockIdx.z];
  const int lane = threadIdx.x & 31;
  const int r = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (r >= q.m) return;
  const bool a_side = blockIdx.y == 0;
  const double2 *src = a_side ? q.L : q.X;
  const long long ld = a_side ? q.ldl : q.ldx;
  const double2 v = lane < q.n ? src[r + (long long)lane * ld] : make_double2(0.0, 0.0);
  int e = bound_exp(v);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) e = max(e, __shfl_xor_sync(0xffffffffu, e, o));
  if (e < -(1 << 28)) e = 0;
  if (lane == 0) (a_side ? q.rexp : q.cexp)[r] = e;
  float dr[kOzS], di[kOzS];
  digits8(v.x, e, dr);
  digits8(a_side ? v.y : -v.y, e, di);
  constexpr int K = kOzKC;
  if (a_side) {
    const size_t rows = 2 * (size_t)q.m;
#pragma unroll
    for (int s = 0; s < kOzS; ++s) {
      *reinterpret_cast<__nv_bfloat162 *>(q.Ap + (s * rows + 2 * (size_t)r) * K + 2 * lane) =
          __floats2bfloat162_rn(dr[s], -di[s]);     // row 2r:   (Re L, -Im L)
      *reinterpret_cast<__nv_bfloat162 *>(q.Ap + (s * rows + 2 * (size_t)r + 1) * K + 2 * lane) =
          __floats2bfloat162_rn(di[s], dr[s]);      // row 2r+1: (Im L,  Re L)
    }
  } else {
#pragma unroll
    for (int s = 0; s < kOzS; ++s)
      *reinterpret_cast<__nv_bfloat162 *>(q.Bp + ((size_t)s * q.m + r) * K + 2 * lane) =
          __floats2bfloat162_rn(dr[s], di[s]);
  }
}

// The entries of dU in the tiles wholly below the diagonal (complex rows
// 64 rt.., columns 32 ct.. with ct < 2 rt; k_oz_update<.., TRI> writes the
// others), every problem of a batch: one column per y, problem in z.
struct OzZeroItem {
  double2 *dU;
  long long ld;
  int m;
};
struct OzZeroTable {
  OzZeroItem p[kMaxProbs];
};
__global__ void k_oz_zero_lower(const __grid_constant__ OzZeroTable t) {
  const OzZeroItem &q = t.p[blockIdx.z];
  for (int c = blockIdx.y; c < q.m; c += gridDim.y) {
    const int r0 = (kOzBM / 2) * ((c / kOzBN) / 2 + 1);
    for (int r = r0 + (int)(blockIdx.x * blockDim.x + threadIdx.x); r < q.m; r += gridDim.x * blockDim.x)
      q.dU[r + (long long)c * q.ld] = make_double2(0.0, 0.0);
  }
}

cudaError_t ozaki_neg_triu_batched(const OzNegTriuItem *items, int count, void *ws, uint32_t *status,
                                   cudaStream_t st) {
  if (count <= 0) return cudaSuccess;
  if (count > kMaxProbs) return cudaErrorInvalidValue;
  std::unique_ptr<OzUpdTab<kMaxProbs>> tb(new OzUpdTab<kMaxProbs>());
  OzZeroTable zt;
  OzAdjSliceTable sl;
  char *cur = static_cast<char *>(ws);
  int k = 0, total = 0, maxm = 0;
  double tiles = 0.0;
  bool one_chunk = true;
  for (int i = 0; i < count; ++i)
    if (items[i].m > 0 && kpad(items[i].n > 0 ? items[i].n : 1) != kOzKC) one_chunk = false;
  if (!one_chunk) return ozaki_neg_triu_chunked(items, count, ws, status, st);
  for (int i = 0; i < count; ++i) {
    const OzNegTriuItem &q = items[i];
    if (q.m <= 0) continue;
    const int m = q.m, n = q.n, K = kpad(n > 0 ? n : 1);
    __nv_bfloat16 *Ap = reinterpret_cast<__nv_bfloat16 *>(cur); cur += a256((size_t)kOzS * 2 * m * K * 2);
    __nv_bfloat16 *Bp = reinterpret_cast<__nv_bfloat16 *>(cur); cur += a256((size_t)kOzS * m * K * 2);
    int *rexp = reinterpret_cast<int *>(cur); cur += a256(4 * (size_t)m);
    int *cexp = reinterpret_cast<int *>(cur); cur += a256(4 * (size_t)m);
    sl.p[k] = OzAdjSliceItem{q.L, q.ldl, q.X, q.ldx, m, n, Ap, Bp, rexp, cexp};
    if (!make_map(&tb->tmA[k], Ap, K, 2 * m, kOzBM, 1) || !make_map(&tb->tmB[k], Bp, K, m, kOzBN, kOzS))
      return cudaErrorNotSupported;
    OzArgs a{};
    a.B = q.dU; a.ldb = q.lddu; a.R = q.dU; a.ldr = q.lddu;
    a.rexp = rexp; a.cexp = cexp;
    a.m = m; a.n = m; a.K = K;
    a.a_x0 = 0;
    a.row_lo = 0; a.row_hi = 2 * m;
    a.col_base = 0; a.ncols = m;
    a.status = ozaki_call_status(status, st);
    tb->args[k] = a;
    const int tn = (m + kOzBN - 1) / kOzBN, tm = (2 * m + kOzBM - 1) / kOzBM;
    int nt = 0;
    for (int rt = 0; rt < tm; ++rt) nt += std::max(0, tn - 2 * rt);   // the tiles meeting the upper triangle
    tb->tiles_n[k] = tn;
    tb->tile_base[k] = total;
    total += nt;
    tiles += nt;
    zt.p[k] = OzZeroItem{q.dU, q.lddu, m};
    maxm = std::max(maxm, m);
    ++k;
  }
  if (k == 0) return cudaGetLastError();
  for (int i = k; i <= kMaxProbs; ++i) tb->tile_base[i] = total;
  tb->tiles_total = total;
  k_oz_slice_adj<<<dim3((maxm + 7) / 8, 2, k), 256, 0, st>>>(sl);
  k_oz_zero_lower<<<dim3(1, std::min(maxm, 65535), k), 256, 0, st>>>(zt);
  count_launches(2);
  cudaError_t e = cudaFuncSetAttribute(k_oz_update<kOzS, kMaxProbs, true>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ozu_smem<kOzS>());
  if (e != cudaSuccess) return e;
  const double mma_flops = tiles * 36.0 * (kOzKC / 16) * 2.0 * kOzBM * kOzBN * 16;
  void *h = trace_on() ? trace_start(2, mma_flops, tiles * kOzS * kOzBN * kOzKC * 2, st) : nullptr;
  e = launch_pdl(k_oz_update<kOzS, kMaxProbs, true>, dim3(std::min(total, kOzPersistentCtas)), dim3(kOzuThreads),
                 ozu_smem<kOzS>(), st, *tb);
  trace_stop(h, st);
  count_launches(1);
  return e != cudaSuccess ? e : cudaGetLastError();
}

}  // namespace msts

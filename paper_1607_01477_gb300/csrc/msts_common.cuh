// msts_common.cuh -- device helpers shared by the libmsts kernels.
//
// Complex numbers are double2 {x = re, y = im} (the layout of msts_z).
// Matrices are column-major: A(r, c) = A[r + c * lda].
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/msts.h"

namespace msts {

// ---------------------------------------------------------------------------
// Constants of the safe variant (Sec. 3).  Omega = 2^kOmegaExp; the pre-check
// |b(i)| / |U(i,i)| >= Omega is made on exponents so it cannot overflow.
// ---------------------------------------------------------------------------
constexpr int kOmegaExp = 960;
constexpr double kEps = 2.220446049250313e-16;        // 2^-52
constexpr double kDblMin = 2.2250738585072014e-308;   // 2^-1022
constexpr int kMaxProbs = 64;                          // problems per launch
constexpr double kRangeLimitU = 281474976710656.0;     // 2^48

__device__ __forceinline__ double omega() { return 0x1p960; }

__device__ __forceinline__ double2 zmake(double re, double im) { return make_double2(re, im); }
__device__ __forceinline__ double2 zadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 zsub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ double2 zconj(double2 a) { return make_double2(a.x, -a.y); }
__device__ __forceinline__ double2 zscale(double2 a, double s) { return make_double2(a.x * s, a.y * s); }
__device__ __forceinline__ double2 zmul(double2 a, double2 b) {
  return make_double2(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}
// a * b and Smith's a / b with every operation rounded on its own (no fused
// multiply-add): the arithmetic of the generalized pivots U(i,i) - s V(i,i)
// and of lambda = T(j,j) / S(j,j), so that exact zeros and the shifts come out
// the same whatever the compiler contracts elsewhere.
__device__ __forceinline__ double2 zmul_rn(double2 a, double2 b) {
  return make_double2(__dsub_rn(__dmul_rn(a.x, b.x), __dmul_rn(a.y, b.y)),
                      __dadd_rn(__dmul_rn(a.x, b.y), __dmul_rn(a.y, b.x)));
}
__device__ __forceinline__ double2 zdiv_rn(double2 a, double2 b) {
  if (fabs(b.x) >= fabs(b.y)) {
    const double r = __ddiv_rn(b.y, b.x);
    const double d = __dadd_rn(b.x, __dmul_rn(b.y, r));
    return make_double2(__ddiv_rn(__dadd_rn(a.x, __dmul_rn(a.y, r)), d),
                        __ddiv_rn(__dsub_rn(a.y, __dmul_rn(a.x, r)), d));
  }
  const double r = __ddiv_rn(b.x, b.y);
  const double d = __dadd_rn(__dmul_rn(b.x, r), b.y);
  return make_double2(__ddiv_rn(__dadd_rn(__dmul_rn(a.x, r), a.y), d),
                      __ddiv_rn(__dsub_rn(__dmul_rn(a.y, r), a.x), d));
}
// acc - a * b, fused.
__device__ __forceinline__ double2 zfms(double2 acc, double2 a, double2 b) {
  acc.x = fma(-a.x, b.x, acc.x);
  acc.x = fma(a.y, b.y, acc.x);
  acc.y = fma(-a.x, b.y, acc.y);
  acc.y = fma(-a.y, b.x, acc.y);
  return acc;
}
// acc + a * b, fused.
__device__ __forceinline__ double2 zfma(double2 acc, double2 a, double2 b) {
  acc.x = fma(a.x, b.x, acc.x);
  acc.x = fma(-a.y, b.y, acc.x);
  acc.y = fma(a.x, b.y, acc.y);
  acc.y = fma(a.y, b.x, acc.y);
  return acc;
}
// acc + conj(a) * b, fused.
__device__ __forceinline__ double2 zfma_cj(double2 acc, double2 a, double2 b) {
  acc.x = fma(a.x, b.x, acc.x);
  acc.x = fma(a.y, b.y, acc.x);
  acc.y = fma(a.x, b.y, acc.y);
  acc.y = fma(-a.y, b.x, acc.y);
  return acc;
}
__device__ __forceinline__ double zabs(double2 a) { return hypot(a.x, a.y); }
__device__ __forceinline__ bool zzero(double2 a) { return a.x == 0.0 && a.y == 0.0; }
__device__ __forceinline__ bool zfinite(double2 a) { return isfinite(a.x) && isfinite(a.y); }

// Complex quotient a / b following Smith's 1962 method: divide through by the
// larger component of b so that no intermediate overflows needlessly.
__device__ __forceinline__ double2 zdiv(double2 a, double2 b) {
  if (fabs(b.x) >= fabs(b.y)) {
    const double r = b.y / b.x;
    const double d = b.x + b.y * r;
    return make_double2((a.x + a.y * r) / d, (a.y - a.x * r) / d);
  }
  const double r = b.x / b.y;
  const double d = b.x * r + b.y;
  return make_double2((a.x * r + a.y) / d, (a.y * r - a.x) / d);
}

__device__ __forceinline__ double2 shfl_z(double2 v, int src) {
  return make_double2(__shfl_sync(0xffffffffu, v.x, src), __shfl_sync(0xffffffffu, v.y, src));
}

__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// Smallest k >= 1 with 2^-k * x < Omega for finite x >= Omega.
__device__ __forceinline__ int choose_k(double x) {
  const int k = ilogb(x) - (kOmegaExp - 1);
  return k < 1 ? 1 : k;
}

// floor(log2(a / b)) for a > 0, b > 0 without forming a / b (which may overflow).
__device__ __forceinline__ int ratio_exponent(double a, double b) {
  const int ea = ilogb(a), eb = ilogb(b);
  const double q = scalbn(a, -ea) / scalbn(b, -eb);
  return ilogb(q) + ea - eb;
}

__device__ __forceinline__ void raise_status(uint32_t *status, uint32_t bits) {
  if (status) atomicOr(reinterpret_cast<unsigned int *>(status), bits);
}

// ----- programmatic dependent launch ------------------------------------------
// A kernel launched by launch_pdl may start while the previous kernel of its
// stream is finishing.  pdl_wait() blocks until that kernel has completed and
// its writes are visible, so it must come before any read of data an earlier
// kernel wrote; pdl_trigger() lets the next launch_pdl kernel start once every
// CTA of this one has called it (or exited).  Plain launches are unaffected.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                              Args... args) {
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, args...);
}

// ----- cheap exact helpers: power-of-two scaling through the exponent field,
// so that the per-row work of the diagonal step stays off the (slow) FP64 pipe
// wherever possible.
__device__ __forceinline__ double pow2i(int k) {            // 2^k, k in [-1022, 1023]
  return __longlong_as_double((long long)(k + 1023) << 52);
}
__device__ __forceinline__ long long absbits(double x) {
  return __double_as_longlong(x) & 0x7fffffffffffffffLL;
}
// floor(log2 max(|Re z|, |Im z|)) clamped to [-1022, 1022] (exponent field).
__device__ __forceinline__ int zexp(double2 z) {
  const long long m = max(absbits(z.x), absbits(z.y));
  const int e = (int)(m >> 52) - 1023;
  return min(max(e, -1022), 1022);
}
__device__ __forceinline__ bool zzero_bits(double2 z) { return (absbits(z.x) | absbits(z.y)) == 0; }

// y / p = y conj(p') / |p'|^2 * 2^-e with p' = p 2^-e (|p'|^2 in [1, 8)): one
// real division and no overflow in the intermediate products.
__device__ __forceinline__ double2 zdiv_fast(double2 y, double2 p) {
  const int e = zexp(p);
  const double s = pow2i(-e);
  const double a = p.x * s, b = p.y * s;
  const double q = 1.0 / fma(a, a, b * b);
  const double wr = fma(y.x, a, y.y * b) * q;
  const double wi = fma(y.y, a, -(y.x * b)) * q;
  return make_double2(wr * s, wi * s);
}
// |z| from the scaled components (one square root).
__device__ __forceinline__ double zabs_fast(double2 z) {
  if (zzero_bits(z)) return 0.0;
  const int e = zexp(z);
  const double s = pow2i(-e);
  const double a = z.x * s, b = z.y * s;
  return sqrt(fma(a, a, b * b)) * pow2i(e);
}
// floor(log2(|y| / |p|)) for y, p != 0 without a division or a square root:
// |y| = sqrt(ny) 2^fy with ny in [1, 4), likewise p.
__device__ __forceinline__ int ratio_exp_fast(double2 y, double2 p) {
  // Subnormal operands are first brought into the normal range (exactly).
  int adj = 0;
  if ((max(absbits(p.x), absbits(p.y)) >> 52) == 0) { p = zscale(p, 0x1p64); adj += 64; }
  if ((max(absbits(y.x), absbits(y.y)) >> 52) == 0) { y = zscale(y, 0x1p64); adj -= 64; }
  int fy = zexp(y), fp = zexp(p);
  const double sy = pow2i(-fy), sp = pow2i(-fp);
  const double ya = y.x * sy, yb = y.y * sy, pa = p.x * sp, pb = p.y * sp;
  double ny = fma(ya, ya, yb * yb), np = fma(pa, pa, pb * pb);
  if (ny >= 4.0) { fy += 1; ny *= 0.25; }
  if (np >= 4.0) { fp += 1; np *= 0.25; }
  return fy - fp - (ny < np ? 1 : 0) + adj;
}
// z * 2^-k for k >= 0 (exact unless the result is subnormal).
__device__ __forceinline__ double2 zshift(double2 z, int k) {
  if (k > 1022) { z = zscale(z, pow2i(-1022)); k -= 1022; }
  const double t = k > 1022 ? 0.0 : pow2i(-k);
  return zscale(z, t);
}
__device__ __forceinline__ double dshift(double x, int k) {
  if (k > 1022) { x *= pow2i(-1022); k -= 1022; }
  return x * (k > 1022 ? 0.0 : pow2i(-k));
}

// ---------------------------------------------------------------------------
// One multi-shift problem as the kernels see it.  Workspace pointers are set
// up by the host driver; the safe-only ones are null for plain solves.
// ---------------------------------------------------------------------------
struct Prob {
  const double2 *U;         // m x m, upper triangle read
  long long ldu;
  const double2 *shifts;    // shift j at shifts[j * shift_stride]
  long long shift_stride;
  double2 *B;               // m x n, overwritten with X
  long long ldb;
  double *scales;           // n (safe)
  int *scale_exp;           // n (safe)
  // safe-variant state (workspace)
  double *G;                // n: growth bound G(j) of Alg. 5
  int *e;                   // n: accumulated exponent, s_j = 2^-e_j
  int *pend;                // n: exponent still owed by B(I0, j) at this step
  int *E;                   // nblk x n: e_j when block b was finished
  double *cin;              // m: within-block column norms (excl. diagonal)
  double *cup;              // m: column norms above the block
  double *cblk;             // nblk: C_blk = sum_k cup[k] over the block
  double *rowsum;           // m: row sums of |U| (for ||U||_inf)
  double *delta;            // 1: zero-pivot replacement
  // generalized problem (appendix): V upper triangular, or null
  const double2 *V;
  long long ldv;
  double *cinV, *cupV, *cblkV;  // as cin, cup, cblk for V (safe)
  double *rowsumV;              // m: row sums of |V| (for ||V||_inf)
  double *deltaV;               // 1: eps ||V||_inf (delta_j = max(delta + |s_j| deltaV, DBL_MIN))
  int m, n, nblk;
  int diag_z;               // TREVC: write Z(j,j) = s_j in the fixup
  // Tensor-core substitution: the diagonal-block step also writes the digit
  // planes of X(I1, jstart..n) (BF16 pairs, plane t, column c at
  // oz_bp[(t * (n - jstart) + c) * oz_kb / 2 + row]) and their exponents.
  uint32_t *oz_bp;
  int *oz_cexp;
  int oz_kb;
};

struct ProbTable {
  int count;
  Prob p[kMaxProbs];
};

// Rows [lo, hi) of block b (blocks cut from the bottom, ragged block on top).
__device__ __forceinline__ void block_range(const Prob &P, int b, int nb, int &lo, int &hi) {
  hi = P.m - b * nb;
  lo = hi - nb < 0 ? 0 : hi - nb;
}

}  // namespace msts

// msts_diag_util.cuh -- exact helpers of the diagonal-block step (both
// kernel layouts): moduli, reciprocals and power-of-two scalings done on the
// IEEE exponent fields where the operands stay normal, and 16-byte
// asynchronous copies to shared memory.
#pragma once
#include <cuda_runtime.h>

#include "msts_common.cuh"

namespace msts {

// |z| with exactly the scaled operands and roundings of zabs_fast, the two
// power-of-two scalings done on the exponent fields (integer operations) when
// every operand stays a normal number; otherwise zabs_fast itself.
__device__ __forceinline__ double zabs_exp(double2 z) {
  const unsigned hx = (unsigned)__double2hiint(z.x) & 0x7fffffffu, lx = (unsigned)__double2loint(z.x);
  const unsigned hy = (unsigned)__double2hiint(z.y) & 0x7fffffffu, ly = (unsigned)__double2loint(z.y);
  const bool zx = (hx | lx) == 0u, zy = (hy | ly) == 0u;
  if (zx && zy) return 0.0;
  const int fx = (int)(hx >> 20), fy = (int)(hy >> 20);   // biased exponent fields
  const int e = max(fx, fy) - 1023;
  const bool ok = max(fx, fy) != 0 && e <= 1021 && (zx || fx - e >= 1) && (zy || fy - e >= 1);
  if (!ok) return zabs_fast(z);
  const double a = zx ? 0.0 : __hiloint2double((int)(hx - ((unsigned)e << 20)), (int)lx);
  const double b = zy ? 0.0 : __hiloint2double((int)(hy - ((unsigned)e << 20)), (int)ly);
  const double r = sqrt(fma(a, a, b * b));              // in [1, 2 sqrt 2)
  return __hiloint2double(__double2hiint(r) + (e << 20), __double2loint(r));
}
// x 2^s, exact unless the result is subnormal or overflows.
__device__ __forceinline__ double dscale(double x, int s) {
  if (s >= 0) {
    if (s > 1023) {
      x *= pow2i(1023);
      s -= 1023;
    }
    return x * pow2i(min(s, 1023));
  }
  return dshift(x, -s);
}
// x >= Omega for x >= 0 (false for NaN), on the exponent field.  (Range
// tests on all bits of a double may be compiled into FP64 comparisons, which
// cost as much as an FP64 multiply here.)
__device__ __forceinline__ bool ge_omega(double x) {
  const unsigned hi = (unsigned)__double2hiint(x);
  const unsigned e = (hi >> 20) & 0x7ffu;
  const bool nan = e == 0x7ffu && (((hi & 0xfffffu) | (unsigned)__double2loint(x)) != 0u);
  return e >= 0x3ffu + kOmegaExp && !nan;
}
// x 2^s for x >= 0 on the exponent field when x and the result are normal,
// else dscale.
__device__ __forceinline__ double dscale_exp(double x, int s) {
  const int hi = __double2hiint(x);
  const int e = (hi >> 20) & 0x7ff;
  if (e == 0 || e == 0x7ff || e + s < 1 || e + s > 0x7fe) return dscale(x, s);
  return __hiloint2double(hi + (s << 20), __double2loint(x));
}
// x 2^s on the exponent field, zero kept as it is (its sign too); otherwise
// as dscale_exp.
__device__ __forceinline__ double dscale_exp0(double x, int s) {
  const int hi = __double2hiint(x);
  if (((hi & 0x7fffffff) | __double2loint(x)) == 0) return x;
  return dscale_exp(x, s);
}
__device__ __forceinline__ double2 zscale_exp(double2 z, int s) {
  return make_double2(dscale_exp0(z.x, s), dscale_exp0(z.y, s));
}
// choose_k for a finite x >= Omega, from the exponent field (the same value as
// ilogb there).
__device__ __forceinline__ int choose_k_exp(double x) {
  const int k = ((__double2hiint(x) >> 20) & 0x7ff) - 1023 - (kOmegaExp - 1);
  return k < 1 ? 1 : k;
}

// Alg. 4's decisions on one block without its serial chain (both layouts).
//
// Write S = G 2^Ka for the running bound G of Alg. 4 and Ka the block's
// cumulative rescale exponent so far.  A rescale changes G and Ka but not S,
// and every addition G += a_i 2^(Kown - Ka) rounds S exactly as it rounds G
// (power-of-two scalings commute with rounding while every value is normal),
// so S_k is the plain running sum of G0 and the a_i 2^Kown, nondecreasing.
// The test "M_i >= Omega" rescales to Ka = em_i - (kOmegaExp - 1), the test
// "G >= Omega" to Ka = e(S_k) - (kOmegaExp - 1) (e: the unbiased exponent),
// each only when that raises Ka.  Ka is therefore a running maximum, and the
// block's final value is
//     Ka = max(0, max_i em_i - (kOmegaExp - 1), e(S_N) - (kOmegaExp - 1)).
// e(S_N) comes from an estimate of S_N accurate to 2^-18 relative (moduli and
// sum in FP32 on the leading significand bits, exponents as integers); it
// decides e(S_N) unless S_N lies within 2^-15 of a power of two.  Blocks where
// it cannot decide, or where some term of the chain could leave the normal
// range, run the chain itself.
constexpr int kBoundNone = -(1 << 28);
// |v| = f 2^e with f in [1, 2) from the leading 23 significand bits (relative
// error below 2^-23); f = 0 for v = 0; odd is set for subnormal, inf and NaN.
__device__ __forceinline__ float dbl_lead_f(double v, int &e, bool &odd) {
  const unsigned hi = (unsigned)__double2hiint(v) & 0x7fffffffu, lo = (unsigned)__double2loint(v);
  const int f = (int)(hi >> 20);
  e = kBoundNone;
  if ((hi | lo) == 0u) return 0.0f;
  if (f == 0 || f == 0x7ff) {
    odd = true;
    return 0.0f;
  }
  e = f - 1023;
  return __uint_as_float(0x3f800000u | ((hi & 0xfffffu) << 3) | (lo >> 29));
}
// f 2^d for f in [1, 8) or 0 and d <= 0, on the exponent field; 0 below 2^-40.
__device__ __forceinline__ float f_scale_down(float f, int d) {
  return (f == 0.0f || d < -40) ? 0.0f : __uint_as_float(__float_as_uint(f) + ((unsigned)d << 23));
}
// |z| as t 2^e with t in [1, 3): FP32 modulus of z's leading bits (relative
// error below 2^-22); t = 0, e = kBoundNone for z = 0.
__device__ __forceinline__ float abs_est(double2 z, int &e, bool &odd) {
  int ex, ey;
  const float fx = dbl_lead_f(z.x, ex, odd), fy = dbl_lead_f(z.y, ey, odd);
  e = max(ex, ey);
  if (e == kBoundNone) return 0.0f;
  const float a = f_scale_down(fx, ex - e), b = f_scale_down(fy, ey - e);   // the larger one is in [1, 2)
  return sqrtf(fmaf(a, a, b * b));
}
// a = |z| c (c >= 0) as t 2^e with t in [1, 6) (relative error below 2^-21);
// t = 0, e = kBoundNone for a = 0.
__device__ __forceinline__ float abs_prod_est(double2 z, double c, int &e, bool &odd) {
  int ez, ec;
  const float tz = abs_est(z, ez, odd), fc = dbl_lead_f(c, ec, odd);
  e = kBoundNone;
  if (fc == 0.0f || tz == 0.0f) return 0.0f;
  e = ez + ec;
  return tz * fc;
}
// floor(log2(|y| / |p|)) from the FP32 moduli (ratio_exp_fast's value, which
// uses FP64 squares): ok is cleared where the quotient lies within 2^-15 of a
// power of two (the estimate is within 2^-20) or an operand is zero,
// subnormal or not finite; the caller then takes ratio_exp_fast.
__device__ __forceinline__ int ratio_exp_est(double2 y, double2 p, bool &ok) {
  bool odd = false;
  int ey, ep;
  const float ty = abs_est(y, ey, odd), tp = abs_est(p, ep, odd);
  if (odd || ty == 0.0f || tp == 0.0f) {
    ok = false;
    return 0;
  }
  const unsigned b = __float_as_uint(__fdividef(ty, tp));
  const unsigned man = b & 0x7fffffu;
  ok = man >= 256u && man <= 0x7fffffu - 256u;
  return ey - ep + (int)(b >> 23) - 127;
}
// One term t 2^e of S into a running (max exponent, min exponent) pair.
__device__ __forceinline__ void alg4_term_exps(float t, int e, int &emax, int &emin) {
  if (t != 0.0f) {
    emax = max(emax, e);
    emin = min(emin, e);
  }
}
// The final Ka from the reduced quantities: em_max, the largest term exponent
// tmax, the smallest tmin, the FP32 sum s of the terms scaled by 2^-tmax
// (s >= 1 when some term is nonzero), odd.  Returns false when the chain must
// decide instead.
__device__ __forceinline__ bool alg4_block_ka(int em_max, int tmax, int tmin, float s, bool odd, int &Ka) {
  Ka = max(0, em_max - (kOmegaExp - 1));
  if (odd) return false;
  if (tmax == kBoundNone) return true;                  // S_N = 0: no "G >= Omega" rescale
  const unsigned b = __float_as_uint(s);
  const unsigned man = b & 0x7fffffu;
  if (man < 256u || man > 0x7fffffu - 256u) return false;   // within 2^-15 of a power of two
  const int eS = tmax + (int)(b >> 23) - 127;
  Ka = max(Ka, eS - (kOmegaExp - 1));
  return tmin - Ka >= -1020;                            // every term and bound stays normal
}

// z == 0 on the bit patterns, word by word.
__device__ __forceinline__ bool zzero_words(double2 z) {
  return ((((unsigned)__double2hiint(z.x) | (unsigned)__double2hiint(z.y)) & 0x7fffffffu) |
          (unsigned)__double2loint(z.x) | (unsigned)__double2loint(z.y)) == 0u;
}

// 1 / p = conj(p') / |p'|^2 2^-e with p' = p 2^-e (one real division); the
// scalings act on the exponent fields when every operand stays normal, with
// the same values as zdiv_fast.
__device__ __forceinline__ double2 zrecip(double2 p) {
  const unsigned hx = (unsigned)__double2hiint(p.x) & 0x7fffffffu, hy = (unsigned)__double2hiint(p.y) & 0x7fffffffu;
  const bool zx = (hx | (unsigned)__double2loint(p.x)) == 0u, zy = (hy | (unsigned)__double2loint(p.y)) == 0u;
  const int fx = (int)(hx >> 20), fy = (int)(hy >> 20);
  const int e = max(fx, fy) - 1023;                      // zexp(p) when unclamped
  const bool ok = max(fx, fy) != 0 && e >= -1021 && e <= 1021 && (zx || fx - e >= 1) && (zy || fy - e >= 1);
  if (!ok) return zdiv_fast(make_double2(1.0, 0.0), p);
  const int sh = e << 20;
  const double a = zx ? 0.0 : __hiloint2double(__double2hiint(p.x) - sh, __double2loint(p.x));
  const double b = zy ? 0.0 : __hiloint2double(__double2hiint(p.y) - sh, __double2loint(p.y));
  const double q = 1.0 / fma(a, a, b * b);               // |p'|^2 in [1, 8)
  const double wr = a * q, wi = -(b * q);                // each zero or of magnitude in (2^-1077, 2]
  // times 2^-e on the exponent fields where the result stays normal
  auto scale = [&](double w) {
    const int f = (__double2hiint(w) >> 20) & 0x7ff;
    if (f == 0) return w * pow2i(-e);                    // zero or subnormal: exact as zdiv_fast
    if (f - e < 1 || f - e > 2046) return w * pow2i(-e);
    return __hiloint2double(__double2hiint(w) - sh, __double2loint(w));
  };
  return make_double2(scale(wr), scale(wi));
}

// 16 bytes from global to shared memory without passing through registers
// (cp.async); when !full the 16 bytes are zero-filled and nothing is read.
// Both addresses are 16-byte aligned (complex arrays are).
__device__ __forceinline__ void cp_async16(void *dst, const void *src, bool full) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 16, %2;\n" ::"r"((unsigned)__cvta_generic_to_shared(dst)),
               "l"(src), "r"(full ? 16 : 0)
               : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

}  // namespace msts

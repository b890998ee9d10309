// msts_digits.cuh -- the error-free splitting of FP64 values into signed
// 7-bit digit planes used by the tensor-core products (the digit planes of a
// row or column share one power-of-two exponent), from the IEEE fields with
// integer operations only.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace msts {

constexpr int kOzS = 8;          // digit planes per operand
constexpr int kOzBits = 7;       // bits per digit

// floor(log2 max(|Re z|, |Im z|)) + 1, or INT_MIN/2 for z == 0, from the
// exponent fields (ilogb of a subnormal from its leading zeros).  Integer
// operations only: FP64 instructions and conversions are slow on this part.
__device__ __forceinline__ int bound_exp(double2 z) {
  const unsigned long long m = (unsigned long long)max(__double_as_longlong(z.x) & 0x7fffffffffffffffLL,
                                                       __double_as_longlong(z.y) & 0x7fffffffffffffffLL);
  if (m == 0ull) return -(1 << 29);
  const int f = (int)(m >> 52);
  return (f != 0 ? f - 1023 : (63 - __clzll((long long)m)) - 1074) + 1;
}

// The 8 signed 7-bit digits of a * 2^-e (|a| < 2^e), most significant first:
// those of M = trunc(|a| 2^(56 - e)), read off the 53-bit significand by a
// shift, each with the sign of a.  A digit c in [0, 127] becomes a float
// exactly through the low mantissa bits of 2^23.
__device__ __forceinline__ void digits8(double a, int e, float (&d)[kOzS]) {
  const unsigned long long bits = (unsigned long long)__double_as_longlong(a);
  const unsigned long long ab = bits & 0x7fffffffffffffffull;
  const int f = (int)(ab >> 52);
  const unsigned long long sig = (ab & 0xfffffffffffffull) | (f != 0 ? (1ull << 52) : 0ull);
  const int sh = max(f, 1) - 1075 + kOzS * kOzBits - e;      // |a| 2^(56 - e) = sig 2^sh
  const unsigned long long M = sh >= 0 ? (sh < 64 ? sig << sh : 0ull) : (sh > -64 ? sig >> -sh : 0ull);
  const bool neg = (bits >> 63) != 0ull;
#pragma unroll
  for (int s = 0; s < kOzS; ++s) {
    const unsigned c = (unsigned)(M >> (kOzBits * (kOzS - 1 - s))) & 127u;
    const float cf = __uint_as_float(0x4B000000u | c) - 8388608.0f;
    d[s] = neg ? -cf : cf;
  }
}

// The digit planes of x (2 x 8 floats: real and imaginary parts) packed as
// BF16 pairs (Re, Im) per plane, the layout of the X planes.
__device__ __forceinline__ void digit_pairs(double2 x, int e, uint32_t (&w)[kOzS]) {
  float dr[kOzS], di[kOzS];
  digits8(x.x, e, dr);
  digits8(x.y, e, di);
#pragma unroll
  for (int t = 0; t < kOzS; ++t)   // digits have <= 7 significant bits: the top half of a float is exact
    w[t] = (__float_as_uint(dr[t]) >> 16) | (__float_as_uint(di[t]) & 0xffff0000u);
}

}  // namespace msts

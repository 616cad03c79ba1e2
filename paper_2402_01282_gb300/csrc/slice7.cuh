// Exact integer slicing of float64 values for the float64-accurate tensor-core GEMMs
// (S2W_FP64_TC): fixed-point rounding, seven balanced base-128 digits as bf16, and the
// integer-only conversions of the epilogues.  Shared by the sliced contractions and the
// sliced DFTs.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <cmath>
#include <cstring>

#include "comp32.cuh"

namespace s2w {
namespace {

constexpr int kSl = 7;   // slices per value
// Digit-pair diagonals i + j = 0 .. 6 of a product of two sliced values are always summed (28
// pairs per K step); diagonal 7 (six more) when the plan asks for it.  The pairs of diagonal 7
// weigh up to ~2^-44 of a term, above the operands' own 47-bit rounding; diagonals 8 and up stay
// below 2^-51.  Accumulator q of diagonal q is exact either way.
constexpr int kDiag = kSl + 1;
// the slices (i, j = qq - i) of diagonal qq, both below kSl
__host__ __device__ constexpr int diag_lo(int qq) { return qq > kSl - 1 ? qq - (kSl - 1) : 0; }
__host__ __device__ constexpr int diag_hi(int qq) { return qq < kSl - 1 ? qq : kSl - 1; }

__device__ __forceinline__ int core16(int r, int k) { return ((r >> 3) * 2 + (k >> 3)) * 64 + (r & 7) * 8 + (k & 7); }

// biased float64 exponent of v (0 for zero and subnormals, which the slicing treats as zero)
__device__ __forceinline__ int bexp(double v) {
  return (int)((unsigned long long)__double_as_longlong(v) >> 52) & 0x7FF;
}

// round(v 2^(47 - e)) for |v| < 2^e, by integer operations on the float64 fields
__device__ __forceinline__ long long fix47(double v, int e) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(v);
  const int E = (int)(u >> 52) & 0x7FF;
  if (E == 0) return 0;
  const int sh = 1028 + e - E;   // >= 6 when |v| < 2^e
  if (sh >= 63) return 0;
  const unsigned long long M = (u & 0xFFFFFFFFFFFFFull) | (1ull << 52);
  const long long X = (long long)((M + (1ull << (sh - 1))) >> sh);
  return (u >> 63) ? -X : X;
}

// round(c r 2^(47 - e)) for |c r| < 2^e: the 106-bit product of the significands by one
// 64 x 64 high multiply (the bits below 2^53 of the product only decide exact ties)
__device__ __forceinline__ long long fix47_prod(double c, double r, int e) {
  const unsigned long long uc = (unsigned long long)__double_as_longlong(c);
  const unsigned long long ur = (unsigned long long)__double_as_longlong(r);
  const int Ec = (int)(uc >> 52) & 0x7FF, Er = (int)(ur >> 52) & 0x7FF;
  if (Ec == 0 || Er == 0) return 0;
  const int s2 = 2050 + e - Ec - Er;   // shift after the high multiply, >= 6 when |c r| < 2^e
  if (s2 >= 63) return 0;
  const unsigned long long Mc = (uc & 0xFFFFFFFFFFFFFull) | (1ull << 52);
  const unsigned long long Mr = (ur & 0xFFFFFFFFFFFFFull) | (1ull << 52);
  const unsigned long long H = __umul64hi(Mc << 11, Mr);   // floor(Mc Mr / 2^53)
  const long long X = (long long)((H + (1ull << (s2 - 1))) >> s2);
  return ((uc ^ ur) >> 63) ? -X : X;
}

// exponent bound of a value (max |v| < 2^e over values is the max of these), offset by 4096 so
// that a zero column (all bounds 0) reads as e = 0
constexpr int kEOff = 4096;
__device__ __forceinline__ int ebound(double v) {
  const int E = bexp(v);
  return E > 0 ? E - 1022 + kEOff : 0;
}
__device__ __forceinline__ int ebound_prod(double c, double r) {   // |c r| < 2^(Ec - 1022) 2^(Er - 1022)
  const int Ec = bexp(c), Er = bexp(r);
  return (Ec > 0 && Er > 0) ? Ec + Er - 2044 + kEOff : 0;
}
__device__ __forceinline__ int e_from(int eb) { return eb > 0 ? eb - kEOff : 0; }

// X (|X| < 2^48) -> seven balanced base-128 digits in [-64, 63], most significant first, as
// the float32 bit patterns of the digit values: the balanced digits are the plain base-128
// digits of X + 64 (128^7 - 1)/127, less 64; each float is exact, and its upper 16 bits are
// the bfloat16 encoding of the same value.
constexpr long long kDigitBias = 283691315109952ll;   // 64 (128^7 - 1)/127
__device__ __forceinline__ void digits7(long long X, uint32_t (&f)[kSl]) {
  const unsigned long long Y = (unsigned long long)(X + kDigitBias);
#pragma unroll
  for (int i = 0; i < kSl; ++i) {
    const unsigned int u = (unsigned int)(Y >> (7 * (kSl - 1 - i))) & 127u;
    f[i] = __float_as_uint(__uint_as_float(0x4B000000u | u) - 8388672.0f);   // u - 64
  }
}

// 2^k x for a float64 x, by the exponent field (zero below the normal range)
__device__ __forceinline__ double scale2(double x, int k) {
  const long long b = __double_as_longlong(x);
  const int E = (int)((unsigned long long)b >> 52) & 0x7FF;
  if (E == 0) return 0.0;
  const int En = E + k;
  if (En <= 0) return 0.0;
  if (En >= 2047) return __longlong_as_double((b & (long long)0x8000000000000000ull) | 0x7FF0000000000000ll);
  return __longlong_as_double(b + ((long long)k << 52));
}

__device__ __forceinline__ double neg(double x) {
  return __longlong_as_double(__double_as_longlong(x) ^ (long long)0x8000000000000000ull);
}

// float -> float64 with integer operations (exact for normal floats; subnormals give 0)
__device__ __forceinline__ double f2d(float f) {
  const unsigned int u = __float_as_uint(f);
  const unsigned int e = (u >> 23) & 0xFFu;
  if (e == 0u) return 0.0;
  const unsigned long long b = ((unsigned long long)(u & 0x80000000u) << 32) |
                               ((unsigned long long)(e + 896u) << 52) | ((unsigned long long)(u & 0x7FFFFFu) << 29);
  return __longlong_as_double((long long)b);
}

// round(x 2^(47 - f)) for a float x with |x| < 2^f, by integer operations on its fields
__device__ __forceinline__ long long fixf(float x, int f) {
  const unsigned int u = __float_as_uint(x);
  const int E = (int)((u >> 23) & 0xFFu);
  if (E == 0) return 0;
  const long long M = (long long)((u & 0x7FFFFFu) | 0x800000u);   // |x| = M 2^(E - 150)
  const int sh = 103 + f - E;                                       // X = M 2^-sh
  long long X;
  if (sh <= 0) X = M << (-sh);
  else if (sh >= 25) X = 0;
  else X = (M + (1ll << (sh - 1))) >> sh;
  return (u >> 31) ? -X : X;
}
// the same for a float pair hi + lo (|hi + lo| < 2^f): the two parts rounded separately
__device__ __forceinline__ long long fixf_pair(float hi, float lo, int f) { return fixf(hi, f) + fixf(lo, f); }
// exponent bound of a float pair hi + lo (renormalised): |hi + lo| < 2^e; 0 for zero
__device__ __forceinline__ int fbound(float hi) {
  const int E = (int)((__float_as_uint(hi) >> 23) & 0xFFu);
  return E > 0 ? E - 126 + kEOff : 0;
}

// host: the seven bf16 slices of round(v 2^(47 - e)) in the device digit convention above
inline void host_digits(double v, int e, uint16_t (&d)[kSl]) {
  const long long X = std::llround(std::ldexp(v, 47 - e));
  const unsigned long long Y = (unsigned long long)(X + kDigitBias);
  for (int i = 0; i < kSl; ++i) {
    const int u = (int)((Y >> (7 * (kSl - 1 - i))) & 127u) - 64;
    const float f = (float)u;
    uint32_t bits;
    std::memcpy(&bits, &f, sizeof(bits));
    d[i] = (uint16_t)(bits >> 16);
  }
}

// a += x exactly as a pair (TwoSum into the high part, the error into the low part)
__device__ __forceinline__ void two_sum_add(Acc& a, float x) {
  const float s = __fadd_rn(a.s, x);
  const float z = __fsub_rn(s, a.s);
  const float t = __fadd_rn(__fsub_rn(a.s, __fsub_rn(s, z)), __fsub_rn(x, z));
  a.s = s;
  a.c = __fadd_rn(a.c, t);
}

}  // namespace
}  // namespace s2w

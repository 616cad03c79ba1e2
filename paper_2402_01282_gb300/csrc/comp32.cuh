// Compensated float32 arithmetic: a value is an unevaluated pair hi + lo of floats
// (~48 significant bits).  Products are split exactly with an FMA (TwoProduct), running
// sums with TwoSum; rounding errors and the cross terms hi*lo + lo*hi are accumulated in a
// float compensation term (the compensated dot product of Ogita, Rump and Oishi, 2005,
// extended to paired inputs).  Explicit _rn intrinsics keep nvcc from contracting the
// error-free transformations into FMAs.
#pragma once
#include <cuda_runtime.h>

namespace s2w {

struct Acc {
  float s, c;   // value s + c
};

// a += (xh + xl) * (wh + wl), dropping only xl*wl (2^-48 relative).
__device__ __forceinline__ void acc_add(Acc& a, float xh, float xl, float wh, float wl) {
  const float p = __fmul_rn(xh, wh);
  const float e = fmaf(xh, wh, -p);               // xh*wh = p + e exactly
  const float s = __fadd_rn(a.s, p);
  const float z = __fsub_rn(s, a.s);
  const float t = __fadd_rn(__fsub_rn(a.s, __fsub_rn(s, z)), __fsub_rn(p, z));   // a.s + p = s + t
  a.s = s;
  a.c = fmaf(xh, wl, fmaf(xl, wh, __fadd_rn(a.c, __fadd_rn(t, e))));
}

// (h, l) with h + l = s + c and |l| <= ulp(h)/2
__device__ __forceinline__ float2 renorm(Acc a) {
  const float h = __fadd_rn(a.s, a.c);
  const float l = __fsub_rn(a.c, __fsub_rn(h, a.s));
  return make_float2(h, l);
}

__device__ __forceinline__ double to_double(Acc a) { return (double)a.s + (double)a.c; }

// float64 -> pair
__device__ __forceinline__ float2 split1(double v) {
  const float h = __double2float_rn(v);
  return make_float2(h, __double2float_rn(v - (double)h));
}

// complex float64 -> (re_hi, re_lo, im_hi, im_lo)
__device__ __forceinline__ float4 split(double2 v) {
  const float2 r = split1(v.x), i = split1(v.y);
  return make_float4(r.x, r.y, i.x, i.y);
}

}  // namespace s2w

namespace s2w {

// float64 -> pair with integer operations only (no conversion on the float64 pipe):
// hi = v truncated to 24 significant bits, lo = the remaining 29 mantissa bits truncated to
// 24, so hi + lo = v to 2^-48 relative.  |v| < 2^-126 returns (0, 0) and lo is dropped once it
// falls below the float range (|v| < ~2^-75): both are far below any term these kernels sum.
// NaN stays NaN, and Inf or a value beyond the float range (|v| >= 2^128) becomes Inf, so that
// a non-finite input stays visible to the checks downstream instead of becoming a finite float.
__device__ __forceinline__ float2 split1_bits(double v) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(v);
  const unsigned int hi32 = (unsigned int)(u >> 32), lo32 = (unsigned int)u;
  const int E = (int)((hi32 >> 20) & 0x7FFu) - 1023;
  if (E < -126) return make_float2(0.f, 0.f);
  const unsigned int sign = hi32 & 0x80000000u;
  if (E >= 128) {
    const bool nan = E == 1024 && ((hi32 & 0xFFFFFu) | lo32) != 0u;
    return make_float2(__uint_as_float(sign | 0x7F800000u | (nan ? 0x400000u : 0u)), 0.f);
  }
  const unsigned int mant23 = ((hi32 & 0xFFFFFu) << 3) | (lo32 >> 29);
  const float h = __uint_as_float(sign | ((unsigned int)(E + 127) << 23) | mant23);
  const unsigned int r = lo32 & 0x1FFFFFFFu;
  float l = 0.f;
  if (r != 0u) {
    const int lead = 31 - __clz((int)r);
    const int field = E - 52 + lead + 127;
    if (field > 0) {
      const unsigned int m = (lead >= 23 ? (r >> (lead - 23)) : (r << (23 - lead))) & 0x7FFFFFu;
      l = __uint_as_float(sign | ((unsigned int)field << 23) | m);
    }
  }
  return make_float2(h, l);
}

}  // namespace s2w

namespace s2w {
// two accumulators (real, imaginary) -> (re_hi, re_lo, im_hi, im_lo)
__device__ __forceinline__ float4 pack_pair(Acc re, Acc im) {
  const float2 r = renorm(re), i = renorm(im);
  return make_float4(r.x, r.y, i.x, i.y);
}
}  // namespace s2w

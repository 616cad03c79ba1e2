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

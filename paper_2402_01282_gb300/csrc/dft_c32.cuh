// Compensated-float32 complex helpers of the azimuthal and gamma DFTs, shared by the
// compensated DFT kernels and the prologue/epilogue of the tensor-core DFTs.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "comp32.cuh"

namespace s2w {
namespace {

// complex pair layout: float4 (re_hi, re_lo, im_hi, im_lo).  PLAIN: ordinary float32
// arithmetic on the hi parts (the reduced-precision modes), otherwise compensated.
template <int SIGN, bool PLAIN>
__device__ __forceinline__ void cmac(Acc& re, Acc& im, const float4 x, const float4 w) {
  const float wih = SIGN > 0 ? w.z : -w.z, wil = SIGN > 0 ? w.w : -w.w;
  if (PLAIN) {
    re.s = fmaf(x.x, w.x, fmaf(-x.z, wih, re.s));
    im.s = fmaf(x.x, wih, fmaf(x.z, w.x, im.s));
    return;
  }
  acc_add(re, x.x, x.y, w.x, w.y);
  acc_add(re, -x.z, -x.w, wih, wil);
  acc_add(im, x.x, x.y, wih, wil);
  acc_add(im, x.z, x.w, w.x, w.y);
}

template <bool PLAIN>
__device__ __forceinline__ float4 pack(Acc re, Acc im) {
  if (PLAIN) return make_float4(re.s, 0.f, im.s, 0.f);
  const float2 r = renorm(re), i = renorm(im);
  return make_float4(r.x, r.y, i.x, i.y);
}

// (ah + al) + (bh + bl) as a renormalised pair
__device__ __forceinline__ float2 add_pair(float ah, float al, float bh, float bl) {
  const float s = __fadd_rn(ah, bh);
  const float z = __fsub_rn(s, ah);
  const float e = __fadd_rn(__fadd_rn(__fsub_rn(ah, __fsub_rn(s, z)), __fsub_rn(bh, z)), __fadd_rn(al, bl));
  const float h = __fadd_rn(s, e);
  return make_float2(h, __fsub_rn(e, __fsub_rn(h, s)));
}

template <bool PLAIN>
__device__ __forceinline__ float4 cadd(float4 x, float4 y, float sy) {   // x + sy * y, sy = +-1
  if (PLAIN) return make_float4(x.x + sy * y.x, 0.f, x.z + sy * y.z, 0.f);
  const float2 r = add_pair(x.x, x.y, sy * y.x, sy * y.y), i = add_pair(x.z, x.w, sy * y.z, sy * y.w);
  return make_float4(r.x, r.y, i.x, i.y);
}

template <bool PLAIN>
__device__ __forceinline__ Acc comb(Acc a, float sb, Acc b) {   // a + sb * b
  if (PLAIN) return Acc{a.s + sb * b.s, 0.f};
  const float2 r = add_pair(a.s, a.c, sb * b.s, sb * b.c);
  return Acc{r.x, r.y};
}

template <bool PLAIN>
__device__ __forceinline__ void racc(Acc& a, float xh, float xl, float wh, float wl) {   // a += x w (real)
  if (PLAIN) a.s = fmaf(xh, wh, a.s);
  else acc_add(a, xh, xl, wh, wl);
}

// ----------------------------------------------------------- gamma on the map side
// SO(3) transforms: the gamma DFT is taken on the map side of the alpha DFT (forward: gamma
// first, inverse: gamma last), so one complex alpha DFT of length n serves each carried n
// instead of one per gamma sample.  For real signals G_{-m,-n} = conj G_{m,n}: one complex
// transform over all n outputs gives both n and -n (m >= 0 of each), so only the n >= 0 values
// are transformed ("jobs").  The gamma sums pair gamma_g with gamma_{Ng-g} like the stages above.
constexpr int kMaxJobs = 64;
constexpr int kJobChunk = 4;   // jobs whose gamma sums share one pass over the samples

__device__ __forceinline__ void make_jobs(const int* nvals, int nact, bool real, int* jn, int* jp, int& nj) {
  nj = 0;
  for (int ni = 0; ni < nact && nj < kMaxJobs; ++ni) {
    const int v = nvals[ni];
    if (real && v < 0) continue;
    int partner = -1;
    if (real && v > 0)
      for (int q = 0; q < nact; ++q)
        if (nvals[q] == -v) partner = q;
    jn[nj] = ni;
    jp[nj] = partner;
    ++nj;
  }
}

__device__ __forceinline__ float4 load_pix(const void* pix, bool real, int64_t i) {
  if (real) {
    const float2 v = split1_bits(((const double*)pix)[i]);
    return make_float4(v.x, v.y, 0.f, 0.f);
  }
  const double2 v = ((const double2*)pix)[i];
  const float2 r = split1_bits(v.x), im = split1_bits(v.y);
  return make_float4(r.x, r.y, im.x, im.y);
}

}  // namespace
}  // namespace s2w

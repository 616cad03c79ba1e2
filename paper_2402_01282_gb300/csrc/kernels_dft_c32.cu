// Azimuthal (alpha/phi) and gamma DFTs (Sec. 5.2, Eq. 48) in compensated float32.
//
// GB300 runs float32 at ~62x its float64 rate, so these fixed-coefficient linear maps
// carry every value as an unevaluated pair hi + lo of floats (~48 significant bits) and
// accumulate with error-free transformations: each product hi*hi is split exactly into
// p + e with an FMA, each running sum is split exactly with TwoSum, and the rounding
// errors plus the cross terms hi*lo + lo*hi go to a float compensation term (the
// compensated dot product of Ogita, Rump and Oishi, extended to paired inputs).  Inputs and
// outputs are float64; twiddles are float64 values split into pairs on the host.
#include <math.h>

#include "comp32.cuh"
#include "s2w_internal.h"

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

template <int SIGN, bool PLAIN>
__device__ void stage1(const float4* x, float4* tmp, const float4* tw, int n, int n1, int n2) {
  for (int idx = threadIdx.x; idx < n; idx += blockDim.x) {
    const int k1 = idx / n2, j2 = idx - k1 * n2;
    const int step = (n2 * k1) % n;
    Acc re{0.f, 0.f}, im{0.f, 0.f};
    int e = 0;
    for (int j1 = 0; j1 < n1; ++j1) {
      cmac<SIGN, PLAIN>(re, im, x[n2 * j1 + j2], tw[e]);
      e += step;
      if (e >= n) e -= n;
    }
    const float4 v = pack<PLAIN>(re, im);
    Acc r2{0.f, 0.f}, i2{0.f, 0.f};
    cmac<SIGN, PLAIN>(r2, i2, v, tw[(j2 * k1) % n]);
    tmp[k1 * n2 + j2] = pack<PLAIN>(r2, i2);
  }
}

template <int SIGN, bool REAL_ONLY, bool PLAIN>
__device__ __forceinline__ void stage2_one(const float4* tmp, const float4* tw, int n, int n1, int n2, int k,
                                           Acc& re, Acc& im) {
  const int k1 = k % n1, k2 = k / n1;
  const int step = (n1 * k2) % n;
  const float4* row = tmp + k1 * n2;
  re = Acc{0.f, 0.f};
  im = Acc{0.f, 0.f};
  int e = 0;
  for (int j2 = 0; j2 < n2; ++j2) {
    const float4 v = row[j2];
    const float4 w = tw[e];
    const float wih = SIGN > 0 ? w.z : -w.z, wil = SIGN > 0 ? w.w : -w.w;
    if (PLAIN) {
      re.s = fmaf(v.x, w.x, fmaf(-v.z, wih, re.s));
      if (!REAL_ONLY) im.s = fmaf(v.x, wih, fmaf(v.z, w.x, im.s));
    } else {
      acc_add(re, v.x, v.y, w.x, w.y);
      acc_add(re, -v.z, -v.w, wih, wil);
      if (!REAL_ONLY) {
        acc_add(im, v.x, v.y, wih, wil);
        acc_add(im, v.z, v.w, w.x, w.y);
      }
    }
    e += step;
    if (e >= n) e -= n;
  }
}

struct DftcArgs {
  const void* pix_in;
  void* pix_out;
  int64_t pix_sb;
  double2* G;           // [B][nact][L][Mc] float64 columns
  int B, nact, Ng, L, Mc, mlo, n, n1, n2;
  const float4* tw;     // [n] exp(+2 pi i e/n) as pairs
  const float4* gph;    // [nact][Ng] exp(+i n gamma_g) as pairs
  double scale;
};

template <bool REAL, bool PLAIN>
__global__ void k_dftc_fwd(DftcArgs a) {
  extern __shared__ float4 s4[];
  const int n = a.n, t = blockIdx.x, b = blockIdx.y;
  float4* tw = s4;
  float4* x = tw + n;
  float4* tmp = x + n;
  float4* H = tmp + n;   // [Ng][Mc]
  for (int i = threadIdx.x; i < n; i += blockDim.x) tw[i] = a.tw[i];
  const int64_t ring = (int64_t)a.L * n;
  for (int g = 0; g < a.Ng; ++g) {
    __syncthreads();
    const int64_t base = (int64_t)b * a.pix_sb + (int64_t)g * ring + (int64_t)t * n;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      if (REAL) x[i] = split(make_double2(((const double*)a.pix_in)[base + i], 0.0));
      else x[i] = split(((const double2*)a.pix_in)[base + i]);
    }
    __syncthreads();
    stage1<-1, PLAIN>(x, tmp, tw, n, a.n1, a.n2);
    __syncthreads();
    for (int mi = threadIdx.x; mi < a.Mc; mi += blockDim.x) {
      int k = a.mlo + mi;
      if (k < 0) k += n;
      Acc re, im;
      stage2_one<-1, false, PLAIN>(tmp, tw, n, a.n1, a.n2, k, re, im);
      H[g * a.Mc + mi] = pack<PLAIN>(re, im);
    }
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < a.nact * a.Mc; idx += blockDim.x) {
    const int ni = idx / a.Mc, mi = idx - ni * a.Mc;
    Acc re{0.f, 0.f}, im{0.f, 0.f};
    for (int g = 0; g < a.Ng; ++g) cmac<-1, PLAIN>(re, im, H[g * a.Mc + mi], a.gph[ni * a.Ng + g]);
    a.G[(((int64_t)b * a.nact + ni) * a.L + t) * a.Mc + mi] =
        make_double2(to_double(re) * a.scale, to_double(im) * a.scale);
  }
}

template <bool REAL, bool PLAIN>
__global__ void k_dftc_inv(DftcArgs a) {
  extern __shared__ float4 s4[];
  const int n = a.n, t = blockIdx.x, b = blockIdx.y;
  float4* tw = s4;
  float4* x = tw + n;
  float4* tmp = x + n;
  float4* Gs = tmp + n;  // [nact][Mc]
  for (int i = threadIdx.x; i < n; i += blockDim.x) tw[i] = a.tw[i];
  for (int idx = threadIdx.x; idx < a.nact * a.Mc; idx += blockDim.x) {
    const int ni = idx / a.Mc, mi = idx - ni * a.Mc;
    Gs[idx] = split(a.G[(((int64_t)b * a.nact + ni) * a.L + t) * a.Mc + mi]);
  }
  const int64_t ring = (int64_t)a.L * n;
  for (int g = 0; g < a.Ng; ++g) {
    __syncthreads();
    for (int mi = threadIdx.x; mi < a.Mc; mi += blockDim.x) {
      Acc re{0.f, 0.f}, im{0.f, 0.f};
      for (int ni = 0; ni < a.nact; ++ni) cmac<1, PLAIN>(re, im, Gs[ni * a.Mc + mi], a.gph[ni * a.Ng + g]);
      const float4 v = pack<PLAIN>(re, im);
      const int m = a.mlo + mi;
      if (REAL) {
        x[m] = v;
        if (m > 0) x[n - m] = make_float4(v.x, v.y, -v.z, -v.w);
      } else {
        x[m < 0 ? m + n : m] = v;
      }
    }
    __syncthreads();
    stage1<1, PLAIN>(x, tmp, tw, n, a.n1, a.n2);
    __syncthreads();
    const int64_t base = (int64_t)b * a.pix_sb + (int64_t)g * ring + (int64_t)t * n;
    for (int k = threadIdx.x; k < n; k += blockDim.x) {
      Acc re, im;
      if (REAL) {
        stage2_one<1, true, PLAIN>(tmp, tw, n, a.n1, a.n2, k, re, im);
        ((double*)a.pix_out)[base + k] = to_double(re);
      } else {
        stage2_one<1, false, PLAIN>(tmp, tw, n, a.n1, a.n2, k, re, im);
        ((double2*)a.pix_out)[base + k] = make_double2(to_double(re), to_double(im));
      }
    }
  }
}

DftcArgs make_args(const GridTables& g, const TransformSpec& t, ColumnArgs c) {
  DftcArgs a;
  a.G = c.G;
  a.B = c.B;
  a.nact = c.nact;
  a.Ng = 2 * t.N - 1;
  a.L = c.L;
  a.Mc = c.Mc;
  a.mlo = c.mlo;
  a.n = g.n;
  a.n1 = g.n1;
  a.n2 = g.n2;
  a.tw = g.tw4;
  a.gph = t.gphase4;
  a.scale = 0.0;
  return a;
}

template <class K>
cudaError_t launch(K kern, dim3 grid, size_t smem, cudaStream_t st, const DftcArgs& a) {
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  kern<<<grid, 256, smem, st>>>(a);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_dftc_forward(const GridTables& g, const TransformSpec& t, const void* pix, int64_t pix_sb,
                                bool real, ColumnArgs c, cudaStream_t st, bool plain) {
  DftcArgs a = make_args(g, t, c);
  a.pix_in = pix;
  a.pix_out = nullptr;
  a.pix_sb = pix_sb;
  a.scale = (2.0 * 3.14159265358979323846 / g.n) * t.gscale;
  const size_t smem = (size_t)(3 * g.n + a.Ng * c.Mc) * sizeof(float4);
  dim3 grid(c.L, c.B);
  if (plain) return real ? launch(k_dftc_fwd<true, true>, grid, smem, st, a) : launch(k_dftc_fwd<false, true>, grid, smem, st, a);
  return real ? launch(k_dftc_fwd<true, false>, grid, smem, st, a) : launch(k_dftc_fwd<false, false>, grid, smem, st, a);
}

cudaError_t launch_dftc_inverse(const GridTables& g, const TransformSpec& t, ColumnArgs c, void* pix,
                                int64_t pix_sb, bool real, cudaStream_t st, bool plain) {
  DftcArgs a = make_args(g, t, c);
  a.pix_in = nullptr;
  a.pix_out = pix;
  a.pix_sb = pix_sb;
  const size_t smem = (size_t)(3 * g.n + c.nact * c.Mc) * sizeof(float4);
  dim3 grid(c.L, c.B);
  if (plain) return real ? launch(k_dftc_inv<true, true>, grid, smem, st, a) : launch(k_dftc_inv<false, true>, grid, smem, st, a);
  return real ? launch(k_dftc_inv<true, false>, grid, smem, st, a) : launch(k_dftc_inv<false, false>, grid, smem, st, a);
}

}  // namespace s2w

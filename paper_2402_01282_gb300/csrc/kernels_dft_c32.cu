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

#include <algorithm>

#include "comp32.cuh"
#include "dft_c32.cuh"
#include "s2w_internal.h"

namespace s2w {
namespace {

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
  double2* G;           // [B][nact][nr][Mc] float64 columns
  int B, nact, Ng, L, nr, Mc, mlo, n, n1, n2;
  const float4* tw;     // [n] exp(+2 pi i e/n) as pairs
  const float4* gph;    // [nact][Ng] exp(+i n gamma_g) as pairs
  const int* nvals;     // [nact] the n values carried
  double scale;
  int jb;               // jobs per pass of the two alpha stages (gamma-side kernels)
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
  const int64_t ring = (int64_t)a.nr * n;
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
    a.G[(((int64_t)b * a.nact + ni) * a.nr + t) * a.Mc + mi] =
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
    Gs[idx] = split(a.G[(((int64_t)b * a.nact + ni) * a.nr + t) * a.Mc + mi]);
  }
  const int64_t ring = (int64_t)a.nr * n;
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

// ------------------------------------------------- symmetric odd-length DFT stages
// Every length here is odd (n = 2L-1 = n1 n2, Ng = 2N-1).  An odd-length DFT
// X(k) = sum_j x_j w^{SIGN j k} (w = exp(2 pi i/p), h = (p-1)/2) pairs index j with p - j:
//   X(0) = sum_j x_j,   X(k), X(p-k) = x_0 + C_k +- SIGN i S_k   (1 <= k <= h)
//   C_k = sum_{j=1..h} a_j cos(2 pi j k/p),  S_k = sum_{j=1..h} b_j sin(2 pi j k/p),
//   a_j = x_j + x_{p-j},  b_j = x_j - x_{p-j},
// so each pair of outputs costs 2h complex-times-real products: a quarter of the direct sum.

// Stage 1: for every column j2, the length-n1 DFT over j1 of x[n2 j1 + j2], times the twiddle
// w_n^{SIGN j2 k1}, into tmp[k1 n2 + j2].  nb transforms at once (x, tmp advance by n per
// transform).  Work items: (transform, j2, output pair).
template <int SIGN, bool PLAIN>
__device__ void stage1_sym(const float4* x0b, float4* tmp0, const float4* tw, int n, int n1, int n2, int nb) {
  const int h1 = (n1 - 1) / 2, per = n2 * (h1 + 1), nit = nb * per;
  for (int it0 = threadIdx.x; it0 < nit; it0 += blockDim.x) {
    const int qb = it0 / per, it = it0 - qb * per;
    const float4* x = x0b + qb * n;
    float4* tmp = tmp0 + qb * n;
    const int j2 = it / (h1 + 1), kk = it - j2 * (h1 + 1);
    const float4 x0 = x[j2];
    if (kk == 0) {
      Acc re{x0.x, x0.y}, im{x0.z, x0.w};
      for (int j = 1; j < n1; ++j) {
        const float4 v = x[n2 * j + j2];
        racc<PLAIN>(re, v.x, v.y, 1.f, 0.f);
        racc<PLAIN>(im, v.z, v.w, 1.f, 0.f);
      }
      tmp[j2] = pack<PLAIN>(re, im);
      continue;
    }
    Acc cr{x0.x, x0.y}, ci{x0.z, x0.w}, sr{0.f, 0.f}, si{0.f, 0.f};
    const int step = (n2 * kk) % n;
    int e = step;
    for (int j = 1; j <= h1; ++j) {
      const float4 u = x[n2 * j + j2], v = x[n2 * (n1 - j) + j2];
      const float4 a = cadd<PLAIN>(u, v, 1.f), b = cadd<PLAIN>(u, v, -1.f);
      const float4 w = tw[e];
      racc<PLAIN>(cr, a.x, a.y, w.x, w.y);
      racc<PLAIN>(ci, a.z, a.w, w.x, w.y);
      racc<PLAIN>(sr, b.x, b.y, w.z, w.w);
      racc<PLAIN>(si, b.z, b.w, w.z, w.w);
      e += step;
      if (e >= n) e -= n;
    }
    const float sg = (float)SIGN;
#pragma unroll
    for (int side = 0; side < 2; ++side) {
      const float t = side == 0 ? sg : -sg;   // X(kk) = C + SIGN i S, X(n1 - kk) = C - SIGN i S
      const Acc xr = comb<PLAIN>(cr, -t, si), xi = comb<PLAIN>(ci, t, sr);
      const int k1 = side == 0 ? kk : n1 - kk;
      Acc r{0.f, 0.f}, i{0.f, 0.f};
      cmac<SIGN, PLAIN>(r, i, make_float4(xr.s, xr.c, xi.s, xi.c), tw[(j2 * k1) % n]);
      tmp[k1 * n2 + j2] = pack<PLAIN>(r, i);
    }
  }
}

// Stage 2: for every row k1, the length-n2 DFT of tmp[k1 n2 + j2] over j2; output k1 + n1 k2
// of transform qb goes to store(qb, k, re, im).  nb transforms at once (tmp and AB advance by
// n per transform); AB receives the row sums and differences first.
template <int SIGN, bool PLAIN, class Store>
__device__ void stage2_sym(const float4* tmp0, float4* AB0, const float4* tw, int n, int n1, int n2, int nb,
                           Store store) {
  const int h2 = (n2 - 1) / 2, pera = n1 * h2;
  for (int it0 = threadIdx.x; it0 < nb * pera; it0 += blockDim.x) {
    const int qb = it0 / pera, it = it0 - qb * pera;
    const int k1 = it / h2, j = it - k1 * h2 + 1;
    const float4* row = tmp0 + qb * n + k1 * n2;
    float4* AB = AB0 + qb * n;
    AB[2 * it] = cadd<PLAIN>(row[j], row[n2 - j], 1.f);
    AB[2 * it + 1] = cadd<PLAIN>(row[j], row[n2 - j], -1.f);
  }
  __syncthreads();
  const int per = n1 * (h2 + 1), nit = nb * per;
  for (int it0 = threadIdx.x; it0 < nit; it0 += blockDim.x) {
    const int qb = it0 / per, it = it0 - qb * per;
    const float4* tmp = tmp0 + qb * n;
    const float4* AB = AB0 + qb * n;
    const int k1 = it / (h2 + 1), kk = it - k1 * (h2 + 1);
    const float4 x0 = tmp[k1 * n2];
    const float4* ab = AB + 2 * k1 * h2;
    if (kk == 0) {
      Acc re{x0.x, x0.y}, im{x0.z, x0.w};
      for (int j = 0; j < h2; ++j) {
        const float4 a = ab[2 * j];
        racc<PLAIN>(re, a.x, a.y, 1.f, 0.f);
        racc<PLAIN>(im, a.z, a.w, 1.f, 0.f);
      }
      store(qb, k1, re, im);
      continue;
    }
    Acc cr{x0.x, x0.y}, ci{x0.z, x0.w}, sr{0.f, 0.f}, si{0.f, 0.f};
    const int step = (n1 * kk) % n;
    if (PLAIN) {
      // float32 arithmetic: the twiddles cos, sin(2 pi p kk/n2) by the rotation recurrence
      // instead of a table load per p, re-seeded from the table every 16 steps so that its error
      // stays ~16 2^-24 whatever the length (a plain recurrence errs ~p 2^-24)
      const float4 w1 = tw[step];
      float wr = w1.x, wi = w1.z;
      int e = step;   // table index of the twiddle of pair p = j + 1
      for (int j = 0; j < h2; ++j) {
        const float4 a = ab[2 * j], b = ab[2 * j + 1];
        cr.s = fmaf(a.x, wr, cr.s);
        ci.s = fmaf(a.z, wr, ci.s);
        sr.s = fmaf(b.x, wi, sr.s);
        si.s = fmaf(b.z, wi, si.s);
        e += step;
        if (e >= n) e -= n;
        if ((j & 15) == 15) {
          const float4 w = tw[e];
          wr = w.x;
          wi = w.z;
        } else {
          const float t = fmaf(wr, w1.x, -wi * w1.z);
          wi = fmaf(wr, w1.z, wi * w1.x);
          wr = t;
        }
      }
    } else {
      int e = step;
      for (int j = 0; j < h2; ++j) {
        const float4 a = ab[2 * j], b = ab[2 * j + 1];
        const float4 w = tw[e];
        racc<PLAIN>(cr, a.x, a.y, w.x, w.y);
        racc<PLAIN>(ci, a.z, a.w, w.x, w.y);
        racc<PLAIN>(sr, b.x, b.y, w.z, w.w);
        racc<PLAIN>(si, b.z, b.w, w.z, w.w);
        e += step;
        if (e >= n) e -= n;
      }
    }
    const float sg = (float)SIGN;
    store(qb, k1 + n1 * kk, comb<PLAIN>(cr, -sg, si), comb<PLAIN>(ci, sg, sr));
    store(qb, k1 + n1 * (n2 - kk), comb<PLAIN>(cr, sg, si), comb<PLAIN>(ci, -sg, sr));
  }
}

template <bool REAL, bool PLAIN>
__global__ void k_dftg_fwd(DftcArgs a) {
  extern __shared__ float4 s4[];
  __shared__ int jn[kMaxJobs], jp[kMaxJobs], njs;
  const int n = a.n, L = a.L, t = blockIdx.x, b = blockIdx.y;
  if (threadIdx.x == 0) {
    int nj;
    make_jobs(a.nvals, a.nact, REAL, jn, jp, nj);
    njs = nj;
  }
  __syncthreads();
  const int nj = njs, JB = a.jb;
  float4* tw = s4;
  float4* HZ = tw + n;        // [jobs][n]
  float4* tmp = HZ + nj * n;  // [JB][n]
  float4* AB = tmp + JB * n;  // [JB][n]
  for (int i = threadIdx.x; i < n; i += blockDim.x) tw[i] = a.tw[i];
  __syncthreads();
  const int Ng = a.Ng, hg = (Ng - 1) / 2;
  const int64_t ring = (int64_t)a.nr * n;
  const int64_t base = (int64_t)b * a.pix_sb + (int64_t)t * n;
  // H_j(alpha) = sum_g W(alpha, gamma_g) exp(-i n_j gamma_g)
  for (int j0 = 0; j0 < nj; j0 += kJobChunk) {
    const int jc = min(kJobChunk, nj - j0);
    for (int al = threadIdx.x; al < n; al += blockDim.x) {
      const float4 w0 = load_pix(a.pix_in, REAL, base + al);
      Acc hr[kJobChunk], hi[kJobChunk];
#pragma unroll
      for (int q = 0; q < kJobChunk; ++q) {
        hr[q] = Acc{w0.x, w0.y};
        hi[q] = Acc{w0.z, w0.w};
      }
      for (int g = 1; g <= hg; ++g) {
        const float4 xp = load_pix(a.pix_in, REAL, base + g * ring + al);
        const float4 xm = load_pix(a.pix_in, REAL, base + (Ng - g) * ring + al);
        const float4 u = cadd<PLAIN>(xp, xm, 1.f), v = cadd<PLAIN>(xp, xm, -1.f);
#pragma unroll
        for (int q = 0; q < kJobChunk; ++q) {
          if (q < jc) {
            const float4 ph = a.gph[jn[j0 + q] * Ng + g];   // cos, sin of n gamma_g
            // u cos - i v sin
            racc<PLAIN>(hr[q], u.x, u.y, ph.x, ph.y);
            racc<PLAIN>(hi[q], v.x, v.y, -ph.z, -ph.w);
            if (!REAL) {
              racc<PLAIN>(hr[q], v.z, v.w, ph.z, ph.w);
              racc<PLAIN>(hi[q], u.z, u.w, ph.x, ph.y);
            }
          }
        }
      }
#pragma unroll
      for (int q = 0; q < kJobChunk; ++q)
        if (q < jc) HZ[(j0 + q) * n + al] = pack<PLAIN>(hr[q], hi[q]);
    }
  }
  // one complex alpha DFT per job, JB jobs per pass of the two stages
  for (int jb0 = 0; jb0 < nj; jb0 += JB) {
    const int nb = min(JB, nj - jb0);
    __syncthreads();
    stage1_sym<-1, PLAIN>(HZ + jb0 * n, tmp, tw, n, a.n1, a.n2, nb);
    __syncthreads();
    const double sc = a.scale;
    const int mlo = a.mlo;
    stage2_sym<-1, PLAIN>(tmp, AB, tw, n, a.n1, a.n2, nb, [&](int qb, int k, Acc re, Acc im) {
      const int ni = jn[jb0 + qb], pi = jp[jb0 + qb];
      double2* Gn = a.G + (((int64_t)b * a.nact + ni) * a.nr + t) * a.Mc;
      double2* Gp = (pi >= 0) ? a.G + (((int64_t)b * a.nact + pi) * a.nr + t) * a.Mc : nullptr;
      const double zr = to_double(re) * sc, zi = to_double(im) * sc;
      if (REAL) {
        if (k < L) Gn[k] = make_double2(zr, zi);                 // G_{m=k, n}
        if (Gp != nullptr) {
          const int mp = (k == 0) ? 0 : n - k;                      // G_{m', -n} = conj Z(-m')
          if (mp < L) Gp[mp] = make_double2(zr, -zi);
        }
      } else {
        const int m = (k < L) ? k : k - n;
        Gn[m - mlo] = make_double2(zr, zi);
      }
    });
  }
}

template <bool REAL, bool PLAIN>
__global__ void k_dftg_inv(DftcArgs a) {
  extern __shared__ float4 s4[];
  __shared__ int jn[kMaxJobs], jp[kMaxJobs], njs;
  const int n = a.n, L = a.L, t = blockIdx.x, b = blockIdx.y;
  if (threadIdx.x == 0) {
    int nj;
    make_jobs(a.nvals, a.nact, REAL, jn, jp, nj);
    njs = nj;
  }
  __syncthreads();
  const int nj = njs, JB = a.jb;
  float4* tw = s4;
  float4* x = tw + n;         // [JB][n] stage-1 input, then stage-2 scratch (AB)
  float4* tmp = x + JB * n;   // [JB][n]
  float4* HZ = tmp + JB * n;  // [jobs][n]
  for (int i = threadIdx.x; i < n; i += blockDim.x) tw[i] = a.tw[i];
  for (int jb0 = 0; jb0 < nj; jb0 += JB) {
    const int nb = min(JB, nj - jb0);
    __syncthreads();
    for (int e = threadIdx.x; e < nb * n; e += blockDim.x) {
      const int qb = e / n, k = e - qb * n;
      const int ni = jn[jb0 + qb], pi = jp[jb0 + qb];
      const double2* Gn = a.G + (((int64_t)b * a.nact + ni) * a.nr + t) * a.Mc;
      const double2* Gp = a.G + (((int64_t)b * a.nact + (pi >= 0 ? pi : ni)) * a.nr + t) * a.Mc;
      double2 v;
      if (REAL) {
        if (k < L) {
          v = Gn[k];
        } else {                      // m = k - n < 0: G_{m,n} = conj G_{-m,-n}
          const double2 w = Gp[n - k];
          v = make_double2(w.x, -w.y);
        }
      } else {
        const int m = (k < L) ? k : k - n;
        v = Gn[m - a.mlo];
      }
      const float2 r = split1_bits(v.x), im = split1_bits(v.y);
      x[qb * n + k] = make_float4(r.x, r.y, im.x, im.y);
    }
    __syncthreads();
    stage1_sym<1, PLAIN>(x, tmp, tw, n, a.n1, a.n2, nb);
    __syncthreads();
    float4* Z = HZ + jb0 * n;
    stage2_sym<1, PLAIN>(tmp, x, tw, n, a.n1, a.n2, nb,
                         [&](int qb, int k, Acc re, Acc im) { Z[qb * n + k] = make_float4(re.s, re.c, im.s, im.c); });
  }
  __syncthreads();
  // W(alpha, gamma_g) = sum_j Z_j(alpha) exp(+i n_j gamma_g); gamma_g and gamma_{Ng-g} share
  // P = sum_j Z_j cos, Q = sum_j Z_j sin.  Real signals: the n, -n pair contributes 2 Re, the
  // n = 0 job Re.
  const int Ng = a.Ng, hg = (Ng - 1) / 2;
  const int64_t ring = (int64_t)a.nr * n;
  const int64_t base = (int64_t)b * a.pix_sb + (int64_t)t * n;
  for (int al = threadIdx.x; al < n; al += blockDim.x) {
    for (int g = 0; g <= hg; ++g) {
      Acc pr{0.f, 0.f}, pim{0.f, 0.f}, qr{0.f, 0.f}, qim{0.f, 0.f};
      for (int j = 0; j < nj; ++j) {
        float4 z = HZ[j * n + al];
        if (REAL && jp[j] >= 0) z = make_float4(2.f * z.x, 2.f * z.y, 2.f * z.z, 2.f * z.w);
        const float4 ph = a.gph[jn[j] * Ng + g];
        racc<PLAIN>(pr, z.x, z.y, ph.x, ph.y);
        if (g > 0) racc<PLAIN>(qim, z.z, z.w, ph.z, ph.w);
        if (!REAL) {
          racc<PLAIN>(pim, z.z, z.w, ph.x, ph.y);
          if (g > 0) racc<PLAIN>(qr, z.x, z.y, ph.z, ph.w);
        }
      }
      if (REAL) {
        double* out = (double*)a.pix_out;
        out[base + g * ring + al] = to_double(comb<PLAIN>(pr, -1.f, qim));            // P - Q
        if (g > 0) out[base + (Ng - g) * ring + al] = to_double(comb<PLAIN>(pr, 1.f, qim));
      } else {
        double2* out = (double2*)a.pix_out;   // P + i Q and P - i Q
        out[base + g * ring + al] =
            make_double2(to_double(comb<PLAIN>(pr, -1.f, qim)), to_double(comb<PLAIN>(pim, 1.f, qr)));
        if (g > 0)
          out[base + (Ng - g) * ring + al] =
              make_double2(to_double(comb<PLAIN>(pr, 1.f, qim)), to_double(comb<PLAIN>(pim, -1.f, qr)));
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
  a.nr = c.nr;
  a.Mc = c.Mc;
  a.mlo = c.mlo;
  a.n = g.n;
  a.n1 = g.n1;
  a.n2 = g.n2;
  a.tw = g.tw4;
  a.gph = t.gphase4;
  a.nvals = t.nvals;
  a.scale = 0.0;
  a.jb = 1;
  return a;
}

// the gamma-side kernels apply when there are several gamma samples, the job list fits and
// the shared memory of one block stays within the opt-in limit
int dftg_jobs(const TransformSpec& t, bool real) {
  int nj = 0;
  for (int v : t.nvals_h)
    if (!real || v >= 0) ++nj;
  return nj;
}
// shared memory of a gamma-side block: twiddles, the jobs' transforms and two stage buffers of
// jb transforms each
size_t dftg_smem_jb(const GridTables& g, int nj, int jb) { return (size_t)(1 + nj + 2 * jb) * g.n * sizeof(float4); }
constexpr size_t kDftgSmemMax = 200 * 1024;
// jobs per pass of the two alpha stages: up to 4 (every thread busy in both stages at the
// headline sizes), fewer when the shared memory would exceed the budget; 0 if even one does
int dftg_jb(const GridTables& g, const TransformSpec& t, bool real) {
  const int nj = dftg_jobs(t, real);
  for (int jb = std::min(nj, 4); jb >= 1; --jb)
    if (dftg_smem_jb(g, nj, jb) <= kDftgSmemMax) return jb;
  return 0;
}
size_t dftg_smem(const GridTables& g, const TransformSpec& t, bool real) {
  return dftg_smem_jb(g, dftg_jobs(t, real), dftg_jb(g, t, real));
}
bool use_dftg(const GridTables& g, const TransformSpec& t, bool real) {
  if (real)   // every negative n needs its partner -n among the carried values
    for (int v : t.nvals_h)
      if (v < 0 && std::find(t.nvals_h.begin(), t.nvals_h.end(), -v) == t.nvals_h.end()) return false;
  return dftg_jobs(t, real) <= kMaxJobs && dftg_jb(g, t, real) >= 1;
}

template <class K>
cudaError_t launch(K kern, dim3 grid, size_t smem, cudaStream_t st, const DftcArgs& a, int threads = 256) {
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  kern<<<grid, threads, smem, st>>>(a);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_dftc_forward(const GridTables& g, const TransformSpec& t, const void* pix, int64_t pix_sb,
                                bool real, ColumnArgs c, cudaStream_t st, bool plain) {
  if (plain && dftf_usable(g, t, real, true)) return launch_dftf_forward(g, t, pix, pix_sb, real, c, st);
  DftcArgs a = make_args(g, t, c);
  a.pix_in = pix;
  a.pix_out = nullptr;
  a.pix_sb = pix_sb;
  a.scale = (2.0 * 3.14159265358979323846 / g.n) * t.gscale;
  dim3 grid(c.nr, c.B);
  if (use_dftg(g, t, real)) {
    const size_t sm = dftg_smem(g, t, real);
    a.jb = dftg_jb(g, t, real);
    const int th = t.dft_threads_fwd;
    if (plain)
      return real ? launch(k_dftg_fwd<true, true>, grid, sm, st, a, th) : launch(k_dftg_fwd<false, true>, grid, sm, st, a, th);
    return real ? launch(k_dftg_fwd<true, false>, grid, sm, st, a, th) : launch(k_dftg_fwd<false, false>, grid, sm, st, a, th);
  }
  const size_t smem = (size_t)(3 * g.n + a.Ng * c.Mc) * sizeof(float4);
  if (plain) return real ? launch(k_dftc_fwd<true, true>, grid, smem, st, a) : launch(k_dftc_fwd<false, true>, grid, smem, st, a);
  return real ? launch(k_dftc_fwd<true, false>, grid, smem, st, a) : launch(k_dftc_fwd<false, false>, grid, smem, st, a);
}

cudaError_t launch_dftc_inverse(const GridTables& g, const TransformSpec& t, ColumnArgs c, void* pix,
                                int64_t pix_sb, bool real, cudaStream_t st, bool plain) {
  if (plain && dftf_usable(g, t, real, false)) return launch_dftf_inverse(g, t, c, pix, pix_sb, real, st);
  DftcArgs a = make_args(g, t, c);
  a.pix_in = nullptr;
  a.pix_out = pix;
  a.pix_sb = pix_sb;
  dim3 grid(c.nr, c.B);
  if (use_dftg(g, t, real)) {
    const size_t sm = dftg_smem(g, t, real);
    a.jb = dftg_jb(g, t, real);
    const int th = t.dft_threads_inv;
    if (plain)
      return real ? launch(k_dftg_inv<true, true>, grid, sm, st, a, th) : launch(k_dftg_inv<false, true>, grid, sm, st, a, th);
    return real ? launch(k_dftg_inv<true, false>, grid, sm, st, a, th) : launch(k_dftg_inv<false, false>, grid, sm, st, a, th);
  }
  const size_t smem = (size_t)(3 * g.n + c.nact * c.Mc) * sizeof(float4);
  if (plain) return real ? launch(k_dftc_inv<true, true>, grid, smem, st, a) : launch(k_dftc_inv<false, true>, grid, smem, st, a);
  return real ? launch(k_dftc_inv<true, false>, grid, smem, st, a) : launch(k_dftc_inv<false, false>, grid, smem, st, a);
}

}  // namespace s2w

// Float64 kernels of the hot path (sm_103a):
//  * k_dft_fwd / k_dft_inv   azimuthal (alpha/phi, length 2L-1) and gamma (length 2N-1)
//                            DFTs between pixel rings and m-columns (Sec. 5.2, Eq. 48);
//  * k_wig_inv               inverse contraction over l against d^l_mn(beta), the
//                            Wigner-d three-term recursion in l fused into the loop, with
//                            the harmonic products (Eq. 27 / Eq. 29) fused as multipliers;
//  * k_wig_fwd               forward contraction: colatitude quadrature matrix applied in
//                            shared memory, then the recursion-generated d tile contracted
//                            against the weighted columns, products fused in the epilogue.
#include <math.h>

#include <algorithm>

#include "comp32.cuh"
#include "s2w_internal.h"
#include "wigner_rec.cuh"

namespace s2w {
namespace {

__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}

// ------------------------------------------------------------------------- DFTs
// y[k] = sum_j x[j] w^(SIGN j k), w = exp(2 pi i/n), n = n1 n2 (Cooley-Tukey split
// j = n2 j1 + j2, k = k1 + n1 k2).  Stage 1 leaves the twiddled length-n1 transforms in
// tmp[k1 n2 + j2]; stage 2 finishes the length-n2 transforms for requested outputs.
template <int SIGN>
__device__ __forceinline__ double2 twid(const double2* tw, int e) {
  double2 t = tw[e];
  if (SIGN < 0) t.y = -t.y;
  return t;
}

template <int SIGN>
__device__ void dft_stage1(const double2* x, double2* tmp, const double2* tw, int n, int n1, int n2) {
  for (int idx = threadIdx.x; idx < n; idx += blockDim.x) {
    const int k1 = idx / n2, j2 = idx - k1 * n2;
    const int step = (n2 * k1) % n;
    double re = 0.0, im = 0.0;
    int e = 0;
    for (int j1 = 0; j1 < n1; ++j1) {
      const double2 xv = x[n2 * j1 + j2];
      const double2 t = twid<SIGN>(tw, e);
      re = fma(xv.x, t.x, fma(-xv.y, t.y, re));
      im = fma(xv.x, t.y, fma(xv.y, t.x, im));
      e += step;
      if (e >= n) e -= n;
    }
    const double2 t = twid<SIGN>(tw, (j2 * k1) % n);
    tmp[k1 * n2 + j2] = make_double2(fma(re, t.x, -im * t.y), fma(re, t.y, im * t.x));
  }
}

// one output of stage 2
template <int SIGN, bool REAL_ONLY>
__device__ __forceinline__ double2 dft_stage2_one(const double2* tmp, const double2* tw, int n, int n1,
                                                  int n2, int k) {
  const int k1 = k % n1, k2 = k / n1;
  const int step = (n1 * k2) % n;
  const double2* row = tmp + k1 * n2;
  double re = 0.0, im = 0.0;
  int e = 0;
  for (int j2 = 0; j2 < n2; ++j2) {
    const double2 v = row[j2];
    const double2 t = twid<SIGN>(tw, e);
    re = fma(v.x, t.x, fma(-v.y, t.y, re));
    if (!REAL_ONLY) im = fma(v.x, t.y, fma(v.y, t.x, im));
    e += step;
    if (e >= n) e -= n;
  }
  return make_double2(re, im);
}

struct DftArgs {
  const void* pix_in;
  void* pix_out;
  int64_t pix_sb;       // elements between maps
  double2* G;           // [B][nact][nr][Mc]
  int B, nact, Ng, L, nr, Mc, mlo, n, n1, n2;
  const double2* tw;
  const double2* gph;   // [nact][Ng] exp(+i n gamma_g)
  double scale;
};

// Pixels [b][g][t][a] -> columns G[b][ni][t][mi].  One block per (ring t, map b).
template <bool REAL>
__global__ void k_dft_fwd(DftArgs a) {
  extern __shared__ double2 sm2[];
  const int n = a.n, t = blockIdx.x, b = blockIdx.y;
  double2* tw = sm2;             // [n]
  double2* x = tw + n;           // [n]
  double2* tmp = x + n;          // [n]
  double2* H = tmp + n;          // [Ng][Mc]
  for (int i = threadIdx.x; i < n; i += blockDim.x) tw[i] = a.tw[i];
  const int64_t ring = (int64_t)a.nr * n;
  for (int g = 0; g < a.Ng; ++g) {
    __syncthreads();
    const int64_t base = (int64_t)b * a.pix_sb + (int64_t)g * ring + (int64_t)t * n;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      if (REAL) x[i] = make_double2(((const double*)a.pix_in)[base + i], 0.0);
      else x[i] = ((const double2*)a.pix_in)[base + i];
    }
    __syncthreads();
    dft_stage1<-1>(x, tmp, tw, n, a.n1, a.n2);
    __syncthreads();
    for (int mi = threadIdx.x; mi < a.Mc; mi += blockDim.x) {
      int k = a.mlo + mi;
      if (k < 0) k += n;
      H[g * a.Mc + mi] = dft_stage2_one<-1, false>(tmp, tw, n, a.n1, a.n2, k);
    }
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < a.nact * a.Mc; idx += blockDim.x) {
    const int ni = idx / a.Mc, mi = idx - ni * a.Mc;
    double re = 0.0, im = 0.0;
    for (int g = 0; g < a.Ng; ++g) {
      const double2 h = H[g * a.Mc + mi];
      const double2 p = a.gph[ni * a.Ng + g];   // conj for the forward sum
      re = fma(h.x, p.x, fma(h.y, p.y, re));
      im = fma(h.y, p.x, fma(-h.x, p.y, im));
    }
    a.G[(((int64_t)b * a.nact + ni) * a.nr + t) * a.Mc + mi] = make_double2(re * a.scale, im * a.scale);
  }
}

// Columns G[b][ni][t][mi] -> pixels [b][g][t][a].  One block per (ring t, map b).
template <bool REAL>
__global__ void k_dft_inv(DftArgs a) {
  extern __shared__ double2 sm2[];
  const int n = a.n, t = blockIdx.x, b = blockIdx.y;
  double2* tw = sm2;
  double2* x = tw + n;
  double2* tmp = x + n;
  double2* Gs = tmp + n;         // [nact][Mc]
  for (int i = threadIdx.x; i < n; i += blockDim.x) tw[i] = a.tw[i];
  for (int idx = threadIdx.x; idx < a.nact * a.Mc; idx += blockDim.x) {
    const int ni = idx / a.Mc, mi = idx - ni * a.Mc;
    Gs[idx] = a.G[(((int64_t)b * a.nact + ni) * a.nr + t) * a.Mc + mi];
  }
  const int64_t ring = (int64_t)a.nr * n;
  for (int g = 0; g < a.Ng; ++g) {
    __syncthreads();
    for (int mi = threadIdx.x; mi < a.Mc; mi += blockDim.x) {
      double re = 0.0, im = 0.0;
      for (int ni = 0; ni < a.nact; ++ni) {
        const double2 v = Gs[ni * a.Mc + mi];
        const double2 p = a.gph[ni * a.Ng + g];
        re = fma(v.x, p.x, fma(-v.y, p.y, re));
        im = fma(v.x, p.y, fma(v.y, p.x, im));
      }
      const int m = a.mlo + mi;
      if (REAL) {
        x[m] = make_double2(re, im);
        if (m > 0) x[n - m] = make_double2(re, -im);
      } else {
        x[m < 0 ? m + n : m] = make_double2(re, im);
      }
    }
    __syncthreads();
    dft_stage1<1>(x, tmp, tw, n, a.n1, a.n2);
    __syncthreads();
    const int64_t base = (int64_t)b * a.pix_sb + (int64_t)g * ring + (int64_t)t * n;
    for (int k = threadIdx.x; k < n; k += blockDim.x) {
      if (REAL) {
        ((double*)a.pix_out)[base + k] = dft_stage2_one<1, true>(tmp, tw, n, a.n1, a.n2, k).x;
      } else {
        ((double2*)a.pix_out)[base + k] = dft_stage2_one<1, false>(tmp, tw, n, a.n1, a.n2, k);
      }
    }
  }
}

struct WigInvArgs {
  const double2* coef;
  int64_t s_b, s_n, s_l;
  int mlo_in;
  const double2* mult;   // [L][nact]
  const int* nvals;
  int nact;
  double2* G;            // [B][nact][nr][Mc]
  int B, L, nr, Mc, mlo;
  int ncol;              // columns launched (grid.x), a sub-range of a row of Mc
  RecTables T;
};

constexpr int kInvThreads = 128;
constexpr int kInvLT = 32;

// C32: the sum over l runs in compensated float32 pairs (comp32.cuh): coefficient tiles are
// split into pairs once per block and each float64 recursion value d^l_mn(beta) is split with
// integer operations, so the float64 pipe only carries the recursion itself.
template <int MB, bool C32>
__global__ void __launch_bounds__(kInvThreads) k_wig_inv(WigInvArgs a) {
  __shared__ double2 Fs[kInvLT * MB];
  __shared__ double cA[kInvLT], cKn[kInvLT], cKs[kInvLT], cC[kInvLT];
  float4* F4 = reinterpret_cast<float4*>(Fs);
  const int mi = blockIdx.x, ni = blockIdx.y;
  const int m = a.mlo + mi, nn = a.nvals[ni];
  const int L = a.L, nr = a.nr;
  const int b = blockIdx.z * blockDim.x + threadIdx.x;
  const int l0 = max(abs(m), abs(nn));
  const double wb = (b < nr) ? a.T.wpole[b] : 0.0;
  const double* cK = (2 * (2 * b + 1) < a.T.den) ? cKn : cKs;
  for (int map0 = 0; map0 < a.B; map0 += MB) {
    double2 acc[C32 ? 1 : MB];
    Acc ar[C32 ? MB : 1], ai[C32 ? MB : 1];
    if (C32) {
#pragma unroll
      for (int k = 0; k < MB; ++k) ar[k] = ai[k] = Acc{0.f, 0.f};
    } else {
#pragma unroll
      for (int k = 0; k < (C32 ? 1 : MB); ++k) acc[k] = make_double2(0.0, 0.0);
    }
    double v = 0.0, vp = 0.0;
    int q = 0;
    if (b < nr && l0 < L) wigner_seed(a.T, b, l0, m, nn, v, q);
    for (int ls = l0; ls < L; ls += kInvLT) {
      const int cnt = min(kInvLT, L - ls);
      __syncthreads();
      for (int idx = threadIdx.x; idx < cnt * MB; idx += blockDim.x) {
        const int i = idx / MB, mp = idx - i * MB, l = ls + i, bm = map0 + mp;
        double2 f = make_double2(0.0, 0.0);
        if (bm < a.B)
          f = cmul(a.coef[(int64_t)bm * a.s_b + (int64_t)ni * a.s_n + (int64_t)l * a.s_l + (m - a.mlo_in)],
                   a.mult[(int64_t)l * a.nact + ni]);
        if (C32) F4[idx] = split(f);
        else Fs[idx] = f;
      }
      for (int i = threadIdx.x; i < cnt; i += blockDim.x) rec_coeffs(ls + i, m, nn, cA[i], cKn[i], cKs[i], cC[i]);
      __syncthreads();
      if (b < nr) {
        for (int i = 0; i < cnt; ++i) {
          if (q == 0) {
            if (C32) {
              const float2 d = split1_bits(v);
#pragma unroll
              for (int k = 0; k < MB; ++k) {
                const float4 f = F4[i * MB + k];
                acc_add(ar[k], f.x, f.y, d.x, d.y);
                acc_add(ai[k], f.z, f.w, d.x, d.y);
              }
            } else {
#pragma unroll
              for (int k = 0; k < (C32 ? 1 : MB); ++k) {
                const double2 f = Fs[i * MB + k];
                acc[k].x = fma(f.x, v, acc[k].x);
                acc[k].y = fma(f.y, v, acc[k].y);
              }
            }
          }
          const double x = fma(cA[i], wb, cK[i]);
          const double vn = fma(x, v, -cC[i] * vp);
          vp = v;
          v = vn;
          if (q > 0 && fabs(v) > kRescaleAt) {
            v *= kRescaleBy;
            vp *= kRescaleBy;
            --q;
          }
        }
      }
    }
    if (b < nr) {
#pragma unroll
      for (int k = 0; k < MB; ++k) {
        const int bm = map0 + k;
        if (bm < a.B) {
          double2 r;
          if (C32) r = make_double2(to_double(ar[k]), to_double(ai[k]));
          else r = acc[C32 ? 0 : k];
          a.G[(((int64_t)bm * a.nact + ni) * nr + b) * a.Mc + mi] = r;
        }
      }
    }
  }
}

struct WigFwdArgs {
  const double2* G;      // [B][nact][nr][Mc]
  int B, L, nr, Mc, mlo;
  int ncol;              // columns launched (grid.x), a sub-range of a row of Mc
  const int* nvals;
  int nact;
  const double2* mult;   // [L][nact]
  double2* out;
  int64_t s_b, s_n, s_l;
  int mlo_out;
  const double* MT;      // MW: [2][L][L]
  const float2* MT2;     // the same as float pairs (compensated quadrature)
  const double* wdiag;   // DH: [nr] ring weights (MT unused)
  int quad;              // 0: skip the quadrature (adjoint of the inverse contraction)
  RecTables T;
};

// C32: the quadrature M^{par} G and the contraction over beta run in compensated float32
// pairs (comp32.cuh); the weighted columns stay as pairs in shared memory and each recursion
// value is split with integer operations.  Without C32 every step is native float64.  The
// Wigner-d recursion is float64 either way.  On DH sampling the quadrature is diagonal and is
// applied in float64 as the columns are loaded.
template <int MB, int LT, bool C32>
__global__ void k_wig_fwd(WigFwdArgs a) {
  extern __shared__ double smd[];
  const int L = a.L, nr = a.nr;
  double2* Gs = (double2*)smd;                  // [nr][MB]
  double* Ds = (double*)(Gs + (size_t)nr * MB); // [LT][nr]
  double* cA = Ds + (size_t)LT * nr;
  double* cKn = cA + LT;
  double* cKs = cKn + LT;
  double* cC = cKs + LT;
  const int mi = blockIdx.x, ni = blockIdx.y;
  const int m = a.mlo + mi, nn = a.nvals[ni];
  const int t = threadIdx.x;
  const int l0 = max(abs(m), abs(nn));
  if (l0 >= L) return;
  const int par = (m + nn) & 1;
  const double* MT = a.MT + (size_t)par * L * L;
  const double wb = (t < nr) ? a.T.wpole[t] : 0.0;
  const double* cK = (2 * (2 * t + 1) < a.T.den) ? cKn : cKs;
  const bool diag = a.quad && a.wdiag != nullptr;
  for (int map0 = 0; map0 < a.B; map0 += MB) {
    __syncthreads();
    for (int idx = threadIdx.x; idx < nr * MB; idx += blockDim.x) {
      const int tt = idx / MB, mp = idx - tt * MB, bm = map0 + mp;
      double2 gv = (bm < a.B) ? a.G[(((int64_t)bm * a.nact + ni) * nr + tt) * a.Mc + mi] : make_double2(0.0, 0.0);
      if (diag) {
        const double w = a.wdiag[tt];
        gv = make_double2(gv.x * w, gv.y * w);
      }
      if (C32) reinterpret_cast<float4*>(Gs)[idx] = split(gv);
      else Gs[idx] = gv;
    }
    __syncthreads();
    // colatitude quadrature (MW): Gs <- M^{par} Gs
    if (!a.quad || diag) {
      // columns enter the beta sum as they are (or were weighted on load)
    } else if (C32) {
      const float2* MT2 = a.MT2 + (size_t)par * L * L;
      const float4* G4 = reinterpret_cast<const float4*>(Gs);
      Acc ar[MB], ai[MB];
#pragma unroll
      for (int k = 0; k < MB; ++k) ar[k] = ai[k] = Acc{0.f, 0.f};
      if (t < L) {
        for (int tp = 0; tp < L; ++tp) {
          const float2 w = MT2[(size_t)tp * L + t];
#pragma unroll
          for (int k = 0; k < MB; ++k) {
            const float4 gv = G4[tp * MB + k];
            acc_add(ar[k], gv.x, gv.y, w.x, w.y);
            acc_add(ai[k], gv.z, gv.w, w.x, w.y);
          }
        }
      }
      __syncthreads();
      if (t < L) {
        float4* G4w = reinterpret_cast<float4*>(Gs);
#pragma unroll
        for (int k = 0; k < MB; ++k) G4w[t * MB + k] = pack_pair(ar[k], ai[k]);
      }
    } else {
      double2 acc[MB];
#pragma unroll
      for (int k = 0; k < MB; ++k) acc[k] = make_double2(0.0, 0.0);
      if (t < L) {
        for (int tp = 0; tp < L; ++tp) {
          const double w = MT[(size_t)tp * L + t];
#pragma unroll
          for (int k = 0; k < MB; ++k) {
            const double2 gv = Gs[tp * MB + k];
            acc[k].x = fma(w, gv.x, acc[k].x);
            acc[k].y = fma(w, gv.y, acc[k].y);
          }
        }
      }
      __syncthreads();
      if (t < L) {
#pragma unroll
        for (int k = 0; k < MB; ++k) Gs[t * MB + k] = acc[k];
      }
    }
    double v = 0.0, vp = 0.0;
    int q = 0;
    if (t < nr) wigner_seed(a.T, t, l0, m, nn, v, q);
    for (int ls = l0; ls < L; ls += LT) {
      const int cnt = min(LT, L - ls);
      __syncthreads();
      for (int i = threadIdx.x; i < cnt; i += blockDim.x) rec_coeffs(ls + i, m, nn, cA[i], cKn[i], cKs[i], cC[i]);
      __syncthreads();
      if (t < nr) {
        for (int i = 0; i < cnt; ++i) {
          if (C32) reinterpret_cast<float2*>(Ds)[i * nr + t] = (q == 0) ? split1_bits(v) : make_float2(0.f, 0.f);
          else Ds[i * nr + t] = (q == 0) ? v : 0.0;
          const double x = fma(cA[i], wb, cK[i]);
          const double vn = fma(x, v, -cC[i] * vp);
          vp = v;
          v = vn;
          if (q > 0 && fabs(v) > kRescaleAt) {
            v *= kRescaleBy;
            vp *= kRescaleBy;
            --q;
          }
        }
      }
      __syncthreads();
      for (int idx = threadIdx.x; idx < cnt * MB; idx += blockDim.x) {
        const int i = idx / MB, mp = idx - i * MB, bm = map0 + mp, l = ls + i;
        double re = 0.0, im = 0.0;
        if (C32) {
          const float2* drow = reinterpret_cast<const float2*>(Ds) + (size_t)i * nr;
          const float4* G4 = reinterpret_cast<const float4*>(Gs);
          Acc ar{0.f, 0.f}, ai{0.f, 0.f};
          for (int bb = 0; bb < nr; ++bb) {
            const float2 d = drow[bb];
            const float4 gv = G4[bb * MB + mp];
            acc_add(ar, gv.x, gv.y, d.x, d.y);
            acc_add(ai, gv.z, gv.w, d.x, d.y);
          }
          re = to_double(ar);
          im = to_double(ai);
        } else {
          const double* drow = Ds + (size_t)i * nr;
          for (int bb = 0; bb < nr; ++bb) {
            const double d = drow[bb];
            const double2 gv = Gs[bb * MB + mp];
            re = fma(d, gv.x, re);
            im = fma(d, gv.y, im);
          }
        }
        if (bm < a.B) {
          const double2 r = cmul(make_double2(re, im), a.mult[(int64_t)l * a.nact + ni]);
          double2* o = a.out + (int64_t)bm * a.s_b + (int64_t)ni * a.s_n + (int64_t)l * a.s_l + (m - a.mlo_out);
          atomicAdd(&o->x, r.x);
          atomicAdd(&o->y, r.y);
        }
      }
    }
  }
}

// ------------------------------------------------- transposed colatitude quadrature
// Adjoint of the forward transforms' quadrature step.  In place: a block owns kQaCols
// columns m of one (map, n) slab, all of one parity of m + n (m = mlo + 2 (kQaCols q + k) +
// cls), reads them whole into shared memory and thread t writes
// sum_t' M^{par}[t'][t] G[t'], reading the row-major matrix along t (coalesced).
constexpr int kQaCols = 8;

struct QuadAdjArgs {
  double2* G;            // [B][nact][L][Mc]
  int B, nact, L, Mc, mlo;
  const int* nvals;
  const double* MR;      // [2][L][L] row-major M[par][t][t']
  const float2* MR2;     // the same as float pairs
};

template <bool C32>
__global__ void k_quad_adj(QuadAdjArgs a) {
  extern __shared__ double smd[];
  double2* Gs = (double2*)smd;                 // [L][kQaCols]
  const int cls = blockIdx.x & 1, q = blockIdx.x >> 1;
  const int ni = blockIdx.y, b = blockIdx.z, L = a.L;
  const int par = (a.mlo + cls + a.nvals[ni]) & 1;
  const int64_t slab = ((int64_t)b * a.nact + ni) * L * a.Mc;
  for (int idx = threadIdx.x; idx < L * kQaCols; idx += blockDim.x) {
    const int tp = idx / kQaCols, k = idx - tp * kQaCols, mi = 2 * (kQaCols * q + k) + cls;
    const double2 gv = (mi < a.Mc) ? a.G[slab + (int64_t)tp * a.Mc + mi] : make_double2(0.0, 0.0);
    if (C32) reinterpret_cast<float4*>(Gs)[idx] = split(gv);
    else Gs[idx] = gv;
  }
  __syncthreads();
  const int t = threadIdx.x;
  if (t >= L) return;
  double2 r[kQaCols];
  if (C32) {
    const float2* M2 = a.MR2 + (size_t)par * L * L;
    const float4* G4 = reinterpret_cast<const float4*>(Gs);
    Acc ar[kQaCols], ai[kQaCols];
#pragma unroll
    for (int k = 0; k < kQaCols; ++k) ar[k] = ai[k] = Acc{0.f, 0.f};
    for (int tp = 0; tp < L; ++tp) {
      const float2 w = M2[(size_t)tp * L + t];
#pragma unroll
      for (int k = 0; k < kQaCols; ++k) {
        const float4 gv = G4[tp * kQaCols + k];
        acc_add(ar[k], gv.x, gv.y, w.x, w.y);
        acc_add(ai[k], gv.z, gv.w, w.x, w.y);
      }
    }
#pragma unroll
    for (int k = 0; k < kQaCols; ++k) r[k] = make_double2(to_double(ar[k]), to_double(ai[k]));
  } else {
    const double* M = a.MR + (size_t)par * L * L;
#pragma unroll
    for (int k = 0; k < kQaCols; ++k) r[k] = make_double2(0.0, 0.0);
    for (int tp = 0; tp < L; ++tp) {
      const double w = M[(size_t)tp * L + t];
#pragma unroll
      for (int k = 0; k < kQaCols; ++k) {
        const double2 gv = Gs[tp * kQaCols + k];
        r[k].x = fma(w, gv.x, r[k].x);
        r[k].y = fma(w, gv.y, r[k].y);
      }
    }
  }
#pragma unroll
  for (int k = 0; k < kQaCols; ++k) {
    const int mi = 2 * (kQaCols * q + k) + cls;
    if (mi < a.Mc) a.G[slab + (int64_t)t * a.Mc + mi] = r[k];
  }
}

// DH: the quadrature is the diagonal of ring weights, its own transpose: G[.][t][.] *= w[t].
__global__ void k_ring_scale(double2* G, int64_t total, int nr, int Mc, const double* w) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const double s = w[(i / Mc) % nr];
    const double2 v = G[i];
    G[i] = make_double2(v.x * s, v.y * s);
  }
}

RecTables rec_tables(const GridTables& g) {
  RecTables T;
  T.wpole = g.wpole;
  T.cpow_m = g.cpow_m;
  T.cpow_e = g.cpow_e;
  T.spow_m = g.spow_m;
  T.spow_e = g.spow_e;
  T.sqrtC = g.sqrtC;
  T.n = g.n;
  T.den = g.den;
  return T;
}

int pick_mb(int B, int cap) {
  int mb = 1;
  while (mb < B && mb < cap) mb *= 2;
  return mb;
}

template <int MB>
cudaError_t launch_inv_mb(const WigInvArgs& a, int nact, bool c32, cudaStream_t st) {
  dim3 grid(a.ncol, nact, (a.nr + kInvThreads - 1) / kInvThreads);
  if (c32) k_wig_inv<MB, true><<<grid, kInvThreads, 0, st>>>(a);
  else k_wig_inv<MB, false><<<grid, kInvThreads, 0, st>>>(a);
  return cudaGetLastError();
}

template <int MB, int LT, bool C32>
cudaError_t launch_fwd_k(const WigFwdArgs& a, int nact, cudaStream_t st) {
  const int threads = ((a.nr + 31) / 32) * 32;
  const size_t smem = (size_t)a.nr * MB * sizeof(double2) + (size_t)LT * a.nr * sizeof(double) + 4 * LT * sizeof(double);
  cudaError_t e = cudaFuncSetAttribute(k_wig_fwd<MB, LT, C32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  dim3 grid(a.ncol, nact);
  k_wig_fwd<MB, LT, C32><<<grid, threads < 32 ? 32 : threads, smem, st>>>(a);
  return cudaGetLastError();
}

template <int MB, int LT>
cudaError_t launch_fwd_mb(const WigFwdArgs& a, int nact, bool c32, cudaStream_t st) {
  return c32 ? launch_fwd_k<MB, LT, true>(a, nact, st) : launch_fwd_k<MB, LT, false>(a, nact, st);
}

}  // namespace

cudaError_t launch_zero(void* p, int64_t bytes, cudaStream_t st) {
  return cudaMemsetAsync(p, 0, (size_t)bytes, st);
}

static DftArgs dft_args(const GridTables& g, const TransformSpec& t, ColumnArgs c) {
  DftArgs a;
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
  a.tw = g.tw;
  a.gph = t.gphase;
  a.scale = 0.0;
  return a;
}

cudaError_t launch_dft_forward(const s2w_plan* P, const GridTables& g, const TransformSpec& t, const void* pix,
                               int64_t pix_sb, bool real, ColumnArgs c, cudaStream_t st) {
  (void)P;
  DftArgs a = dft_args(g, t, c);
  a.pix_in = pix;
  a.pix_out = nullptr;
  a.pix_sb = pix_sb;
  a.scale = (2.0 * 3.14159265358979323846 / g.n) * t.gscale;
  const size_t smem = (size_t)(3 * g.n + a.Ng * c.Mc) * sizeof(double2);
  dim3 grid(c.nr, c.B);
  cudaError_t e;
  if (real) {
    e = cudaFuncSetAttribute(k_dft_fwd<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_dft_fwd<true><<<grid, 256, smem, st>>>(a);
  } else {
    e = cudaFuncSetAttribute(k_dft_fwd<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_dft_fwd<false><<<grid, 256, smem, st>>>(a);
  }
  return cudaGetLastError();
}

cudaError_t launch_dft_inverse(const s2w_plan* P, const GridTables& g, const TransformSpec& t, ColumnArgs c,
                               void* pix, int64_t pix_sb, bool real, cudaStream_t st) {
  (void)P;
  DftArgs a = dft_args(g, t, c);
  a.pix_in = nullptr;
  a.pix_out = pix;
  a.pix_sb = pix_sb;
  const size_t smem = (size_t)(3 * g.n + c.nact * c.Mc) * sizeof(double2);
  dim3 grid(c.nr, c.B);
  cudaError_t e;
  if (real) {
    e = cudaFuncSetAttribute(k_dft_inv<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_dft_inv<true><<<grid, 256, smem, st>>>(a);
  } else {
    e = cudaFuncSetAttribute(k_dft_inv<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_dft_inv<false><<<grid, 256, smem, st>>>(a);
  }
  return cudaGetLastError();
}

cudaError_t launch_wigner_inverse(const s2w_plan* P, const GridTables& g, const TransformSpec& t, CoefArgs in,
                                  ColumnArgs out, cudaStream_t st) {
  WigInvArgs a;
  a.coef = in.coef;
  a.s_b = in.s_b;
  a.s_n = in.s_n;
  a.s_l = in.s_l;
  a.mlo_in = in.mlo;
  a.mult = t.mult_inv;
  a.nvals = t.nvals;
  a.nact = t.nact;
  a.G = out.G;
  a.B = out.B;
  a.L = out.L;
  a.nr = out.nr;
  a.Mc = out.Mc;
  a.mlo = out.mlo;
  a.ncol = out.ncol > 0 ? out.ncol : out.Mc;
  a.T = rec_tables(g);
  switch (pick_mb(out.B, t.inv_mb)) {
    case 1: return launch_inv_mb<1>(a, t.nact, !P->native64, st);
    case 2: return launch_inv_mb<2>(a, t.nact, !P->native64, st);
    case 4: return launch_inv_mb<4>(a, t.nact, !P->native64, st);
    case 8: return launch_inv_mb<8>(a, t.nact, !P->native64, st);
    default: return launch_inv_mb<16>(a, t.nact, !P->native64, st);
  }
}

cudaError_t launch_wigner_forward(const s2w_plan* P, const GridTables& g, const TransformSpec& t, ColumnArgs in,
                                  CoefArgs out, cudaStream_t st, bool quad) {
  WigFwdArgs a;
  a.quad = quad ? 1 : 0;
  a.G = in.G;
  a.B = in.B;
  a.L = in.L;
  a.nr = in.nr;
  a.Mc = in.Mc;
  a.mlo = in.mlo;
  a.ncol = in.ncol > 0 ? in.ncol : in.Mc;
  a.nvals = t.nvals;
  a.nact = t.nact;
  a.mult = t.mult_fwd;
  a.out = const_cast<double2*>(out.coef);
  a.s_b = out.s_b;
  a.s_n = out.s_n;
  a.s_l = out.s_l;
  a.mlo_out = out.mlo;
  a.MT = g.MT;
  a.MT2 = g.MT2;
  a.wdiag = g.wdiag;
  a.T = rec_tables(g);
  const bool c32 = !P->native64;
  // Compensated blocks use 16-row recursion tiles so that two blocks fit on an SM (one
  // block's float64 recursion phase overlaps the other's float32 contraction phase).  Shapes
  // follow the ring count (one thread per ring; shared memory grows with it).
  if (in.nr <= 256) {
    if (c32) {
      switch (pick_mb(in.B, 16)) {
        case 1: return launch_fwd_mb<1, 16>(a, t.nact, c32, st);
        case 2: return launch_fwd_mb<2, 16>(a, t.nact, c32, st);
        case 4: return launch_fwd_mb<4, 16>(a, t.nact, c32, st);
        case 8: return launch_fwd_mb<8, 16>(a, t.nact, c32, st);
        default: return launch_fwd_mb<16, 16>(a, t.nact, c32, st);
      }
    }
    switch (pick_mb(in.B, 16)) {
      case 1: return launch_fwd_mb<1, 32>(a, t.nact, c32, st);
      case 2: return launch_fwd_mb<2, 32>(a, t.nact, c32, st);
      case 4: return launch_fwd_mb<4, 32>(a, t.nact, c32, st);
      case 8: return launch_fwd_mb<8, 32>(a, t.nact, c32, st);
      default: return launch_fwd_mb<16, 32>(a, t.nact, c32, st);
    }
  } else if (in.nr <= 512) {
    switch (pick_mb(in.B, 8)) {
      case 1: return launch_fwd_mb<1, 32>(a, t.nact, c32, st);
      case 2: return launch_fwd_mb<2, 32>(a, t.nact, c32, st);
      case 4: return launch_fwd_mb<4, 32>(a, t.nact, c32, st);
      default: return launch_fwd_mb<8, 32>(a, t.nact, c32, st);
    }
  } else {
    switch (pick_mb(in.B, 4)) {
      case 1: return launch_fwd_mb<1, 16>(a, t.nact, c32, st);
      case 2: return launch_fwd_mb<2, 16>(a, t.nact, c32, st);
      default: return launch_fwd_mb<4, 16>(a, t.nact, c32, st);
    }
  }
}

cudaError_t launch_quad_adjoint(const s2w_plan* P, const GridTables& g, const TransformSpec& t, ColumnArgs c,
                                cudaStream_t st) {
  if (g.wdiag != nullptr) {
    const int64_t total = (int64_t)c.B * c.nact * c.nr * c.Mc;
    const int blocks = (int)std::min<int64_t>((total + 255) / 256, 152 * 16);
    k_ring_scale<<<blocks, 256, 0, st>>>(c.G, total, c.nr, c.Mc, g.wdiag);
    return cudaGetLastError();
  }
  QuadAdjArgs a;
  a.G = c.G;
  a.B = c.B;
  a.nact = c.nact;
  a.L = c.L;
  a.Mc = c.Mc;
  a.mlo = c.mlo;
  a.nvals = t.nvals;
  a.MR = g.MR;
  a.MR2 = g.MR2;
  const int nq = ((c.Mc + 1) / 2 + kQaCols - 1) / kQaCols;   // column tiles per parity class
  const int threads = ((c.L + 31) / 32) * 32;
  const size_t smem = (size_t)c.L * kQaCols * sizeof(double2);
  dim3 grid(2 * nq, c.nact, c.B);
  cudaError_t e;
  if (P->native64) {
    e = cudaFuncSetAttribute(k_quad_adj<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_quad_adj<false><<<grid, threads, smem, st>>>(a);
  } else {
    e = cudaFuncSetAttribute(k_quad_adj<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_quad_adj<true><<<grid, threads, smem, st>>>(a);
  }
  return cudaGetLastError();
}

}  // namespace s2w

// Azimuthal (alpha/phi) and gamma DFTs (Sec. 5.2, Eq. 48) in plain float32, for the
// reduced-precision modes.
//
// One block per (ring, map), the carried n values ("jobs", see dft_c32.cuh) in chunks of up to
// four.  The length n = 2L-1 transform is split n = n1 n2 (Cooley-Tukey, twiddles between the
// stages) and both stages take the symmetric odd-length form: with a_j = x_j + x_{p-j},
// b_j = x_j - x_{p-j} (j = 1..h, h = (p-1)/2),
//   X(kk), X(p-kk) = x_0 + sum_j a_j cos(2 pi j kk/p)  +-  SIGN i sum_j b_j sin(2 pi j kk/p).
// The long stage (length n2, every row k1 of every job) is a small real matrix product of the
// (a, b) rows against cos/sin tables held in shared memory: each thread owns one row and four
// consecutive kk, so one pass over j loads two complex operands and two float4 table entries
// for sixteen multiply-adds.  The short stage forms the (a, b) rows directly, so the
// twiddled intermediate never exists as an array.  Complex values are float2 throughout.
#include <stdint.h>

#include <algorithm>

#include "dft_c32.cuh"
#include "s2w_internal.h"

namespace s2w {
namespace {

constexpr int kFKT = 4;   // long-stage outputs kk per thread
constexpr int kFVB = 4;   // jobs per chunk, at most

struct DftfArgs {
  const void* pix_in;
  void* pix_out;
  int64_t pix_sb;
  double2* G;            // [B][nact][nr][Mc] float64 columns
  int nact, Ng, L, nr, Mc, mlo, n, n1, n2;
  const float4* tw;      // [n] exp(+2 pi i e/n) as pairs (the hi parts are used)
  const float4* gph;     // [nact][Ng] exp(+i n gamma_g) as pairs
  const int* nvals;      // [nact]
  double scale;          // forward normalisation
  int vb;                // jobs per chunk
};

// Shared-memory layout, in float2 units (the cos/sin tables first, so that they are
// 16-byte aligned for float4 reads).
struct FLayout {
  int h1, h2, Q, R, Rp;
  int cs, tw, gp, Z, X, T0, A, B, total;
};

__host__ __device__ inline FLayout f_layout(int n, int n1, int n2, int nj, int Ng, int vb, bool zall) {
  FLayout l;
  l.h1 = (n1 - 1) / 2;
  l.h2 = (n2 - 1) / 2;
  l.Q = (l.h2 + kFKT) / kFKT;        // ceil((h2 + 1) / 4)
  l.R = vb * n1;
  l.Rp = l.R | 1;                    // odd row stride: the short stage's scattered stores do not collide
  l.cs = 0;                          // [2][h2][Q] float4: cos, then sin
  l.tw = l.cs + 2 * l.h2 * l.Q * 2;
  l.gp = l.tw + n;                   // [nj][Ng] (cos, sin) of n_j gamma_g
  l.Z = l.gp + nj * Ng;              // inverse: [nj][n] the alpha-synthesised jobs
  l.X = l.Z + (zall ? nj * n : 0);   // [vb][n] chunk input (and the forward's output staging)
  l.T0 = l.X + vb * n;               // [Rp] row constants x_0
  l.A = l.T0 + l.Rp;                 // [h2][Rp] sums a_j
  l.B = l.A + l.h2 * l.Rp;           // [h2][Rp] differences b_j
  l.total = l.B + l.h2 * l.Rp;
  return l;
}

__device__ __forceinline__ float2 f2add(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 f2sub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
// a * omega_n^{SIGN e} for the table entry w = exp(+2 pi i e/n)
template <int SIGN>
__device__ __forceinline__ float2 f2tw(float2 a, float2 w) {
  const float s = SIGN > 0 ? w.y : -w.y;
  return make_float2(fmaf(a.x, w.x, -a.y * s), fmaf(a.x, s, a.y * w.x));
}

// Tables of the long stage: cos and sin of 2 pi j kk / n2 for j = 1..h2 and kk = 0..4Q-1
// (zero past h2), from the twiddle table (2 pi j kk / n2 = 2 pi (n1 j kk) / n).
__device__ void f_tables(const FLayout& l, float2* s2, const float4* tw_g, int n, int n1) {
  float2* tw = s2 + l.tw;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const float4 w = tw_g[i];
    tw[i] = make_float2(w.x, w.z);
  }
  float* cs = reinterpret_cast<float*>(s2 + l.cs);
  const int per = l.h2 * l.Q * kFKT;
  for (int i = threadIdx.x; i < per; i += blockDim.x) {
    const int j = i / (l.Q * kFKT) + 1, kk = i % (l.Q * kFKT);
    float c = 0.f, s = 0.f;
    if (kk <= l.h2) {
      const float4 w = tw_g[(int)(((int64_t)n1 * j * kk) % n)];
      c = w.x;
      s = w.z;
    }
    cs[i] = c;
    cs[per + i] = s;
  }
}

// Short stage for a chunk of vb transforms x[v][n] (input index n2 j1 + j2): the length-n1 DFTs
// over j1 of the columns j2 = p and n2 - p, twiddled by omega_n^{SIGN j2 k1}, then combined into
// the long stage's rows: T0 = column 0, A = sum, B = difference of the column pair.
template <int SIGN>
__device__ void f_stage1(const FLayout& l, float2* s2, int n, int n1, int n2, int vb) {
  const float2* x0 = s2 + l.X;
  const float2* tw = s2 + l.tw;
  float2* T0 = s2 + l.T0;
  float2* A = s2 + l.A;
  float2* B = s2 + l.B;
  const int per = l.h2 + 1;
  for (int it = threadIdx.x; it < vb * per; it += blockDim.x) {
    const int v = it / per, p = it - v * per;
    const int q = p == 0 ? 0 : n2 - p;
    const float2* x = x0 + v * n;
    const int row0 = v * n1;
    auto emit = [&](int k1, float2 yp, float2 yq) {
      if (p == 0) {
        T0[row0 + k1] = yp;   // column 0: twiddle 1
      } else {
        const float2 tp = f2tw<SIGN>(yp, tw[p * k1]), tq = f2tw<SIGN>(yq, tw[q * k1]);   // p k1, q k1 < n
        A[(p - 1) * l.Rp + row0 + k1] = f2add(tp, tq);
        B[(p - 1) * l.Rp + row0 + k1] = f2sub(tp, tq);
      }
    };
    {
      float2 sp = make_float2(0.f, 0.f), sq = sp;
      for (int j1 = 0; j1 < n1; ++j1) {
        sp = f2add(sp, x[n2 * j1 + p]);
        sq = f2add(sq, x[n2 * j1 + q]);
      }
      emit(0, sp, sq);
    }
    const float sg = (float)SIGN;
    for (int kk = 1; kk <= l.h1; ++kk) {
      const int step = n2 * kk;   // < n
      float2 cp = x[p], cq = x[q], sp = make_float2(0.f, 0.f), sq = sp;
      int e = step;
      for (int j = 1; j <= l.h1; ++j) {
        const float2 w = tw[e];   // cos, sin of 2 pi j kk / n1
        const float2 u = x[n2 * j + p], uu = x[n2 * (n1 - j) + p];
        const float2 r = x[n2 * j + q], rr = x[n2 * (n1 - j) + q];
        cp.x = fmaf(u.x + uu.x, w.x, cp.x);
        cp.y = fmaf(u.y + uu.y, w.x, cp.y);
        sp.x = fmaf(u.x - uu.x, w.y, sp.x);
        sp.y = fmaf(u.y - uu.y, w.y, sp.y);
        cq.x = fmaf(r.x + rr.x, w.x, cq.x);
        cq.y = fmaf(r.y + rr.y, w.x, cq.y);
        sq.x = fmaf(r.x - rr.x, w.y, sq.x);
        sq.y = fmaf(r.y - rr.y, w.y, sq.y);
        e += step;
        if (e >= n) e -= n;
      }
      // y(kk) = C + SIGN i S, y(n1 - kk) = C - SIGN i S
      emit(kk, make_float2(cp.x - sg * sp.y, cp.y + sg * sp.x), make_float2(cq.x - sg * sq.y, cq.y + sg * sq.x));
      emit(n1 - kk, make_float2(cp.x + sg * sp.y, cp.y - sg * sp.x), make_float2(cq.x + sg * sq.y, cq.y - sg * sq.x));
    }
  }
}

// Long stage: for every row r = (v, k1) of the chunk, the length-n2 DFT over j2; output
// k1 + n1 k2 of transform v goes to store(v, k, value).
template <int SIGN, class Store>
__device__ void f_stage2(const FLayout& l, const float2* s2, int n1, int n2, int vb, Store store) {
  const float4* cs = reinterpret_cast<const float4*>(s2 + l.cs);
  const float4* sn = cs + l.h2 * l.Q;
  const float2* T0 = s2 + l.T0;
  const float2* A = s2 + l.A;
  const float2* B = s2 + l.B;
  const float sg = (float)SIGN;
  const int R = vb * n1;   // rows of this chunk (l.R is the widest chunk's)
  for (int it = threadIdx.x; it < l.Q * R; it += blockDim.x) {
    const int qg = it / R, r = it - qg * R;
    const float2 t0 = T0[r];
    float cr[kFKT], ci[kFKT], sr[kFKT], si[kFKT];
#pragma unroll
    for (int u = 0; u < kFKT; ++u) {
      cr[u] = t0.x;
      ci[u] = t0.y;
      sr[u] = 0.f;
      si[u] = 0.f;
    }
#pragma unroll 2
    for (int j = 0; j < l.h2; ++j) {
      const float2 a = A[j * l.Rp + r], b = B[j * l.Rp + r];
      const float4 c4 = cs[j * l.Q + qg], s4 = sn[j * l.Q + qg];
      const float c[kFKT] = {c4.x, c4.y, c4.z, c4.w}, s[kFKT] = {s4.x, s4.y, s4.z, s4.w};
#pragma unroll
      for (int u = 0; u < kFKT; ++u) {
        cr[u] = fmaf(a.x, c[u], cr[u]);
        ci[u] = fmaf(a.y, c[u], ci[u]);
        sr[u] = fmaf(b.x, s[u], sr[u]);
        si[u] = fmaf(b.y, s[u], si[u]);
      }
    }
    const int v = r / n1, k1 = r - v * n1;
#pragma unroll
    for (int u = 0; u < kFKT; ++u) {
      const int kk = qg * kFKT + u;
      if (kk > l.h2) break;
      store(v, k1 + n1 * kk, make_float2(cr[u] - sg * si[u], ci[u] + sg * sr[u]));
      if (kk > 0) store(v, k1 + n1 * (n2 - kk), make_float2(cr[u] + sg * si[u], ci[u] - sg * sr[u]));
    }
  }
}

__device__ __forceinline__ float2 f_pix(const void* pix, bool real, int64_t i) {
  if (real) return make_float2((float)((const double*)pix)[i], 0.f);
  const double2 v = ((const double2*)pix)[i];
  return make_float2((float)v.x, (float)v.y);
}

template <bool REAL>
__global__ void __launch_bounds__(512) k_dftf_fwd(DftfArgs a) {
  extern __shared__ float4 s4f[];
  float2* s2 = reinterpret_cast<float2*>(s4f);
  __shared__ int jn[kMaxJobs], jp[kMaxJobs], njs;
  const int n = a.n, L = a.L, t = blockIdx.x, b = blockIdx.y;
  if (threadIdx.x == 0) {
    int nj;
    make_jobs(a.nvals, a.nact, REAL, jn, jp, nj);
    njs = nj;
  }
  __syncthreads();
  const int nj = njs, Ng = a.Ng, hg = (Ng - 1) / 2;
  const FLayout l = f_layout(n, a.n1, a.n2, nj, Ng, a.vb, false);
  f_tables(l, s2, a.tw, n, a.n1);
  float2* gp = s2 + l.gp;
  for (int i = threadIdx.x; i < nj * Ng; i += blockDim.x) {
    const int j = i / Ng, g = i - j * Ng;
    const float4 ph = a.gph[jn[j] * Ng + g];
    gp[i] = make_float2(ph.x, ph.z);
  }
  float2* X = s2 + l.X;
  const int64_t ring = (int64_t)a.nr * n;
  const int64_t base = (int64_t)b * a.pix_sb + (int64_t)t * n;
  const double sc = a.scale;
  for (int j0 = 0; j0 < nj; j0 += a.vb) {
    const int vb = min(a.vb, nj - j0);
    __syncthreads();   // tables ready; the previous chunk's write-out has read X
    // H_j(alpha) = sum_g W(alpha, gamma_g) exp(-i n_j gamma_g), gamma_g paired with gamma_{Ng-g}
    for (int al = threadIdx.x; al < n; al += blockDim.x) {
      const float2 w0 = f_pix(a.pix_in, REAL, base + al);
      float hr[kFVB], hi[kFVB];
#pragma unroll
      for (int q = 0; q < kFVB; ++q) {
        hr[q] = w0.x;
        hi[q] = w0.y;
      }
#pragma unroll 4
      for (int g = 1; g <= hg; ++g) {
        const float2 xp = f_pix(a.pix_in, REAL, base + g * ring + al);
        const float2 xm = f_pix(a.pix_in, REAL, base + (Ng - g) * ring + al);
        const float2 u = f2add(xp, xm), v = f2sub(xp, xm);
#pragma unroll
        for (int q = 0; q < kFVB; ++q) {
          if (q < vb) {
            const float2 ph = gp[(j0 + q) * Ng + g];   // cos, sin of n gamma_g
            hr[q] = fmaf(u.x, ph.x, hr[q]);           // u cos - i v sin
            hi[q] = fmaf(-v.x, ph.y, hi[q]);
            if (!REAL) {
              hr[q] = fmaf(v.y, ph.y, hr[q]);
              hi[q] = fmaf(u.y, ph.x, hi[q]);
            }
          }
        }
      }
#pragma unroll
      for (int q = 0; q < kFVB; ++q)
        if (q < vb) X[q * n + al] = make_float2(hr[q], hi[q]);
    }
    __syncthreads();
    f_stage1<-1>(l, s2, n, a.n1, a.n2, vb);
    __syncthreads();
    f_stage2<-1>(l, s2, a.n1, a.n2, vb, [&](int v, int k, float2 z) { X[v * n + k] = z; });
    __syncthreads();
    // write-out: G_{m,n} = scale Z(m); real signals also give G_{m',-n} = conj Z(-m')
    for (int e = threadIdx.x; e < vb * n; e += blockDim.x) {
      const int v = e / n, k = e - v * n;
      const int ni = jn[j0 + v], pi = jp[j0 + v];
      const float2 z = X[e];
      const double zr = (double)z.x * sc, zi = (double)z.y * sc;
      double2* Gn = a.G + (((int64_t)b * a.nact + ni) * a.nr + t) * a.Mc;
      if (REAL) {
        if (k < L) Gn[k] = make_double2(zr, zi);
        if (pi >= 0) {
          const int mp = (k == 0) ? 0 : n - k;
          if (mp < L) a.G[(((int64_t)b * a.nact + pi) * a.nr + t) * a.Mc + mp] = make_double2(zr, -zi);
        }
      } else {
        const int m = (k < L) ? k : k - n;
        Gn[m - a.mlo] = make_double2(zr, zi);
      }
    }
  }
}

template <bool REAL>
__global__ void __launch_bounds__(512) k_dftf_inv(DftfArgs a) {
  extern __shared__ float4 s4f[];
  float2* s2 = reinterpret_cast<float2*>(s4f);
  __shared__ int jn[kMaxJobs], jp[kMaxJobs], njs;
  const int n = a.n, L = a.L, t = blockIdx.x, b = blockIdx.y;
  if (threadIdx.x == 0) {
    int nj;
    make_jobs(a.nvals, a.nact, REAL, jn, jp, nj);
    njs = nj;
  }
  __syncthreads();
  const int nj = njs, Ng = a.Ng, hg = (Ng - 1) / 2;
  const FLayout l = f_layout(n, a.n1, a.n2, nj, Ng, a.vb, true);
  f_tables(l, s2, a.tw, n, a.n1);
  float2* gp = s2 + l.gp;
  for (int i = threadIdx.x; i < nj * Ng; i += blockDim.x) {
    const int j = i / Ng, g = i - j * Ng;
    const float4 ph = a.gph[jn[j] * Ng + g];
    gp[i] = make_float2(ph.x, ph.z);
  }
  float2* X = s2 + l.X;
  float2* Z = s2 + l.Z;
  for (int j0 = 0; j0 < nj; j0 += a.vb) {
    const int vb = min(a.vb, nj - j0);
    // chunk input x_v(k), k = 0..n-1: m = k for k < L, m = k - n otherwise; real signals take
    // G_{m,n} = conj G_{-m,-n} for m < 0
    for (int e = threadIdx.x; e < vb * n; e += blockDim.x) {
      const int v = e / n, k = e - v * n;
      const int ni = jn[j0 + v], pi = jp[j0 + v];
      const double2* Gn = a.G + (((int64_t)b * a.nact + ni) * a.nr + t) * a.Mc;
      double2 z;
      if (REAL) {
        if (k < L) {
          z = Gn[k];
        } else {
          const double2 w = a.G[(((int64_t)b * a.nact + (pi >= 0 ? pi : ni)) * a.nr + t) * a.Mc + (n - k)];
          z = make_double2(w.x, -w.y);
        }
      } else {
        const int m = (k < L) ? k : k - n;
        z = Gn[m - a.mlo];
      }
      X[e] = make_float2((float)z.x, (float)z.y);
    }
    __syncthreads();   // X loaded; the previous chunk's long stage has read T0/A/B
    f_stage1<1>(l, s2, n, a.n1, a.n2, vb);
    __syncthreads();
    f_stage2<1>(l, s2, a.n1, a.n2, vb, [&](int v, int k, float2 z) { Z[(j0 + v) * n + k] = z; });
  }
  __syncthreads();
  // W(alpha, gamma_g) = sum_j Z_j(alpha) exp(+i n_j gamma_g); gamma_g and gamma_{Ng-g} share
  // P = sum_j Z_j cos, Q = sum_j Z_j sin.  Real signals: the n, -n pair gives 2 Re, n = 0 Re.
  const int64_t ring = (int64_t)a.nr * n;
  const int64_t base = (int64_t)b * a.pix_sb + (int64_t)t * n;
  for (int al = threadIdx.x; al < n; al += blockDim.x) {
    for (int g = 0; g <= hg; ++g) {
      float pr = 0.f, pim = 0.f, qr = 0.f, qim = 0.f;
      for (int j = 0; j < nj; ++j) {
        float2 z = Z[j * n + al];
        if (REAL && jp[j] >= 0) z = make_float2(2.f * z.x, 2.f * z.y);
        const float2 ph = gp[j * Ng + g];
        pr = fmaf(z.x, ph.x, pr);
        qim = fmaf(z.y, ph.y, qim);
        if (!REAL) {
          pim = fmaf(z.y, ph.x, pim);
          qr = fmaf(z.x, ph.y, qr);
        }
      }
      if (REAL) {
        double* out = (double*)a.pix_out;
        out[base + g * ring + al] = (double)(pr - qim);
        if (g > 0) out[base + (Ng - g) * ring + al] = (double)(pr + qim);
      } else {
        double2* out = (double2*)a.pix_out;   // P + i Q and P - i Q
        out[base + g * ring + al] = make_double2((double)(pr - qim), (double)(pim + qr));
        if (g > 0) out[base + (Ng - g) * ring + al] = make_double2((double)(pr + qim), (double)(pim - qr));
      }
    }
  }
}

constexpr size_t kDftfSmemMax = 74 * 1024;   // three blocks per SM

int dftf_jobs(const TransformSpec& t, bool real) {
  int nj = 0;
  for (int v : t.nvals_h)
    if (!real || v >= 0) ++nj;
  return nj;
}

size_t dftf_bytes(const GridTables& g, const TransformSpec& t, bool real, int vb, bool zall) {
  const FLayout l = f_layout(g.n, g.n1, g.n2, dftf_jobs(t, real), 2 * t.N - 1, vb, zall);
  return (size_t)l.total * sizeof(float2);
}

// jobs per chunk: the largest of 4, 2, 1 whose shared memory fits three blocks per SM, else the
// smallest that fits the opt-in limit; 0 if none does
int dftf_vb(const GridTables& g, const TransformSpec& t, bool real, bool zall) {
  const int nj = dftf_jobs(t, real);
  if (nj < 1 || nj > kMaxJobs) return 0;
  for (int vb = std::min(nj, kFVB); vb >= 1; vb /= 2)
    if (dftf_bytes(g, t, real, vb, zall) <= kDftfSmemMax) return vb;
  return dftf_bytes(g, t, real, 1, zall) <= 200 * 1024 ? 1 : 0;
}

bool dftf_ok(const GridTables& g, const TransformSpec& t, bool real) {
  if (real)   // every negative n needs its partner -n among the carried values
    for (int v : t.nvals_h)
      if (v < 0) {
        bool found = false;
        for (int w : t.nvals_h) found = found || (w == -v);
        if (!found) return false;
      }
  return g.n >= 1 && g.n % 2 == 1 && (2 * t.N - 1) % 2 == 1;
}

DftfArgs f_args(const GridTables& g, const TransformSpec& t, ColumnArgs c) {
  DftfArgs a;
  a.pix_in = nullptr;
  a.pix_out = nullptr;
  a.pix_sb = 0;
  a.G = c.G;
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
  a.vb = 1;
  return a;
}

template <class K>
cudaError_t f_launch(K kern, dim3 grid, size_t smem, int threads, cudaStream_t st, const DftfArgs& a) {
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  kern<<<grid, threads, smem, st>>>(a);
  return cudaGetLastError();
}

}  // namespace

bool dftf_usable(const GridTables& g, const TransformSpec& t, bool real, bool fwd) {
  return dftf_ok(g, t, real) && dftf_vb(g, t, real, !fwd) >= 1;
}

cudaError_t launch_dftf_forward(const GridTables& g, const TransformSpec& t, const void* pix, int64_t pix_sb,
                                bool real, ColumnArgs c, cudaStream_t st) {
  if (!dftf_usable(g, t, real, true)) return cudaErrorInvalidValue;
  const int vb = dftf_vb(g, t, real, false);
  DftfArgs a = f_args(g, t, c);
  a.pix_in = pix;
  a.pix_sb = pix_sb;
  a.scale = (2.0 * 3.14159265358979323846 / g.n) * t.gscale;
  a.vb = vb;
  const size_t smem = dftf_bytes(g, t, real, vb, false);
  const dim3 grid(c.nr, c.B);
  return real ? f_launch(k_dftf_fwd<true>, grid, smem, t.dft_threads_fwd, st, a)
              : f_launch(k_dftf_fwd<false>, grid, smem, t.dft_threads_fwd, st, a);
}

cudaError_t launch_dftf_inverse(const GridTables& g, const TransformSpec& t, ColumnArgs c, void* pix, int64_t pix_sb,
                                bool real, cudaStream_t st) {
  if (!dftf_usable(g, t, real, false)) return cudaErrorInvalidValue;
  const int vb = dftf_vb(g, t, real, true);
  DftfArgs a = f_args(g, t, c);
  a.pix_out = pix;
  a.pix_sb = pix_sb;
  a.vb = vb;
  const size_t smem = dftf_bytes(g, t, real, vb, true);
  const dim3 grid(c.nr, c.B);
  return real ? f_launch(k_dftf_inv<true>, grid, smem, t.dft_threads_inv, st, a)
              : f_launch(k_dftf_inv<false>, grid, smem, t.dft_threads_inv, st, a);
}

}  // namespace s2w

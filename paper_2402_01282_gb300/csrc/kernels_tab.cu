// Float64-accurate l-contractions against precomputed Wigner-d tables (S2W_FP64 with
// precompute = 1; the paper's precomputed mode, Sec. 4.2).  The tables are built once per
// plan from the same float64 recursion as the on-the-fly kernels and stored as float pairs
// (hi + lo, ~48 bits); the contractions are compensated-float32 GEMMs (comp32.cuh).
//
//  * k_tab_build   T_inv[(m,n)][l - l0a][beta] (l0a = max(|m|,|n|) rounded down to a multiple of 8) = d^l_mn(beta_b): one thread per beta runs the
//                  recursion over l (wigner_rec.cuh), zero outside l0 <= l < L, beta < nr (rings).
//  * k_tab_fold    T_fwd[(m,n)][beta'][l - l0a] = sum_beta M^{par(m+n)}[beta][beta'] d^l_mn(beta):
//                  the colatitude quadrature of the forward transforms folded into the table
//                  (F_l = sum_beta d^l (M G)(beta) = sum_beta' (M^T d^l)(beta') G(beta')), float64;
//                  on DH sampling M is the diagonal of ring weights, T_fwd = w(beta') d^l_mn(beta').
//  * k_tab_inv     G[b][n][beta][m] = sum_l T_inv[l][beta] (mult_inv f)(b, l, m)
//  * k_tab_fwd     out(b, l, m) += mult_fwd[l][n] sum_beta' T_fwd[beta'][l] G[b][n][beta'][m]
// Both GEMM kernels: one block per (64-row tile, m, n), 128 threads, a 4 x 4 micro-tile per
// thread (4 rows x 2 maps x re/im), 32-deep reduction chunks staged in shared memory with
// the reduction index outermost (tables are stored that way, so the loads are coalesced).
#include <math.h>

#include "comp32.cuh"
#include "s2w_internal.h"
#include "wigner_rec.cuh"

namespace s2w {
namespace {

constexpr int kRows = 64;      // output rows per block
constexpr int kK = 32;         // reduction chunk
constexpr int kMaps = 16;      // maps per pass (32 real columns)
constexpr int kThreads = 128;  // 16 row groups x 8 column groups

__device__ __forceinline__ double2 cmul2(double2 a, double2 b) {
  return make_double2(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}

struct TabBuildArgs {
  RecTables T;
  const int* nvals;
  int nact, L, nr, Mc, mlo, Lp;
  const int64_t* off_inv;
  const int* kp;
  float2* inv;
};

__global__ void k_tab_build(TabBuildArgs a) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  const int mi = blockIdx.y, ni = blockIdx.z;
  if (b >= a.Lp) return;
  const int idx = mi * a.nact + ni, kp = a.kp[idx];
  if (kp == 0) return;
  const int m = a.mlo + mi, nn = a.nvals[ni], L = a.L;
  const int l0 = max(abs(m), abs(nn)), l0a = l0 & ~7;
  float2* out = a.inv + a.off_inv[idx] + b;
  for (int ll = 0; ll < l0 - l0a; ++ll) out[(int64_t)ll * a.Lp] = make_float2(0.f, 0.f);
  for (int ll = L - l0a; ll < kp; ++ll) out[(int64_t)ll * a.Lp] = make_float2(0.f, 0.f);
  if (b >= a.nr) {
    for (int ll = l0 - l0a; ll < L - l0a; ++ll) out[(int64_t)ll * a.Lp] = make_float2(0.f, 0.f);
    return;
  }
  const double wb = a.T.wpole[b];
  const bool north = 2 * (2 * b + 1) < a.T.den;
  double v = 0.0, vp = 0.0;
  int q = 0;
  wigner_seed(a.T, b, l0, m, nn, v, q);
  for (int l = l0; l < L; ++l) {
    out[(int64_t)(l - l0a) * a.Lp] = (q == 0) ? split1(v) : make_float2(0.f, 0.f);
    double A, Kn, Ks, C;
    rec_coeffs(l, m, nn, A, Kn, Ks, C);
    const double x = fma(A, wb, north ? Kn : Ks);
    const double vn = fma(x, v, -C * vp);
    vp = v;
    v = vn;
    if (q > 0 && fabs(v) > kRescaleAt) {
      v *= kRescaleBy;
      vp *= kRescaleBy;
      --q;
    }
  }
}

struct TabFoldArgs {
  const int* nvals;
  int nact, L, nr, Mc, mlo, Lp, Lk;
  const int64_t* off_inv;
  const int64_t* off_fwd;
  const int* kp;
  const float2* inv;
  float2* fwd;
  const double* MR;      // MW: [2][L][L] row-major M[par][t][t']
  const double* wdiag;   // DH: [nr] ring weights (MR unused)
};

constexpr int kFoldL = 32, kFoldB = 64, kFoldThreads = 256;

// block: (32-l chunk x 256-beta' tile, m, n); thread = beta'
__global__ void __launch_bounds__(kFoldThreads) k_tab_fold(TabFoldArgs a) {
  __shared__ double Ds[kFoldL][kFoldB];
  const int nbt = (a.Lk + kFoldThreads - 1) / kFoldThreads;
  const int lc = blockIdx.x / nbt, bt = blockIdx.x - lc * nbt, mi = blockIdx.y, ni = blockIdx.z;
  const int idx = mi * a.nact + ni, kp = a.kp[idx];
  if (lc * kFoldL >= kp) return;
  const int m = a.mlo + mi, nn = a.nvals[ni], L = a.L;
  const float2* Tin = a.inv + a.off_inv[idx];
  float2* Tout = a.fwd + a.off_fwd[idx];
  const int bp = bt * kFoldThreads + threadIdx.x;
  if (a.wdiag != nullptr) {   // DH: T_fwd[beta'][l] = w(beta') d^l(beta')
    if (bp < a.Lk) {
      const double w = (bp < a.nr) ? a.wdiag[bp] : 0.0;
      for (int j = 0; j < kFoldL; ++j) {
        float2 r = make_float2(0.f, 0.f);
        if (bp < a.nr) {
          const float2 p = Tin[(int64_t)(lc * kFoldL + j) * a.Lp + bp];
          r = split1(((double)p.x + (double)p.y) * w);
        }
        Tout[(int64_t)bp * kp + lc * kFoldL + j] = r;
      }
    }
    return;
  }
  const int par = (m + nn) & 1;
  const double* M = a.MR + (size_t)par * L * L;
  double acc[kFoldL];
#pragma unroll
  for (int j = 0; j < kFoldL; ++j) acc[j] = 0.0;
  for (int b0 = 0; b0 < L; b0 += kFoldB) {
    __syncthreads();
    for (int i = threadIdx.x; i < kFoldL * kFoldB; i += blockDim.x) {
      const int j = i / kFoldB, bb = i - j * kFoldB, beta = b0 + bb;
      double d = 0.0;
      if (beta < L) {
        const float2 p = Tin[(int64_t)(lc * kFoldL + j) * a.Lp + beta];
        d = (double)p.x + (double)p.y;
      }
      Ds[j][bb] = d;
    }
    __syncthreads();
    if (bp < L) {
      const int cnt = min(kFoldB, L - b0);
      for (int bb = 0; bb < cnt; ++bb) {
        const double w = M[(size_t)(b0 + bb) * L + bp];
#pragma unroll
        for (int j = 0; j < kFoldL; ++j) acc[j] = fma(w, Ds[j][bb], acc[j]);
      }
    }
  }
  if (bp < a.Lk) {
#pragma unroll
    for (int j = 0; j < kFoldL; ++j)
      Tout[(int64_t)bp * kp + lc * kFoldL + j] = (bp < L) ? split1(acc[j]) : make_float2(0.f, 0.f);
  }
}

// 4 rows x (2 maps x re/im) compensated multiply-adds for one reduction index k
__device__ __forceinline__ void mac_tile(Acc (&acc)[4][4], const float4* Ak, const float4* Bk, int ty, int tx) {
  const float4 a01 = Ak[2 * ty], a23 = Ak[2 * ty + 1];
  const float4 b0 = Bk[2 * tx], b1 = Bk[2 * tx + 1];
  const float2 av[4] = {make_float2(a01.x, a01.y), make_float2(a01.z, a01.w), make_float2(a23.x, a23.y),
                        make_float2(a23.z, a23.w)};
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    acc_add(acc[r][0], b0.x, b0.y, av[r].x, av[r].y);
    acc_add(acc[r][1], b0.z, b0.w, av[r].x, av[r].y);
    acc_add(acc[r][2], b1.x, b1.y, av[r].x, av[r].y);
    acc_add(acc[r][3], b1.z, b1.w, av[r].x, av[r].y);
  }
}

// asynchronous 16-byte global -> shared copies (one group per reduction chunk)
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((uint32_t)__cvta_generic_to_shared(smem)),
               "l"(gmem)
               : "memory");
}
__device__ __forceinline__ void cp_async16_zfill(void* smem, const void* gmem, int src_bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"((uint32_t)__cvta_generic_to_shared(smem)),
               "l"(gmem), "r"(src_bytes)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// complex float64 -> (re_hi, re_lo, im_hi, im_lo) with integer operations only
__device__ __forceinline__ float4 split_bits(double2 v) {
  const float2 r = split1_bits(v.x), i = split1_bits(v.y);
  return make_float4(r.x, r.y, i.x, i.y);
}

// Copies the 32 x 64 table tile (k rows k0.., row columns row0..) into As: 1024 granules of
// 16 bytes, 8 per thread.  `ld` = row stride of the table in float2.
// Columns row0 + 2c >= rows_valid are zero-filled without a read (source size 0).
__device__ __forceinline__ void issue_tile(float4 (*As)[kRows / 2], const float2* T, int64_t ld, int k0, int row0,
                                           int tid, int rows_valid) {
#pragma unroll
  for (int q = 0; q < (kK * kRows / 2) / kThreads; ++q) {
    const int gi = tid + q * kThreads, k = gi / (kRows / 2), c = gi - k * (kRows / 2);
    const bool ok = row0 + 2 * c < rows_valid;
    cp_async16_zfill(&As[k][c], ok ? T + (int64_t)(k0 + k) * ld + row0 + 2 * c : T, ok ? 16 : 0);
  }
  cp_async_commit();
}

constexpr int kBPer = kK * kMaps / kThreads;   // B entries per thread per chunk (4)

struct TabInvArgs {
  const double2* coef;
  int64_t s_b, s_n, s_l;
  int mlo_in;
  const double* mult_r;   // [L][nact] real factor of the inverse multiplier
  double2 phase;          // its constant complex phase
  const int* nvals;
  int nact;
  const int64_t* off;
  const int* kp;
  int Lp;
  const float2* tab;
  double2* G;
  int B, L, nr, Mc, mlo;
};

// Double-buffered: the table tile of chunk c+1 is copied asynchronously and its data
// operand is fetched into registers while chunk c is contracted.
__global__ void __launch_bounds__(kThreads) k_tab_inv(TabInvArgs a) {
  __shared__ __align__(16) float4 As[2][kK][kRows / 2];   // [k][row] pairs
  __shared__ __align__(16) float4 Bs[2][kK][kMaps];       // [k][map] (re_hi, re_lo, im_hi, im_lo)
  const int rt = blockIdx.x, mi = blockIdx.y, ni = blockIdx.z;
  const int L = a.L, nr = a.nr, row0 = rt * kRows;
  if (row0 >= nr) return;
  const int m = a.mlo + mi, nn = a.nvals[ni];
  const int idx = mi * a.nact + ni, kp = a.kp[idx];
  const int l0 = max(abs(m), abs(nn)), l0a = l0 & ~7;
  const int nch = kp == 0 ? 0 : (L - l0a + kK - 1) / kK;
  const float2* T = a.tab + a.off[idx];
  const int tid = threadIdx.x, ty = tid >> 3, tx = tid & 7;
  const bool warp_live = row0 + 16 * (tid >> 5) < nr;   // a warp owns 16 rows beta
  auto load_b = [&](int c, int map0, double2 (&f)[kBPer]) {
#pragma unroll
    for (int q = 0; q < kBPer; ++q) {
      const int i = tid + q * kThreads, k = i / kMaps, mp = i - k * kMaps;
      const int l = l0a + c * kK + k, bm = map0 + mp;
      f[q] = make_double2(0.0, 0.0);
      if (l >= l0 && l < L && bm < a.B) {
        const double2 v = a.coef[(int64_t)bm * a.s_b + (int64_t)ni * a.s_n + (int64_t)l * a.s_l + (m - a.mlo_in)];
        const double r = a.mult_r[(int64_t)l * a.nact + ni];
        f[q] = make_double2(v.x * r, v.y * r);
      }
    }
  };
  for (int map0 = 0; map0 < a.B; map0 += kMaps) {
    Acc acc[4][4];
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
      for (int c = 0; c < 4; ++c) acc[r][c] = Acc{0.f, 0.f};
    double2 f[kBPer];
    if (nch > 0) {
      issue_tile(As[0], T, a.Lp, 0, row0, tid, a.Lp);
      load_b(0, map0, f);
    }
    for (int c = 0; c < nch; ++c) {
      const int buf = c & 1;
#pragma unroll
      for (int q = 0; q < kBPer; ++q) {
        const int i = tid + q * kThreads;
        Bs[buf][i / kMaps][i % kMaps] = split_bits(f[q]);
      }
      if (c + 1 < nch) {
        issue_tile(As[buf ^ 1], T, a.Lp, (c + 1) * kK, row0, tid, a.Lp);
        load_b(c + 1, map0, f);
        cp_async_wait<1>();
      } else {
        cp_async_wait<0>();
      }
      __syncthreads();
      if (warp_live) {
        const int kend = min(kK, L - l0a - c * kK);   // the last chunk stops at l = L - 1
#pragma unroll 4
        for (int k = 0; k < kend; ++k) mac_tile(acc, As[buf][k], Bs[buf][k], ty, tx);
      }
      __syncthreads();
    }
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const int beta = row0 + 4 * ty + r;
      if (beta >= nr) continue;
#pragma unroll
      for (int p = 0; p < 2; ++p) {
        const int bm = map0 + 2 * tx + p;
        if (bm < a.B) {
          const double x = to_double(acc[r][2 * p]), y = to_double(acc[r][2 * p + 1]);
          a.G[(((int64_t)bm * a.nact + ni) * nr + beta) * a.Mc + mi] =
              make_double2(fma(x, a.phase.x, -y * a.phase.y), fma(x, a.phase.y, y * a.phase.x));
        }
      }
    }
  }
}

struct TabFwdArgs {
  const double2* G;
  int B, L, nr, Mc, mlo;
  const int* nvals;
  int nact;
  const double2* mult;
  double2* out;
  int64_t s_b, s_n, s_l;
  int mlo_out;
  const int64_t* off;
  const int* kp;
  int Lk;
  const float2* tab;
};

__global__ void __launch_bounds__(kThreads) k_tab_fwd(TabFwdArgs a) {
  __shared__ __align__(16) float4 As[2][kK][kRows / 2];   // [k = beta'][row = l] pairs
  __shared__ __align__(16) float4 Bs[2][kK][kMaps];       // [k = beta'][map]
  const int rt = blockIdx.x, mi = blockIdx.y, ni = blockIdx.z;
  const int idx = mi * a.nact + ni, kp = a.kp[idx];
  const int row0 = rt * kRows;
  if (row0 >= kp) return;
  const int L = a.L, nr = a.nr, m = a.mlo + mi, nn = a.nvals[ni];
  const int l0 = max(abs(m), abs(nn)), l0a = l0 & ~7;
  const int nch = (nr + kK - 1) / kK;   // reduction over the rings beta'
  const float2* T = a.tab + a.off[idx];
  const int tid = threadIdx.x, ty = tid >> 3, tx = tid & 7;
  // a warp owns 16 rows l; it skips the products when none of them lies in [l0, L)
  const int wl0 = l0a + row0 + 16 * (tid >> 5);
  const bool warp_live = wl0 + 16 > l0 && wl0 < L;
  auto load_b = [&](int c, int map0, double2 (&f)[kBPer]) {
#pragma unroll
    for (int q = 0; q < kBPer; ++q) {
      const int i = tid + q * kThreads, k = i / kMaps, mp = i - k * kMaps;
      const int beta = c * kK + k, bm = map0 + mp;
      f[q] = (beta < nr && bm < a.B) ? a.G[(((int64_t)bm * a.nact + ni) * nr + beta) * a.Mc + mi]
                                     : make_double2(0.0, 0.0);
    }
  };
  for (int map0 = 0; map0 < a.B; map0 += kMaps) {
    Acc acc[4][4];
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
      for (int c = 0; c < 4; ++c) acc[r][c] = Acc{0.f, 0.f};
    double2 f[kBPer];
    issue_tile(As[0], T, kp, 0, row0, tid, kp);
    load_b(0, map0, f);
    for (int c = 0; c < nch; ++c) {
      const int buf = c & 1;
#pragma unroll
      for (int q = 0; q < kBPer; ++q) {
        const int i = tid + q * kThreads;
        Bs[buf][i / kMaps][i % kMaps] = split_bits(f[q]);
      }
      if (c + 1 < nch) {
        issue_tile(As[buf ^ 1], T, kp, (c + 1) * kK, row0, tid, kp);
        load_b(c + 1, map0, f);
        cp_async_wait<1>();
      } else {
        cp_async_wait<0>();
      }
      __syncthreads();
      if (warp_live) {
        const int kend = min(kK, nr - c * kK);
#pragma unroll 4
        for (int k = 0; k < kend; ++k) mac_tile(acc, As[buf][k], Bs[buf][k], ty, tx);
      }
      __syncthreads();
    }
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const int l = l0a + row0 + 4 * ty + r;
      if (l < l0 || l >= L) continue;
      const double2 u = a.mult[(int64_t)l * a.nact + ni];
#pragma unroll
      for (int p = 0; p < 2; ++p) {
        const int bm = map0 + 2 * tx + p;
        if (bm < a.B) {
          const double2 v = cmul2(make_double2(to_double(acc[r][2 * p]), to_double(acc[r][2 * p + 1])), u);
          double2* o = a.out + (int64_t)bm * a.s_b + (int64_t)ni * a.s_n + (int64_t)l * a.s_l + (m - a.mlo_out);
          atomicAdd(&o->x, v.x);
          atomicAdd(&o->y, v.y);
        }
      }
    }
  }
}

RecTables rec_tables_tab(const GridTables& g) {
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

}  // namespace

cudaError_t launch_tab_build(const GridTables& g, const TransformSpec& t, const TabTable& tab, int Mc, int mlo,
                             cudaStream_t st) {
  TabBuildArgs a;
  a.T = rec_tables_tab(g);
  a.nvals = t.nvals;
  a.nact = t.nact;
  a.L = t.L;
  a.nr = g.nr;
  a.Mc = Mc;
  a.mlo = mlo;
  a.Lp = tab.Lp;
  a.off_inv = tab.off_inv;
  a.kp = tab.kp;
  a.inv = tab.inv;
  dim3 grid((tab.Lp + 127) / 128, Mc, t.nact);
  k_tab_build<<<grid, 128, 0, st>>>(a);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  TabFoldArgs f;
  f.nvals = t.nvals;
  f.nact = t.nact;
  f.L = t.L;
  f.nr = g.nr;
  f.Mc = Mc;
  f.mlo = mlo;
  f.Lp = tab.Lp;
  f.Lk = tab.Lk;
  f.off_inv = tab.off_inv;
  f.off_fwd = tab.off_fwd;
  f.kp = tab.kp;
  f.inv = tab.inv;
  f.fwd = tab.fwd;
  f.MR = g.MR;
  f.wdiag = g.wdiag;
  dim3 fgrid((tab.kpmax / kFoldL) * ((tab.Lk + kFoldThreads - 1) / kFoldThreads), Mc, t.nact);
  k_tab_fold<<<fgrid, kFoldThreads, 0, st>>>(f);
  return cudaGetLastError();
}

cudaError_t launch_tab_inverse(const GridTables& g, const TransformSpec& t, CoefArgs in, ColumnArgs out,
                               cudaStream_t st) {
  (void)g;
  const TabTable& tab = *t.tab;
  TabInvArgs a;
  a.coef = in.coef;
  a.s_b = in.s_b;
  a.s_n = in.s_n;
  a.s_l = in.s_l;
  a.mlo_in = in.mlo;
  a.mult_r = t.minv_r;
  a.phase = t.minv_phase;
  a.nvals = t.nvals;
  a.nact = t.nact;
  a.off = tab.off_inv;
  a.kp = tab.kp;
  a.Lp = tab.Lp;
  a.tab = tab.inv;
  a.G = out.G;
  a.B = out.B;
  a.L = out.L;
  a.nr = out.nr;
  a.Mc = out.Mc;
  a.mlo = out.mlo;
  dim3 grid(tab.Lp / kRows, out.Mc, t.nact);
  k_tab_inv<<<grid, kThreads, 0, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_tab_forward(const GridTables& g, const TransformSpec& t, ColumnArgs in, CoefArgs out,
                               cudaStream_t st) {
  (void)g;
  const TabTable& tab = *t.tab;
  TabFwdArgs a;
  a.G = in.G;
  a.B = in.B;
  a.L = in.L;
  a.nr = in.nr;
  a.Mc = in.Mc;
  a.mlo = in.mlo;
  a.nvals = t.nvals;
  a.nact = t.nact;
  a.mult = t.mult_fwd;
  a.out = const_cast<double2*>(out.coef);
  a.s_b = out.s_b;
  a.s_n = out.s_n;
  a.s_l = out.s_l;
  a.mlo_out = out.mlo;
  a.off = tab.off_fwd;
  a.kp = tab.kp;
  a.Lk = tab.Lk;
  a.tab = tab.fwd;
  dim3 grid((tab.kpmax + kRows - 1) / kRows, in.Mc, t.nact);
  k_tab_fwd<<<grid, kThreads, 0, st>>>(a);
  return cudaGetLastError();
}

}  // namespace s2w

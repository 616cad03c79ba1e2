// Reduced-precision contractions on the 5th-generation tensor cores (tcgen05):
// precomputed Wigner-d tiles (built once per plan from the float64 recursion) contracted
// against the harmonic coefficients (inverse) or the colatitude-weighted columns (forward),
// with float32 accumulation in TMEM.
//
// Two precisions, both with every operand a pair hi + lo and three MMAs per K step
// (hi*hi + hi*lo + lo*hi, the lo*lo term dropped): "split" in fp16 (scaled by a power of two
// into the fp16 range; 22 bits per pair, ~2^-22 per product) and "bf16" in bf16 (16 bits per
// pair, ~2^-17 per product; no range scaling needed, the tables are scaled the same way).
//
// Tiles are stored in the non-swizzled core-matrix layout (see tc_sm100.cuh) so a tile is
// one contiguous chunk that a single bulk asynchronous copy (TMA engine) brings to shared
// memory:
//   inverse table  (rows beta, K = l):  [beta/128][beta%128/8][(l-l0a)/8][8][8]
//   forward table  (rows l,    K = beta): [(l-l0a)/128][(l-l0a)%128/8][beta/8][8][8]
//   quadrature     (rows beta, K = beta'): [parity][beta/128][beta%128/8][beta'/8][8][8]
// where l0a = max(|m|,|n|) rounded down to a multiple of 16, the l extent kl is rounded up to a
// multiple of 128 and the beta extent Lb = L rounded up to 128; entries outside the
// transform are zero.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "s2w_internal.h"
#include "tc_sm100.cuh"
#include "wigner_rec.cuh"

namespace s2w {
namespace {

constexpr double kDScale = 256.0;   // d^l_mn scaled by 2^8 in the tables

// SPLIT selects fp16 (split mode) or bf16 (bf16 mode) elements; PAIR writes hi and lo.
template <bool SPLIT, bool PAIR>
__device__ __forceinline__ void put16(uint16_t* hi, uint16_t* lo, int64_t i, double x) {
  if (SPLIT) {
    const __half h = __double2half(x);
    hi[i] = __half_as_ushort(h);
    if (PAIR) lo[i] = __half_as_ushort(__double2half(x - (double)__half2float(h)));
  } else {
    const __nv_bfloat16 h = __double2bfloat16(x);
    hi[i] = __bfloat16_as_ushort(h);
    if (PAIR) lo[i] = __bfloat16_as_ushort(__double2bfloat16(x - (double)__bfloat162float(h)));
  }
}

__device__ __forceinline__ int64_t inv_index(int beta, int ll, int kl) {
  const int t = beta >> 7, r = beta & 127;
  return (int64_t)t * 128 * kl + (int64_t)(((r >> 3) * (kl >> 3) + (ll >> 3)) * 64 + (r & 7) * 8 + (ll & 7));
}
__device__ __forceinline__ int64_t fwd_index(int beta, int ll, int Lb) {
  const int u = ll >> 7, rr = ll & 127;
  return (int64_t)u * 128 * Lb + (int64_t)(((rr >> 3) * (Lb >> 3) + (beta >> 3)) * 64 + (rr & 7) * 8 + (beta & 7));
}

struct BuildArgs {
  RecTables T;
  int L, Lb, Mc, mlo, nact;
  const int* nvals;
  const int64_t* off;   // [Mc * nact]
  const int* kl;        // [Mc * nact]
  uint16_t *inv_hi, *inv_lo, *fwd_hi, *fwd_lo;
};

// One block per (m, n), one thread per beta row (Lb threads): the float64 recursion writes
// 2^8 d^l_mn(beta) into both packed tables (zeros outside the transform).
template <bool SPLIT>
__global__ void k_tc_build(BuildArgs a) {
  __shared__ double cA[1024], cKn[1024], cKs[1024], cC[1024];
  const int mi = blockIdx.x, ni = blockIdx.y, beta = threadIdx.x;
  const int tile = mi * a.nact + ni;
  const int kl = a.kl[tile];
  if (kl == 0) return;
  const int m = a.mlo + mi, n = a.nvals[ni];
  const int l0 = max(abs(m), abs(n)), l0a = l0 & ~15, L = a.L;
  const int64_t off = a.off[tile];
  for (int l = l0 + threadIdx.x; l < L; l += blockDim.x) rec_coeffs(l, m, n, cA[l], cKn[l], cKs[l], cC[l]);
  __syncthreads();
  double v = 0.0, vp = 0.0;
  int q = 0;
  const bool live = beta < L;
  double wb = 0.0;
  const double* cK = cKn;
  if (live) {
    wigner_seed(a.T, beta, l0, m, n, v, q);
    wb = a.T.wpole[beta];
    cK = (2 * (2 * beta + 1) < a.T.n) ? cKn : cKs;
  }
  for (int ll = 0; ll < kl; ++ll) {
    const int l = l0a + ll;
    double x = 0.0;
    if (live && l >= l0 && l < L) {
      x = (q == 0) ? kDScale * v : 0.0;
      const double c = fma(cA[l], wb, cK[l]);
      const double vn = fma(c, v, -cC[l] * vp);
      vp = v;
      v = vn;
      if (q > 0 && fabs(v) > kRescaleAt) {
        v *= kRescaleBy;
        vp *= kRescaleBy;
        --q;
      }
    }
    put16<SPLIT, true>(a.inv_hi + off, a.inv_lo + off, inv_index(beta, ll, kl), x);
    put16<SPLIT, true>(a.fwd_hi + off, a.fwd_lo + off, fwd_index(beta, ll, a.Lb), x);
  }
}

// Quadrature matrices M^par (rows beta, K = beta'), scaled by sM, packed per 128-row tile.
template <bool SPLIT>
__global__ void k_tc_build_quad(const double* MT, int L, int Lb, double sM, uint16_t* hi, uint16_t* lo) {
  const int par = blockIdx.y, beta = blockIdx.x;
  for (int bp = threadIdx.x; bp < Lb; bp += blockDim.x) {
    const double x = (beta < L && bp < L) ? sM * MT[(size_t)par * L * L + (size_t)bp * L + beta] : 0.0;
    const int t = beta >> 7, r = beta & 127;
    const int64_t i = (int64_t)par * Lb * Lb + (int64_t)t * 128 * Lb +
                      (((r >> 3) * (Lb >> 3) + (bp >> 3)) * 64 + (r & 7) * 8 + (bp & 7));
    put16<SPLIT, true>(hi, lo, i, x);
  }
}

constexpr int kTcThreads = 128;
constexpr int kTcN = 32;               // MMA N: 16 maps x (re, im)
constexpr uint32_t kWaitIter = 1u << 26;

// 2^(14 - ceil(log2 mx)): scales a block whose largest magnitude is mx below 2^14.
__device__ __forceinline__ double pow2_scale(double mx) {
  if (!(mx > 0.0)) return 1.0;
  int e;
  frexp(mx, &e);
  return ldexp(1.0, 14 - e);
}

__device__ double block_max(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  const int w = threadIdx.x >> 5;
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[w] = v;
  __syncthreads();
  double r = red[0];
  for (int i = 1; i < (int)(blockDim.x >> 5); ++i) r = fmax(r, red[i]);
  return r;
}

// element (row, k) of a K-major packed operand with K extent K
__device__ __forceinline__ int pk(int row, int k, int K) {
  return ((row >> 3) * (K >> 3) + (k >> 3)) * 64 + (row & 7) * 8 + (k & 7);
}

// data operands are always pairs (fp16 in split mode, bf16 in bf16 mode)
template <bool SPLIT>
__device__ __forceinline__ void put_s(uint16_t* hi, uint16_t* lo, int i, float x) {
  if (SPLIT) {
    const __half h = __float2half_rn(x);
    hi[i] = __half_as_ushort(h);
    lo[i] = __half_as_ushort(__float2half_rn(x - __half2float(h)));
  } else {
    const __nv_bfloat16 h = __float2bfloat16_rn(x);
    hi[i] = __bfloat16_as_ushort(h);
    lo[i] = __bfloat16_as_ushort(__float2bfloat16_rn(x - __bfloat162float(h)));
  }
}

// acc = A[128 x K] B[N x K]^T with B a pair (hi, lo) and A a pair (a_pair) or a single value:
// per K step Ahi*Bhi + Ahi*Blo (+ Alo*Bhi)
__device__ __forceinline__ void issue_mmas(uint32_t tmem, const uint16_t* Ahi, const uint16_t* Alo,
                                           const uint16_t* Bhi, const uint16_t* Blo, int K, uint32_t idesc,
                                           bool a_pair) {
  const uint32_t sbo = (uint32_t)(K >> 3) * 128u;
  const uint32_t ah = tc::smem_u32(Ahi), al = tc::smem_u32(Alo), bh = tc::smem_u32(Bhi), bl = tc::smem_u32(Blo);
  for (int s = 0; s < (K >> 4); ++s) {
    const uint32_t o = (uint32_t)s * 256u;
    tc::mma_f16(tmem, tc::make_sdesc(ah + o, 128, sbo), tc::make_sdesc(bh + o, 128, sbo), idesc, s > 0);
    tc::mma_f16(tmem, tc::make_sdesc(ah + o, 128, sbo), tc::make_sdesc(bl + o, 128, sbo), idesc, 1);
    if (a_pair) tc::mma_f16(tmem, tc::make_sdesc(al + o, 128, sbo), tc::make_sdesc(bh + o, 128, sbo), idesc, 1);
  }
}

struct TcInvArgs {
  const uint16_t *A_hi, *A_lo;   // inverse table
  const int64_t* off;
  const int* kl;
  const double2* coef;
  int64_t s_b, s_n, s_l;
  int mlo_in;
  const double2* mult;           // [L][nact]
  const int* nvals;
  int nact;
  double2* G;                    // [B][nact][L][Mc]
  int B, L, Lb, Mc, mlo, klmax;
  int* err;
};

// G[b][n][beta][m] = sum_l d^l_mn(beta) * coef(b, n, l, m) mult[l][n] for one (m, n) and one
// 128-row beta tile; maps in chunks of 16 (N = 32 columns: re, im).
template <bool SPLIT>
__global__ void __launch_bounds__(kTcThreads) k_tc_inv(TcInvArgs a) {
  extern __shared__ __align__(1024) uint8_t smem[];
  __shared__ __align__(8) uint64_t bar_ld, bar_mma;
  __shared__ uint32_t tbase;
  __shared__ double red[kTcThreads / 32];
  const int mi = blockIdx.x, ni = blockIdx.y, t = blockIdx.z;
  const int tile = mi * a.nact + ni, kl = a.kl[tile];
  const int m = a.mlo + mi, n = a.nvals[ni], L = a.L;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (kl == 0) {   // l0 >= L: this (m, n) column is zero
    for (int idx = tid; idx < a.B * 128; idx += kTcThreads) {
      const int b = idx >> 7, beta = t * 128 + (idx & 127);
      if (beta < L) a.G[(((int64_t)b * a.nact + ni) * L + beta) * a.Mc + mi] = make_double2(0.0, 0.0);
    }
    return;
  }
  const int l0 = max(abs(m), abs(n)), l0a = l0 & ~15;
  uint16_t* Ah = reinterpret_cast<uint16_t*>(smem);
  uint16_t* Al = Ah + 128 * a.klmax;
  uint16_t* Bh = Al + 128 * a.klmax;
  uint16_t* Bl = Bh + kTcN * a.klmax;   // data operand is a pair in both modes
  if (tid == 0) {
    tc::mbar_init(&bar_ld, 1);
    tc::mbar_init(&bar_mma, 1);
  }
  if (warp == 0) tc::tmem_alloc(&tbase, 32);
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = tbase;
  if (tid == 0) {
    const uint32_t bytes = 128u * kl * 2u;
    tc::mbar_expect_tx(&bar_ld, 2 * bytes);
    const int64_t src = a.off[tile] + (int64_t)t * 128 * kl;
    tc::bulk_g2s(Ah, a.A_hi + src, bytes, &bar_ld);
    tc::bulk_g2s(Al, a.A_lo + src, bytes, &bar_ld);
  }
  const uint32_t idesc = tc::make_idesc(128, kTcN, SPLIT ? 0 : 1, 0, 0);
  bool ok = true;
  for (int map0 = 0, chunk = 0; map0 < a.B && ok; map0 += kTcN / 2, ++chunk) {
    // coefficient operand F[j][l - l0a], j = 2 (map - map0) + (re, im), scaled into fp16 range
    double mx = 0.0;
    for (int idx = tid; idx < kTcN * kl; idx += kTcThreads) {
      const int j = idx / kl, ll = idx - j * kl, l = l0a + ll, bm = map0 + (j >> 1);
      if (l >= l0 && l < L && bm < a.B) {
        const double2 c = a.coef[(int64_t)bm * a.s_b + (int64_t)ni * a.s_n + (int64_t)l * a.s_l + (m - a.mlo_in)];
        const double2 u = a.mult[(int64_t)l * a.nact + ni];
        const double f = (j & 1) ? fma(c.x, u.y, c.y * u.x) : fma(c.x, u.x, -c.y * u.y);
        mx = fmax(mx, fabs(f));
      }
    }
    const double sF = pow2_scale(block_max(mx, red));
    for (int idx = tid; idx < kTcN * kl; idx += kTcThreads) {
      const int j = idx / kl, ll = idx - j * kl, l = l0a + ll, bm = map0 + (j >> 1);
      double f = 0.0;
      if (l >= l0 && l < L && bm < a.B) {
        const double2 c = a.coef[(int64_t)bm * a.s_b + (int64_t)ni * a.s_n + (int64_t)l * a.s_l + (m - a.mlo_in)];
        const double2 u = a.mult[(int64_t)l * a.nact + ni];
        f = (j & 1) ? fma(c.x, u.y, c.y * u.x) : fma(c.x, u.x, -c.y * u.y);
      }
      put_s<SPLIT>(Bh, Bl, pk(j, ll, kl), (float)(f * sF));
    }
    tc::fence_proxy_async();
    __syncthreads();
    if (tid == 0) {
      if (chunk == 0 && !tc::mbar_wait(&bar_ld, 0, kWaitIter)) {
        atomicExch(a.err, (int)S2W_ETIMEOUT);
        ok = false;
      }
      if (ok) {
        tc::fence_after_sync();
        issue_mmas(tmem, Ah, Al, Bh, Bl, kl, idesc, true);
        tc::mma_commit(&bar_mma);
      }
    }
    __syncwarp();
    if (!tc::mbar_wait(&bar_mma, chunk & 1, kWaitIter)) {
      if (tid == 0) atomicExch(a.err, (int)S2W_ETIMEOUT);
      ok = false;
    }
    ok = __syncthreads_and(ok);
    if (!ok) break;
    tc::fence_after_sync();
    float v[32];
    tc::tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16), v);
    const int beta = t * 128 + warp * 32 + lane;
    const double un = 1.0 / (sF * kDScale);
    if (beta < L) {
#pragma unroll
      for (int p = 0; p < kTcN / 2; ++p) {
        const int bm = map0 + p;
        if (bm < a.B)
          a.G[(((int64_t)bm * a.nact + ni) * L + beta) * a.Mc + mi] = make_double2(v[2 * p] * un, v[2 * p + 1] * un);
      }
    }
    tc::fence_before_sync();
    __syncthreads();   // TMEM and B are reused by the next chunk
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tmem, 32);
}

struct TcFwdArgs {
  const uint16_t *Q_hi, *Q_lo;   // quadrature tiles [2][Lb/128][128 x Lb]
  const uint16_t *E_hi, *E_lo;   // forward table
  const int64_t* off;
  const int* kl;
  const double2* G;              // [B][nact][L][Mc]
  int B, L, Lb, Mc, mlo;
  const int* nvals;
  int nact;
  const double2* mult;           // [L][nact]
  double2* out;
  int64_t s_b, s_n, s_l;
  int mlo_out;
  double inv_sM;                 // 1 / quadrature scale
  int* err;
};

// out(b, n, l, m) += mult[l][n] sum_beta d^l_mn(beta) (M^par G_mn)(beta) for one (m, n):
// GEMM 1 (quadrature, TMEM columns [32 t, 32 t + 32) per 128-row beta tile t), then GEMM 2
// against the forward table (TMEM columns from 32 Lb/128 on, per 128-row l tile).
template <bool SPLIT>
__global__ void __launch_bounds__(kTcThreads) k_tc_fwd(TcFwdArgs a) {
  extern __shared__ __align__(1024) uint8_t smem[];
  __shared__ __align__(8) uint64_t bar_ld, bar_mma;
  __shared__ uint32_t tbase;
  __shared__ double red[kTcThreads / 32];
  const int mi = blockIdx.x, ni = blockIdx.y;
  const int tile = mi * a.nact + ni, kl = a.kl[tile];
  if (kl == 0) return;
  const int m = a.mlo + mi, n = a.nvals[ni], L = a.L, Lb = a.Lb;
  const int l0 = max(abs(m), abs(n)), l0a = l0 & ~15;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int nbt = Lb >> 7, nlt = kl >> 7;
  uint16_t* Ah = reinterpret_cast<uint16_t*>(smem);
  uint16_t* Al = Ah + 128 * Lb;           // quadrature tiles are pairs in both modes
  uint16_t* B1h = Al + 128 * Lb;
  uint16_t* B1l = B1h + kTcN * Lb;
  uint16_t* B2h = B1l + kTcN * Lb;
  uint16_t* B2l = B2h + kTcN * Lb;
  if (tid == 0) {
    tc::mbar_init(&bar_ld, 1);
    tc::mbar_init(&bar_mma, 1);
  }
  if (warp == 0) tc::tmem_alloc(&tbase, 128);
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = tbase;
  const int par = (m + n) & 1;
  const uint32_t idesc = tc::make_idesc(128, kTcN, SPLIT ? 0 : 1, 0, 0);
  const uint32_t abytes = 128u * Lb * 2u;
  uint32_t ph_ld = 0, ph_mma = 0;
  bool ok = true;
  // thread 0: copy one 128-row A tile, wait, issue its MMAs, commit and wait for them
  auto run_tile = [&](const uint16_t* src_hi, const uint16_t* src_lo, const uint16_t* Bh, const uint16_t* Bl,
                      uint32_t tcol, bool a_pair) {
    if (tid != 0 || !ok) return;
    tc::mbar_expect_tx(&bar_ld, a_pair ? 2 * abytes : abytes);
    tc::bulk_g2s(Ah, src_hi, abytes, &bar_ld);
    if (a_pair) tc::bulk_g2s(Al, src_lo, abytes, &bar_ld);
    if (!tc::mbar_wait(&bar_ld, ph_ld, kWaitIter)) {
      atomicExch(a.err, (int)S2W_ETIMEOUT);
      ok = false;
      return;
    }
    ph_ld ^= 1u;
    tc::fence_after_sync();
    issue_mmas(tmem + tcol, Ah, Al, Bh, Bl, Lb, idesc, a_pair);
    tc::mma_commit(&bar_mma);
    if (!tc::mbar_wait(&bar_mma, ph_mma, kWaitIter)) {
      atomicExch(a.err, (int)S2W_ETIMEOUT);
      ok = false;
      return;
    }
    ph_mma ^= 1u;
  };
  for (int map0 = 0; map0 < a.B; map0 += kTcN / 2) {
    // B1[j][beta] = G (scaled, split)
    double mx = 0.0;
    for (int idx = tid; idx < kTcN * L; idx += kTcThreads) {
      const int j = idx / L, beta = idx - j * L, bm = map0 + (j >> 1);
      if (bm < a.B) {
        const double2 g = a.G[(((int64_t)bm * a.nact + ni) * L + beta) * a.Mc + mi];
        mx = fmax(mx, fabs((j & 1) ? g.y : g.x));
      }
    }
    const double sG = pow2_scale(block_max(mx, red));
    for (int idx = tid; idx < kTcN * Lb; idx += kTcThreads) {
      const int j = idx / Lb, beta = idx - j * Lb, bm = map0 + (j >> 1);
      double g = 0.0;
      if (bm < a.B && beta < L) {
        const double2 gv = a.G[(((int64_t)bm * a.nact + ni) * L + beta) * a.Mc + mi];
        g = (j & 1) ? gv.y : gv.x;
      }
      put_s<SPLIT>(B1h, B1l, pk(j, beta, Lb), (float)(g * sG));
    }
    tc::fence_proxy_async();
    __syncthreads();
    for (int bt = 0; bt < nbt; ++bt) {
      const int64_t q = ((int64_t)par * nbt + bt) * 128 * Lb;
      run_tile(a.Q_hi + q, a.Q_lo + q, B1h, B1l, 32u * bt, true);
    }
    ok = __syncthreads_and(ok);
    if (!ok) break;
    tc::fence_after_sync();
    // weighted columns M G: TMEM -> registers -> B2 (scaled, split)
    float w[2][32];
    double wm = 0.0;
    const double un1 = a.inv_sM / sG;
    for (int bt = 0; bt < nbt; ++bt) {
      tc::tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + 32u * bt, w[bt]);
#pragma unroll
      for (int j = 0; j < 32; ++j) wm = fmax(wm, fabs((double)w[bt][j] * un1));
    }
    const double sW = pow2_scale(block_max(wm, red));
    for (int bt = 0; bt < nbt; ++bt) {
      const int beta = bt * 128 + warp * 32 + lane;
#pragma unroll
      for (int j = 0; j < 32; ++j) put_s<SPLIT>(B2h, B2l, pk(j, beta, Lb), (float)((double)w[bt][j] * un1 * sW));
    }
    tc::fence_proxy_async();
    tc::fence_before_sync();
    __syncthreads();
    for (int u = 0; u < nlt; ++u) {
      const int64_t e = a.off[tile] + (int64_t)u * 128 * Lb;
      run_tile(a.E_hi + e, a.E_lo + e, B2h, B2l, 32u * (nbt + u), true);
    }
    ok = __syncthreads_and(ok);
    if (!ok) break;
    tc::fence_after_sync();
    const double un2 = 1.0 / (sW * kDScale);
    for (int u = 0; u < nlt; ++u) {
      float v[32];
      tc::tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + 32u * (nbt + u), v);
      const int l = l0a + u * 128 + warp * 32 + lane;
      if (l >= l0 && l < L) {
        const double2 mu = a.mult[(int64_t)l * a.nact + ni];
#pragma unroll
        for (int p = 0; p < kTcN / 2; ++p) {
          const int bm = map0 + p;
          if (bm >= a.B) break;
          const double re = v[2 * p] * un2, im = v[2 * p + 1] * un2;
          double2* o = a.out + (int64_t)bm * a.s_b + (int64_t)ni * a.s_n + (int64_t)l * a.s_l + (m - a.mlo_out);
          atomicAdd(&o->x, fma(re, mu.x, -im * mu.y));
          atomicAdd(&o->y, fma(re, mu.y, im * mu.x));
        }
      }
    }
    tc::fence_before_sync();
    __syncthreads();
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tmem, 128);
}

}  // namespace

size_t tc_inv_smem(bool split, int klmax) {
  (void)split;
  return (size_t)(2 * 128 + 2 * kTcN) * klmax * sizeof(uint16_t);
}
size_t tc_fwd_smem(bool split, int Lb) {
  (void)split;
  return (size_t)(2 * 128 + 4 * kTcN) * Lb * sizeof(uint16_t);
}

cudaError_t launch_tc_build(const GridTables& g, const TransformSpec& t, const TcTable& tab, int Mc, int mlo,
                            bool split, cudaStream_t st) {
  BuildArgs a;
  a.T.wpole = g.wpole;
  a.T.cpow_m = g.cpow_m;
  a.T.cpow_e = g.cpow_e;
  a.T.spow_m = g.spow_m;
  a.T.spow_e = g.spow_e;
  a.T.sqrtC = g.sqrtC;
  a.T.n = g.n;
  a.L = t.L;
  a.Lb = tab.Lb;
  a.Mc = Mc;
  a.mlo = mlo;
  a.nact = t.nact;
  a.nvals = t.nvals;
  a.off = tab.off;
  a.kl = tab.kl;
  a.inv_hi = tab.inv_hi;
  a.inv_lo = tab.inv_lo;
  a.fwd_hi = tab.fwd_hi;
  a.fwd_lo = tab.fwd_lo;
  dim3 grid(Mc, t.nact);
  if (split) k_tc_build<true><<<grid, tab.Lb, 0, st>>>(a);
  else k_tc_build<false><<<grid, tab.Lb, 0, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_tc_build_quad(const GridTables& g, bool split, cudaStream_t st) {
  dim3 grid(g.Lb, 2);
  if (split) k_tc_build_quad<true><<<grid, 256, 0, st>>>(g.MT, g.L, g.Lb, g.qscale, g.Q_hi, g.Q_lo);
  else k_tc_build_quad<false><<<grid, 256, 0, st>>>(g.MT, g.L, g.Lb, g.qscale, g.Q_hi, g.Q_lo);
  return cudaGetLastError();
}

cudaError_t launch_tc_inverse(const s2w_plan* P, const GridTables& g, const TransformSpec& t, CoefArgs in,
                              ColumnArgs out, cudaStream_t st) {
  const TcTable& tab = *t.tc;
  TcInvArgs a;
  a.A_hi = tab.inv_hi;
  a.A_lo = tab.inv_lo;
  a.off = tab.off;
  a.kl = tab.kl;
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
  a.Lb = tab.Lb;
  a.Mc = out.Mc;
  a.mlo = out.mlo;
  a.klmax = tab.klmax;
  a.err = P->err_word;
  const bool split = P->p.precision == S2W_FP32_SPLIT;
  const size_t smem = tc_inv_smem(split, tab.klmax);
  dim3 grid(out.Mc, t.nact, tab.Lb / 128);
  cudaError_t e;
  if (split) {
    e = cudaFuncSetAttribute(k_tc_inv<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_tc_inv<true><<<grid, kTcThreads, smem, st>>>(a);
  } else {
    e = cudaFuncSetAttribute(k_tc_inv<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_tc_inv<false><<<grid, kTcThreads, smem, st>>>(a);
  }
  return cudaGetLastError();
}

cudaError_t launch_tc_forward(const s2w_plan* P, const GridTables& g, const TransformSpec& t, ColumnArgs in,
                              CoefArgs out, cudaStream_t st) {
  const TcTable& tab = *t.tc;
  TcFwdArgs a;
  a.Q_hi = g.Q_hi;
  a.Q_lo = g.Q_lo;
  a.E_hi = tab.fwd_hi;
  a.E_lo = tab.fwd_lo;
  a.off = tab.off;
  a.kl = tab.kl;
  a.G = in.G;
  a.B = in.B;
  a.L = in.L;
  a.Lb = tab.Lb;
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
  a.inv_sM = 1.0 / g.qscale;
  a.err = P->err_word;
  const bool split = P->p.precision == S2W_FP32_SPLIT;
  const size_t smem = tc_fwd_smem(split, tab.Lb);
  dim3 grid(in.Mc, t.nact);
  cudaError_t e;
  if (split) {
    e = cudaFuncSetAttribute(k_tc_fwd<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_tc_fwd<true><<<grid, kTcThreads, smem, st>>>(a);
  } else {
    e = cudaFuncSetAttribute(k_tc_fwd<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_tc_fwd<false><<<grid, kTcThreads, smem, st>>>(a);
  }
  return cudaGetLastError();
}

}  // namespace s2w

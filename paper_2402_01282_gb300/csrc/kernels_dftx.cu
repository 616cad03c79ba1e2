// Azimuthal (alpha/phi) DFTs of the float64-accurate tensor-core mode (S2W_FP64_TC) on the
// 5th-generation tensor cores, by the same exact integer slicing as the l-contractions
// (slice7.cuh; Ozaki, Ogita, Oishi and Rump, Numer. Algorithms 59, 2012).
//
// Every DFT length here is odd, n = 2L - 1, h = L - 1.  The symmetric form of an odd-length
// DFT (Sec. 5.2, Eq. 48 evaluated on the MW azimuthal samples) pairs index p with n - p:
//   a_p = x_p + x_{n-p},  b_p = x_p - x_{n-p}  (1 <= p <= h),   a_0 = x_0,  b_0 = 0,
//   C_k = sum_{p=0..h} a_p cos(2 pi p k/n),   S_k = sum_{p=0..h} b_p sin(2 pi p k/n),
//   X(k) = C_k + SIGN i S_k,   X(n-k) = C_k - SIGN i S_k   (0 <= k <= h),
// so the whole transform is two real GEMMs with M = K = L (frequencies k x index pairs p),
// shared by every ring, map and carried n: the columns.  Both GEMMs run exactly on bf16
// tensor cores with float32 accumulators in TMEM: the twiddle tables (plan time) and the
// folded data (every call) are cut into seven balanced base-128 digits of a 47-bit fixed-point
// value, and the 28 digit-pair products with i + i' <= 6 (34 with i + i' = 7 where the plan asks
// for it) are summed exactly (K <= 512).
//
// Per call and direction, two kernels:
//   k_dftx_fwd_prep / k_dftx_inv_prep (one block per ring and map): the gamma DFT on the map side
//     (forward only, compensated float32 as in kernels_dft_c32.cu: one complex alpha transform
//     per carried n >= 0 for real maps), the fold a, b in the integer domain, the column
//     exponents and the seven slices of every column;
//   k_dftx_gemm (one CTA per 128 frequencies and 32 columns): the cos GEMM, then the sin GEMM,
//     through a three-stage bulk-copy pipeline into seven (eight) 128 x 32 TMEM accumulators; the
//     epilogue forms X(k), X(n-k) and writes the columns G (forward) or, after the gamma
//     synthesis over the carried n (inverse), the pixels.
// Columns: ring (map b, ring t) and job q (a carried n, with its -n partner for real maps) give
// the complex column pair (re, im); cpr = 2 nj rounded up to a power of two columns per ring,
// 32 / cpr rings per CTA, so the inverse epilogue holds every job of its rings.
#include <math.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <vector>

#include "comp32.cuh"
#include "dft_c32.cuh"
#include "s2w_internal.h"
#include "slice7.cuh"
#include "tc_sm100.cuh"

namespace s2w {
namespace {

constexpr int kXT = 256;                  // GEMM threads (8 warps: 2 per TMEM lane quarter)
constexpr int kXN = 32;                   // columns per CTA (MMA N)
constexpr int kXKc = 16;                  // K chunk (one MMA deep)
constexpr int kXATile = 128 * kXKc;       // elements of one table slice chunk
constexpr int kXBTile = kXN * kXKc;       // elements of one data slice chunk
constexpr int kXAChunk = kSl * kXATile;   // 14336
constexpr int kXBChunk = kSl * kXBTile;   // 3584
constexpr int kXStage = kXAChunk + kXBChunk;
constexpr int kXStages = 3;
constexpr size_t kXSmem = (size_t)kXStages * kXStage * sizeof(uint16_t);   // 107520 B
constexpr uint32_t kXWait = 1u << 20;     // bounded mbarrier polls
constexpr int kXTmem = 256;               // 8 accumulators x 32 columns
constexpr int kXMaxJobs = 16;             // jobs per ring (cpr <= 32)
static_assert((size_t)kXN / 2 * 2 * 128 * sizeof(float4) <= kXSmem, "inverse epilogue staging");


struct XArgs {
  // prep
  const void* pix_in;
  int64_t pix_sb;
  const double2* Gin;
  // gemm outputs
  double2* Gout;
  void* pix_out;
  // geometry
  const int* nvals;
  int nact, Ng, n, L, nr, B, Mc, mlo;
  const float4* gph;        // [nact][Ng] exp(+i n gamma_g) as pairs
  int Kp, nkc, Mt;          // reduction extent (L rounded up to 16), its chunks, row tiles
  int cpr, rpg, ngroups;    // columns per ring, rings per CTA, CTAs along the columns
  int g0;                   // first column group of this launch
  uint16_t* ops;            // data slices: [group][a|b][chunk][slice][512]
  int* fexp;                // [B * nr][16] column exponents
  const uint16_t *tcos, *tsin;
  int e_tw;                 // table row exponent
  uint32_t idesc;
  int* err;
  int ndiag;   // digit-pair diagonals summed: 7 (28 pairs per K step) or 8 (34)
};

// 8 consecutive values (index pairs p0 .. p0+7) of one column -> one 16-byte core-matrix row per
// slice of chunk p0/16 of column j of CTA group g, operand ab (0: a, 1: b)
__device__ __forceinline__ void store_slices(const XArgs& a, int g, int ab, int j, int p0, const long long (&X)[8]) {
  uint32_t w[kSl][4];
#pragma unroll
  for (int u = 0; u < 8; u += 2) {
    uint32_t d0[kSl], d1[kSl];
    digits7(X[u], d0);
    digits7(X[u + 1], d1);
#pragma unroll
    for (int s = 0; s < kSl; ++s) w[s][u / 2] = __byte_perm(d0[s], d1[s], 0x7632);
  }
  const int64_t o = ((int64_t)(g * 2 + ab) * a.nkc + (p0 >> 4)) * kXBChunk + ((p0 & 15) >> 3) * 64 + (j >> 3) * 128 +
                    (j & 7) * 8;
#pragma unroll
  for (int s = 0; s < kSl; ++s)
    *reinterpret_cast<uint4*>(a.ops + o + (int64_t)s * kXBTile) = make_uint4(w[s][0], w[s][1], w[s][2], w[s][3]);
}

// ------------------------------------------------------------------ forward: pixels -> slices
// Block (ring t, map b).  H_q(alpha) = sum_g W(alpha, gamma_g) exp(-i n_q gamma_g) for every job
// q, then the fold of H_q over alpha and its slices; one exponent per (ring, job).
template <bool REAL>
__global__ void k_dftx_fwd_prep(XArgs a) {
  extern __shared__ float4 HZ[];   // [nj][n]
  __shared__ int jn[kMaxJobs], jp[kMaxJobs], njs;
  __shared__ int emax[kXMaxJobs];
  const int n = a.n, t = blockIdx.x, b = blockIdx.y;
  if (threadIdx.x == 0) {
    int nj;
    make_jobs(a.nvals, a.nact, REAL, jn, jp, nj);
    njs = nj;
  }
  if (threadIdx.x < kXMaxJobs) emax[threadIdx.x] = 0;
  __syncthreads();
  const int nj = njs;
  const int Ng = a.Ng, hg = (Ng - 1) / 2;
  const int64_t ring = (int64_t)a.nr * n;
  const int64_t base = (int64_t)b * a.pix_sb + (int64_t)t * n;
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
        const float4 u = cadd<false>(xp, xm, 1.f), v = cadd<false>(xp, xm, -1.f);
#pragma unroll
        for (int q = 0; q < kJobChunk; ++q) {
          if (q < jc) {
            const float4 ph = a.gph[jn[j0 + q] * Ng + g];   // cos, sin of n gamma_g
            racc<false>(hr[q], u.x, u.y, ph.x, ph.y);        // u cos - i v sin
            racc<false>(hi[q], v.x, v.y, -ph.z, -ph.w);
            if (!REAL) {
              racc<false>(hr[q], v.z, v.w, ph.z, ph.w);
              racc<false>(hi[q], u.z, u.w, ph.x, ph.y);
            }
          }
        }
      }
#pragma unroll
      for (int q = 0; q < kJobChunk; ++q)
        if (q < jc) {
          const float4 z = pack<false>(hr[q], hi[q]);
          HZ[(j0 + q) * n + al] = z;
          const int e = max(fbound(z.x), fbound(z.z));
          if (e > 0) atomicMax(&emax[j0 + q], e);
          // a NaN or Inf sample (exponent field all ones) would be sliced as a finite integer
          if ((__float_as_uint(z.x) & 0x7F800000u) == 0x7F800000u || (__float_as_uint(z.z) & 0x7F800000u) == 0x7F800000u)
            atomicCAS(a.err, 0, (int)S2W_ENONFINITE);
        }
    }
  }
  __syncthreads();
  const int hc = a.cpr / 2, h = (n - 1) / 2;
  const int rf = b * a.nr + t, g = rf / a.rpg, r = rf % a.rpg;
  if (threadIdx.x < hc)   // the fold doubles the bound
    a.fexp[(int64_t)rf * kXMaxJobs + threadIdx.x] =
        (threadIdx.x < nj && emax[threadIdx.x] > 0) ? e_from(emax[threadIdx.x]) + 1 : 0;
  // items (component c, job q, group of 8 index pairs, operand ab), c and q fastest: the 2 hc
  // columns of this ring and the two k halves of a chunk form 2 x cpr 16-byte rows that are
  // contiguous in each slice, so consecutive threads store whole sectors
  const int npg = a.Kp / 8, nit = hc * 4 * npg;
  for (int it = threadIdx.x; it < nit; it += blockDim.x) {
    const int c = it & 1, q = (it >> 1) % hc, rest = (it >> 1) / hc, pg = rest % npg, ab = rest / npg;
    const bool live = q < nj && emax[q] > 0;   // emax = 0: an all-zero column (f may be any integer)
    const int f = live ? e_from(emax[q]) + 1 : 0;
    long long X[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int p = pg * 8 + u;
      X[u] = 0;
      if (!live || p > h) continue;
      const float4 z1 = HZ[q * n + p];
      const float h1 = c ? z1.z : z1.x, l1 = c ? z1.w : z1.y;
      const long long x1 = fixf(h1, f) + fixf(l1, f);
      if (p == 0) {
        X[u] = ab ? 0 : x1;
        continue;
      }
      const float4 z2 = HZ[q * n + n - p];
      const float h2 = c ? z2.z : z2.x, l2 = c ? z2.w : z2.y;
      const long long x2 = fixf(h2, f) + fixf(l2, f);
      X[u] = ab ? x1 - x2 : x1 + x2;
    }
    store_slices(a, g, ab, r * a.cpr + 2 * q + c, pg * 8, X);
  }
}

// ------------------------------------------------------------------ inverse: columns -> slices
// Block (ring t, map b).  x_m = G_{m, n} over the full m range of every job (m < 0 from the -n
// partner for real maps: G_{m,n} = conj G_{-m,-n}), folded and sliced with one exponent per ring.
template <bool REAL>
__global__ void k_dftx_inv_prep(XArgs a) {
  extern __shared__ double2 Gs[];   // [nact][Mc]
  __shared__ int jn[kMaxJobs], jp[kMaxJobs], njs;
  __shared__ int emax;
  const int t = blockIdx.x, b = blockIdx.y, Mc = a.Mc;
  if (threadIdx.x == 0) {
    int nj;
    make_jobs(a.nvals, a.nact, REAL, jn, jp, nj);
    njs = nj;
    emax = 0;
  }
  __syncthreads();
  const int nj = njs;
  int e = 0;
  bool bad = false;
  for (int i = threadIdx.x; i < a.nact * Mc; i += blockDim.x) {
    const int ni = i / Mc, mi = i - ni * Mc;
    const double2 v = a.Gin[(((int64_t)b * a.nact + ni) * a.nr + t) * Mc + mi];
    Gs[i] = v;
    e = max(e, max(ebound(v.x), ebound(v.y)));
    bad |= (bexp(v.x) == 0x7FF) | (bexp(v.y) == 0x7FF);   // NaN or Inf: sliced as a finite integer otherwise
  }
  if (bad) atomicCAS(a.err, 0, (int)S2W_ENONFINITE);
  if (e > 0) atomicMax(&emax, e);
  __syncthreads();
  const int f = emax > 0 ? e_from(emax) + 1 : 0;   // the fold doubles the bound
  const int hc = a.cpr / 2, h = (a.n - 1) / 2;
  const int rf = b * a.nr + t, g = rf / a.rpg, r = rf % a.rpg;
  if (threadIdx.x < hc) a.fexp[(int64_t)rf * kXMaxJobs + threadIdx.x] = f;
  const int npg = a.Kp / 8, nit = hc * 4 * npg;
  for (int it = threadIdx.x; it < nit; it += blockDim.x) {   // c, q fastest (see k_dftx_fwd_prep)
    const int c = it & 1, q = (it >> 1) % hc, rest = (it >> 1) / hc, pg = rest % npg, ab = rest / npg;
    long long X[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int p = pg * 8 + u;
      X[u] = 0;
      if (q >= nj || p > h || emax == 0) continue;   // emax = 0: an all-zero ring
      const double2* Gn = Gs + jn[q] * Mc;
      if (REAL) {
        // x_p = Gn[p], x_{n-p} = conj Gp[p] (Gp = Gn for the n = 0 job)
        const double2* Gp = Gs + (jp[q] >= 0 ? jp[q] : jn[q]) * Mc;
        const double2 u1 = Gn[p];
        if (p == 0) {
          X[u] = ab ? 0 : fix47(c ? u1.y : u1.x, f);
          continue;
        }
        const double2 u2 = Gp[p];
        const long long x1 = fix47(c ? u1.y : u1.x, f), x2 = fix47(c ? u2.y : u2.x, f);
        // a: (re1 + re2, im1 - im2), b: (re1 - re2, im1 + im2)
        X[u] = (ab ^ c) ? x1 - x2 : x1 + x2;
      } else {
        const double2 u1 = Gn[p - a.mlo];
        if (p == 0) {
          X[u] = ab ? 0 : fix47(c ? u1.y : u1.x, f);
          continue;
        }
        const double2 u2 = Gn[-p - a.mlo];
        const long long x1 = fix47(c ? u1.y : u1.x, f), x2 = fix47(c ? u2.y : u2.x, f);
        X[u] = ab ? x1 - x2 : x1 + x2;
      }
    }
    store_slices(a, g, ab, r * a.cpr + 2 * q + c, pg * 8, X);
  }
}

// ------------------------------------------------------------------ GEMM + epilogue
// float pair (s, c) -> float64 times 2^k, integer operations and one float64 add
__device__ __forceinline__ double pair_to_double(float s, float c, int k) {
  return scale2(f2d(s), k) + scale2(f2d(c), k);
}

// Combine C +- i S for the pair (xr, xi) of C and (yr, yi) of S: (xr - sg yi, xi + sg yr)
__device__ __forceinline__ void combine(const Acc& xr, const Acc& xi, const Acc& yr, const Acc& yi, float sg,
                                        float2& re, float2& im) {
  re = add_pair(xr.s, xr.c, -sg * yi.s, -sg * yi.c);
  im = add_pair(xi.s, xi.c, sg * yr.s, sg * yr.c);
}

template <bool FWD, bool REAL>
__global__ void __launch_bounds__(kXT) k_dftx_gemm(XArgs a) {
  extern __shared__ __align__(1024) uint8_t smem[];
  __shared__ __align__(8) uint64_t bar_ld[kXStages], bar_mma[kXStages];
  __shared__ uint32_t tbase;
  __shared__ int jn[kMaxJobs], jp[kMaxJobs], njs;
  __shared__ int fx[kXN / 2];
  // the row tiles of one column group are neighbours in the grid, so the second reads the
  // group's data slices from L2
  const int kt = blockIdx.x, g = a.g0 + blockIdx.y;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  // warp w reads TMEM lanes 32 (w % 4) .. (its lane quarter) and columns 16 (w / 4) .. of every
  // accumulator: rows (frequencies) 32 (w % 4) + lane, column pairs 8 (w / 4) .. 8 (w / 4) + 7
  const int quarter = warp & 3, half = warp >> 2;
  const int hc = a.cpr / 2, nkc = a.nkc, rings = a.B * a.nr;
  // every CTA walks the K chunks from its own starting point (the integer sums are exact in
  // any order), so concurrent CTAs do not all fetch the same twiddle chunk at once
  const int rot = g % nkc;
  if (tid == 0) {
    int nj;
    make_jobs(a.nvals, a.nact, REAL, jn, jp, nj);
    njs = nj;
    for (int s = 0; s < kXStages; ++s) {
      tc::mbar_init(&bar_ld[s], 1);
      tc::mbar_init(&bar_mma[s], 1);
    }
    tc::fence_mbar_init();
  }
  __syncwarp();
  if (warp == 0) tc::tmem_alloc(&tbase, kXTmem);
  if (tid < kXN / 2) {
    const int r = tid / hc, q = tid % hc, rf = g * a.rpg + r;
    fx[tid] = rf < rings ? a.fexp[(int64_t)rf * kXMaxJobs + q] : 0;
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = tbase;
  const int nj = njs;
  uint16_t* const stage0 = reinterpret_cast<uint16_t*>(smem);
  constexpr uint32_t stage_bytes = (uint32_t)kXStage * 2u;
  uint32_t ph_ld[kXStages] = {0u, 0u, 0u}, ph_mma[kXStages] = {0u, 0u, 0u};
  unsigned pend_ld = 0u, pend_mma = 0u;   // thread 0: stages with copies / MMAs not yet waited for
  bool ok = true;

  // Thread 0 drives both GEMMs (phase 0: cos table x a slices, phase 1: sin table x b slices) as
  // one sequence of 2 nkc chunks over the three stages (chunk gc = phase nkc + c uses stage gc % 3).
  auto load = [&](int phase, int c, int s) {
    const uint16_t* A = (phase ? a.tsin : a.tcos) + (int64_t)kt * nkc * kXAChunk;
    const uint16_t* Bq = a.ops + (int64_t)(g * 2 + phase) * nkc * kXBChunk;
    uint16_t* S = stage0 + s * kXStage;
    const int cc = c + rot < nkc ? c + rot : c + rot - nkc;
    tc::mbar_expect_tx(&bar_ld[s], stage_bytes);
    tc::bulk_g2s(S, A + (int64_t)cc * kXAChunk, kXAChunk * 2u, &bar_ld[s]);
    tc::bulk_g2s(S + kXAChunk, Bq + (int64_t)cc * kXBChunk, kXBChunk * 2u, &bar_ld[s]);
    pend_ld |= 1u << s;
  };
  auto wait_ld = [&](int s) {
    if (!ok) return;
    if (!tc::mbar_wait(&bar_ld[s], ph_ld[s], kXWait)) {
      atomicExch(a.err, (int)S2W_ETIMEOUT);
      ok = false;
      return;
    }
    ph_ld[s] ^= 1u;
    pend_ld &= ~(1u << s);
  };
  auto wait_mma = [&](int s) {
    if (!ok) return;
    if (!tc::mbar_wait(&bar_mma[s], ph_mma[s], kXWait)) {
      atomicExch(a.err, (int)S2W_ETIMEOUT);
      ok = false;
      return;
    }
    ph_mma[s] ^= 1u;
    pend_mma &= ~(1u << s);
  };
  auto prologue = [&](int phase) {   // the first two chunks of a phase (their stages are free)
    for (int c = 0; c < kXStages - 1 && c < nkc; ++c) load(phase, c, (phase * nkc + c) % kXStages);
  };
  auto run = [&](int phase) {
    for (int c = 0; c < nkc && ok; ++c) {
      const int s = (phase * nkc + c) % kXStages;
      wait_ld(s);
      if (!ok) break;
      tc::fence_after_sync();
      const uint32_t A0 = tc::smem_u32(stage0 + s * kXStage), B0 = A0 + kXAChunk * 2u;
      // the slice operands of a stage differ only in their start address: descriptors by offset
      // (address field = byte address / 16)
      const uint64_t dA = tc::make_sdesc(A0, 128, 256), dB = tc::make_sdesc(B0, 128, 256);
      const uint32_t acc0 = c > 0 ? 1u : 0u;
      // one MMA per twiddle slice sa against the data slices 0 .. 6 - sa side by side (contiguous
      // 32-row blocks: one N = 32 (7 - sa) operand), pair (sa, sb) into accumulator sa + sb at
      // TMEM columns 32 (sa + sb); diagonal 7 as in kernels_tcx.cu (pair (1, 6) first, alone)
      const bool d7 = a.ndiag > kSl;   // uniform
#pragma unroll
      for (int sa = 0; sa < kSl; ++sa) {
        const uint64_t dAs = dA + (uint64_t)(sa * (kXATile * 2 / 16));
        if (d7 && sa == 1)
          tc::mma_f16(tmem + (uint32_t)(32 * kSl), dAs, dB + (uint64_t)((kSl - 1) * (kXBTile * 2 / 16)),
                      tc::make_idesc(128, kXN, 1, 0, 0), acc0);
        const int nb = kSl - sa + ((d7 && sa >= 2) ? 1 : 0);
        tc::mma_f16(tmem + (uint32_t)(32 * sa), dAs, dB, tc::make_idesc(128, kXN * nb, 1, 0, 0), sa > 0 ? 1u : acc0);
      }
      tc::mma_commit(&bar_mma[s]);
      pend_mma |= 1u << s;
      if (c + kXStages - 1 < nkc) {
        // the stage of chunk c + 2 last held chunk c - 1 (waited for here) or, for c = 0, a chunk
        // of the previous phase (waited for at its end)
        const int sn = (phase * nkc + c + kXStages - 1) % kXStages;
        if (c >= 1) wait_mma(sn);
        if (!ok) break;
        load(phase, c + kXStages - 1, sn);
      }
    }
    // the MMAs of this phase still outstanding: chunks max(0, nkc - 3) .. nkc - 1
    for (int c = nkc > kXStages ? nkc - kXStages : 0; c < nkc && ok; ++c) wait_mma((phase * nkc + c) % kXStages);
  };
  auto settle = [&]() {   // after a timeout: let this CTA's own copies and MMAs in flight land (bounded)
    for (int s = 0; s < kXStages; ++s) {
      if (pend_ld & (1u << s)) tc::mbar_wait(&bar_ld[s], ph_ld[s], kXWait);
      if (pend_mma & (1u << s)) tc::mbar_wait(&bar_mma[s], ph_mma[s], kXWait);
    }
  };
  // TMEM -> this thread's 16 compensated column values: sum_q 2^(-7 q) D_q, smallest weight first
  auto drain = [&](Acc (&acc)[kXN / 2]) {
#pragma unroll
    for (int j = 0; j < kXN / 2; ++j) acc[j] = Acc{0.f, 0.f};
    for (int qq = a.ndiag - 1; qq >= 0; --qq) {
      float v[16];
      tc::tmem_ld16(tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(32 * qq + 16 * half), v);
      const float w = __uint_as_float((uint32_t)(127 - 7 * qq) << 23);   // 2^(-7 qq)
#pragma unroll
      for (int j = 0; j < kXN / 2; ++j) two_sum_add(acc[j], v[j] * w);
    }
  };

  Acc C[kXN / 2], S[kXN / 2];
  if (tid == 0) {
    prologue(0);
    run(0);
    if (ok) prologue(1);   // the sin GEMM's first copies overlap the drain of the cos GEMM
  }
  ok = __syncthreads_and(ok);
  if (ok) {
    tc::fence_after_sync();
    drain(C);
    tc::fence_before_sync();
  }
  __syncthreads();   // every TMEM read is done before the sin GEMM overwrites the accumulators
  if (ok && tid == 0) {
    tc::fence_after_sync();
    run(1);
  }
  if (!ok && tid == 0) settle();
  ok = __syncthreads_and(ok);
  if (ok) {
    tc::fence_after_sync();
    drain(S);
  }
  const int n = a.n, h = (n - 1) / 2;
  const int row = quarter * 32 + lane, k = kt * 128 + row;
  const float sg = FWD ? -1.f : 1.f;
  if (ok && FWD && k <= h) {
#pragma unroll
    for (int ii = 0; ii < kXN / 4; ++ii) {
      const int i = half * (kXN / 4) + ii;   // column pair
      const int r = i / hc, q = i % hc, rf = g * a.rpg + r;
      if (rf >= rings || q >= nj) continue;
      const int bb = rf / a.nr, t = rf - bb * a.nr;
      const int ke = a.e_tw + fx[i] - 10;
      float2 re1, im1, re2, im2;
      combine(C[2 * ii], C[2 * ii + 1], S[2 * ii], S[2 * ii + 1], sg, re1, im1);    // X(k)
      combine(C[2 * ii], C[2 * ii + 1], S[2 * ii], S[2 * ii + 1], -sg, re2, im2);   // X(n - k)
      const double2 xk = make_double2(pair_to_double(re1.x, re1.y, ke), pair_to_double(im1.x, im1.y, ke));
      const double2 xm = make_double2(pair_to_double(re2.x, re2.y, ke), pair_to_double(im2.x, im2.y, ke));
      double2* Gn = a.Gout + (((int64_t)bb * a.nact + jn[q]) * a.nr + t) * a.Mc;
      if (REAL) {
        Gn[k] = xk;                                           // G_{m=k, n}
        if (jp[q] >= 0) {                                     // G_{k, -n} = conj X(n - k)
          double2* Gp = a.Gout + (((int64_t)bb * a.nact + jp[q]) * a.nr + t) * a.Mc;
          Gp[k] = make_double2(xm.x, -xm.y);
        }
      } else {
        Gn[k - a.mlo] = xk;
        if (k > 0) Gn[-k - a.mlo] = xm;
      }
    }
  }
  if (!FWD) {
    // Z_q(alpha) for alpha = k (slot 0) and n - k (slot 1) of every column pair, in the ring's
    // common scale, to shared memory (the stages are idle now): Zs[i][slot][row]; then the
    // phases exp(+i n_q gamma_g) of the jobs after them when they fit
    float4* Zs = reinterpret_cast<float4*>(smem);
    float4* Ph = Zs + (kXN / 2) * 2 * 128;
    const int Ng = a.Ng;
    const bool ph_smem = nj * Ng * sizeof(float4) + (size_t)(kXN / 2) * 2 * 128 * sizeof(float4) <= kXSmem;
    if (ok) {
#pragma unroll
      for (int ii = 0; ii < kXN / 4; ++ii) {
        const int i = half * (kXN / 4) + ii;
        float2 re1, im1, re2, im2;
        combine(C[2 * ii], C[2 * ii + 1], S[2 * ii], S[2 * ii + 1], sg, re1, im1);
        combine(C[2 * ii], C[2 * ii + 1], S[2 * ii], S[2 * ii + 1], -sg, re2, im2);
        Zs[(i * 2 + 0) * 128 + row] = make_float4(re1.x, re1.y, im1.x, im1.y);
        Zs[(i * 2 + 1) * 128 + row] = make_float4(re2.x, re2.y, im2.x, im2.y);
      }
      if (ph_smem)
        for (int e = tid; e < nj * Ng; e += kXT) Ph[e] = a.gph[jn[e / Ng] * Ng + e % Ng];
    }
    ok = __syncthreads_and(ok);
    if (ok) {
      // W(alpha, gamma_g) = sum_q Z_q(alpha) exp(+i n_q gamma_g); gamma_g and gamma_{Ng-g} share
      // P = sum_q Z_q cos, Q = sum_q Z_q sin.  Real maps: the n, -n pair contributes 2 Re, n = 0 Re.
      const int hg = (Ng - 1) / 2;
      const int64_t ringlen = (int64_t)a.nr * n;
      for (int it = tid; it < a.rpg * 2 * 128; it += kXT) {
        const int rw = it & 127, slot = (it >> 7) & 1, r = it >> 8;
        const int kk = kt * 128 + rw, rf = g * a.rpg + r;
        if (kk > h || rf >= rings || (slot == 1 && kk == 0)) continue;
        const int al = slot ? n - kk : kk;
        const int bb = rf / a.nr, t = rf - bb * a.nr;
        const int ke = a.e_tw + fx[r * hc] - 10;   // one exponent per ring
        const int64_t base = (int64_t)bb * a.pix_sb + (int64_t)t * n + al;
        for (int gg = 0; gg <= hg; ++gg) {
          Acc pr{0.f, 0.f}, pim{0.f, 0.f}, qr{0.f, 0.f}, qim{0.f, 0.f};
          for (int q = 0; q < nj; ++q) {
            float4 z = Zs[((r * hc + q) * 2 + slot) * 128 + rw];
            if (REAL && jp[q] >= 0) z = make_float4(2.f * z.x, 2.f * z.y, 2.f * z.z, 2.f * z.w);
            const float4 ph = ph_smem ? Ph[q * Ng + gg] : a.gph[jn[q] * Ng + gg];
            racc<false>(pr, z.x, z.y, ph.x, ph.y);
            if (gg > 0) racc<false>(qim, z.z, z.w, ph.z, ph.w);
            if (!REAL) {
              racc<false>(pim, z.z, z.w, ph.x, ph.y);
              if (gg > 0) racc<false>(qr, z.x, z.y, ph.z, ph.w);
            }
          }
          if (REAL) {
            double* out = (double*)a.pix_out;
            const Acc w0 = comb<false>(pr, -1.f, qim), w1 = comb<false>(pr, 1.f, qim);   // P - Q, P + Q
            out[base + gg * ringlen] = pair_to_double(w0.s, w0.c, ke);
            if (gg > 0) out[base + (Ng - gg) * ringlen] = pair_to_double(w1.s, w1.c, ke);
          } else {
            double2* out = (double2*)a.pix_out;   // P + i Q and P - i Q
            const Acc r0 = comb<false>(pr, -1.f, qim), i0 = comb<false>(pim, 1.f, qr);
            out[base + gg * ringlen] = make_double2(pair_to_double(r0.s, r0.c, ke), pair_to_double(i0.s, i0.c, ke));
            if (gg > 0) {
              const Acc r1 = comb<false>(pr, 1.f, qim), i1 = comb<false>(pim, -1.f, qr);
              out[base + (Ng - gg) * ringlen] =
                  make_double2(pair_to_double(r1.s, r1.c, ke), pair_to_double(i1.s, i1.c, ke));
            }
          }
        }
      }
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tmem, kXTmem);
}

int jobs_of(const TransformSpec& t, bool real) {
  int nj = 0;
  for (int v : t.nvals_h)
    if (!real || v >= 0) ++nj;
  return nj;
}

int cols_per_ring(int nj) {
  int c = 2;
  while (c < 2 * nj) c *= 2;
  return c;
}

XArgs make_xargs(const s2w_plan* P, const GridTables& g, const TransformSpec& t, const DftxTable& tab, ColumnArgs c,
                 bool real) {
  XArgs a{};
  a.nvals = t.nvals;
  a.nact = t.nact;
  a.Ng = 2 * t.N - 1;
  a.n = g.n;
  a.L = c.L;
  a.nr = c.nr;
  a.B = c.B;
  a.Mc = c.Mc;
  a.mlo = c.mlo;
  a.gph = t.gphase4;
  a.Kp = tab.Kp;
  a.nkc = tab.Kp / kXKc;
  a.Mt = tab.Mt;
  a.cpr = cols_per_ring(jobs_of(t, real));
  a.rpg = kXN / a.cpr;
  a.ngroups = (c.B * c.nr + a.rpg - 1) / a.rpg;
  a.ops = P->dftx_ops;
  a.fexp = P->dftx_fexp;
  a.tcos = tab.cos;
  a.tsin = tab.sin;
  a.e_tw = tab.e;
  a.idesc = tc::make_idesc(128, kXN, 1, 0, 0);   // bf16 slices
  a.err = P->err_word;
  a.ndiag = P->slice_diag7 ? kDiag : kDiag - 1;
  return a;
}

template <class K>
cudaError_t launch_x(K kern, dim3 grid, int threads, size_t smem, cudaStream_t st, const XArgs& a) {
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  kern<<<grid, threads, smem, st>>>(a);
  return cudaGetLastError();
}

// grid (row tiles, column groups), in launches of at most 65535 groups
template <class K>
cudaError_t launch_gemm(K kern, cudaStream_t st, XArgs a) {
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kXSmem);
  if (e != cudaSuccess) return e;
  for (int g0 = 0; g0 < a.ngroups; g0 += 65535) {
    a.g0 = g0;
    kern<<<dim3(a.Mt, std::min(65535, a.ngroups - g0)), kXT, kXSmem, st>>>(a);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

int host_core16(int r, int k) { return ((r >> 3) * 2 + (k >> 3)) * 64 + (r & 7) * 8 + (k & 7); }

}  // namespace

bool dftx_shape_ok(const TransformSpec& t, bool real) {
  const int nj = jobs_of(t, real);
  if (nj < 1 || nj > kXMaxJobs || t.L > 512) return false;
  if (real)   // every carried n != 0 needs its partner -n
    for (int v : t.nvals_h)
      if (v != 0 && std::find(t.nvals_h.begin(), t.nvals_h.end(), -v) == t.nvals_h.end()) return false;
  const size_t n = 2 * (size_t)t.L - 1, Mc = real ? t.L : n, lim = 200 * 1024;
  return (size_t)nj * n * sizeof(float4) <= lim && (size_t)t.nact * Mc * sizeof(double2) <= lim;
}

int64_t dftx_ops_elems(const TransformSpec& t, bool real, int B, int nr) {
  const int cpr = cols_per_ring(jobs_of(t, real)), rpg = kXN / cpr;
  const int64_t ng = ((int64_t)B * nr + rpg - 1) / rpg;
  const int nkc = ((t.L + kXKc - 1) / kXKc);
  return ng * 2 * nkc * kXBChunk;
}

int64_t dftx_fexp_elems(int B, int nr) { return (int64_t)B * nr * kXMaxJobs; }

// Sliced twiddle tables for length n = 2L - 1 with every entry times `scale`.
void build_dftx_table(int L, double scale, DftxTable* tab, std::vector<uint16_t>& hcos, std::vector<uint16_t>& hsin) {
  const int n = 2 * L - 1, h = L - 1;
  tab->L = L;
  tab->scale = scale;
  tab->Kp = ((L + kXKc - 1) / kXKc) * kXKc;
  tab->Mt = (L + 127) / 128;
  tab->e = std::ilogb(scale) + 1;   // |scale cos|, |scale sin| <= scale < 2^e
  const int nkc = tab->Kp / kXKc;
  const size_t elems = (size_t)tab->Mt * nkc * kXAChunk;
  hcos.assign(elems, 0);
  hsin.assign(elems, 0);
  const double w = 2.0 * 3.14159265358979323846 / n;
  for (int k = 0; k < tab->Mt * 128; ++k)
    for (int p = 0; p < tab->Kp; ++p) {
      double vc = 0.0, vs = 0.0;
      if (k <= h && p <= h) {
        const int e = (int)(((long long)p * k) % n);
        vc = scale * std::cos(w * e);
        vs = scale * std::sin(w * e);
      }
      uint16_t dc[kSl], ds[kSl];
      host_digits(vc, tab->e, dc);
      host_digits(vs, tab->e, ds);
      const size_t o = ((size_t)((k >> 7) * nkc + (p >> 4)) * kSl) * kXATile + host_core16(k & 127, p & 15);
      for (int s = 0; s < kSl; ++s) {
        hcos[o + (size_t)s * kXATile] = dc[s];
        hsin[o + (size_t)s * kXATile] = ds[s];
      }
    }
}

cudaError_t launch_dftx_forward(const s2w_plan* P, const GridTables& g, const TransformSpec& t, const void* pix,
                                int64_t pix_sb, bool real, ColumnArgs c, cudaStream_t st) {
  XArgs a = make_xargs(P, g, t, *t.dftx_fwd, c, real);
  a.pix_in = pix;
  a.pix_sb = pix_sb;
  a.Gout = c.G;
  const int nj = jobs_of(t, real);
  const size_t psm = (size_t)nj * g.n * sizeof(float4);
  const dim3 pg(c.nr, c.B);
  const int th = t.dft_threads_fwd;
  cudaError_t e = real ? launch_x(k_dftx_fwd_prep<true>, pg, th, psm, st, a)
                       : launch_x(k_dftx_fwd_prep<false>, pg, th, psm, st, a);
  if (e != cudaSuccess) return e;
  return real ? launch_gemm(k_dftx_gemm<true, true>, st, a) : launch_gemm(k_dftx_gemm<true, false>, st, a);
}

cudaError_t launch_dftx_inverse(const s2w_plan* P, const GridTables& g, const TransformSpec& t, ColumnArgs c,
                                void* pix, int64_t pix_sb, bool real, cudaStream_t st) {
  XArgs a = make_xargs(P, g, t, *t.dftx_inv, c, real);
  a.Gin = c.G;
  a.pix_out = pix;
  a.pix_sb = pix_sb;
  const size_t psm = (size_t)t.nact * c.Mc * sizeof(double2);
  const dim3 pg(c.nr, c.B);
  const int th = t.dft_threads_inv;
  cudaError_t e = real ? launch_x(k_dftx_inv_prep<true>, pg, th, psm, st, a)
                       : launch_x(k_dftx_inv_prep<false>, pg, th, psm, st, a);
  if (e != cudaSuccess) return e;
  return real ? launch_gemm(k_dftx_gemm<false, true>, st, a) : launch_gemm(k_dftx_gemm<false, false>, st, a);
}

}  // namespace s2w

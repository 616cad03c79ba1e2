// Azimuthal (alpha/phi) DFTs of the float64-accurate tensor-core mode (S2W_FP64_TC) by the
// prime-factor (Good-Thomas) split of the odd length n = 2L - 1 = n1 n2 (gcd(n1, n2) = 1, e.g.
// 511 = 7 x 73, 255 = 5 x 51): the n2-point stage an exact sliced GEMM on the tcgen05 tensor cores
// (seven bf16 digits per value, slice7.cuh; Ozaki, Ogita, Oishi and Rump, Numer. Algorithms 59,
// 2012), the n1-point stage in compensated float32 straight from the accumulators.  (Sec. 5.2,
// Eq. 48: the D-matrix factorisation leaves a 2-D DFT over (alpha, gamma); gamma is taken on the
// map side.)
//
// Prime-factor split (no twiddle factors between the stages): with the input index map
// p = (n2 p1 + n1 p2) mod n and the output index map k = (k1 e1 + k2 e2) mod n (e1 = n2 (n2^-1
// mod n1), e2 = n1 (n1^-1 mod n2), so k = k1 mod n1 and k = k2 mod n2),
//   X(k) = sum_p1 w_n1^(S p1 k1) [ sum_p2 w_n2^(S p2 k2) x(p) ],   w_m = exp(2 pi i/m), S = -+1.
// The inner n2-point DFT of every column (ring, job, p1, re|im) is one GEMM against a table of
// n2 + 1 rows: row 2j holds s cos(2 pi p2 j/n2), row 2j + 1 holds s sin(2 pi p2 j/n2), j <= (n2-1)/2
// (s = the transform's normalisation), so the accumulator rows 2j and 2j + 1 of a column are C_j
// and S_j; lane 2j forms Y(j) and lane 2j + 1 forms Y(n2 - j) after exchanging their rows with a
// shuffle, then each lane takes the n1-point DFT over p1 of its Y values: n1 outputs per lane.
//
// Exactness of the GEMM: the table (scale s < 2^e_tw) and the data (one exponent f per ring,
// max |x| < 2^f) are rounded to 47-bit fixed point and cut into seven balanced base-128 digits;
// the 28 digit pairs with i + i' = q <= 6 of a K step (10 MMAs: one per table slice and group of
// up to four data slices side by side) go to accumulator q (seven 128 x 64 float32 accumulators
// in TMEM), whose partial sums are integers below 2^24 (K <= 128), so every accumulator is exact
// (plans that also sum the diagonal i + i' = 7 use the direct form);
// C = 2^(e_tw + f - 10) sum_q 2^(-7q) D_q, summed smallest weight first in compensated float32.
//
// GEMM columns come in passes of 64: slots of W = 2 n1 rounded up to a power of two columns
// (one ring and job each: p1 < n1, re|im), S = 64/W slots, rpp = S/nj rings per pass.  Per call:
//   forward  k_dftp_fwd_prep (block per ring): the gamma DFT on the map side (compensated, as in
//            kernels_dft_c32.cu), the ring exponent and the slices of the ring's columns, in pass
//            order; k_dftp_tc (persistent): bulk copies of each pass's slices through a stage
//            pipeline, the MMAs, and 8 TMEM warps draining the accumulators, taking the n1-point
//            DFT and writing the columns G through shared memory (coalesced);
//   inverse  k_dftp_inv_prep (block per ring): the ring's columns, exponent and slices;
//            k_dftp_tc: as above, writing Z_q(alpha) (unscaled pairs) through shared memory;
//            k_dftp_synth (block per ring): the gamma synthesis of Z to the pixels.
// The SIMT stages run at full occupancy in the per-ring kernels; the persistent kernel keeps the
// table resident in shared memory and streams only the data slices.
#include <math.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <type_traits>
#include <vector>

#include "comp32.cuh"
#include "dft_c32.cuh"
#include "s2w_internal.h"
#include "slice7.cuh"
#include "tc_sm100.cuh"

namespace s2w {
namespace {

constexpr int kPN = 64;                 // GEMM columns per pass (MMA N)
constexpr int kPBTile = kPN * 16;       // elements of one data slice chunk (64 x 16)
constexpr int kPChunk = kSl * kPBTile;  // elements of one K chunk of a pass (7 slices)
constexpr int kPStages = 4;             // bulk-copy stages of the persistent kernel
constexpr int kPTmemWarps = 16;         // warps 0-15 of the persistent kernel (lane quarter w % 4, chunk w / 4)
constexpr int kPT = (kPTmemWarps + 1) * 32;   // + the issuing warp
constexpr uint32_t kPWait = 1u << 20;   // bounded mbarrier polls
constexpr int kPMaxRpp = 32;            // rings per pass (n1 = 1: 32 slots of 2 columns)
constexpr int kPMaxSmem = 200 * 1024;   // dynamic shared memory limit used for the plan choice
constexpr int kPMaxNg = 15;             // gamma samples 2N - 1 (N <= 8)

template <int N1>
struct SlotShape {
  static constexpr int W = N1 == 1 ? 2 : (N1 == 3 ? 8 : 16);   // columns per slot
  static constexpr int SPC = 16 / W;                             // slots per 16-column chunk
};

struct PArgs {
  const void* pix_in;
  void* pix_out;
  int64_t pix_sb;
  const double2* Gin;
  double2* Gout;
  const int* nvals;
  int nact, Ng, n, n1, n2, R, Rs, nkc, nr, B, Mc, mlo;
  int e1, e2, W, rpp, npass;
  const float4* gph;        // [nact][Ng] exp(+i n gamma_g) as pairs
  const uint16_t* tab;      // sliced n2-point table, [chunk][slice][Rs x 16 core-matrix layout]
  int e_tw;
  float4 tw1[8];            // cos, sin (2 pi m/n1) as pairs (hi, lo, hi, lo), m < n1
  uint32_t idesc;
  uint16_t* ops;            // data slices in pass order: [pass][chunk][slice][64 x 16]
  int* fexp;                // [rings] ring exponents (0: an all-zero ring)
  float4* zbuf;             // inverse: [rings][job][n] Z_q(alpha), unscaled pairs
  int* err;
};

// n1-point DFT X(k) = sum_p Y(p) w^(SIGN p k), w = exp(2 pi i/N1), of compensated complex values
// in the symmetric odd-length form (index pairs p, N1 - p).  Y, X as (re, im) Acc pairs.
template <int N1, int SIGN>
__device__ __forceinline__ void dft_small(const Acc (&yr)[N1], const Acc (&yi)[N1], const float4* tw, Acc (&xr)[N1],
                                          Acc (&xi)[N1]) {
  if (N1 == 1) {
    xr[0] = yr[0];
    xi[0] = yi[0];
    return;
  }
  constexpr int H = (N1 - 1) / 2;
  float2 ar[H + 1], ai[H + 1], br[H + 1], bi[H + 1];   // index 1..H used
#pragma unroll
  for (int p = 1; p <= H; ++p) {
    ar[p] = add_pair(yr[p].s, yr[p].c, yr[N1 - p].s, yr[N1 - p].c);
    ai[p] = add_pair(yi[p].s, yi[p].c, yi[N1 - p].s, yi[N1 - p].c);
    br[p] = add_pair(yr[p].s, yr[p].c, -yr[N1 - p].s, -yr[N1 - p].c);
    bi[p] = add_pair(yi[p].s, yi[p].c, -yi[N1 - p].s, -yi[N1 - p].c);
  }
  Acc s0r = yr[0], s0i = yi[0];
#pragma unroll
  for (int p = 1; p <= H; ++p) {
    s0r = comb<false>(s0r, 1.f, Acc{ar[p].x, ar[p].y});
    s0i = comb<false>(s0i, 1.f, Acc{ai[p].x, ai[p].y});
  }
  xr[0] = s0r;
  xi[0] = s0i;
#pragma unroll
  for (int k = 1; k <= H; ++k) {
    Acc cr = yr[0], ci = yi[0], sr{0.f, 0.f}, si{0.f, 0.f};
#pragma unroll
    for (int p = 1; p <= H; ++p) {
      const float4 w = tw[(p * k) % N1];
      racc<false>(cr, ar[p].x, ar[p].y, w.x, w.y);
      racc<false>(ci, ai[p].x, ai[p].y, w.x, w.y);
      racc<false>(sr, br[p].x, br[p].y, w.z, w.w);
      racc<false>(si, bi[p].x, bi[p].y, w.z, w.w);
    }
    // X(k) = C + SIGN i S, X(N1 - k) = C - SIGN i S, i S = (-S_im, S_re)
    const float sg = (float)SIGN;
    xr[k] = comb<false>(cr, -sg, si);
    xi[k] = comb<false>(ci, sg, sr);
    xr[N1 - k] = comb<false>(cr, sg, si);
    xi[N1 - k] = comb<false>(ci, -sg, sr);
  }
}



// float pair (s, c) -> float64 times 2^k
__device__ __forceinline__ double pair_dbl(const Acc& a, int k) { return scale2(f2d(a.s), k) + scale2(f2d(a.c), k); }

// 8 consecutive reduction indices of one column as seven 16-byte core-matrix rows, pass order
__device__ __forceinline__ void store_pass_slices(const PArgs& a, int pass, int col, int kg, const long long (&X)[8]) {
  uint32_t w[kSl][4];
#pragma unroll
  for (int u = 0; u < 8; u += 2) {
    uint32_t d0[kSl], d1[kSl];
    digits7(X[u], d0);
    digits7(X[u + 1], d1);
#pragma unroll
    for (int s = 0; s < kSl; ++s) w[s][u / 2] = __byte_perm(d0[s], d1[s], 0x7632);
  }
  const int64_t o = ((int64_t)pass * a.nkc + (kg >> 1)) * kPChunk + ((col >> 3) * 2 + (kg & 1)) * 64 + (col & 7) * 8;
#pragma unroll
  for (int s = 0; s < kSl; ++s)
    *reinterpret_cast<uint4*>(a.ops + o + (int64_t)s * kPBTile) = make_uint4(w[s][0], w[s][1], w[s][2], w[s][3]);
}

// ------------------------------------------------------------------ forward prologue
// Block (ring t, map b).  H_q(alpha) = sum_g W(alpha, gamma_g) exp(-i n_q gamma_g) for every job q,
// the ring exponent, then the slices of the ring's columns (job q, p1, re|im) over p2.
// (64 registers for real maps: four 256-thread blocks per SM instead of three; the complex
// variant keeps its 128)
template <bool REAL>
__global__ void __launch_bounds__(512, REAL ? 2 : 1) k_dftp_fwd_prep(PArgs a) {
  extern __shared__ float4 HZ[];   // [nj][n]
  __shared__ int jn[kMaxJobs], jp[kMaxJobs], njs, emax;
  const int n = a.n, t = blockIdx.x, b = blockIdx.y;
  if (threadIdx.x == 0) {
    int nj;
    make_jobs(a.nvals, a.nact, REAL, jn, jp, nj);
    njs = nj;
    emax = 0;
  }
  __syncthreads();
  const int nj = njs;
  const int Ng = a.Ng, hg = (Ng - 1) / 2;
  const int64_t ring = (int64_t)a.nr * n;
  const int64_t base = (int64_t)b * a.pix_sb + (int64_t)t * n;
  int e = 0;
  bool bad = false;
  constexpr int HG = (kPMaxNg - 1) / 2;
  using Raw = typename std::conditional<REAL, double, double2>::type;
  const Raw* pin = static_cast<const Raw*>(a.pix_in);
  auto to_pair = [](Raw v) -> float4 {
    if constexpr (REAL) {
      const float2 r = split1_bits(v);
      return make_float4(r.x, r.y, 0.f, 0.f);
    } else {
      const float2 r = split1_bits(v.x), i = split1_bits(v.y);
      return make_float4(r.x, r.y, i.x, i.y);
    }
  };
  for (int al = threadIdx.x; al < n; al += blockDim.x) {
    // every sample of this alpha in flight before the arithmetic
    Raw rp[HG], rm[HG];
    const Raw r0 = pin[base + al];
#pragma unroll
    for (int g = 1; g <= HG; ++g)
      if (g <= hg) {
        rp[g - 1] = pin[base + g * ring + al];
        rm[g - 1] = pin[base + (Ng - g) * ring + al];
      }
    const float4 w0 = to_pair(r0);
    Acc hr[kJobChunk], hi[kJobChunk];
#pragma unroll
    for (int q = 0; q < kJobChunk; ++q) {
      hr[q] = Acc{w0.x, w0.y};
      hi[q] = Acc{w0.z, w0.w};
    }
#pragma unroll
    for (int g = 1; g <= HG; ++g) {
      if (g > hg) break;
      const float4 xp = to_pair(rp[g - 1]), xm = to_pair(rm[g - 1]);
      const float4 u = cadd<false>(xp, xm, 1.f), v = cadd<false>(xp, xm, -1.f);
#pragma unroll
      for (int q = 0; q < kJobChunk; ++q) {
        if (q < nj) {
          const float4 ph = a.gph[jn[q] * Ng + g];   // cos, sin of n gamma_g
          racc<false>(hr[q], u.x, u.y, ph.x, ph.y);   // u cos - i v sin
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
      if (q < nj) {
        const float4 z = pack<false>(hr[q], hi[q]);
        HZ[q * n + al] = z;
        e = max(e, max(fbound(z.x), fbound(z.z)));
        bad |= ((__float_as_uint(z.x) & 0x7F800000u) == 0x7F800000u) |
               ((__float_as_uint(z.z) & 0x7F800000u) == 0x7F800000u);
      }
  }
  if (bad) atomicCAS(a.err, 0, (int)S2W_ENONFINITE);   // a NaN or Inf would be sliced as a finite integer
  if (e > 0) atomicMax(&emax, e);
  __syncthreads();
  const int f = emax > 0 ? e_from(emax) : 0;
  const int rf = b * a.nr + t, pass = rf / a.rpp, rip = rf - pass * a.rpp;
  if (threadIdx.x == 0) a.fexp[rf] = f;
  // items (column of this ring's slots, group of 8 indices p2); consecutive threads take
  // consecutive columns, so a warp stores whole 128-byte runs
  const int W = a.W, cols = nj * W, nit = cols * 2 * a.nkc;
  for (int it = threadIdx.x; it < nit; it += blockDim.x) {
    const int cl = it % cols, kg = it / cols;
    const int q = cl / W, p1 = (cl % W) >> 1, c = cl & 1;
    const int col = (rip * nj + q) * W + (cl % W);
    long long X[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int p2 = kg * 8 + u;
      X[u] = 0;
      if (p1 >= a.n1 || p2 >= a.n2) continue;
      const int pp = a.n2 * p1 + a.n1 * p2, p = pp >= n ? pp - n : pp;
      const float4 z = HZ[q * n + p];
      X[u] = c ? fixf_pair(z.z, z.w, f) : fixf_pair(z.x, z.y, f);
    }
    store_pass_slices(a, pass, col, kg, X);
  }
}

// ------------------------------------------------------------------ inverse prologue
// Block (ring t, map b).  x_q(m) = G_{m, n_q} over the full m range of every job (m < 0 from the
// -n partner for real maps: G_{m,n} = conj G_{-m,-n}), the ring exponent, the slices.
template <bool REAL>
__global__ void k_dftp_inv_prep(PArgs a) {
  extern __shared__ double2 Gs[];   // [nact][Mc]
  __shared__ int jn[kMaxJobs], jp[kMaxJobs], njs, emax;
  const int t = blockIdx.x, b = blockIdx.y, Mc = a.Mc, n = a.n, h = (n - 1) / 2;
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
  // the ring's columns: nact contiguous runs of Mc values; four loads in flight per thread
  const int total = a.nact * Mc;
  for (int i0 = threadIdx.x; i0 < total; i0 += 4 * blockDim.x) {
    double2 v[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int i = i0 + u * blockDim.x;
      if (i < total) {
        const int ni = i / Mc, mi = i - ni * Mc;
        v[u] = a.Gin[(((int64_t)b * a.nact + ni) * a.nr + t) * Mc + mi];
      }
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int i = i0 + u * blockDim.x;
      if (i < total) {
        Gs[i] = v[u];
        e = max(e, max(ebound(v[u].x), ebound(v[u].y)));
        bad |= (bexp(v[u].x) == 0x7FF) | (bexp(v[u].y) == 0x7FF);
      }
    }
  }
  if (bad) atomicCAS(a.err, 0, (int)S2W_ENONFINITE);
  if (e > 0) atomicMax(&emax, e);
  __syncthreads();
  const int f = emax > 0 ? e_from(emax) : 0;
  const int rf = b * a.nr + t, pass = rf / a.rpp, rip = rf - pass * a.rpp;
  if (threadIdx.x == 0) a.fexp[rf] = f;
  const int W = a.W, cols = nj * W, nit = cols * 2 * a.nkc;
  for (int it = threadIdx.x; it < nit; it += blockDim.x) {
    const int cl = it % cols, kg = it / cols;
    const int q = cl / W, p1 = (cl % W) >> 1, c = cl & 1;
    const int col = (rip * nj + q) * W + (cl % W);
    long long X[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int p2 = kg * 8 + u;
      X[u] = 0;
      if (p1 >= a.n1 || p2 >= a.n2 || emax == 0) continue;
      const int pp = a.n2 * p1 + a.n1 * p2, p = pp >= n ? pp - n : pp;
      double2 v;
      if (REAL) {
        if (p <= h) {
          v = Gs[jn[q] * Mc + p];
        } else {   // x_p = conj G_{n-p, -n} (the job's own column for the n = 0 job)
          v = Gs[(jp[q] >= 0 ? jp[q] : jn[q]) * Mc + (n - p)];
          v.y = -v.y;
        }
      } else {
        v = Gs[jn[q] * Mc + ((p <= h ? p : p - n) - a.mlo)];
      }
      X[u] = fix47(c ? v.y : v.x, f);
    }
    store_pass_slices(a, pass, col, kg, X);
  }
}

// ------------------------------------------------------------------ persistent tensor-core kernel
// One CTA per SM over the passes; warp 16 (one thread) streams each pass's slices through
// kPStages bulk-copy stages and issues the MMAs; warps 0-15 drain the accumulators (warp w: TMEM
// lane quarter w % 4, 16-column chunk w / 4), take the n1-point DFT and stage the outputs in
// shared memory, then write them out coalesced (forward: the columns G; inverse: Z).
template <bool FWD, bool REAL, int N1>
__global__ void __launch_bounds__(kPT, 1) k_dftp_tc(PArgs a) {
  using SS = SlotShape<N1>;
  extern __shared__ __align__(1024) uint8_t smem[];
  __shared__ __align__(8) uint64_t full[kPStages], freeb[kPStages], acc_full, acc_empty;
  __shared__ uint32_t tbase;
  __shared__ int jn[kMaxJobs], jp[kMaxJobs], njs;
  __shared__ volatile int s_abort;   // the issuer or a TMEM warp: a wait ran out
  __shared__ int t_abort;            // the TMEM warps' common decision
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int abytes = a.nkc * kSl * a.Rs * 32;
  const int boff = (abytes + 1023) & ~1023;
  const int n = a.n, h = (n - 1) / 2, rings = a.B * a.nr, rpp = a.rpp, Mc = a.Mc;
  uint16_t* const As = reinterpret_cast<uint16_t*>(smem);
  uint16_t* const Bs = reinterpret_cast<uint16_t*>(smem + boff);
  // output staging of one pass: forward double2 columns, inverse float4 pairs, [slot][n]
  uint8_t* const OUT = smem + boff + (size_t)kPStages * kPChunk * 2;
  if (tid == 0) {
    int nj;
    make_jobs(a.nvals, a.nact, REAL, jn, jp, nj);
    njs = nj;
    for (int s = 0; s < kPStages; ++s) {
      tc::mbar_init(&full[s], 1);
      tc::mbar_init(&freeb[s], 1);
    }
    tc::mbar_init(&acc_full, 1);
    tc::mbar_init(&acc_empty, kPTmemWarps);
    s_abort = 0;
    t_abort = 0;
    tc::fence_mbar_init();
  }
  // the sliced table, resident for the whole kernel (plain 16-byte loads)
  for (int i = tid; i < abytes / 16; i += kPT)
    reinterpret_cast<uint4*>(As)[i] = reinterpret_cast<const uint4*>(a.tab)[i];
  if (warp == kPTmemWarps) tc::tmem_alloc(&tbase, 512);
  tc::fence_proxy_async();   // generic-proxy writes of the table, read by the MMAs
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = tbase;
  const int nj = njs;
  const int G = gridDim.x, my = (a.npass - (int)blockIdx.x + G - 1) / G;   // passes of this CTA
  auto on_timeout = [&]() {
    atomicExch(a.err, (int)S2W_ETIMEOUT);
    s_abort = 1;
  };

  if (warp == kPTmemWarps) {
    // ------------------------------------------------------------ bulk copies and MMAs
    if (lane == 0) {
      const uint32_t A0 = tc::smem_u32(As);
      const uint32_t atile = (uint32_t)a.Rs * 32u, btile = (uint32_t)kPBTile * 2u;
      const int nkc = a.nkc, T = my * nkc;   // chunks of this CTA, in order
      // chunk gc uses stage gc % kPStages for the (gc / kPStages)-th time: phase parity of both
      // barriers of the stage.  Copies issued for chunks < loaded, their arrival waited for chunks
      // < seen; MMAs committed for chunks < mma, their completion waited for chunks < done.
      int loaded = 0, seen = 0, mma = 0, done = 0;
      bool ok = true;
      auto par = [](int gc) { return (uint32_t)((gc / kPStages) & 1); };
      auto load = [&](int gc) {
        const int i = gc / nkc, c = gc - i * nkc, s = gc % kPStages;
        tc::mbar_expect_tx(&full[s], (uint32_t)kPChunk * 2u);
        tc::bulk_g2s(Bs + s * kPChunk, a.ops + ((int64_t)((int)blockIdx.x + i * G) * nkc + c) * kPChunk,
                     (uint32_t)kPChunk * 2u, &full[s]);
        loaded = gc + 1;
      };
      auto wait = [&](uint64_t* bar, uint32_t parity) {
        if (!ok) return;
        if (s_abort || !tc::mbar_wait(bar, parity, kPWait)) {
          if (!s_abort) on_timeout();
          ok = false;
        }
      };
      for (int gc = 0; gc < kPStages - 1 && gc < T; ++gc) load(gc);
      for (int gc = 0; gc < T && ok; ++gc) {
        const int i = gc / nkc, c = gc - i * nkc, s = gc % kPStages;
        wait(&full[s], par(gc));
        if (!ok) break;
        seen = gc + 1;
        if (c == 0 && i > 0) wait(&acc_empty, (uint32_t)((i - 1) & 1));   // pass i-1 drained
        if (!ok) break;
        tc::fence_after_sync();
        const uint32_t ab = A0 + (uint32_t)(c * kSl) * atile, bb = tc::smem_u32(Bs + s * kPChunk);
        // one MMA per table slice sa and group of at most four data slices side by side (the 64-row
        // slices are contiguous with one row-group stride: N = 64 x group size <= 256); pair
        // (sa, sb) lands in accumulator sa + sb at TMEM columns 64 (sa + sb): 10 MMAs per K chunk
        // for the 28 pairs, each table slice read once or twice
#pragma unroll
        for (int sa = 0; sa < kSl; ++sa)
#pragma unroll
          for (int g0 = 0; g0 < kSl - sa; g0 += 4) {
            const int gn = (kSl - sa - g0) < 4 ? (kSl - sa - g0) : 4;
            tc::mma_f16(tmem + (uint32_t)(64 * (sa + g0)), tc::make_sdesc(ab + (uint32_t)sa * atile, 128, 256),
                        tc::make_sdesc(bb + (uint32_t)g0 * btile, 128, 256), tc::make_idesc(128, kPN * gn, 1, 0, 0),
                        (c > 0 || sa > 0) ? 1u : 0u);
          }
        tc::mma_commit(&freeb[s]);
        mma = gc + 1;
        if (c == nkc - 1) tc::mma_commit(&acc_full);
        // the stage of chunk gc + kPStages - 1 last held chunk gc - 1: its MMAs must be done
        const int gn = gc + kPStages - 1;
        if (gn < T) {
          if (gc >= 1) {
            wait(&freeb[(gc - 1) % kPStages], par(gc - 1));
            if (!ok) break;
            done = gc;
          }
          load(gn);
        }
      }
      if (!ok) {
        // after an abort: let this CTA's own copies and MMAs in flight land (bounded waits on the
        // exact phases still pending) before TMEM is freed
        for (int gc = seen; gc < loaded; ++gc) tc::mbar_wait(&full[gc % kPStages], par(gc), kPWait);
        if (mma > done) tc::mbar_wait(&freeb[(mma - 1) % kPStages], par(mma - 1), kPWait);
      }
    }
  } else {
    // ------------------------------------------------------------ TMEM warps
    const int quarter = warp & 3, chunk = warp >> 2;
    const int row = 32 * quarter + lane, j = row >> 1, sd = row & 1;
    const bool warp_live = 32 * quarter < a.R;
    const bool live = row < a.R && !(j == 0 && sd == 1);   // rows that produce an output
    const int k2 = sd == 0 ? j : a.n2 - j;
    // Y_re = C_re - sg S_im, Y_im = C_im + sg S_re: sg = SIGN on a cos row (frequency j), -SIGN on a
    // sin row (its partner computes the mirrored frequency n2 - j)
    const float sg = (FWD ? -1.f : 1.f) * (sd == 0 ? 1.f : -1.f);
    // output index k = (k1 e1 + k2 e2) mod n = ka[k1] + kb, less n once if it reaches n
    const int kb = (int)(((int64_t)k2 * a.e2) % n);
    int ka[N1];
#pragma unroll
    for (int k1 = 0; k1 < N1; ++k1) ka[k1] = (int)(((int64_t)k1 * a.e1) % n);
    // one thread polls (a plain bounded try-wait: nothing else polls, so it need not back off);
    // the named barrier after it releases the other TMEM warps
    auto poll_wait = [&](uint64_t* bar, uint32_t parity) -> bool {
      if (s_abort) return false;
      if (!tc::mbar_wait(bar, parity, kPWait)) {
        on_timeout();
        return false;
      }
      return true;
    };
    // the seven accumulators of one 16-column chunk, smallest weight first: two halves of 8
    // columns, each with its 7 loads in flight before one wait
    auto drain = [&](int chunk, Acc (&acc)[16]) {
#pragma unroll
      for (int hf = 0; hf < 2; ++hf) {
        uint32_t r[kSl][8];
#pragma unroll
        for (int qq = 0; qq < kSl; ++qq)
          tc::tmem_ld8_nowait(tmem + ((uint32_t)(32 * quarter) << 16) + (uint32_t)(64 * qq + 16 * chunk + 8 * hf),
                              r[qq]);
        tc::tmem_wait_ld();
#pragma unroll
        for (int qq = 0; qq < kSl; ++qq) tc::tmem_regs_ready(r[qq]);
#pragma unroll
        for (int u = 0; u < 8; ++u) acc[8 * hf + u] = Acc{0.f, 0.f};
#pragma unroll
        for (int qq = kSl - 1; qq >= 0; --qq) {
          const float wq = __uint_as_float((uint32_t)(127 - 7 * qq) << 23);   // 2^(-7 qq)
#pragma unroll
          for (int u = 0; u < 8; ++u) two_sum_add(acc[8 * hf + u], __uint_as_float(r[qq][u]) * wq);
        }
      }
    };
    // row exchange, n1-point DFT and staged outputs of the slots of one 16-column chunk
    auto stage_b = [&](int gp, int chunk, const Acc (&acc)[16]) {
#pragma unroll
      for (int u = 0; u < SS::SPC; ++u) {
        const int sl = chunk * SS::SPC + u;
        if (sl >= rpp * nj) continue;   // warp-uniform
        const int rip = sl / nj, rf = gp * rpp + rip;
        Acc yr[N1], yi[N1];
#pragma unroll
        for (int p1 = 0; p1 < N1; ++p1) {
          const Acc own_r = acc[u * SS::W + 2 * p1], own_i = acc[u * SS::W + 2 * p1 + 1];
          Acc oth_r, oth_i;
          oth_r.s = __shfl_xor_sync(0xFFFFFFFFu, own_r.s, 1);
          oth_r.c = __shfl_xor_sync(0xFFFFFFFFu, own_r.c, 1);
          oth_i.s = __shfl_xor_sync(0xFFFFFFFFu, own_i.s, 1);
          oth_i.c = __shfl_xor_sync(0xFFFFFFFFu, own_i.c, 1);
          const Acc Cr = sd == 0 ? own_r : oth_r, Ci = sd == 0 ? own_i : oth_i;
          const Acc Sr = sd == 0 ? oth_r : own_r, Si = sd == 0 ? oth_i : own_i;
          yr[p1] = comb<false>(Cr, -sg, Si);
          yi[p1] = comb<false>(Ci, sg, Sr);
        }
        if (rf >= rings || !live) continue;
        Acc xr[N1], xi[N1];
        dft_small<N1, FWD ? -1 : 1>(yr, yi, a.tw1, xr, xi);
        if (FWD) {
          const int ke = a.e_tw + a.fexp[rf] - 10;
          double2* const o = reinterpret_cast<double2*>(OUT) + (size_t)sl * (n + 1);
#pragma unroll
          for (int k1 = 0; k1 < N1; ++k1) {
            const int k = ka[k1] + kb >= n ? ka[k1] + kb - n : ka[k1] + kb;
            const double2 v = make_double2(pair_dbl(xr[k1], ke), pair_dbl(xi[k1], ke));
            if (REAL) {
              // staged as the two columns the write-out copies whole: A[m] = X(m), m <= h
              // (column n) and B[m] = conj X((n - m) mod n), m <= h (column -n), at o[0..h] and
              // o[h+1 .. 2h+1]
              if (k <= h) o[k] = v;
              if (k == 0 || k > h) o[h + 1 + (k == 0 ? 0 : n - k)] = make_double2(v.x, -v.y);
            } else {
              const int mm = k + h >= n ? k + h - n : k + h;   // m = k or k - n, stored at m + h
              o[mm] = v;
            }
          }
        } else {
          float4* const o = reinterpret_cast<float4*>(OUT) + (size_t)sl * (n + 1);
#pragma unroll
          for (int k1 = 0; k1 < N1; ++k1) {
            const int k = ka[k1] + kb >= n ? ka[k1] + kb - n : ka[k1] + kb;
            o[k] = make_float4(xr[k1].s, xr[k1].c, xi[k1].s, xi[k1].c);
          }
        }
      }
    };
    const int tt = tid;   // 0 .. 511 over the TMEM warps
    for (int i = 0; i < my; ++i) {
      const int gp = (int)blockIdx.x + i * G;
      // the TMEM warps meet at named barriers below: one abort decision for all of them, taken
      // after a barrier from flags written before it
      if (tt == 0) {
        if (!poll_wait(&acc_full, (uint32_t)(i & 1))) t_abort = 1;
        tc::bulk_wait_read0();   // the previous pass's copies have read OUT
      }
      asm volatile("bar.sync 1, %0;" ::"n"(kPTmemWarps * 32) : "memory");
      if (t_abort) break;
      tc::fence_after_sync();
      Acc acc[16];
      if (warp_live) drain(chunk, acc);
      // every accumulator value this warp needs is in registers: release TMEM to the next pass
      tc::fence_before_sync();
      __syncwarp();
      if (lane == 0) tc::mbar_arrive(&acc_empty);
      if (warp_live) stage_b(gp, chunk, acc);
      tc::fence_proxy_async();   // this thread's OUT writes before the copies' async-proxy reads
      asm volatile("bar.sync 1, %0;" ::"n"(kPTmemWarps * 32) : "memory");
      // the pass's staged outputs to global memory as bulk copies of whole columns, issued by one
      // thread while the others go on to the next pass; that pass rewrites OUT only after these
      // copies have read it (the wait at its top, before its first barrier)
      if (tt == 0) {
        for (int sl = 0; sl < rpp * nj; ++sl) {
          const int rip = sl / nj, q = sl - rip * nj, rf = gp * rpp + rip;
          if (rf >= rings) break;
          const int bb = rf / a.nr, t = rf - bb * a.nr;
          if (FWD) {
            const double2* o = reinterpret_cast<const double2*>(OUT) + (size_t)sl * (n + 1);
            double2* Gn = a.Gout + (((int64_t)bb * a.nact + jn[q]) * a.nr + t) * Mc;
            if (REAL) {
              // G_{m, n} = X(m) and G_{m, -n} = conj X((n - m) mod n), m <= h
              tc::bulk_s2g(Gn, o, (uint32_t)(h + 1) * 16u);
              if (jp[q] >= 0)
                tc::bulk_s2g(a.Gout + (((int64_t)bb * a.nact + jp[q]) * a.nr + t) * Mc, o + h + 1,
                             (uint32_t)(h + 1) * 16u);
            } else {
              tc::bulk_s2g(Gn, o, (uint32_t)n * 16u);   // m = -h .. h at m + h
            }
          } else {
            tc::bulk_s2g(a.zbuf + ((int64_t)rf * nj + q) * n,
                         reinterpret_cast<const float4*>(OUT) + (size_t)sl * (n + 1), (uint32_t)n * 16u);
          }
        }
        tc::bulk_commit();
      }
    }
    if (tt == 0) tc::bulk_wait_read0();   // OUT stays allocated until the last copies have read it
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == kPTmemWarps) {
    __syncwarp();
    tc::tmem_dealloc(tmem, 512);
  }
}

// ------------------------------------------------------------------ inverse gamma synthesis
// Block (ring t, map b): W(alpha, gamma_g) = sum_q Z_q(alpha) exp(+i n_q gamma_g) (real maps: the
// n, -n pair contributes 2 Re, n = 0 Re), scaled by the ring's exponent.
template <bool REAL>
__global__ void __launch_bounds__(512, 2) k_dftp_synth(PArgs a) {
  extern __shared__ float4 Zs[];   // [nj][n]
  __shared__ int jn[kMaxJobs], jp[kMaxJobs], njs;
  __shared__ float4 Ph[kJobChunk * kPMaxNg];
  const int t = blockIdx.x, b = blockIdx.y, n = a.n, Ng = a.Ng, hg = (Ng - 1) / 2;
  if (threadIdx.x == 0) {
    int nj;
    make_jobs(a.nvals, a.nact, REAL, jn, jp, nj);
    njs = nj;
  }
  __syncthreads();
  const int nj = njs, rf = b * a.nr + t;
  for (int i = threadIdx.x; i < nj * n; i += blockDim.x) Zs[i] = a.zbuf[(int64_t)rf * nj * n + i];
  for (int i = threadIdx.x; i < nj * Ng; i += blockDim.x) Ph[(i / Ng) * kPMaxNg + i % Ng] = a.gph[jn[i / Ng] * Ng + i % Ng];
  __syncthreads();
  const int ke = a.e_tw + a.fexp[rf] - 10;
  const int64_t ringlen = (int64_t)a.nr * n;
  for (int al = threadIdx.x; al < n; al += blockDim.x) {
    float4 z[kJobChunk];
#pragma unroll
    for (int q = 0; q < kJobChunk; ++q)
      if (q < nj) {
        z[q] = Zs[q * n + al];
        if (REAL && jp[q] >= 0) z[q] = make_float4(2.f * z[q].x, 2.f * z[q].y, 2.f * z[q].z, 2.f * z[q].w);
      }
    const int64_t base = (int64_t)b * a.pix_sb + (int64_t)t * n + al;
    for (int gg = 0; gg <= hg; ++gg) {
      Acc pr{0.f, 0.f}, pim{0.f, 0.f}, qr{0.f, 0.f}, qim{0.f, 0.f};
#pragma unroll
      for (int q = 0; q < kJobChunk; ++q)
        if (q < nj) {
          const float4 ph = Ph[q * kPMaxNg + gg];
          racc<false>(pr, z[q].x, z[q].y, ph.x, ph.y);
          if (gg > 0) racc<false>(qim, z[q].z, z[q].w, ph.z, ph.w);
          if (!REAL) {
            racc<false>(pim, z[q].z, z[q].w, ph.x, ph.y);
            if (gg > 0) racc<false>(qr, z[q].x, z[q].y, ph.z, ph.w);
          }
        }
      if (REAL) {
        double* out = (double*)a.pix_out;
        const Acc w0 = comb<false>(pr, -1.f, qim), w1 = comb<false>(pr, 1.f, qim);   // P - Q, P + Q
        out[base + gg * ringlen] = pair_dbl(w0, ke);
        if (gg > 0) out[base + (Ng - gg) * ringlen] = pair_dbl(w1, ke);
      } else {
        double2* out = (double2*)a.pix_out;
        const Acc r0 = comb<false>(pr, -1.f, qim), i0 = comb<false>(pim, 1.f, qr);
        out[base + gg * ringlen] = make_double2(pair_dbl(r0, ke), pair_dbl(i0, ke));
        if (gg > 0) {
          const Acc r1 = comb<false>(pr, 1.f, qim), i1 = comb<false>(pim, -1.f, qr);
          out[base + (Ng - gg) * ringlen] = make_double2(pair_dbl(r1, ke), pair_dbl(i1, ke));
        }
      }
    }
  }
}

int jobs_of_p(const TransformSpec& t, bool real) {
  int nj = 0;
  for (int v : t.nvals_h)
    if (!real || v >= 0) ++nj;
  return nj;
}

int slot_width(int n1) { return n1 == 1 ? 2 : (n1 == 3 ? 8 : 16); }

int gcd_i(int x, int y) {
  while (y) {
    const int r = x % y;
    x = y;
    y = r;
  }
  return x;
}

// inverse of a modulo m (gcd 1), m >= 1
int inv_mod(int a, int m) {
  if (m == 1) return 0;
  for (int x = 1; x < m; ++x)
    if ((int64_t)a * x % m == 1) return x;
  return 0;
}

// dynamic shared memory of the persistent kernel: table, data stages, output staging
size_t tc_smem_bytes(int n, int n1, int nj) {
  const int n2 = n / n1, Rs = ((n2 + 1 + 7) / 8) * 8, nkc = (n2 + 15) / 16;
  const int rpp = (kPN / slot_width(n1)) / nj;
  const size_t abytes = (size_t)nkc * kSl * Rs * 32, boff = (abytes + 1023) & ~(size_t)1023;
  return boff + (size_t)kPStages * kPChunk * 2 + (size_t)rpp * nj * (n + 1) * 16;   // OUT: n + 1 per slot
}

int num_sms() {
  static int nsm = 0;
  if (nsm == 0) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
      nsm = 148;
  }
  return nsm;
}

PArgs make_pargs(const s2w_plan* P, const GridTables& g, const TransformSpec& t, const DftpTable& tab, ColumnArgs c,
                 bool real) {
  PArgs a{};
  a.nvals = t.nvals;
  a.nact = t.nact;
  a.Ng = 2 * t.N - 1;
  a.n = g.n;
  a.n1 = tab.n1;
  a.n2 = tab.n2;
  a.R = tab.n2 + 1;
  a.Rs = tab.Rs;
  a.nkc = tab.nkc;
  a.nr = c.nr;
  a.B = c.B;
  a.Mc = c.Mc;
  a.mlo = c.mlo;
  a.e1 = tab.e1;
  a.e2 = tab.e2;
  const int nj = jobs_of_p(t, real);
  a.W = slot_width(tab.n1);
  a.rpp = (kPN / a.W) / nj;
  a.npass = (c.B * c.nr + a.rpp - 1) / a.rpp;
  a.gph = t.gphase4;
  a.tab = tab.tab;
  a.e_tw = tab.e;
  for (int m = 0; m < 8; ++m) {
    const double th = 2.0 * 3.14159265358979323846 * (double)(m % std::max(tab.n1, 1)) / (double)std::max(tab.n1, 1);
    const double cs = std::cos(th), sn = std::sin(th);
    const float ch = (float)cs, sh = (float)sn;
    a.tw1[m] = make_float4(ch, (float)(cs - (double)ch), sh, (float)(sn - (double)sh));
  }
  a.idesc = tc::make_idesc(128, kPN, 1, 0, 0);   // bf16 slices, M = 128, N = 64
  a.ops = P->dftp_ops;
  a.fexp = P->dftp_fexp;
  a.zbuf = P->dftp_z;
  a.err = P->err_word;
  return a;
}

template <class K>
cudaError_t launch_k(K kern, dim3 grid, int threads, size_t smem, cudaStream_t st, const PArgs& a) {
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  kern<<<grid, threads, smem, st>>>(a);
  return cudaGetLastError();
}

template <bool FWD, bool REAL>
cudaError_t launch_tc(int n1, size_t smem, cudaStream_t st, const PArgs& a) {
  const dim3 grid(std::min(a.npass, num_sms()));
  switch (n1) {
    case 1: return launch_k(k_dftp_tc<FWD, REAL, 1>, grid, kPT, smem, st, a);
    case 3: return launch_k(k_dftp_tc<FWD, REAL, 3>, grid, kPT, smem, st, a);
    case 5: return launch_k(k_dftp_tc<FWD, REAL, 5>, grid, kPT, smem, st, a);
    case 7: return launch_k(k_dftp_tc<FWD, REAL, 7>, grid, kPT, smem, st, a);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace

// Factorisation n = 2L - 1 = n1 n2 for the prime-factor tensor-core DFTs: the smallest n1 in
// {1, 3, 5, 7} with gcd(n1, n2) = 1, n2 + 1 <= 128 table rows and the persistent kernel's shared
// memory within the limit for the transform's job count; false if none fits, or where the jobs do
// not: at most four (the prologue's gamma DFT pass) and every carried n != 0 with its -n partner
// for real maps, and 2N - 1 <= 15 gamma samples.
bool dftp_shape(const TransformSpec& t, bool real, int* n1_out, int* n2_out) {
  const int nj = jobs_of_p(t, real);
  if (nj < 1 || nj > kJobChunk || t.L < 2 || 2 * t.N - 1 > kPMaxNg) return false;
  if (real)
    for (int v : t.nvals_h)
      if (v != 0 && std::find(t.nvals_h.begin(), t.nvals_h.end(), -v) == t.nvals_h.end()) return false;
  const int n = 2 * t.L - 1;
  const size_t lim = 200 * 1024;   // the prologues' shared memory (one ring's gamma DFT or columns)
  const size_t Mc = real ? t.L : n;
  if ((size_t)nj * n * sizeof(float4) > lim || (size_t)t.nact * Mc * sizeof(double2) > lim) return false;
  for (int n1 : {1, 3, 5, 7}) {
    if (n % n1 != 0) continue;
    const int n2 = n / n1;
    if (gcd_i(n1, n2) != 1 || n2 + 1 > 128 || n2 < 2) continue;
    if (nj > kPN / slot_width(n1) || (kPN / slot_width(n1)) / nj > kPMaxRpp) continue;
    if (tc_smem_bytes(n, n1, nj) > (size_t)kPMaxSmem) continue;
    *n1_out = n1;
    *n2_out = n2;
    return true;
  }
  return false;
}

// Workspace of the prime-factor DFTs of one transform for B maps on nr rings: the pass-ordered
// slices (uint16 elements), the ring exponents and the inverse's Z staging (float4 elements).
void dftp_ws_elems(const TransformSpec& t, bool real, int n1, int B, int nr, int64_t* ops, int64_t* fexp, int64_t* z) {
  const int nj = jobs_of_p(t, real), n = 2 * t.L - 1, n2 = n / n1;
  const int rpp = (kPN / slot_width(n1)) / nj, nkc = (n2 + 15) / 16;
  const int64_t rings = (int64_t)B * nr, npass = (rings + rpp - 1) / rpp;
  *ops = npass * nkc * kPChunk;
  *fexp = rings;
  *z = rings * nj * n;
}

// The sliced n2-point table: rows 2j (s cos(2 pi p2 j/n2)) and 2j + 1 (s sin(2 pi p2 j/n2)) for
// j <= (n2-1)/2, reduction index p2 < n2, zero elsewhere; seven bf16 digits of
// round(v 2^(47 - e)), e = ilogb(s) + 1, in [chunk][slice][Rs rows x 16] core-matrix tiles.
void build_dftp_table(int L, int n1, int n2, double scale, DftpTable* tab, std::vector<uint16_t>& h) {
  const int n = 2 * L - 1;
  tab->n = n;
  tab->n1 = n1;
  tab->n2 = n2;
  tab->Rs = ((n2 + 1 + 7) / 8) * 8;
  tab->nkc = (n2 + 15) / 16;
  tab->scale = scale;
  tab->e = std::ilogb(scale) + 1;
  tab->e1 = n1 == 1 ? 0 : (int)((int64_t)n2 * inv_mod(n2 % n1, n1) % n);
  tab->e2 = (int)((int64_t)n1 * inv_mod(n1 % n2, n2) % n);
  const int tile = tab->Rs * 16;
  h.assign((size_t)tab->nkc * kSl * tile, 0);
  const double w = 2.0 * 3.14159265358979323846 / n2;
  for (int r = 0; r < tab->Rs; ++r)
    for (int k = 0; k < tab->nkc * 16; ++k) {
      double v = 0.0;
      const int jj = r >> 1;
      if (r < n2 + 1 && k < n2) {
        const int e = (int)(((long long)k * jj) % n2);
        v = scale * ((r & 1) ? std::sin(w * e) : std::cos(w * e));
      }
      uint16_t d[kSl];
      host_digits(v, tab->e, d);
      const size_t o = (size_t)(k >> 4) * kSl * tile + (size_t)(((r >> 3) * 2 + ((k & 15) >> 3)) * 64 + (r & 7) * 8 + (k & 7));
      for (int s = 0; s < kSl; ++s) h[o + (size_t)s * tile] = d[s];
    }
}

cudaError_t launch_dftp_forward(const s2w_plan* P, const GridTables& g, const TransformSpec& t, const void* pix,
                                int64_t pix_sb, bool real, ColumnArgs c, cudaStream_t st) {
  const DftpTable& tab = *t.dftp_fwd;
  PArgs a = make_pargs(P, g, t, tab, c, real);
  a.pix_in = pix;
  a.pix_sb = pix_sb;
  a.Gout = c.G;
  const int nj = jobs_of_p(t, real);
  const dim3 pg(c.nr, c.B);
  const size_t psm = (size_t)nj * g.n * sizeof(float4);
  const int th = t.dft_threads_fwd;
  cudaError_t e = real ? launch_k(k_dftp_fwd_prep<true>, pg, th, psm, st, a)
                       : launch_k(k_dftp_fwd_prep<false>, pg, th, psm, st, a);
  if (e != cudaSuccess) return e;
  const size_t smem = tc_smem_bytes(g.n, tab.n1, nj);
  return real ? launch_tc<true, true>(tab.n1, smem, st, a) : launch_tc<true, false>(tab.n1, smem, st, a);
}

cudaError_t launch_dftp_inverse(const s2w_plan* P, const GridTables& g, const TransformSpec& t, ColumnArgs c,
                                void* pix, int64_t pix_sb, bool real, cudaStream_t st) {
  const DftpTable& tab = *t.dftp_inv;
  PArgs a = make_pargs(P, g, t, tab, c, real);
  a.Gin = c.G;
  a.pix_out = pix;
  a.pix_sb = pix_sb;
  const int nj = jobs_of_p(t, real);
  const dim3 pg(c.nr, c.B);
  const int th = t.dft_threads_inv;
  const size_t gsm = (size_t)t.nact * c.Mc * sizeof(double2);
  cudaError_t e = real ? launch_k(k_dftp_inv_prep<true>, pg, th, gsm, st, a)
                       : launch_k(k_dftp_inv_prep<false>, pg, th, gsm, st, a);
  if (e != cudaSuccess) return e;
  const size_t smem = tc_smem_bytes(g.n, tab.n1, nj);
  e = real ? launch_tc<false, true>(tab.n1, smem, st, a) : launch_tc<false, false>(tab.n1, smem, st, a);
  if (e != cudaSuccess) return e;
  const size_t zsm = (size_t)nj * g.n * sizeof(float4);
  return real ? launch_k(k_dftp_synth<true>, pg, th, zsm, st, a) : launch_k(k_dftp_synth<false>, pg, th, zsm, st, a);
}

}  // namespace s2w

// Radial maps of the ball (Sec. 2.3, Eqs. 7-8: the Fourier-Laguerre transform and its inverse;
// Sec. 3.2: the per-scale radial filters of the ball wavelets) on the 5th-generation tensor
// cores, float64-accurate by exact integer slicing (slice7.cuh; Ozaki, Ogita, Oishi and Rump,
// Numer. Algorithms 59, 2012):
//   out[b][o][c] (+)= wo[o][l] sum_q R[o][q] wi[q][l] in[b][q][c],   c = l Mc + m,
// a real Pout x Pin matrix R (P <= 256 radial nodes or coefficients) applied to every complex
// angular coefficient column, with optional per-(row, l) weights before (wi) and after (wo).
//
// The radial matrices span a huge dynamic range along the node index (the Gauss-Laguerre weights
// grow like e^{x_i}, the basis decays like e^{-x_i/2}), so both operands are first balanced by an
// exact power-of-two scale per reduction index q: R f = (R D)(D^-1 f) with D = diag 2^{k_q},
// k_q = -ilogb(max_o |R[o][q]|), so every column of R D has its largest entry in [1, 2); a zero
// column of R takes no part in the data's exponent.  The sums then err by ~2^-54 of their largest
// term, as float64 does, instead of by a fixed fraction of max|R| max|f|.
// Eight digits (54-bit fixed point), not the seven of the other sliced GEMMs: the chain of maps a
// ball wavelet scale takes (the Laguerre transform of the field, then the top radial filter's
// synthesis at a node where the filtered basis is small) amplifies the forward map's noise floor
// about a hundredfold, and 47-bit operands would leave it near 1e-13 where float64 reaches 1e-15.
// R D is sliced once at plan time (one exponent per row, eight bf16 digits of a 54-bit fixed-point
// value, [row tile][K chunk][slice][128 x 16] core-matrix tiles); per call, k_radx_prep gives
// every data column (batch, c, re|im) its exponent over the K nodes and its eight slices
// ([column group of 16 complex][K chunk][slice][32 x 16]); k_radx_gemm sums the 36 digit pairs
// of a K step with eight MMAs (one per table slice, N = 256 .. 32 over the data slices side by
// side) into eight exact float32 accumulators (a pair sums to <= 2^12 K <= 2^20, eight pairs
// <= 2^23) through a two-stage bulk-copy pipeline (two CTAs per SM), and the epilogue forms
// 2^(e_row + f_col - 10) sum_q 2^(-7q) D_q in compensated float32, applies wo and writes or
// accumulates.  Every mbarrier wait is bounded; a timeout sets the plan's error word.
#include <cmath>
#include <cstring>
#include <vector>

#include "comp32.cuh"
#include "s2w_internal.h"
#include "slice7.cuh"
#include "tc_sm100.cuh"

namespace s2w {
namespace {

constexpr int kRSl = 8;   // slices per value
// kexp of a zero column of R: its data is left out of the exponent and the slices
constexpr int kRZeroCol = 1 << 20;

// round(c r 2^(54 - e)) for |c r| < 2^e: floor(Mc Mr / 2^52) by one 64 x 64 high multiply, then a
// rounding shift s = 2044 + e - Ec - Er >= 0 (at s = 0 the truncated bits below 2^52 of the
// 106-bit product are dropped: an error below one unit of 2^(e - 54))
__device__ __forceinline__ long long fix54_prod(double c, double r, int e) {
  const unsigned long long uc = (unsigned long long)__double_as_longlong(c);
  const unsigned long long ur = (unsigned long long)__double_as_longlong(r);
  const int Ec = (int)(uc >> 52) & 0x7FF, Er = (int)(ur >> 52) & 0x7FF;
  if (Ec == 0 || Er == 0) return 0;
  const int sh = 2044 + e - Ec - Er;
  if (sh >= 63) return 0;
  const unsigned long long Mc = (uc & 0xFFFFFFFFFFFFFull) | (1ull << 52);
  const unsigned long long Mr = (ur & 0xFFFFFFFFFFFFFull) | (1ull << 52);
  const unsigned long long H = __umul64hi(Mc << 11, Mr << 1);   // floor(Mc Mr / 2^52)
  const long long X = (long long)(sh > 0 ? (H + (1ull << (sh - 1))) >> sh : H);
  return ((uc ^ ur) >> 63) ? -X : X;
}

// X (|X| <= 2^54) -> eight balanced base-128 digits in [-64, 63], most significant first, as float32
// bit patterns (upper 16 bits = the bfloat16 of the same value): the plain base-128 digits of
// X + 64 (128^8 - 1)/127, less 64.
constexpr long long kDigitBias8 = 36312488334073920ll;   // 64 (128^8 - 1)/127
__device__ __forceinline__ void digits8(long long X, uint32_t (&f)[kRSl]) {
  const unsigned long long Y = (unsigned long long)(X + kDigitBias8);
#pragma unroll
  for (int i = 0; i < kRSl; ++i) {
    const unsigned int u = (unsigned int)(Y >> (7 * (kRSl - 1 - i))) & 127u;
    f[i] = __float_as_uint(__uint_as_float(0x4B000000u | u) - 8388672.0f);   // u - 64
  }
}

// host: the eight bf16 slices of round(v 2^(54 - e)) for |v| < 2^e, in the device convention
inline void host_digits8(double v, int e, uint16_t (&d)[kRSl]) {
  const long long X = std::llround(std::ldexp(v, 54 - e));
  const unsigned long long Y = (unsigned long long)(X + kDigitBias8);
  for (int i = 0; i < kRSl; ++i) {
    const int u = (int)((Y >> (7 * (kRSl - 1 - i))) & 127u) - 64;
    const float f = (float)u;
    uint32_t bits;
    std::memcpy(&bits, &f, sizeof(bits));
    d[i] = (uint16_t)(bits >> 16);
  }
}

constexpr int kRT = 128;                       // GEMM threads: one per output row of a tile
constexpr int kRN = 32;                        // GEMM columns per CTA: 16 complex (re, im)
constexpr int kRATile = 128 * 16;              // one table slice chunk
constexpr int kRBTile = kRN * 16;              // one data slice chunk
constexpr int kRAChunk = kRSl * kRATile;
constexpr int kRBChunk = kRSl * kRBTile;
constexpr int kRStage = kRAChunk + kRBChunk;
constexpr int kRStages = 2;   // 80 KB: two CTAs (and 2 x 256 TMEM columns) per SM
constexpr size_t kRSmem = (size_t)kRStages * kRStage * sizeof(uint16_t);   // 81920 B
constexpr uint32_t kRWait = 1u << 20;

struct RArgs {
  const double2* in;
  double2* out;
  int B, Pin, Pout, L, Mc, nkc, cg;   // cg: column groups of 16 complex columns per map
  int64_t ncol;
  const double *wi, *wo;
  int accumulate;
  const uint16_t* tab;
  const int* rexp;
  const int* kexp;  // [Pin] the balancing exponents k_q (table column scaled by 2^k_q, data by 2^-k_q)
  uint16_t* ops;   // [B * cg][nkc][8][32 x 16]
  int* fexp;       // [B][ncol][2] column exponents (re, im)
  uint32_t idesc;
  int* err;
};

// One thread per complex column (b, c): its exponent over the Pin nodes (re and im separately),
// then its slices, 8 nodes per 16-byte core-matrix row.
__global__ void __launch_bounds__(128) k_radx_prep(RArgs a) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int b = blockIdx.y;
  if (c >= a.ncol) return;
  const int l = (int)(c / a.Mc);
  const double2* inb = a.in + (int64_t)b * a.Pin * a.ncol + c;
  int er = 0, ei = 0;
  bool bad = false;
  for (int q = 0; q < a.Pin; ++q) {
    const double2 v = inb[(int64_t)q * a.ncol];
    const double w = a.wi != nullptr ? a.wi[(int64_t)q * a.L + l] : 1.0;
    const int kq = a.kexp[q];
    bad |= (bexp(v.x) == 0x7FF) | (bexp(v.y) == 0x7FF);
    if (kq == kRZeroCol) continue;
    const int br = ebound_prod(v.x, w), bi = ebound_prod(v.y, w);
    if (br > 0) er = max(er, br - kq);   // |v w 2^-k_q| < 2^(bound - k_q)
    if (bi > 0) ei = max(ei, bi - kq);
  }
  if (bad) atomicCAS(a.err, 0, (int)S2W_ENONFINITE);
  const int fr = e_from(er), fi = e_from(ei);
  int* fx = a.fexp + ((int64_t)b * a.ncol + c) * 2;
  fx[0] = fr;
  fx[1] = fi;
  const int64_t gg = (int64_t)b * a.cg + c / 16;
  const int jr = (int)(c % 16) * 2, ji = jr + 1;
  for (int kg = 0; kg < a.nkc * 2; ++kg) {
    uint32_t wr[kRSl][4], wim[kRSl][4];
#pragma unroll
    for (int u = 0; u < 8; u += 2) {
      long long xr[2], xi[2];
#pragma unroll
      for (int v2 = 0; v2 < 2; ++v2) {
        const int q = kg * 8 + u + v2;
        xr[v2] = xi[v2] = 0;
        if (q < a.Pin && a.kexp[q] != kRZeroCol) {
          const double2 v = inb[(int64_t)q * a.ncol];
          const double w = a.wi != nullptr ? a.wi[(int64_t)q * a.L + l] : 1.0;
          const int kq = a.kexp[q];   // round(v w 2^-k_q 2^(54 - f)) = fix54_prod(v, w, f + k_q)
          xr[v2] = fix54_prod(v.x, w, fr + kq);
          xi[v2] = fix54_prod(v.y, w, fi + kq);
        }
      }
      uint32_t d0[kRSl], d1[kRSl], e0[kRSl], e1[kRSl];
      digits8(xr[0], d0);
      digits8(xr[1], d1);
      digits8(xi[0], e0);
      digits8(xi[1], e1);
#pragma unroll
      for (int s = 0; s < kRSl; ++s) {
        wr[s][u / 2] = __byte_perm(d0[s], d1[s], 0x7632);
        wim[s][u / 2] = __byte_perm(e0[s], e1[s], 0x7632);
      }
    }
    const int64_t o = (gg * a.nkc + (kg >> 1)) * kRBChunk + (kg & 1) * 64;
#pragma unroll
    for (int s = 0; s < kRSl; ++s) {
      *reinterpret_cast<uint4*>(a.ops + o + (int64_t)s * kRBTile + (jr >> 3) * 128 + (jr & 7) * 8) =
          make_uint4(wr[s][0], wr[s][1], wr[s][2], wr[s][3]);
      *reinterpret_cast<uint4*>(a.ops + o + (int64_t)s * kRBTile + (ji >> 3) * 128 + (ji & 7) * 8) =
          make_uint4(wim[s][0], wim[s][1], wim[s][2], wim[s][3]);
    }
  }
}

// CTA (row tile, column group, map): thread 0 streams the K chunks (table and data slices) through
// two stages and issues eight MMAs (the 36 digit pairs) per chunk into eight 128 x 32 accumulators;
// then every thread
// converts its row's 32 columns.
__global__ void __launch_bounds__(kRT) k_radx_gemm(RArgs a) {
  extern __shared__ __align__(1024) uint8_t smem[];
  __shared__ __align__(8) uint64_t bar_ld[kRStages], bar_mma[kRStages];
  __shared__ uint32_t tbase;
  __shared__ int fx_s[kRN];
  const int rt = blockIdx.x, g = blockIdx.y, b = blockIdx.z;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int64_t gg = (int64_t)b * a.cg + g;
  if (tid == 0) {
    for (int s = 0; s < kRStages; ++s) {
      tc::mbar_init(&bar_ld[s], 1);
      tc::mbar_init(&bar_mma[s], 1);
    }
    tc::fence_mbar_init();
  }
  if (tid < kRN) {
    const int64_t c = (int64_t)g * 16 + tid / 2;
    fx_s[tid] = c < a.ncol ? a.fexp[((int64_t)b * a.ncol + c) * 2 + (tid & 1)] : 0;
  }
  if (warp == 0) tc::tmem_alloc(&tbase, 256);
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = tbase;
  uint16_t* const stage0 = reinterpret_cast<uint16_t*>(smem);
  const int nkc = a.nkc;
  bool ok = true;
  if (tid == 0) {
    uint32_t ph_ld[kRStages] = {}, ph_mma[kRStages] = {};
    unsigned pend_ld = 0u, pend_mma = 0u;
    const uint16_t* A = a.tab + (int64_t)rt * nkc * kRAChunk;
    const uint16_t* Bq = a.ops + gg * nkc * kRBChunk;
    auto load = [&](int c, int s) {
      uint16_t* S = stage0 + s * kRStage;
      tc::mbar_expect_tx(&bar_ld[s], (uint32_t)kRStage * 2u);
      tc::bulk_g2s(S, A + (int64_t)c * kRAChunk, kRAChunk * 2u, &bar_ld[s]);
      tc::bulk_g2s(S + kRAChunk, Bq + (int64_t)c * kRBChunk, kRBChunk * 2u, &bar_ld[s]);
      pend_ld |= 1u << s;
    };
    auto wait = [&](uint64_t* bar, uint32_t& ph, unsigned& pend, int s) {
      if (!ok) return;
      if (!tc::mbar_wait(bar, ph, kRWait)) {
        atomicExch(a.err, (int)S2W_ETIMEOUT);
        ok = false;
        return;
      }
      ph ^= 1u;
      pend &= ~(1u << s);
    };
    for (int c = 0; c < kRStages - 1 && c < nkc; ++c) load(c, c);
    for (int c = 0; c < nkc && ok; ++c) {
      const int s = c % kRStages;
      wait(&bar_ld[s], ph_ld[s], pend_ld, s);
      if (!ok) break;
      tc::fence_after_sync();
      const uint32_t A0 = tc::smem_u32(stage0 + s * kRStage), B0 = A0 + kRAChunk * 2u;
      const uint64_t dA = tc::make_sdesc(A0, 128, 256), dB = tc::make_sdesc(B0, 128, 256);
      // one MMA per table slice sa against the data slices 0 .. 7 - sa side by side (contiguous
      // 32-row blocks: one N = 32 (8 - sa) operand), pair (sa, sb) into accumulator sa + sb at TMEM
      // columns 32 (sa + sb): eight MMAs per K chunk for the 36 digit pairs
#pragma unroll
      for (int sa = 0; sa < kRSl; ++sa)
        tc::mma_f16(tmem + (uint32_t)(32 * sa), dA + (uint64_t)(sa * (kRATile * 2 / 16)), dB,
                    tc::make_idesc(128, kRN * (kRSl - sa), 1, 0, 0), (c > 0 || sa > 0) ? 1u : 0u);
      tc::mma_commit(&bar_mma[s]);
      pend_mma |= 1u << s;
      if (c + kRStages - 1 < nkc) {
        const int sn = (c + kRStages - 1) % kRStages;   // last held chunk c - 1
        if (c >= 1) wait(&bar_mma[sn], ph_mma[sn], pend_mma, sn);
        if (!ok) break;
        load(c + kRStages - 1, sn);
      }
    }
    for (int c = nkc > kRStages ? nkc - kRStages : 0; c < nkc && ok; ++c) {
      const int s = c % kRStages;
      if (pend_mma & (1u << s)) wait(&bar_mma[s], ph_mma[s], pend_mma, s);
    }
    if (!ok)   // let this CTA's own copies and MMAs in flight land (bounded)
      for (int s = 0; s < kRStages; ++s) {
        if (pend_ld & (1u << s)) tc::mbar_wait(&bar_ld[s], ph_ld[s], kRWait);
        if (pend_mma & (1u << s)) tc::mbar_wait(&bar_mma[s], ph_mma[s], kRWait);
      }
  }
  ok = __syncthreads_and(ok);
  if (ok) {
    tc::fence_after_sync();
    Acc acc[kRN];
#pragma unroll
    for (int j = 0; j < kRN; ++j) acc[j] = Acc{0.f, 0.f};
    for (int qq = kRSl - 1; qq >= 0; --qq) {
      float v[32];
      tc::tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(32 * qq), v);
      const float w = __uint_as_float((uint32_t)(127 - 7 * qq) << 23);   // 2^(-7 qq)
#pragma unroll
      for (int j = 0; j < kRN; ++j) two_sum_add(acc[j], v[j] * w);
    }
    const int o = rt * 128 + warp * 32 + lane;
    if (o < a.Pout) {
      const int er = a.rexp[o];
      double2* outb = a.out + ((int64_t)b * a.Pout + o) * a.ncol;
#pragma unroll
      for (int p = 0; p < kRN / 2; ++p) {
        const int64_t c = (int64_t)g * 16 + p;
        if (c >= a.ncol) break;
        const int kr = er + fx_s[2 * p] - 10, ki = er + fx_s[2 * p + 1] - 10;
        double x = scale2(f2d(acc[2 * p].s), kr) + scale2(f2d(acc[2 * p].c), kr);
        double y = scale2(f2d(acc[2 * p + 1].s), ki) + scale2(f2d(acc[2 * p + 1].c), ki);
        if (a.wo != nullptr) {
          const double w = a.wo[(int64_t)o * a.L + (int)(c / a.Mc)];
          x *= w;
          y *= w;
        }
        if (a.accumulate) {
          const double2 prev = outb[c];
          x += prev.x;
          y += prev.y;
        }
        outb[c] = make_double2(x, y);
      }
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tmem, 256);
}

}  // namespace

// Host: the balancing exponents k_q = -ilogb(max_o |M[o][q]|) (kRZeroCol for a zero column) and the sliced
// table of the row-major Pout x Pin float64 matrix M D, D = diag 2^{k_q} (row exponents e_o with
// max_q |(M D)[o][q]| < 2^e_o; zero rows get e = 0).
void build_radx(const std::vector<double>& M, int Pout, int Pin, RadxMap* map, std::vector<uint16_t>& tab,
                std::vector<int>& rexp, std::vector<int>& kexp) {
  map->Pout = Pout;
  map->Pin = Pin;
  map->Mt = (Pout + 127) / 128;
  map->nkc = (Pin + 15) / 16;
  tab.assign((size_t)map->Mt * map->nkc * kRAChunk, 0);
  rexp.assign((size_t)map->Mt * 128, 0);
  kexp.assign((size_t)Pin, 0);
  for (int q = 0; q < Pin; ++q) {
    double mx = 0.0;
    for (int o = 0; o < Pout; ++o) mx = std::max(mx, std::fabs(M[(size_t)o * Pin + q]));
    kexp[q] = mx > 0.0 ? -std::ilogb(mx) : kRZeroCol;
  }
  auto scaled = [&](int o, int q) {   // exact; a zero column stays zero
    return kexp[q] == kRZeroCol ? 0.0 : std::ldexp(M[(size_t)o * Pin + q], kexp[q]);
  };
  for (int o = 0; o < map->Mt * 128; ++o) {
    int e = 0;
    if (o < Pout) {
      double mx = 0.0;
      for (int q = 0; q < Pin; ++q) mx = std::max(mx, std::fabs(scaled(o, q)));
      if (mx > 0.0) e = std::ilogb(mx) + 1;   // mx < 2^e
    }
    rexp[o] = e;
    for (int q = 0; q < map->nkc * 16; ++q) {
      const double v = (o < Pout && q < Pin) ? scaled(o, q) : 0.0;
      uint16_t d[kRSl];
      host_digits8(v, e, d);
      const size_t base = ((size_t)(o >> 7) * map->nkc + (q >> 4)) * kRAChunk;
      const size_t in = (size_t)((((o & 127) >> 3) * 2 + ((q & 15) >> 3)) * 64 + (o & 7) * 8 + (q & 7));
      for (int s = 0; s < kRSl; ++s) tab[base + (size_t)s * kRATile + in] = d[s];
    }
  }
}

int64_t radx_ops_elems(int B, int Pin, int64_t ncol) {
  return (int64_t)B * ((ncol + 15) / 16) * ((Pin + 15) / 16) * kRBChunk;
}

cudaError_t launch_radx(const RadxMap& R, const double2* in, double2* out, int B, int L, int Mc, const double* wi,
                        const double* wo, bool accumulate, uint16_t* ops, int* fexp, int* err, cudaStream_t st) {
  if (R.Pin > 256) return cudaErrorInvalidValue;   // eight pair sums of K <= 256 terms stay below 2^24
  RArgs a{};
  a.in = in;
  a.out = out;
  a.B = B;
  a.Pin = R.Pin;
  a.Pout = R.Pout;
  a.L = L;
  a.Mc = Mc;
  a.nkc = R.nkc;
  a.ncol = (int64_t)L * Mc;
  a.cg = (int)((a.ncol + 15) / 16);
  a.wi = wi;
  a.wo = wo;
  a.accumulate = accumulate ? 1 : 0;
  a.tab = R.tab;
  a.rexp = R.rexp;
  a.kexp = R.kexp;
  a.ops = ops;
  a.fexp = fexp;
  a.idesc = tc::make_idesc(128, kRN, 1, 0, 0);   // bf16 slices
  a.err = err;
  k_radx_prep<<<dim3((unsigned)((a.ncol + 127) / 128), B), 128, 0, st>>>(a);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_radx_gemm, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kRSmem);
  if (e != cudaSuccess) return e;
  k_radx_gemm<<<dim3(R.Mt, a.cg, B), kRT, kRSmem, st>>>(a);
  return cudaGetLastError();
}

}  // namespace s2w

// Reduced-precision l-contractions on the 5th-generation tensor cores (tcgen05), float32
// accumulation in TMEM, against precomputed Wigner-d tables.
//
// Precision: every operand is a pair hi + lo and each K step issues three MMAs (hi*hi +
// hi*lo + lo*hi, the lo*lo term dropped): "split" in fp16 (values scaled by powers of two into
// the fp16 range; 22 bits per pair) and "bf16" (split-bf16, 16 bits per pair).
//
// Both directions are one GEMM per (m, n) pair: rows x 32 columns (16 maps x re/im), in K
// chunks of 32:
//   inverse  rows beta, K = l:   G[beta][map] = sum_l 2^8 d^l_mn(beta) * s F[l][map]
//   forward  rows l, K = beta':  F[l][map]    = sum_b' 2^10 (M^T d^l_mn)(beta') * s G[beta'][map]
// The forward tables carry the colatitude quadrature folded in (as the float64 table mode
// does), so the forward transform needs no second GEMM.  The tables are packed from the
// float64-accurate float-pair tables of kernels_tab.cu (built and folded there, then freed).
//
// k_tcp: the data operand of every (m, n) and 16-map chunk, prepared once in float32 (a
// power-of-two scale per operand into the fp16 range, the hi/lo split) into a plan workspace.
// k_tc_gemm: one CTA of 128 threads per (row tile of 128, m, n); thread 0 runs a two-stage
// pipeline of bulk asynchronous copies (TMA engine, 20 KB per stage: table hi/lo + operand
// hi/lo) and MMAs; 40 KB of shared memory lets five CTAs share an SM, so that the short CTAs
// (at most eight K chunks each) overlap one another's pipeline fill and epilogue; every
// mbarrier wait is bounded and a timeout sets the plan's error word.
//
// Packed layouts (core matrices of 8 rows x 8 elements, K-major, no swizzle; see tc_sm100.cuh):
//   table chunk (row tile t, K chunk c): 128 x 32 elements, element (r, k) at
//     ((r / 8) * 4 + k / 8) * 64 + (r % 8) * 8 + k % 8, chunks ordered [t][c]
//   operand chunk c: 32 x 32 elements, element (j, k) at ((j / 8) * 4 + k / 8) * 64 + (j % 8) * 8 + k % 8
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "comp32.cuh"
#include "s2w_internal.h"
#include "tc_sm100.cuh"

namespace s2w {
namespace {

constexpr double kInvScale = 256.0;    // inverse tables hold 2^8 d
constexpr double kFwdScale = 1024.0;   // forward tables hold 2^10 M^T d
constexpr int kTcThreads = 128;
constexpr int kTcN = 32;               // MMA N: 16 maps x (re, im)
constexpr int kKc = 32;                // K chunk (the K extents are multiples of 64)
constexpr int kTileElems = 128 * kKc;  // table chunk elements
constexpr int kOpElems = kTcN * kKc;   // operand chunk elements
constexpr uint32_t kWaitIter = 1u << 26;

constexpr uint32_t kSbo = (kKc / 8) * 128;   // bytes between 8-row core-matrix groups
__device__ __forceinline__ int tile_index(int r, int k) {
  return ((r >> 3) * (kKc / 8) + (k >> 3)) * 64 + (r & 7) * 8 + (k & 7);
}

// hi and lo of x in fp16 (FP16 = true) or bf16
template <bool FP16>
__device__ __forceinline__ void put_pair(uint16_t* hi, uint16_t* lo, int64_t i, float x) {
  if (FP16) {
    const __half h = __float2half_rn(x);
    hi[i] = __half_as_ushort(h);
    lo[i] = __half_as_ushort(__float2half_rn(x - __half2float(h)));
  } else {
    const __nv_bfloat16 h = __float2bfloat16_rn(x);
    hi[i] = __bfloat16_as_ushort(h);
    lo[i] = __bfloat16_as_ushort(__float2bfloat16_rn(x - __bfloat162float(h)));
  }
}

// hi and lo of a float64 value (plan-time table packing)
template <bool FP16>
__device__ __forceinline__ void put_pair_d(uint16_t* hi, uint16_t* lo, int64_t i, double v) {
  if (FP16) {
    const __half h = __double2half(v);
    hi[i] = __half_as_ushort(h);
    lo[i] = __half_as_ushort(__double2half(v - (double)__half2float(h)));
  } else {
    const __nv_bfloat16 h = __double2bfloat16(v);
    hi[i] = __bfloat16_as_ushort(h);
    lo[i] = __bfloat16_as_ushort(__double2bfloat16(v - (double)__bfloat162float(h)));
  }
}

// float64 -> float without the float64 pipe (hi part of the integer split, 2^-24 relative)
__device__ __forceinline__ float to_f(double x) { return split1_bits(x).x; }

// float -> float64 with integer operations (exact for normal floats; subnormals give 0; Inf and
// NaN carried over)
__device__ __forceinline__ double f2d(float f) {
  const unsigned int u = __float_as_uint(f);
  const unsigned int e = (u >> 23) & 0xFFu;
  if (e == 0u) return 0.0;
  const unsigned long long b = ((unsigned long long)(u & 0x80000000u) << 32) |
                               ((unsigned long long)(e == 0xFFu ? 0x7FFu : e + 896u) << 52) | ((unsigned long long)(u & 0x7FFFFFu) << 29);
  return __longlong_as_double((long long)b);
}

__device__ float block_max_f(float v, float* red) {
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  float r = red[0];
  for (int i = 1; i < (int)(blockDim.x >> 5); ++i) r = fmaxf(r, red[i]);
  return r;
}

// 2^(14 - e) with mx = f 2^e, f in [0.5, 1): scales a block whose largest magnitude is mx below 2^14
__device__ __forceinline__ float pow2_scale_f(float mx) {
  if (!(mx > 0.f)) return 1.f;
  int e;
  frexpf(mx, &e);
  return ldexpf(1.f, 14 - e);
}

// ------------------------------------------------------------------ table packing
struct PackArgs {
  const int* nvals;
  int nact, L, nr, Mc, mlo;
  const int64_t *toff_i, *toff_f;   // float-pair tables (kernels_tab.cu layout)
  const int* tkp;
  int tLp, tLk;
  const float2 *tinv, *tfwd;
  const int64_t *off_i, *off_f;     // packed tensor-core tables
  const int *kli, *klf;
  int Lb, Lk;
  uint16_t *inv_hi, *inv_lo, *fwd_hi, *fwd_lo;
};

// block (m, n), threads over the tile elements
template <bool FP16>
__global__ void k_tc_pack(PackArgs a) {
  const int mi = blockIdx.x, ni = blockIdx.y, idx = mi * a.nact + ni;
  const int m = a.mlo + mi, nn = a.nvals[ni], L = a.L;
  const int l0 = max(abs(m), abs(nn)), l0a = l0 & ~7;
  const int kli = a.kli[idx], klf = a.klf[idx];
  if (kli == 0) return;
  const float2* Ti = a.tinv + a.toff_i[idx];   // [kp][tLp]
  const float2* Tf = a.tfwd + a.toff_f[idx];   // [tLk][kp]
  const int kp = a.tkp[idx];
  const int nkci = kli / kKc;
  for (int64_t e = threadIdx.x; e < (int64_t)a.Lb * kli; e += blockDim.x) {
    const int beta = (int)(e / kli), ll = (int)(e - (int64_t)beta * kli), l = l0a + ll;
    double v = 0.0;
    if (beta < a.nr && l >= l0 && l < L && ll < kp) {
      const float2 p = Ti[(int64_t)ll * a.tLp + beta];
      v = ((double)p.x + (double)p.y) * kInvScale;
    }
    const int64_t o = a.off_i[idx] + ((int64_t)(beta >> 7) * nkci + ll / kKc) * kTileElems + tile_index(beta & 127, ll % kKc);
    put_pair_d<FP16>(a.inv_hi, a.inv_lo, o, v);
  }
  const int nkcf = a.Lk / kKc;
  for (int64_t e = threadIdx.x; e < (int64_t)klf * a.Lk; e += blockDim.x) {
    const int ll = (int)(e / a.Lk), bp = (int)(e - (int64_t)ll * a.Lk), l = l0a + ll;
    double v = 0.0;
    if (bp < a.nr && l >= l0 && l < L && ll < kp) {
      const float2 p = Tf[(int64_t)bp * kp + ll];
      v = ((double)p.x + (double)p.y) * kFwdScale;
    }
    const int64_t o = a.off_f[idx] + ((int64_t)(ll >> 7) * nkcf + bp / kKc) * kTileElems + tile_index(ll & 127, bp % kKc);
    put_pair_d<FP16>(a.fwd_hi, a.fwd_lo, o, v);
  }
}

// ------------------------------------------------------------------ operand preparation
struct PrepArgs {
  const int* nvals;
  int nact, L, nr, Mc, mlo, B;
  const int* kl;          // inverse: K extent per tile (0 = empty); forward: row extent (0 = empty)
  const int64_t* off_i;   // inverse table offsets (operand offset = off_i / Lb * 32)
  int Lb, Lk;
  const double2* coef;    // inverse source: coefficients and multiplier
  int64_t s_b, s_n, s_l;
  int mlo_in;
  const double2* mult;
  const double2* G;       // forward source: columns
  uint16_t *hi, *lo;      // destination
  float* scale;           // [q][Mc * nact]
  int64_t qstride;        // operand elements per 16-map chunk
};

template <bool FWD>
__device__ __forceinline__ float prep_value(const PrepArgs& a, int mi, int ni, int m, int l0, int l0a, int j, int k,
                                            int map0) {
  const int bm = map0 + (j >> 1);
  if (bm >= a.B) return 0.f;
  if (FWD) {
    if (k >= a.nr) return 0.f;
    const double2 g = a.G[(((int64_t)bm * a.nact + ni) * a.nr + k) * a.Mc + mi];
    return to_f((j & 1) ? g.y : g.x);
  }
  const int l = l0a + k;
  if (l < l0 || l >= a.L) return 0.f;
  const double2 c = a.coef[(int64_t)bm * a.s_b + (int64_t)ni * a.s_n + (int64_t)l * a.s_l + (m - a.mlo_in)];
  const double2 u = a.mult[(int64_t)l * a.nact + ni];
  const float cx = to_f(c.x), cy = to_f(c.y), ux = to_f(u.x), uy = to_f(u.y);
  return (j & 1) ? fmaf(cx, uy, cy * ux) : fmaf(cx, ux, -cy * uy);
}

// block (m, n, 16-map chunk); 256 threads
template <bool FWD, bool FP16>
__global__ void k_tcp(PrepArgs a) {
  __shared__ float red[8];
  const int mi = blockIdx.x, ni = blockIdx.y, q = blockIdx.z, idx = mi * a.nact + ni;
  const int kl = a.kl[idx];
  if (kl == 0) return;
  const int m = a.mlo + mi, nn = a.nvals[ni];
  const int l0 = max(abs(m), abs(nn)), l0a = l0 & ~7;
  const int K = FWD ? a.Lk : kl;
  const int map0 = q * (kTcN / 2);
  float mx = 0.f;
  for (int e = threadIdx.x; e < kTcN * K; e += blockDim.x) {
    const int j = e / K, k = e - j * K;
    mx = fmaxf(mx, fabsf(prep_value<FWD>(a, mi, ni, m, l0, l0a, j, k, map0)));
  }
  const float s = pow2_scale_f(block_max_f(mx, red));
  if (threadIdx.x == 0) a.scale[(int64_t)q * a.Mc * a.nact + idx] = s;
  const int64_t base = (int64_t)q * a.qstride + (FWD ? (int64_t)idx * a.Lk * kTcN : a.off_i[idx] / a.Lb * kTcN);
  for (int e = threadIdx.x; e < kTcN * K; e += blockDim.x) {
    const int j = e / K, k = e - j * K;
    const float v = prep_value<FWD>(a, mi, ni, m, l0, l0a, j, k, map0) * s;
    put_pair<FP16>(a.hi, a.lo, base + (int64_t)(k / kKc) * kOpElems + tile_index(j, k % kKc), v);
  }
}

// The same in one pass over the source: each thread holds its kTcpVpt values in registers
// between the block maximum and the scaled write, and issues all of its loads before the first
// use (the sources are read with a stride of a whole row, so the two-pass form waited on one
// L2 or DRAM latency per value, twice).  MP = 2: a block prepares the operands of two adjacent
// m (thread pairs read the two neighbouring complex values of one 32-byte sector instead of one
// value per sector); thread t serves m0 + t % MP throughout.  TH * kTcpVpt >= MP * 32 K
// (host-checked).
constexpr int kTcpVpt = 32;
template <bool FWD, bool FP16, int TH, int MP>
__global__ void __launch_bounds__(TH) k_tcp1(PrepArgs a) {
  __shared__ float red[TH / 32][MP];
  __shared__ int kmax_s;
  const int ni = blockIdx.y, q = blockIdx.z, sub = threadIdx.x % MP;
  const int mi = blockIdx.x * MP + sub, nn = a.nvals[ni];
  int Kmax = 0;
#pragma unroll
  for (int s = 0; s < MP; ++s) {
    const int ms = blockIdx.x * MP + s;
    const int kls = ms < a.Mc ? a.kl[ms * a.nact + ni] : 0;
    Kmax = max(Kmax, kls == 0 ? 0 : (FWD ? a.Lk : kls));
  }
  if (Kmax == 0) return;
  const int idx = mi * a.nact + ni;
  const int kl = mi < a.Mc ? a.kl[idx] : 0;
  const int K = kl == 0 ? 0 : (FWD ? a.Lk : kl);   // this thread's m
  const int m = a.mlo + mi;
  const int l0 = max(abs(m), abs(nn)), l0a = l0 & ~7;
  const int map0 = q * (kTcN / 2);
  // value i of this thread is element e = tq + i TH/MP = j Kmax + k of its m; (j, k) are stepped
  // instead of divided (e < total exactly when j < kTcN)
  const int tq = threadIdx.x / MP, sj = (TH / MP) / Kmax, sk = (TH / MP) - sj * Kmax;
  float v[kTcpVpt];
  {
    int j = tq / Kmax, k = tq - j * Kmax;
#pragma unroll
    for (int i = 0; i < kTcpVpt; ++i) {
      v[i] = (j < kTcN && k < K) ? prep_value<FWD>(a, mi, ni, m, l0, l0a, j, k, map0) : 0.f;
      k += sk;
      j += sj;
      if (k >= Kmax) {
        k -= Kmax;
        ++j;
      }
    }
  }
  float mx = 0.f;
#pragma unroll
  for (int i = 0; i < kTcpVpt; ++i) mx = fmaxf(mx, fabsf(v[i]));
  for (int o = 16; o >= MP; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if ((threadIdx.x & 31) < MP) red[threadIdx.x >> 5][sub] = mx;
  if (threadIdx.x == 0) kmax_s = Kmax;
  __syncthreads();
  // the write loop recomputes its indices from the shared copy of the extent, so that the load
  // loop's addresses need not stay live across the barrier (they would double the registers)
  const int Kw = kmax_s, swj = (TH / MP) / Kw, swk = (TH / MP) - swj * Kw;
  float bm = red[0][sub];
  for (int w = 1; w < TH / 32; ++w) bm = fmaxf(bm, red[w][sub]);
  if (K == 0) return;
  const float sc = pow2_scale_f(bm);
  if (threadIdx.x < MP) a.scale[(int64_t)q * a.Mc * a.nact + idx] = sc;
  const int64_t base = (int64_t)q * a.qstride + (FWD ? (int64_t)idx * a.Lk * kTcN : a.off_i[idx] / a.Lb * kTcN);
  int j = tq / Kw, k = tq - j * Kw;
#pragma unroll
  for (int i = 0; i < kTcpVpt; ++i) {
    if (j < kTcN && k < K)
      put_pair<FP16>(a.hi, a.lo, base + (int64_t)(k / kKc) * kOpElems + tile_index(j, k % kKc), v[i] * sc);
    k += swk;
    j += swj;
    if (k >= Kw) {
      k -= Kw;
      ++j;
    }
  }
}

// operand preparation with the largest K extent kmax: the one-pass kernel where its registers
// hold a block's values (two m per block up to K = 256), else the two-pass one
template <bool FWD>
void launch_tcp(const PrepArgs& pa, int Mc, int nact, int nq, int kmax, bool fp16, cudaStream_t st) {
  const dim3 g1(Mc, nact, nq), g2((Mc + 1) / 2, nact, nq);
  if (2 * kTcN * kmax <= 256 * kTcpVpt) {
    if (fp16) k_tcp1<FWD, true, 256, 2><<<g2, 256, 0, st>>>(pa);
    else k_tcp1<FWD, false, 256, 2><<<g2, 256, 0, st>>>(pa);
  } else if (2 * kTcN * kmax <= 512 * kTcpVpt) {
    if (fp16) k_tcp1<FWD, true, 512, 2><<<g2, 512, 0, st>>>(pa);
    else k_tcp1<FWD, false, 512, 2><<<g2, 512, 0, st>>>(pa);
  } else if (kTcN * kmax <= 512 * kTcpVpt) {
    if (fp16) k_tcp1<FWD, true, 512, 1><<<g1, 512, 0, st>>>(pa);
    else k_tcp1<FWD, false, 512, 1><<<g1, 512, 0, st>>>(pa);
  } else {
    if (fp16) k_tcp<FWD, true><<<g1, 256, 0, st>>>(pa);
    else k_tcp<FWD, false><<<g1, 256, 0, st>>>(pa);
  }
}

// ------------------------------------------------------------------ GEMM
struct GemmArgs {
  const uint16_t *A_hi, *A_lo;
  const int64_t* off;     // table offsets (inverse off_i or forward off_f)
  const int64_t* off_i;   // inverse offsets (operand placement of the inverse)
  const int* kl;          // inverse: K extent; forward: row extent
  const uint16_t *B_hi, *B_lo;
  const float* scale;
  int64_t qstride;
  const int* nvals;
  int nact, L, nr, Lb, Lk, Mc, mlo, B;
  double2* G;             // inverse output
  const double2* mult;    // forward multiplier
  double2* out;           // forward output (accumulated)
  int64_t s_b, s_n, s_l;
  int mlo_out;
  uint32_t idesc, idesc2;   // N = 32 and N = 64 (the operand's hi and lo tiles side by side)
  int* err;
};

template <bool FWD>
__global__ void __launch_bounds__(kTcThreads) k_tc_gemm(GemmArgs a) {
  extern __shared__ __align__(1024) uint8_t smem[];
  __shared__ __align__(8) uint64_t bar_ld[2], bar_mma[2];
  __shared__ uint32_t tbase;
  const int rt = blockIdx.x, mi = blockIdx.y, ni = blockIdx.z, idx = mi * a.nact + ni;
  const int kl = a.kl[idx], L = a.L, nr = a.nr;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int m = a.mlo + mi, nn = a.nvals[ni];
  const int l0 = max(abs(m), abs(nn)), l0a = l0 & ~7;
  if (!FWD && kl == 0) {   // l0 >= L: this (m, n) column of every map is zero
    for (int e = tid; e < a.B * 128; e += kTcThreads) {
      const int b = e >> 7, beta = rt * 128 + (e & 127);
      if (beta < nr) a.G[(((int64_t)b * a.nact + ni) * nr + beta) * a.Mc + mi] = make_double2(0.0, 0.0);
    }
    return;
  }
  if (FWD && rt * 128 >= kl) return;
  const int K = FWD ? a.Lk : kl, nkc = K / kKc;
  // stage s at element offset s * (2 * kTileElems + 2 * kOpElems): A hi, A lo, B hi, B lo
  uint16_t* const stage0 = reinterpret_cast<uint16_t*>(smem);
  constexpr int kStageElems = 2 * kTileElems + 2 * kOpElems;
  if (tid == 0) {
    for (int s = 0; s < 2; ++s) {
      tc::mbar_init(&bar_ld[s], 1);
      tc::mbar_init(&bar_mma[s], 1);
    }
  }
  if (warp == 0) tc::tmem_alloc(&tbase, 64);   // hi*hi + lo*hi at columns 0..31, hi*lo at 32..63
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = tbase;
  const int64_t aoff = a.off[idx] + (int64_t)rt * nkc * kTileElems;
  const int64_t boff = FWD ? (int64_t)idx * a.Lk * kTcN : a.off_i[idx] / a.Lb * kTcN;
  const uint32_t stage_bytes = (uint32_t)kStageElems * 2u;
  uint32_t ph_ld[2] = {0u, 0u}, ph_mma[2] = {0u, 0u};
  bool ok = true;
  for (int map0 = 0, q = 0; map0 < a.B && ok; map0 += kTcN / 2, ++q) {
    if (tid == 0) {
      const uint16_t* bh = a.B_hi + (int64_t)q * a.qstride + boff;
      const uint16_t* bl = a.B_lo + (int64_t)q * a.qstride + boff;
      auto load = [&](int c, int s) {
        uint16_t* S = stage0 + s * kStageElems;
        tc::mbar_expect_tx(&bar_ld[s], stage_bytes);
        tc::bulk_g2s(S, a.A_hi + aoff + (int64_t)c * kTileElems, kTileElems * 2u, &bar_ld[s]);
        tc::bulk_g2s(S + kTileElems, a.A_lo + aoff + (int64_t)c * kTileElems, kTileElems * 2u, &bar_ld[s]);
        tc::bulk_g2s(S + 2 * kTileElems, bh + (int64_t)c * kOpElems, kOpElems * 2u, &bar_ld[s]);
        tc::bulk_g2s(S + 2 * kTileElems + kOpElems, bl + (int64_t)c * kOpElems, kOpElems * 2u, &bar_ld[s]);
      };
      auto wait = [&](uint64_t* bar, uint32_t& ph) {
        if (!ok) return;
        if (!tc::mbar_wait(bar, ph, kWaitIter)) {
          atomicExch(a.err, (int)S2W_ETIMEOUT);
          ok = false;
          return;
        }
        ph ^= 1u;
      };
      load(0, 0);
      for (int c = 0; c < nkc && ok; ++c) {
        const int s = c & 1;
        wait(&bar_ld[s], ph_ld[s]);
        if (!ok) break;
        tc::fence_after_sync();
        const uint32_t A0 = tc::smem_u32(stage0 + s * kStageElems), A1 = A0 + kTileElems * 2u;
        const uint32_t B0 = A1 + kTileElems * 2u;   // operand hi, then lo one 32-row block further
        for (int ks = 0; ks < kKc / 16; ++ks) {
          const uint32_t o = (uint32_t)ks * 256u;
          const uint32_t acc = (c > 0 || ks > 0) ? 1u : 0u;
          // the operand's hi and lo tiles are adjacent 32-row blocks with one row-group stride: one
          // N = 64 MMA of the table's hi against both (hi*hi into columns 0..31, hi*lo into 32..63),
          // then lo*hi into columns 0..31; the epilogue adds the two halves
          tc::mma_f16(tmem, tc::make_sdesc(A0 + o, 128, kSbo), tc::make_sdesc(B0 + o, 128, kSbo), a.idesc2, acc);
          tc::mma_f16(tmem, tc::make_sdesc(A1 + o, 128, kSbo), tc::make_sdesc(B0 + o, 128, kSbo), a.idesc, 1);
        }
        tc::mma_commit(&bar_mma[s]);
        if (c + 1 < nkc) {
          if (c >= 1) wait(&bar_mma[s ^ 1], ph_mma[s ^ 1]);   // chunk c-1 no longer reads stage s^1
          if (!ok) break;
          load(c + 1, s ^ 1);
        }
      }
      // the MMAs of the last two chunks
      for (int c = nkc >= 2 ? nkc - 2 : 0; c < nkc; ++c) wait(&bar_mma[c & 1], ph_mma[c & 1]);
    }
    ok = __syncthreads_and(ok);
    if (!ok) break;
    tc::fence_after_sync();
    float v[32], w[32];
    tc::tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16), v);
    tc::tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + 32u, w);
#pragma unroll
    for (int j = 0; j < 32; ++j) v[j] += w[j];
    const float sc = a.scale[(int64_t)q * a.Mc * a.nact + idx];
    const float un = 1.f / (sc * (float)(FWD ? kFwdScale : kInvScale));   // a power of two
    const int row = rt * 128 + warp * 32 + lane;
    if (!FWD) {
      if (row < nr) {
#pragma unroll
        for (int p = 0; p < kTcN / 2; ++p) {
          const int bm = map0 + p;
          if (bm < a.B)
            a.G[(((int64_t)bm * a.nact + ni) * nr + row) * a.Mc + mi] = make_double2(f2d(v[2 * p] * un), f2d(v[2 * p + 1] * un));
        }
      }
    } else {
      const int l = l0a + row;
      if (l >= l0 && l < L) {
        const double2 mu = a.mult[(int64_t)l * a.nact + ni];
#pragma unroll
        for (int p = 0; p < kTcN / 2; ++p) {
          const int bm = map0 + p;
          if (bm >= a.B) break;
          const double re = f2d(v[2 * p] * un), im = f2d(v[2 * p + 1] * un);
          double2* o = a.out + (int64_t)bm * a.s_b + (int64_t)ni * a.s_n + (int64_t)l * a.s_l + (m - a.mlo_out);
          atomicAdd(&o->x, fma(re, mu.x, -im * mu.y));
          atomicAdd(&o->y, fma(re, mu.y, im * mu.x));
        }
      }
    }
    tc::fence_before_sync();
    __syncthreads();   // TMEM is rewritten by the next map chunk
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tmem, 64);
}

constexpr size_t kGemmSmem = 2 * (2 * kTileElems + 2 * kOpElems) * sizeof(uint16_t);   // 40 KB

PrepArgs prep_args(const s2w_plan* P, const TransformSpec& t, const TcTable& tab, int nr, int Mc, int mlo, int B) {
  PrepArgs a{};
  a.nvals = t.nvals;
  a.nact = t.nact;
  a.L = t.L;
  a.nr = nr;
  a.Mc = Mc;
  a.mlo = mlo;
  a.B = B;
  a.off_i = tab.off_i;
  a.Lb = tab.Lb;
  a.Lk = tab.Lk;
  a.hi = P->tc_b_hi;
  a.lo = P->tc_b_lo;
  a.scale = P->tc_scale;
  return a;
}

GemmArgs gemm_args(const s2w_plan* P, const TransformSpec& t, const TcTable& tab, int nr, int Mc, int mlo, int B,
                   bool fp16) {
  GemmArgs a{};
  a.nr = nr;
  a.off_i = tab.off_i;
  a.B_hi = P->tc_b_hi;
  a.B_lo = P->tc_b_lo;
  a.scale = P->tc_scale;
  a.nvals = t.nvals;
  a.nact = t.nact;
  a.L = t.L;
  a.Lb = tab.Lb;
  a.Lk = tab.Lk;
  a.Mc = Mc;
  a.mlo = mlo;
  a.B = B;
  a.idesc = tc::make_idesc(128, kTcN, fp16 ? 0 : 1, 0, 0);
  a.idesc2 = tc::make_idesc(128, 2 * kTcN, fp16 ? 0 : 1, 0, 0);
  a.err = P->err_word;
  return a;
}

}  // namespace

cudaError_t launch_tc_pack(const TransformSpec& t, const TcTable& tab, const TabTable& src, int nr, int Mc, int mlo,
                           bool fp16, cudaStream_t st) {
  PackArgs a;
  a.nvals = t.nvals;
  a.nact = t.nact;
  a.L = t.L;
  a.nr = nr;
  a.Mc = Mc;
  a.mlo = mlo;
  a.toff_i = src.off_inv;
  a.toff_f = src.off_fwd;
  a.tkp = src.kp;
  a.tLp = src.Lp;
  a.tLk = src.Lk;
  a.tinv = src.inv;
  a.tfwd = src.fwd;
  a.off_i = tab.off_i;
  a.off_f = tab.off_f;
  a.kli = tab.kli;
  a.klf = tab.klf;
  a.Lb = tab.Lb;
  a.Lk = tab.Lk;
  a.inv_hi = tab.inv_hi;
  a.inv_lo = tab.inv_lo;
  a.fwd_hi = tab.fwd_hi;
  a.fwd_lo = tab.fwd_lo;
  dim3 grid(Mc, t.nact);
  if (fp16) k_tc_pack<true><<<grid, 256, 0, st>>>(a);
  else k_tc_pack<false><<<grid, 256, 0, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_tc_inverse(const s2w_plan* P, const GridTables& g, const TransformSpec& t, CoefArgs in,
                              ColumnArgs out, cudaStream_t st) {
  (void)g;
  const TcTable& tab = *t.tc;
  const bool fp16 = P->p.precision == S2W_FP32_SPLIT;
  const int nq = (out.B + kTcN / 2 - 1) / (kTcN / 2);
  PrepArgs pa = prep_args(P, t, tab, out.nr, out.Mc, out.mlo, out.B);
  pa.kl = tab.kli;
  pa.coef = in.coef;
  pa.s_b = in.s_b;
  pa.s_n = in.s_n;
  pa.s_l = in.s_l;
  pa.mlo_in = in.mlo;
  pa.mult = t.mult_inv;
  pa.qstride = tab.op_i;
  launch_tcp<false>(pa, out.Mc, t.nact, nq, (t.L + 63) / 64 * 64, fp16, st);   // inverse K extents: at most L rounded up to 64
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  GemmArgs a = gemm_args(P, t, tab, out.nr, out.Mc, out.mlo, out.B, fp16);
  a.A_hi = tab.inv_hi;
  a.A_lo = tab.inv_lo;
  a.off = tab.off_i;
  a.kl = tab.kli;
  a.qstride = tab.op_i;
  a.G = out.G;
  e = cudaFuncSetAttribute(k_tc_gemm<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kGemmSmem);
  if (e != cudaSuccess) return e;
  dim3 grid(tab.Lb / 128, out.Mc, t.nact);
  k_tc_gemm<false><<<grid, kTcThreads, kGemmSmem, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_tc_forward(const s2w_plan* P, const GridTables& g, const TransformSpec& t, ColumnArgs in,
                              CoefArgs out, cudaStream_t st) {
  (void)g;
  const TcTable& tab = *t.tc;
  const bool fp16 = P->p.precision == S2W_FP32_SPLIT;
  const int nq = (in.B + kTcN / 2 - 1) / (kTcN / 2);
  PrepArgs pa = prep_args(P, t, tab, in.nr, in.Mc, in.mlo, in.B);
  pa.kl = tab.klf;
  pa.G = in.G;
  pa.qstride = tab.op_f;
  launch_tcp<true>(pa, in.Mc, t.nact, nq, tab.Lk, fp16, st);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  GemmArgs a = gemm_args(P, t, tab, in.nr, in.Mc, in.mlo, in.B, fp16);
  a.A_hi = tab.fwd_hi;
  a.A_lo = tab.fwd_lo;
  a.off = tab.off_f;
  a.kl = tab.klf;
  a.qstride = tab.op_f;
  a.mult = t.mult_fwd;
  a.out = const_cast<double2*>(out.coef);
  a.s_b = out.s_b;
  a.s_n = out.s_n;
  a.s_l = out.s_l;
  a.mlo_out = out.mlo;
  e = cudaFuncSetAttribute(k_tc_gemm<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kGemmSmem);
  if (e != cudaSuccess) return e;
  dim3 grid(tab.klf_max / 128, in.Mc, t.nact);
  k_tc_gemm<true><<<grid, kTcThreads, kGemmSmem, st>>>(a);
  return cudaGetLastError();
}

}  // namespace s2w

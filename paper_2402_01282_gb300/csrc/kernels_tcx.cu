// Float64-accurate l-contractions on the 5th-generation tensor cores (S2W_FP64_TC) by exact
// integer slicing of both operands (the error-free splitting of Ozaki, Ogita, Oishi and Rump,
// "Error-free transformations of matrix multiplication by using fast routines of matrix
// multiplication and its applications", Numer. Algorithms 59, 2012).
//
// Slicing.  Every value v of a table row or of a data column, whose row/column exponent e
// bounds it (max |v| < 2^e), is rounded to the fixed-point integer X = round(v 2^(47 - e)),
// |X| < 2^47, and X is written as seven balanced base-128 digits s_0..s_6 in [-64, 63]
// (X = sum_i s_i 128^(6 - i), s_0 most significant).  Digits are exact in bf16 and the
// product of two digits (|s t| <= 2^12) is exact in the MMA.
//
// Exact accumulation.  The pairs (i, i') of slices with i + i' = q (q = 0..6, 28 pairs) are
// summed into one float32 TMEM accumulator D_q: over K <= 512 reduction terms one pair sums
// to |.| <= 2^21 and at most seven pairs share an accumulator, so every partial sum is an
// integer below 2^24 and float32 holds it exactly, whatever the order of the additions.  The
// six pairs of diagonal 7 can reach ~2^-44 of a term together, above the operands' own 47-bit
// rounding: they are summed where the plan asks for it (the ball's sphere plans), else dropped
// with the pairs i + i' >= 8 (below ~2^-51).  Then
//   C[r][j] = 2^(e_r + f_j - 10) sum_q 2^(-7 q) D_q[r][j]
// (e_r: table row exponent, f_j: data column exponent), summed from the smallest weight up in
// compensated float32 and converted to float64: each output carries ~2^-44 (2^-47 with diagonal
// 7) of max_k|A[r][k]| max_k|B[k][j]| per reduction term, the float64 accuracy class of the
// rest of the path.
//
// The GEMMs are those of the reduced modes (one per (m, n), 128-row tiles, 32 columns = 16
// maps x re/im): inverse rows beta, K = l (tables d^l_mn(beta)); forward rows l, K = beta'
// (tables with the colatitude quadrature folded in).  Layouts, K chunks of 16, seven slices
// contiguous per chunk (core matrices of 8 x 8 16-bit elements, K-major, no swizzle):
//   table  (row tile t, chunk c, slice s): element (r, k) at
//          ((t nkc + c) 7 + s) 2048 + ((r/8) 2 + k/8) 64 + (r%8) 8 + k%8
//   data   (chunk c, slice s): element (j, k) at (c 7 + s) 512 + ((j/8) 2 + k/8) 64 + (j%8) 8 + k%8
// k_tcx_gemm: one CTA of 128 threads per (row tile, m, n); thread 0 drives a three-stage
// pipeline of bulk copies (35 KB per stage: 7 table slices + 7 data slices) and seven MMAs per
// chunk (one per table slice, N = 224 .. 32 over the data slices side by side: the 28 pairs; 8
// MMAs for the 34 with diagonal 7); 105 KB of shared memory and 256 TMEM columns per CTA let two CTAs share an SM; every
// mbarrier wait is bounded and a timeout sets the plan's error word.
#include "comp32.cuh"
#include "s2w_internal.h"
#include "tc_sm100.cuh"
#include "slice7.cuh"

namespace s2w {
namespace {

constexpr int kThreads = 128;
constexpr int kN = 32;                         // MMA N: 16 maps x (re, im)
constexpr int kKc = 16;                        // K chunk (one MMA deep)
constexpr int kATile = 128 * kKc;              // elements of one table slice chunk
constexpr int kBTile = kN * kKc;               // elements of one data slice chunk
constexpr int kAChunk = kSl * kATile;          // 14336
constexpr int kBChunk = kSl * kBTile;          // 3584
constexpr int kStageElems = kAChunk + kBChunk;
constexpr int kStages = 3;
constexpr size_t kSmem = (size_t)kStages * kStageElems * sizeof(uint16_t);   // 107520 B
constexpr uint32_t kWaitIter = 1u << 20;   // bounded mbarrier polls (far above any legitimate wait)
constexpr uint32_t kInjectIter = 1u << 10;  // polls of the injected wait (s2w_plan_inject_timeout)
constexpr int kTmemCols = 256;                 // 8 accumulators x 32 columns


// ------------------------------------------------------------------ table packing (plan time)
struct PackArgs {
  const int* nvals;
  int nact, L, nr, Mc, mlo, lmin;
  const int64_t *toff_i, *toff_f;   // float-pair tables (kernels_tab.cu layout)
  const int* tkp;
  int tLp;
  const float2 *tinv, *tfwd;
  const int64_t *off_i, *off_f;
  const int *kli, *klf;
  int Lb, Lk, klf_max;
  int *rexp_i, *rexp_f;
  uint16_t *inv, *fwd;
};

// block (m, n), one thread per table row
__global__ void k_tcx_pack(PackArgs a) {
  const int mi = blockIdx.x, ni = blockIdx.y, idx = mi * a.nact + ni;
  const int kli = a.kli[idx], klf = a.klf[idx];
  if (kli == 0) return;
  const int m = a.mlo + mi, nn = a.nvals[ni], L = a.L;
  const int l0 = max(abs(m), abs(nn)), l0s = l0 & ~7;   // the float-pair tables start at l0s
  const int lb = max(l0, a.lmin), la = lb & ~7;         // the sliced tables at la
  const int kp = a.tkp[idx];
  const float2* Ti = a.tinv + a.toff_i[idx];   // [kp][tLp]
  const float2* Tf = a.tfwd + a.toff_f[idx];   // [tLk][kp]
  // inverse: rows beta, K = l - la
  const int nkci = kli / kKc;
  for (int r = threadIdx.x; r < a.Lb; r += blockDim.x) {
    auto val = [&](int k) -> double {
      const int l = la + k, ks = l - l0s;
      if (r >= a.nr || l < lb || l >= L || ks >= kp) return 0.0;
      const float2 p = Ti[(int64_t)ks * a.tLp + r];
      return (double)p.x + (double)p.y;
    };
    int eb = 0;
    for (int k = 0; k < kli; ++k) eb = max(eb, ebound(val(k)));
    const int e = e_from(eb);
    a.rexp_i[(int64_t)idx * a.Lb + r] = e;
    uint32_t d[kSl];
    for (int k = 0; k < kli; ++k) {
      digits7(fix47(val(k), e), d);
      const int64_t o = a.off_i[idx] + ((int64_t)(r >> 7) * nkci + (k >> 4)) * kAChunk + core16(r & 127, k & 15);
#pragma unroll
      for (int s = 0; s < kSl; ++s) a.inv[o + (int64_t)s * kATile] = (uint16_t)(d[s] >> 16);
    }
  }
  // forward: rows l - la, K = beta'
  const int nkcf = a.Lk / kKc;
  for (int r = threadIdx.x; r < klf; r += blockDim.x) {
    const int l = la + r, rs = l - l0s;
    auto val = [&](int k) -> double {
      if (k >= a.nr || l < lb || l >= L || rs >= kp) return 0.0;
      const float2 p = Tf[(int64_t)k * kp + rs];
      return (double)p.x + (double)p.y;
    };
    int eb = 0;
    for (int k = 0; k < a.Lk; ++k) eb = max(eb, ebound(val(k)));
    const int e = e_from(eb);
    a.rexp_f[(int64_t)idx * a.klf_max + r] = e;
    uint32_t d[kSl];
    for (int k = 0; k < a.Lk; ++k) {
      digits7(fix47(val(k), e), d);
      const int64_t o = a.off_f[idx] + ((int64_t)(r >> 7) * nkcf + (k >> 4)) * kAChunk + core16(r & 127, k & 15);
#pragma unroll
      for (int s = 0; s < kSl; ++s) a.fwd[o + (int64_t)s * kATile] = (uint16_t)(d[s] >> 16);
    }
  }
}

// ------------------------------------------------------------------ data slicing (every call)
struct PrepArgs {
  const int* nvals;
  int nact, L, nr, Mc, mlo, B, lmin;
  const int* kl;             // inverse: K extent (0 = empty); forward: row extent (0 = empty)
  const int64_t* opoff_i;    // inverse: operand offset of (m, n) within a 16-map chunk
  int Lk;
  const double2* coef;       // inverse source
  int64_t s_b, s_n, s_l;
  int mlo_in;
  const double* mult_r;      // inverse: real multiplier (factored) ...
  const double2* mult;       // ... or the full complex one (mult_r == nullptr)
  const double2* G;          // forward source: columns [B][nact][nr][Mc]
  uint16_t* ops;             // destination slices
  int* fexp;                 // [q][Mc * nact][32] column exponent bounds (+ kEOff; 0 = zero column)
  int64_t qstride;           // operand elements per 16-map chunk
  int* err;                  // plan error word: k_tcxe records S2W_ENONFINITE for a NaN or Inf value
};

// Source of the data operand at reduction index k of column (mi, ni) for map bm: the pair
// (re, im) and, for the inverse with a factored multiplier, the real factor r (value = pair r);
// otherwise r = 1 and the pair is the value.  Zero outside the data.
template <bool FWD>
__device__ __forceinline__ double2 prep_pair(const PrepArgs& a, int mi, int ni, int m, int l0, int l0a, int bm,
                                             int k, double& r) {
  r = 1.0;
  if (bm >= a.B) return make_double2(0.0, 0.0);
  if (FWD) {
    if (k >= a.nr) return make_double2(0.0, 0.0);
    return a.G[(((int64_t)bm * a.nact + ni) * a.nr + k) * a.Mc + mi];
  }
  const int l = l0a + k;
  if (l < l0 || l >= a.L) return make_double2(0.0, 0.0);
  const double2 c = a.coef[(int64_t)bm * a.s_b + (int64_t)ni * a.s_n + (int64_t)l * a.s_l + (m - a.mlo_in)];
  if (a.mult_r != nullptr) {
    r = a.mult_r[(int64_t)l * a.nact + ni];
    return c;
  }
  const double2 u = a.mult[(int64_t)l * a.nact + ni];
  return make_double2(fma(c.x, u.x, -c.y * u.y), fma(c.x, u.y, c.y * u.x));
}

// Two passes over the data, each a grid of blocks (8 consecutive m, n, 16-map chunk, 64-wide
// slice of K) of 256 threads, so that every block does the same short amount of work whatever
// the K extent of its m.  Work item (m, map, group of 8 reduction indices): the 8 m of a group
// read 128 contiguous bytes per (map, k).
//   k_tcxe: column exponent bounds (for a product c r the bound of |c| |r|), reduced in
//           registers, then shared memory, then one global atomicMax per column and block into
//           fexp (zeroed before; 0 = zero column, else exponent + kEOff);
//   k_tcxs: the seven slices, the product c r formed in the integer domain; the slices of 8
//           consecutive k of one column form one 16-byte row of a core matrix (one vector store
//           per slice).
constexpr int kPrepM = 8;
constexpr int kPrepK = 16;   // reduction indices per block (two or more waves of blocks at the top scales)

template <bool FWD>
__global__ void __launch_bounds__(256) k_tcxe(PrepArgs a, int ks_n) {
  __shared__ int colE[kPrepM][kN];
  const int mi0 = blockIdx.x * kPrepM, ni = blockIdx.y, q = blockIdx.z / ks_n, ks = blockIdx.z % ks_n;
  const int t = threadIdx.x, ml = t % kPrepM, p = (t / kPrepM) % (kN / 2), kg0 = t / (kPrepM * kN / 2);
  constexpr int kGStride = 256 / (kPrepM * kN / 2);
  const int mi = mi0 + ml;
  const int idx = mi * a.nact + ni;
  const bool live = mi < a.Mc && a.kl[min(idx, a.Mc * a.nact - 1)] != 0;
  const int m = a.mlo + mi, nn = a.nvals[ni];
  const int l0 = max(max(abs(m), abs(nn)), a.lmin), l0a = l0 & ~7;   // first l with a nonzero term
  const int K = live ? min(FWD ? a.Lk : a.kl[idx], (ks + 1) * kPrepK) : 0;
  const int bm = q * (kN / 2) + p;
  colE[t / kN][t % kN] = 0;
  __syncthreads();
  int er = 0, ei = 0;
  bool bad = false;   // a NaN or Inf (exponent field all ones) among the values read
  for (int kg = ks * (kPrepK / 8) + kg0; kg * 8 < K; kg += kGStride) {
    double2 v[8];
    double r[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) v[u] = prep_pair<FWD>(a, mi, ni, m, l0, l0a, bm, kg * 8 + u, r[u]);
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      er = max(er, ebound_prod(v[u].x, r[u]));
      ei = max(ei, ebound_prod(v[u].y, r[u]));
      bad |= (bexp(v[u].x) == 0x7FF) | (bexp(v[u].y) == 0x7FF) | (bexp(r[u]) == 0x7FF);
    }
  }
  if (bad) atomicCAS(a.err, 0, (int)S2W_ENONFINITE);   // the first recorded status is kept
  if (er > 0) atomicMax(&colE[ml][2 * p], er);
  if (ei > 0) atomicMax(&colE[ml][2 * p + 1], ei);
  __syncthreads();
  const int j = t % kN, mj = t / kN;   // one thread per (m, column)
  const int idxj = (mi0 + mj) * a.nact + ni;
  if (mi0 + mj < a.Mc && colE[mj][j] > 0)
    atomicMax(a.fexp + ((int64_t)q * a.Mc * a.nact + idxj) * kN + j, colE[mj][j]);
}

template <bool FWD>
__global__ void __launch_bounds__(256) k_tcxs(PrepArgs a, int ks_n) {
  const int mi0 = blockIdx.x * kPrepM, ni = blockIdx.y, q = blockIdx.z / ks_n, ks = blockIdx.z % ks_n;
  const int t = threadIdx.x, ml = t % kPrepM, p = (t / kPrepM) % (kN / 2), kg0 = t / (kPrepM * kN / 2);
  constexpr int kGStride = 256 / (kPrepM * kN / 2);
  const int mi = mi0 + ml;
  if (mi >= a.Mc) return;
  const int idx = mi * a.nact + ni;
  if (a.kl[idx] == 0) return;
  const int m = a.mlo + mi, nn = a.nvals[ni];
  const int l0 = max(max(abs(m), abs(nn)), a.lmin), l0a = l0 & ~7;   // first l with a nonzero term
  const int K = min(FWD ? a.Lk : a.kl[idx], (ks + 1) * kPrepK);
  const int bm = q * (kN / 2) + p;
  const int* fx = a.fexp + ((int64_t)q * a.Mc * a.nact + idx) * kN;
  const int fr = e_from(fx[2 * p]), fi = e_from(fx[2 * p + 1]);
  const int64_t base = (int64_t)q * a.qstride + (FWD ? (int64_t)idx * a.Lk * kN * kSl : a.opoff_i[idx]);
  const int jr = 2 * p, ji = 2 * p + 1;
  for (int kg = ks * (kPrepK / 8) + kg0; kg * 8 < K; kg += kGStride) {
    double2 v[8];
    double rr[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) v[u] = prep_pair<FWD>(a, mi, ni, m, l0, l0a, bm, kg * 8 + u, rr[u]);
    uint32_t wr[kSl][4], wi[kSl][4];
#pragma unroll
    for (int u = 0; u < 8; u += 2) {
      uint32_t d0[kSl], d1[kSl], e0[kSl], e1[kSl];
      digits7(fix47_prod(v[u].x, rr[u], fr), d0);
      digits7(fix47_prod(v[u + 1].x, rr[u + 1], fr), d1);
      digits7(fix47_prod(v[u].y, rr[u], fi), e0);
      digits7(fix47_prod(v[u + 1].y, rr[u + 1], fi), e1);
#pragma unroll
      for (int sl = 0; sl < kSl; ++sl) {
        wr[sl][u / 2] = __byte_perm(d0[sl], d1[sl], 0x7632);   // bf16(k+u) | bf16(k+u+1) << 16
        wi[sl][u / 2] = __byte_perm(e0[sl], e1[sl], 0x7632);
      }
    }
    const int k = kg * 8;
    // element (j, k..k+7) of chunk k/16: one 16-byte core-matrix row per slice
    const int64_t o = base + (int64_t)(k >> 4) * kBChunk + ((k & 15) >> 3) * 64;
#pragma unroll
    for (int sl = 0; sl < kSl; ++sl) {
      *reinterpret_cast<uint4*>(a.ops + o + (int64_t)sl * kBTile + (jr >> 3) * 128 + (jr & 7) * 8) =
          make_uint4(wr[sl][0], wr[sl][1], wr[sl][2], wr[sl][3]);
      *reinterpret_cast<uint4*>(a.ops + o + (int64_t)sl * kBTile + (ji >> 3) * 128 + (ji & 7) * 8) =
          make_uint4(wi[sl][0], wi[sl][1], wi[sl][2], wi[sl][3]);
    }
  }
}

// ------------------------------------------------------------------ GEMM
struct GemmArgs {
  const uint16_t* A;
  const int64_t* off;       // table offsets (inverse off_i or forward off_f)
  const int* kl;            // inverse: K extent; forward: row extent
  const int* rexp;          // row exponents
  int rstride;              // rows per (m, n) in rexp (Lb or klf_max)
  const int64_t* opoff_i;   // inverse operand offsets
  const uint16_t* ops;
  const int* fexp;
  int64_t qstride;
  const int* nvals;
  int nact, L, nr, Lk, Mc, mlo, B, lmin;
  double2* G;               // inverse output
  int phase_mode;           // inverse: 0 general, 1: +1, 2: -1, 3: +i, 4: -i
  double2 phase;
  const double2* mult;      // forward multiplier
  double2* out;             // forward output (accumulated)
  int64_t s_b, s_n, s_l;
  int mlo_out;
  uint32_t idesc;
  int* err;
  int inject_timeout;       // test hook (s2w_plan_inject_timeout): make a bounded wait run out
  int ndiag;                // digit-pair diagonals summed: 7 (28 pairs per K step) or 8 (34)
};

template <bool FWD>
__global__ void __launch_bounds__(kThreads) k_tcx_gemm(GemmArgs a) {
  extern __shared__ __align__(1024) uint8_t smem[];
  __shared__ __align__(8) uint64_t bar_ld[kStages], bar_mma[kStages], bar_never;
  __shared__ uint32_t tbase;
  __shared__ int fexp_s[kN];
  const int rt = blockIdx.x, mi = blockIdx.y, ni = blockIdx.z, idx = mi * a.nact + ni;
  const int kl = a.kl[idx], L = a.L, nr = a.nr;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int m = a.mlo + mi, nn = a.nvals[ni];
  const int l0 = max(max(abs(m), abs(nn)), a.lmin), l0a = l0 & ~7;   // first l with a nonzero term
  if (!FWD && kl == 0) {   // l0 >= L: this (m, n) column of every map is zero
    for (int e = tid; e < a.B * 128; e += kThreads) {
      const int b = e >> 7, beta = rt * 128 + (e & 127);
      if (beta < nr) a.G[(((int64_t)b * a.nact + ni) * nr + beta) * a.Mc + mi] = make_double2(0.0, 0.0);
    }
    return;
  }
  if (FWD && rt * 128 >= kl) return;
  const int K = FWD ? a.Lk : kl, nkc = K / kKc;
  uint16_t* const stage0 = reinterpret_cast<uint16_t*>(smem);
  if (tid == 0) {
    for (int s = 0; s < kStages; ++s) {
      tc::mbar_init(&bar_ld[s], 1);
      tc::mbar_init(&bar_mma[s], 1);
    }
    tc::mbar_init(&bar_never, 1);   // nothing arrives on it: the injected timeout waits here
  }
  if (warp == 0) tc::tmem_alloc(&tbase, kTmemCols);
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = tbase;
  const int64_t aoff = a.off[idx] + (int64_t)rt * nkc * kAChunk;
  const int64_t boff = FWD ? (int64_t)idx * a.Lk * kN * kSl : a.opoff_i[idx];
  constexpr uint32_t stage_bytes = (uint32_t)kStageElems * 2u;
  uint32_t ph_ld[kStages] = {0u, 0u, 0u}, ph_mma[kStages] = {0u, 0u, 0u};
  unsigned pend_ld = 0u, pend_mma = 0u;   // thread 0: stages with copies / MMAs not yet waited for
  const int row = rt * 128 + warp * 32 + lane;
  const int e_r = a.rexp[(int64_t)idx * a.rstride + row];
  bool ok = true;
  for (int map0 = 0, q = 0; map0 < a.B && ok; map0 += kN / 2, ++q) {
    if (tid < kN) fexp_s[tid] = e_from(a.fexp[((int64_t)q * a.Mc * a.nact + idx) * kN + tid]);
    if (tid == 0) {
      const uint16_t* bq = a.ops + (int64_t)q * a.qstride + boff;
      auto load = [&](int c, int s) {
        uint16_t* S = stage0 + s * kStageElems;
        tc::mbar_expect_tx(&bar_ld[s], stage_bytes);
        tc::bulk_g2s(S, a.A + aoff + (int64_t)c * kAChunk, kAChunk * 2u, &bar_ld[s]);
        tc::bulk_g2s(S + kAChunk, bq + (int64_t)c * kBChunk, kBChunk * 2u, &bar_ld[s]);
        pend_ld |= 1u << s;
      };
      // bounded wait; `bit` marks the stage's pending copies (pend_ld) or MMAs (pend_mma)
      auto wait = [&](uint64_t* bar, uint32_t& ph, unsigned& pend, int s) {
        if (!ok) return;
        if (!tc::mbar_wait(bar, ph, kWaitIter)) {
          atomicExch(a.err, (int)S2W_ETIMEOUT);
          ok = false;
          return;
        }
        ph ^= 1u;
        pend &= ~(1u << s);
      };
      for (int c = 0; c < kStages - 1 && c < nkc; ++c) load(c, c);
      if (a.inject_timeout && q == 0 && !tc::mbar_wait(&bar_never, 0u, kInjectIter)) {
        // injected failure: a wait that nothing completes runs out (after a short poll limit, so
        // that a test does not wait for the full one) with copies in flight, and the timeout path
        // below (error word, settling the copies, freeing TMEM) is the one exercised
        atomicExch(a.err, (int)S2W_ETIMEOUT);
        ok = false;
      }
      for (int c = 0; c < nkc && ok; ++c) {
        const int s = c % kStages;
        wait(&bar_ld[s], ph_ld[s], pend_ld, s);
        if (!ok) break;
        tc::fence_after_sync();
        const uint32_t A0 = tc::smem_u32(stage0 + s * kStageElems), B0 = A0 + kAChunk * 2u;
        // the slice operands of a stage differ only in their start address: descriptors by
        // offset (address field = byte address / 16)
        const uint64_t dA = tc::make_sdesc(A0, 128, 256), dB = tc::make_sdesc(B0, 128, 256);
        const uint32_t acc0 = c > 0 ? 1u : 0u;
        // One MMA per table slice sa against the data slices 0 .. 6 - sa side by side: the data
        // slices of a chunk are contiguous 32-row blocks with one row-group stride, so they form one
        // N = 32 (7 - sa) operand, and pair (sa, sb) lands in accumulator sa + sb at TMEM columns
        // 32 (sa + sb).  Seven MMAs per K chunk read each table slice once (the 28 pairs, exactly).
        // Diagonal 7 (ndiag = 8): slices sa >= 2 take one more data slice (7 - sa); pair (1, 6)
        // goes first, alone, so that it initialises accumulator 7 at the first chunk.
        const bool d7 = a.ndiag > kSl;   // uniform
#pragma unroll
        for (int sa = 0; sa < kSl; ++sa) {
          const uint64_t dAs = dA + (uint64_t)(sa * (kATile * 2 / 16));
          if (d7 && sa == 1)
            tc::mma_f16(tmem + (uint32_t)(32 * kSl), dAs, dB + (uint64_t)((kSl - 1) * (kBTile * 2 / 16)),
                        tc::make_idesc(128, kN, 1, 0, 0), acc0);
          const int nb = kSl - sa + ((d7 && sa >= 2) ? 1 : 0);
          tc::mma_f16(tmem + (uint32_t)(32 * sa), dAs, dB, tc::make_idesc(128, kN * nb, 1, 0, 0), sa > 0 ? 1u : acc0);
        }
        tc::mma_commit(&bar_mma[s]);
        pend_mma |= 1u << s;
        if (c + kStages - 1 < nkc) {
          // the stage of chunk c + 2 last held chunk c - 1: its MMAs must be done
          const int sn = (c + kStages - 1) % kStages;
          if (c >= 1) wait(&bar_mma[sn], ph_mma[sn], pend_mma, sn);
          if (!ok) break;
          load(c + kStages - 1, sn);
        }
      }
      // the MMAs still outstanding: chunks max(0, nkc - 3) .. nkc - 1 (every earlier chunk was
      // waited for before its stage was reloaded)
      for (int c = nkc > kStages ? nkc - kStages : 0; c < nkc && ok; ++c)
        wait(&bar_mma[c % kStages], ph_mma[c % kStages], pend_mma, c % kStages);
      if (!ok) {
        // after a timeout: let this CTA's own copies and MMAs in flight land (bounded) before
        // the CTA frees its TMEM and exits
        for (int s = 0; s < kStages; ++s) {
          if (pend_ld & (1u << s)) tc::mbar_wait(&bar_ld[s], ph_ld[s], kWaitIter);
          if (pend_mma & (1u << s)) tc::mbar_wait(&bar_mma[s], ph_mma[s], kWaitIter);
        }
      }
    }
    ok = __syncthreads_and(ok);
    if (!ok) break;
    tc::fence_after_sync();
    Acc acc[kN];
#pragma unroll
    for (int j = 0; j < kN; ++j) acc[j] = Acc{0.f, 0.f};
    for (int qq = a.ndiag - 1; qq >= 0; --qq) {
      float v[32];
      tc::tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(32 * qq), v);
      const float w = __uint_as_float((uint32_t)(127 - 7 * qq) << 23);   // 2^(-7 qq)
#pragma unroll
      for (int j = 0; j < kN; ++j) two_sum_add(acc[j], v[j] * w);
    }
    if (!FWD) {
      if (row < nr) {
#pragma unroll
        for (int p = 0; p < kN / 2; ++p) {
          const int bm = map0 + p;
          if (bm >= a.B) break;
          const int kr = e_r + fexp_s[2 * p] - 10, ki = e_r + fexp_s[2 * p + 1] - 10;
          double x = scale2(f2d(acc[2 * p].s), kr) + scale2(f2d(acc[2 * p].c), kr);
          double y = scale2(f2d(acc[2 * p + 1].s), ki) + scale2(f2d(acc[2 * p + 1].c), ki);
          double2 r;
          switch (a.phase_mode) {
            case 1: r = make_double2(x, y); break;
            case 2: r = make_double2(neg(x), neg(y)); break;
            case 3: r = make_double2(neg(y), x); break;
            case 4: r = make_double2(y, neg(x)); break;
            default: r = make_double2(fma(x, a.phase.x, -y * a.phase.y), fma(x, a.phase.y, y * a.phase.x));
          }
          a.G[(((int64_t)bm * a.nact + ni) * nr + row) * a.Mc + mi] = r;
        }
      }
    } else {
      const int l = l0a + row;
      if (l >= l0 && l < L) {
        const double2 mu = a.mult[(int64_t)l * a.nact + ni];
#pragma unroll
        for (int p = 0; p < kN / 2; ++p) {
          const int bm = map0 + p;
          if (bm >= a.B) break;
          const int kr = e_r + fexp_s[2 * p] - 10, ki = e_r + fexp_s[2 * p + 1] - 10;
          const double x = scale2(f2d(acc[2 * p].s), kr) + scale2(f2d(acc[2 * p].c), kr);
          const double y = scale2(f2d(acc[2 * p + 1].s), ki) + scale2(f2d(acc[2 * p + 1].c), ki);
          double2* o = a.out + (int64_t)bm * a.s_b + (int64_t)ni * a.s_n + (int64_t)l * a.s_l + (m - a.mlo_out);
          atomicAdd(&o->x, fma(x, mu.x, -y * mu.y));
          atomicAdd(&o->y, fma(x, mu.y, y * mu.x));
        }
      }
    }
    tc::fence_before_sync();
    __syncthreads();   // TMEM and fexp_s are rewritten by the next map chunk
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tmem, kTmemCols);
}

int phase_mode(double2 ph) {
  if (ph.y == 0.0 && ph.x == 1.0) return 1;
  if (ph.y == 0.0 && ph.x == -1.0) return 2;
  if (ph.x == 0.0 && ph.y == 1.0) return 3;
  if (ph.x == 0.0 && ph.y == -1.0) return 4;
  return 0;
}

}  // namespace

cudaError_t launch_tcx_pack(const TransformSpec& t, const TcxTable& tab, const TabTable& src, int nr, int Mc, int mlo,
                            cudaStream_t st) {
  PackArgs a;
  a.nvals = t.nvals;
  a.nact = t.nact;
  a.L = t.L;
  a.nr = nr;
  a.Mc = Mc;
  a.mlo = mlo;
  a.lmin = tab.lmin;
  a.toff_i = src.off_inv;
  a.toff_f = src.off_fwd;
  a.tkp = src.kp;
  a.tLp = src.Lp;
  a.tinv = src.inv;
  a.tfwd = src.fwd;
  a.off_i = tab.off_i;
  a.off_f = tab.off_f;
  a.kli = tab.kli;
  a.klf = tab.klf;
  a.Lb = tab.Lb;
  a.Lk = tab.Lk;
  a.klf_max = tab.klf_max;
  a.rexp_i = tab.rexp_i;
  a.rexp_f = tab.rexp_f;
  a.inv = tab.inv;
  a.fwd = tab.fwd;
  k_tcx_pack<<<dim3(Mc, t.nact), 128, 0, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_tcx_inverse(const s2w_plan* P, const GridTables& g, const TransformSpec& t, CoefArgs in,
                               ColumnArgs out, cudaStream_t st) {
  (void)g;
  const TcxTable& tab = *t.tcx;
  const int nq = (out.B + kN / 2 - 1) / (kN / 2);
  PrepArgs pa{};
  pa.nvals = t.nvals;
  pa.nact = t.nact;
  pa.L = t.L;
  pa.nr = out.nr;
  pa.Mc = out.Mc;
  pa.mlo = out.mlo;
  pa.B = out.B;
  pa.kl = tab.kli;
  pa.lmin = tab.lmin;
  pa.opoff_i = tab.opoff_i;
  pa.Lk = tab.Lk;
  pa.coef = in.coef;
  pa.s_b = in.s_b;
  pa.s_n = in.s_n;
  pa.s_l = in.s_l;
  pa.mlo_in = in.mlo;
  pa.mult_r = t.minv_factored ? t.minv_r : nullptr;
  pa.mult = t.mult_inv;
  pa.ops = P->tcx_ops;
  pa.fexp = P->tcx_fexp;
  pa.qstride = tab.op_i;
  pa.err = P->err_word;
  const int ksn = (tab.kli_max + kPrepK - 1) / kPrepK;   // 0 when every multiplier is zero
  cudaError_t e = cudaMemsetAsync(pa.fexp, 0, (size_t)nq * out.Mc * t.nact * kN * sizeof(int), st);
  if (e != cudaSuccess) return e;
  if (ksn > 0) {
    const dim3 pg((out.Mc + kPrepM - 1) / kPrepM, t.nact, nq * ksn);
    k_tcxe<false><<<pg, 256, 0, st>>>(pa, ksn);
    k_tcxs<false><<<pg, 256, 0, st>>>(pa, ksn);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  GemmArgs a{};
  a.A = tab.inv;
  a.off = tab.off_i;
  a.kl = tab.kli;
  a.rexp = tab.rexp_i;
  a.rstride = tab.Lb;
  a.opoff_i = tab.opoff_i;
  a.ops = P->tcx_ops;
  a.fexp = P->tcx_fexp;
  a.qstride = tab.op_i;
  a.nvals = t.nvals;
  a.nact = t.nact;
  a.L = t.L;
  a.nr = out.nr;
  a.Lk = tab.Lk;
  a.Mc = out.Mc;
  a.mlo = out.mlo;
  a.B = out.B;
  a.G = out.G;
  a.phase = t.minv_factored ? t.minv_phase : make_double2(1.0, 0.0);
  a.phase_mode = phase_mode(a.phase);
  a.idesc = tc::make_idesc(128, kN, 1, 0, 0);   // bf16 slices
  a.lmin = tab.lmin;
  a.err = P->err_word;
  a.inject_timeout = P->inject_timeout;
  a.ndiag = P->slice_diag7 ? kDiag : kDiag - 1;
  e = cudaFuncSetAttribute(k_tcx_gemm<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmem);
  if (e != cudaSuccess) return e;
  k_tcx_gemm<false><<<dim3(tab.Lb / 128, out.Mc, t.nact), kThreads, kSmem, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_tcx_forward(const s2w_plan* P, const GridTables& g, const TransformSpec& t, ColumnArgs in,
                               CoefArgs out, cudaStream_t st) {
  (void)g;
  const TcxTable& tab = *t.tcx;
  const int nq = (in.B + kN / 2 - 1) / (kN / 2);
  PrepArgs pa{};
  pa.nvals = t.nvals;
  pa.nact = t.nact;
  pa.L = t.L;
  pa.nr = in.nr;
  pa.Mc = in.Mc;
  pa.mlo = in.mlo;
  pa.B = in.B;
  pa.kl = tab.klf;
  pa.lmin = tab.lmin;
  pa.Lk = tab.Lk;
  pa.G = in.G;
  pa.ops = P->tcx_ops;
  pa.fexp = P->tcx_fexp;
  pa.qstride = tab.op_f;
  pa.err = P->err_word;
  const int ksn = (tab.Lk + kPrepK - 1) / kPrepK;
  cudaError_t e = cudaMemsetAsync(pa.fexp, 0, (size_t)nq * in.Mc * t.nact * kN * sizeof(int), st);
  if (e != cudaSuccess) return e;
  const dim3 pg((in.Mc + kPrepM - 1) / kPrepM, t.nact, nq * ksn);
  k_tcxe<true><<<pg, 256, 0, st>>>(pa, ksn);
  k_tcxs<true><<<pg, 256, 0, st>>>(pa, ksn);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  GemmArgs a{};
  a.A = tab.fwd;
  a.off = tab.off_f;
  a.kl = tab.klf;
  a.rexp = tab.rexp_f;
  a.rstride = tab.klf_max;
  a.ops = P->tcx_ops;
  a.fexp = P->tcx_fexp;
  a.qstride = tab.op_f;
  a.nvals = t.nvals;
  a.nact = t.nact;
  a.L = t.L;
  a.nr = in.nr;
  a.Lk = tab.Lk;
  a.Mc = in.Mc;
  a.mlo = in.mlo;
  a.B = in.B;
  a.mult = t.mult_fwd;
  a.out = const_cast<double2*>(out.coef);
  a.s_b = out.s_b;
  a.s_n = out.s_n;
  a.s_l = out.s_l;
  a.mlo_out = out.mlo;
  a.idesc = tc::make_idesc(128, kN, 1, 0, 0);   // bf16 slices
  a.lmin = tab.lmin;
  a.err = P->err_word;
  a.inject_timeout = P->inject_timeout;
  a.ndiag = P->slice_diag7 ? kDiag : kDiag - 1;
  e = cudaFuncSetAttribute(k_tcx_gemm<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmem);
  if (e != cudaSuccess) return e;
  if (tab.klf_max == 0) return cudaSuccess;
  k_tcx_gemm<true><<<dim3(tab.klf_max / 128, in.Mc, t.nact), kThreads, kSmem, st>>>(a);
  return cudaGetLastError();
}

}  // namespace s2w

// Azimuthal (alpha/phi) DFTs of the float64-accurate tensor-core mode (S2W_FP64_TC) as one
// persistent, warp-specialised kernel per direction: the prime-factor (Good-Thomas) split of
// the odd length n = 2L - 1 = n1 n2 (gcd(n1, n2) = 1, e.g. 511 = 7 x 73, 255 = 5 x 51), with the
// n2-point stage an exact sliced GEMM on the tcgen05 tensor cores (seven bf16 digits per value,
// slice7.cuh; Ozaki, Ogita, Oishi and Rump, Numer. Algorithms 59, 2012) and the n1-point stage
// in compensated float32 straight from the accumulators.  (Sec. 5.2, Eq. 48: the D-matrix
// factorisation leaves a 2-D DFT over (alpha, gamma); here gamma is taken on the map side.)
//
// Prime-factor split (no twiddle factors between the stages): with the input index map
// p = (n2 p1 + n1 p2) mod n and the output index map k = (k1 e1 + k2 e2) mod n (e1 = n2 (n2^-1
// mod n1), e2 = n1 (n1^-1 mod n2), so k = k1 mod n1 and k = k2 mod n2),
//   X(k) = sum_p1 w_n1^(S p1 k1) [ sum_p2 w_n2^(S p2 k2) x(p) ],   w_m = exp(2 pi i/m), S = -+1.
// The inner n2-point DFT of every column (ring, job, p1, re|im) is one GEMM against a table of
// n2 + 1 rows: row 2j holds s cos(2 pi p2 j/n2), row 2j + 1 holds s sin(2 pi p2 j/n2), j <= (n2-1)/2
// (s = the transform's normalisation), so the accumulator rows 2j and 2j + 1 of a column are C_j
// and S_j; Y(j) and Y(n2 - j) follow from (C, S) by one add each, lane 2j computing Y(j) and
// lane 2j + 1 computing Y(n2 - j) after exchanging their rows with a shuffle.  Each lane then
// takes the n1-point DFT over p1 of its Y values and writes its n1 outputs.
//
// Exactness of the GEMM: the table (scale s < 2^e_tw) and the data (one exponent f per ring,
// max |x| < 2^f) are rounded to 47-bit fixed point and cut into seven balanced base-128 digits;
// the 28 digit-pair MMAs with i + i' = q <= 6 of a K step go to accumulator q (seven 128 x 64
// float32 accumulators in TMEM), whose partial sums are integers below 2^24 (K <= 128), so every
// accumulator is exact; C = 2^(e_tw + f - 10) sum_q 2^(-7q) D_q, summed smallest weight first in
// compensated float32.
//
// One CTA per SM, persistent over passes; a pass is 64 GEMM columns: slots of W = 2 n1 rounded up
// to a power of two columns (ring, job), S = 64/W slots, rpp = S/nj rings per pass.
//   warps 0-7  (TMEM warps): warp w reads TMEM lane quarter w % 4 and column chunks 2 (w/4),
//              2 (w/4) + 1 (16 columns each): drain, row exchange, n1-point DFT, outputs
//              (forward: the columns G; inverse: Z_q(alpha) into shared memory);
//   warp 8     issues the 28 x K/16 MMAs of a pass (one thread) and owns the TMEM allocation;
//   warps 9-15 (producers): forward: the gamma DFT of the pass's rings (compensated, as in
//              kernels_dft_c32.cu) into shared memory, the ring exponents, the slices; inverse: the
//              ring exponents and slices from the columns, and the gamma synthesis of the previous
//              pass from Z to the pixels.
// Handshakes are mbarriers (b_full/b_empty: the data slices; acc_full/acc_empty: the accumulators;
// z_full/z_empty: the inverse staging), every wait bounded; a timeout sets the plan's error word
// and an abort flag that every role checks, so the CTA always reaches its exit and frees TMEM.
// Shared memory: the table, resident for the whole kernel; one buffer of data slices; the
// gamma-DFT (forward) or Z (inverse) staging of one pass.
#include <math.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "comp32.cuh"
#include "dft_c32.cuh"
#include "s2w_internal.h"
#include "slice7.cuh"
#include "tc_sm100.cuh"

namespace s2w {
namespace {

constexpr int kPT = 512;                        // threads per CTA
constexpr int kPTmemWarps = 8;                  // warps 0-7
constexpr int kPMmaWarp = 8;                    // warp 8
constexpr int kPProdWarp0 = 9;                  // warps 9-15
constexpr int kPProd = kPT - kPProdWarp0 * 32;  // 224 producer threads
constexpr int kPN = 64;                         // GEMM columns per pass (MMA N)
constexpr int kPBTile = kPN * 16;               // elements of one data slice chunk (64 x 16)
constexpr uint32_t kPWait = 1u << 20;           // bounded mbarrier polls
constexpr int kPMaxRpp = 32;                    // rings per pass (n1 = 1: 32 slots of 2 columns)
constexpr int kPMaxSmem = 220 * 1024;           // dynamic shared memory limit used for the plan choice
constexpr int kPMaxNg = 15;                     // gamma samples 2N - 1 (N <= 8)
constexpr int kPSlots = 4;                      // per-pass tables, by pass index mod 4

struct PArgs {
  const void* pix_in;
  void* pix_out;
  int64_t pix_sb;
  const double2* Gin;
  double2* Gout;
  const int* nvals;
  int nact, Ng, n, n1, n2, R, Rs, nkc, nr, B, Mc, mlo;
  int e1, e2, rpp, npass;
  int hz_bytes;             // bytes of the gamma / Z staging of one pass
  int gstage;               // inverse: the pass's columns are staged in shared memory by bulk copies
  const float4* gph;        // [nact][Ng] exp(+i n gamma_g) as pairs
  const uint16_t* tab;      // sliced table, [chunk][slice][Rs x 16 core-matrix layout]
  int e_tw;
  float4 tw1[8];            // cos, sin (2 pi m/n1) as pairs (hi, lo, hi, lo), m < n1
  uint32_t idesc;
  int* err;
};

__device__ __forceinline__ void pbar() { asm volatile("bar.sync 1, %0;" ::"n"(kPProd) : "memory"); }

template <int N1>
struct SlotShape {
  static constexpr int W = N1 == 1 ? 2 : (N1 == 3 ? 8 : 16);   // columns per slot
  static constexpr int SPC = 16 / W;                             // slots per 16-column chunk
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

template <bool FWD, bool REAL, int N1>
__global__ void __launch_bounds__(kPT, 1) k_dftp(PArgs a) {
  using SS = SlotShape<N1>;
  extern __shared__ __align__(1024) uint8_t smem[];
  __shared__ __align__(8) uint64_t b_full, b_empty, acc_full, acc_empty, z_full, z_empty, g_full;
  __shared__ uint32_t tbase;
  __shared__ int jn[kMaxJobs], jp[kMaxJobs], njs;
  __shared__ uint8_t slot_rip[64], slot_q[64];   // slot -> (ring of the pass, job)
  __shared__ float4 ph_s[kJobChunk * kPMaxNg];   // exp(+i n_q gamma_g) of the jobs, [q][g]
  __shared__ int emax_s[kPMaxRpp];
  // per pass, by pass index mod 4: ring exponent, map and ring (bb < 0: past the last ring).  The
  // producers fill pass i's exponents and pass i + 1's rings after MMA(i-1) has completed, when
  // the TMEM warps (which read them in stage B, after releasing TMEM) can still be on pass i - 2
  __shared__ int fr_s[kPSlots][kPMaxRpp], rbb_s[kPSlots][kPMaxRpp], rt_s[kPSlots][kPMaxRpp];
  __shared__ volatile int s_abort;   // any role: a wait ran out, every role stops
  __shared__ int p_abort;            // the producers' copy, written by one producer before a named barrier
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int abytes = a.nkc * kSl * a.Rs * 32;
  const int boff = (abytes + 1023) & ~1023;
  const int n = a.n, h = (n - 1) / 2, rings = a.B * a.nr, rpp = a.rpp, Mc = a.Mc, nact = a.nact;
  uint16_t* const As = reinterpret_cast<uint16_t*>(smem);
  uint16_t* const Bs = reinterpret_cast<uint16_t*>(smem + boff);
  float4* const HZ = reinterpret_cast<float4*>(smem + boff + a.nkc * kSl * kPBTile * 2);
  // inverse: the columns of the pass's rings, [ring][n index][Mc], when a.gstage
  double2* const Gs = reinterpret_cast<double2*>(reinterpret_cast<uint8_t*>(HZ) + (size_t)a.hz_bytes);
  if (tid == 0) {
    int nj;
    make_jobs(a.nvals, nact, REAL, jn, jp, nj);
    njs = nj;
    tc::mbar_init(&b_full, 1);
    tc::mbar_init(&b_empty, 1);
    tc::mbar_init(&acc_full, 1);
    tc::mbar_init(&acc_empty, kPTmemWarps);
    tc::mbar_init(&z_full, kPTmemWarps);
    tc::mbar_init(&z_empty, 1);
    tc::mbar_init(&g_full, 1);
    s_abort = 0;
    p_abort = 0;
    tc::fence_mbar_init();
  }
  // the sliced table, resident for the whole kernel (plain 16-byte loads)
  for (int i = tid; i < abytes / 16; i += kPT)
    reinterpret_cast<uint4*>(As)[i] = reinterpret_cast<const uint4*>(a.tab)[i];
  if (warp == kPMmaWarp) tc::tmem_alloc(&tbase, 512);
  tc::fence_proxy_async();   // generic-proxy writes of the table, read by the MMAs
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = tbase;
  const int nj = njs;
  if (tid < 64) {
    slot_rip[tid] = (uint8_t)(tid / nj);
    slot_q[tid] = (uint8_t)(tid % nj);
  }
  for (int i = tid; i < kJobChunk * kPMaxNg; i += kPT) {
    const int q = i / kPMaxNg, g = i - q * kPMaxNg;
    ph_s[i] = (q < nj && g < a.Ng) ? a.gph[jn[q] * a.Ng + g] : make_float4(0.f, 0.f, 0.f, 0.f);
  }
  __syncthreads();
  const int G = gridDim.x, my = (a.npass - (int)blockIdx.x + G - 1) / G;   // passes of this CTA
  const int64_t ringlen = (int64_t)a.nr * n;

  // bounded waits: `wait` polls (the MMA issuer, latency-critical), `wait_bo` backs off with
  // nanosleep (the other roles)
  auto on_timeout = [&]() {
    atomicExch(a.err, (int)S2W_ETIMEOUT);
    s_abort = 1;
  };
  auto wait = [&](uint64_t* bar, uint32_t parity) -> bool {
    if (s_abort) return false;
    if (!tc::mbar_wait(bar, parity, kPWait)) return on_timeout(), false;
    return true;
  };
  auto wait_bo = [&](uint64_t* bar, uint32_t parity) -> bool {
    if (s_abort) return false;
    if (!tc::mbar_wait_backoff(bar, parity, kPWait)) return on_timeout(), false;
    return true;
  };

  if (warp == kPMmaWarp) {
    // ------------------------------------------------------------ MMA issue (one thread)
    if (lane == 0) {
      const uint32_t A0 = tc::smem_u32(As), B0 = tc::smem_u32(Bs);
      const uint32_t atile = (uint32_t)a.Rs * 32u, btile = (uint32_t)kPBTile * 2u;
      int issued = -1;
      for (int i = 0; i < my; ++i) {
        if (!wait(&b_full, (uint32_t)(i & 1))) break;
        if (i > 0 && !wait(&acc_empty, (uint32_t)((i - 1) & 1))) break;
        tc::fence_after_sync();
        for (int c = 0; c < a.nkc; ++c) {
          const uint32_t ab = A0 + (uint32_t)(c * kSl) * atile, bb = B0 + (uint32_t)(c * kSl) * btile;
#pragma unroll
          for (int qq = 0; qq < kSl; ++qq)
#pragma unroll
            for (int sa = 0; sa <= qq; ++sa)
              tc::mma_f16(tmem + (uint32_t)(64 * qq), tc::make_sdesc(ab + (uint32_t)sa * atile, 128, 256),
                          tc::make_sdesc(bb + (uint32_t)(qq - sa) * btile, 128, 256), a.idesc,
                          (c > 0 || sa > 0) ? 1u : 0u);
        }
        tc::mma_commit(&b_empty);
        tc::mma_commit(&acc_full);
        issued = i;
      }
      // after an abort: let the last issued MMAs land before TMEM is freed (bounded)
      if (s_abort && issued >= 0) tc::mbar_wait(&b_empty, (uint32_t)(issued & 1), kPWait);
    }
  } else if (warp < kPTmemWarps) {
    // ------------------------------------------------------------ TMEM warps
    const int quarter = warp & 3, grp = warp >> 2;
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
    // bounded wait by lane 0, the outcome broadcast so that the warp stays converged
    auto warp_wait = [&](uint64_t* bar, uint32_t parity) -> bool {
      int ok = 1;
      if (lane == 0) ok = wait_bo(bar, parity) ? 1 : 0;
      return __shfl_sync(0xFFFFFFFFu, ok, 0) != 0;
    };
    // the seven accumulators of one 16-column chunk, summed smallest weight first: two halves of
    // 8 columns, each with its 7 loads in flight before one wait
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
    // row exchange, n1-point DFT and outputs of the slots of one 16-column chunk
    auto stage_b = [&](int i, int chunk, const Acc (&acc)[16]) {
      const int i3 = i % kPSlots;
#pragma unroll
      for (int u = 0; u < SS::SPC; ++u) {
        const int sl = chunk * SS::SPC + u;
        const bool slot_ok = sl < rpp * nj;   // warp-uniform
        if (!slot_ok) continue;
        const int rip = slot_rip[sl], q = slot_q[sl];
        const int bb = rbb_s[i3][rip], t = rt_s[i3][rip];
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
        if (bb < 0 || !live) continue;
        Acc xr[N1], xi[N1];
        dft_small<N1, FWD ? -1 : 1>(yr, yi, a.tw1, xr, xi);
        if (FWD) {
          const int ke = a.e_tw + fr_s[i3][rip] - 10;
          double2* const Gn = a.Gout + (((int64_t)bb * nact + jn[q]) * a.nr + t) * Mc;
          double2* const Gp = jp[q] >= 0 ? a.Gout + (((int64_t)bb * nact + jp[q]) * a.nr + t) * Mc : nullptr;
#pragma unroll
          for (int k1 = 0; k1 < N1; ++k1) {
            const int k = ka[k1] + kb >= n ? ka[k1] + kb - n : ka[k1] + kb;
            const double2 x = make_double2(pair_dbl(xr[k1], ke), pair_dbl(xi[k1], ke));
            if (REAL) {
              // G_{m, n} = X(m) for m = k <= h; the partner column G_{m', -n} = conj X(n - m') for
              // m' = n - k in 1..h, and G_{0, -n} = conj X(0)
              if (k <= h) Gn[k] = x;
              if (Gp != nullptr && (k > h || k == 0)) Gp[k == 0 ? 0 : n - k] = make_double2(x.x, -x.y);
            } else {
              Gn[(k <= h ? k : k - n) - a.mlo] = x;
            }
          }
        } else {
#pragma unroll
          for (int k1 = 0; k1 < N1; ++k1) {
            const int k = ka[k1] + kb >= n ? ka[k1] + kb - n : ka[k1] + kb;
            HZ[(rip * nj + q) * n + k] = make_float4(xr[k1].s, xr[k1].c, xi[k1].s, xi[k1].c);
          }
        }
      }
    };
    for (int i = 0; i < my; ++i) {
      if (!warp_wait(&acc_full, (uint32_t)(i & 1))) break;
      tc::fence_after_sync();
      if (!warp_live) {   // no accumulator row of this lane quarter carries data
        __syncwarp();
        if (lane == 0) tc::mbar_arrive(&acc_empty);
        if (!FWD) {
          if (i > 0 && !warp_wait(&z_empty, (uint32_t)((i - 1) & 1))) break;
          if (lane == 0) tc::mbar_arrive(&z_full);
        }
        continue;
      }
      Acc acc[16];
      drain(2 * grp, acc);
      // the inverse writes Z into the staging the producers read for pass i - 1
      if (!FWD && i > 0 && !warp_wait(&z_empty, (uint32_t)((i - 1) & 1))) break;
      stage_b(i, 2 * grp, acc);
      drain(2 * grp + 1, acc);
      // every accumulator value this warp needs is in registers: release TMEM to the next pass
      tc::fence_before_sync();
      __syncwarp();
      if (lane == 0) tc::mbar_arrive(&acc_empty);
      stage_b(i, 2 * grp + 1, acc);
      if (!FWD) {
        __threadfence_block();
        __syncwarp();
        if (lane == 0) tc::mbar_arrive(&z_full);
      }
    }
  } else {
    // ------------------------------------------------------------ producers
    const int pt = tid - kPProdWarp0 * 32;
    const int Ng = a.Ng, hg = (Ng - 1) / 2;
    auto slice_store = [&](int col, int kg, const long long (&X)[8]) {
      uint32_t w[kSl][4];
#pragma unroll
      for (int u = 0; u < 8; u += 2) {
        uint32_t d0[kSl], d1[kSl];
        digits7(X[u], d0);
        digits7(X[u + 1], d1);
#pragma unroll
        for (int s = 0; s < kSl; ++s) w[s][u / 2] = __byte_perm(d0[s], d1[s], 0x7632);
      }
      const int o = (kg >> 1) * kSl * kPBTile + ((col >> 3) * 2 + (kg & 1)) * 64 + (col & 7) * 8;
#pragma unroll
      for (int s = 0; s < kSl; ++s)
        *reinterpret_cast<uint4*>(Bs + o + s * kPBTile) = make_uint4(w[s][0], w[s][1], w[s][2], w[s][3]);
    };
    // the ring table of pass i
    auto rings_of_pass = [&](int i) {
      if (pt < rpp) {
        const int rf = ((int)blockIdx.x + i * G) * rpp + pt;
        const int bb = rf < rings ? rf / a.nr : -1;
        rbb_s[i % kPSlots][pt] = bb;
        rt_s[i % kPSlots][pt] = bb < 0 ? 0 : rf - bb * a.nr;
      }
    };
    int g_pending = -1;   // producer 0: the pass whose column copies are in flight
    // inverse: the columns of pass i's rings into Gs by bulk copies (one producer thread)
    auto fetch_cols = [&](int i) {
      if (pt != 0) return;
      const int i3 = i % kPSlots;
      g_pending = i;
      uint32_t bytes = 0;
      for (int r = 0; r < rpp; ++r)
        if (rbb_s[i3][r] >= 0) bytes += (uint32_t)(nact * Mc * 16);
      tc::mbar_expect_tx(&g_full, bytes);
      for (int r = 0; r < rpp; ++r) {
        const int bb = rbb_s[i3][r], t = rt_s[i3][r];
        if (bb < 0) continue;
        for (int ni = 0; ni < nact; ++ni)
          tc::bulk_g2s(Gs + ((int64_t)r * nact + ni) * Mc, a.Gin + (((int64_t)bb * nact + ni) * a.nr + t) * Mc,
                       (uint32_t)(Mc * 16), &g_full);
      }
    };
    auto gval = [&](int i3, int rip, int ni, int m) -> double2 {
      if (a.gstage) return Gs[((int64_t)rip * nact + ni) * Mc + m];
      return a.Gin[(((int64_t)rbb_s[i3][rip] * nact + ni) * a.nr + rt_s[i3][rip]) * Mc + m];
    };
    // gamma synthesis of pass ip (inverse): W(alpha, gamma_g) = sum_q Z_q(alpha) exp(+i n_q gamma_g)
    auto synth = [&](int ip) -> bool {
      if (pt == 0) {
        wait_bo(&z_full, (uint32_t)(ip & 1));
        p_abort = s_abort;
      }
      pbar();
      if (p_abort) return false;
      const int i3 = ip % kPSlots;
      for (int rip = 0; rip < rpp; ++rip) {
        const int bb = rbb_s[i3][rip];
        if (bb < 0) break;   // rings are in order: the rest of the pass is past the end too
        const int ke = a.e_tw + fr_s[i3][rip] - 10;
        const int64_t base0 = (int64_t)bb * a.pix_sb + (int64_t)rt_s[i3][rip] * n;
        for (int al = pt; al < n; al += kPProd) {
          float4 z[kJobChunk];
#pragma unroll
          for (int q = 0; q < kJobChunk; ++q)
            if (q < nj) {
              z[q] = HZ[(rip * nj + q) * n + al];
              if (REAL && jp[q] >= 0) z[q] = make_float4(2.f * z[q].x, 2.f * z[q].y, 2.f * z[q].z, 2.f * z[q].w);
            }
          const int64_t base = base0 + al;
          for (int gg = 0; gg <= hg; ++gg) {
            Acc pr{0.f, 0.f}, pim{0.f, 0.f}, qr{0.f, 0.f}, qim{0.f, 0.f};
#pragma unroll
            for (int q = 0; q < kJobChunk; ++q)
              if (q < nj) {
                const float4 ph = ph_s[q * kPMaxNg + gg];
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
      pbar();
      if (pt == 0) tc::mbar_arrive(&z_empty);
      return true;
    };
    const int ncols = rpp * nj * SS::W;   // columns carrying data (the rest are sliced as zeros)
    if (my > 0) {
      rings_of_pass(0);
      pbar();
      if (!FWD && a.gstage) fetch_cols(0);
    }
    for (int i = 0; i < my; ++i) {
      const int i3 = i % kPSlots;
      if (pt < rpp) emax_s[pt] = 0;
      if (!FWD && a.gstage) {
        if (pt == 0) {
          if (wait_bo(&g_full, (uint32_t)(i & 1))) g_pending = -1;
          p_abort = s_abort;
        }
      }
      pbar();
      if (p_abort) break;
      bool bad = false;
      if (FWD) {
        // gamma DFT of every ring of the pass: H_q(alpha) = sum_g W(alpha, gamma_g) exp(-i n_q gamma_g)
        for (int rip = 0; rip < rpp; ++rip) {
          const int bb = rbb_s[i3][rip];
          const int64_t base0 = bb < 0 ? 0 : (int64_t)bb * a.pix_sb + (int64_t)rt_s[i3][rip] * n;
          for (int al = pt; al < n; al += kPProd) {
            Acc hr[kJobChunk], hi[kJobChunk];
#pragma unroll
            for (int q = 0; q < kJobChunk; ++q) hr[q] = hi[q] = Acc{0.f, 0.f};
            if (bb >= 0) {
              // the samples of this alpha in flight in batches of up to four pairs gamma_g,
              // gamma_{Ng-g} before their arithmetic (more at once spills registers)
              constexpr int HG = (kPMaxNg - 1) / 2, BAT = 2;
              const float4 x0 = load_pix(a.pix_in, REAL, base0 + al);
#pragma unroll
              for (int q = 0; q < kJobChunk; ++q) {
                hr[q] = Acc{x0.x, x0.y};
                hi[q] = Acc{x0.z, x0.w};
              }
#pragma unroll
              for (int g0 = 1; g0 <= HG; g0 += BAT) {
                if (g0 > hg) break;
                float4 xpa[BAT], xma[BAT];
#pragma unroll
                for (int u = 0; u < BAT; ++u)
                  if (g0 + u <= hg) {
                    xpa[u] = load_pix(a.pix_in, REAL, base0 + (g0 + u) * ringlen + al);
                    xma[u] = load_pix(a.pix_in, REAL, base0 + (Ng - g0 - u) * ringlen + al);
                  }
#pragma unroll
              for (int u = 0; u < BAT; ++u) {
                const int g = g0 + u;
                if (g > hg) break;
                const float4 xp = xpa[u], xm = xma[u];
                const float4 uu = cadd<false>(xp, xm, 1.f), vv = cadd<false>(xp, xm, -1.f);
#pragma unroll
                for (int q = 0; q < kJobChunk; ++q) {
                  if (q < nj) {
                    const float4 ph = ph_s[q * kPMaxNg + g];
                    racc<false>(hr[q], uu.x, uu.y, ph.x, ph.y);   // u cos - i v sin
                    racc<false>(hi[q], vv.x, vv.y, -ph.z, -ph.w);
                    if (!REAL) {
                      racc<false>(hr[q], vv.z, vv.w, ph.z, ph.w);
                      racc<false>(hi[q], uu.z, uu.w, ph.x, ph.y);
                    }
                  }
                }
              }
              }
            }
            int e = 0;
#pragma unroll
            for (int q = 0; q < kJobChunk; ++q)
              if (q < nj) {
                const float4 z = pack<false>(hr[q], hi[q]);
                HZ[(rip * nj + q) * n + al] = z;
                e = max(e, max(fbound(z.x), fbound(z.z)));
                bad |= ((__float_as_uint(z.x) & 0x7F800000u) == 0x7F800000u) |
                        ((__float_as_uint(z.z) & 0x7F800000u) == 0x7F800000u);
              }
            if (e > 0) atomicMax(&emax_s[rip], e);
          }
        }
      } else {
        // ring exponents over every column value of the pass's rings
        for (int rip = 0; rip < rpp; ++rip) {
          if (rbb_s[i3][rip] < 0) break;
          int e = 0;
          for (int it = pt; it < nact * Mc; it += kPProd) {
            const int ni = it / Mc, m = it - ni * Mc;
            const double2 v = gval(i3, rip, ni, m);
            e = max(e, max(ebound(v.x), ebound(v.y)));
            bad |= (bexp(v.x) == 0x7FF) | (bexp(v.y) == 0x7FF);
          }
          if (e > 0) atomicMax(&emax_s[rip], e);
        }
      }
      if (bad) atomicCAS(a.err, 0, (int)S2W_ENONFINITE);
      pbar();
      if (pt == 0) {
        if (i > 0) wait_bo(&b_empty, (uint32_t)((i - 1) & 1));   // the MMAs of pass i - 1 read B
        p_abort = s_abort;   // one decision for all producers (they meet at named barriers)
      }
      pbar();
      if (p_abort) break;
      // after MMA(i-1): every TMEM warp has finished pass i-3 (it drained pass i-2), whose ring
      // tables share this slot
      if (pt < rpp) fr_s[i3][pt] = emax_s[pt] > 0 ? e_from(emax_s[pt]) : 0;
      pbar();
      // the seven slices of every column: item (column, group of 8 reduction indices p2)
      for (int it = pt; it < kPN * 2 * a.nkc; it += kPProd) {
        const int col = it & (kPN - 1), kg = it >> 6;
        const int sl = col / SS::W, p1 = (col % SS::W) >> 1, c = col & 1;
        long long X[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) X[u] = 0;
        if (col < ncols && p1 < N1) {
          const int rip = slot_rip[sl], q = slot_q[sl];
          const int f = fr_s[i3][rip];
          const int pa = a.n2 * p1;   // < n; p = (n2 p1 + n1 p2) mod n with n1 p2 < n
          if (rbb_s[i3][rip] >= 0) {
#pragma unroll
            for (int u = 0; u < 8; ++u) {
              const int p2 = kg * 8 + u;
              if (p2 >= a.n2) continue;
              const int p = pa + a.n1 * p2 >= n ? pa + a.n1 * p2 - n : pa + a.n1 * p2;
              if (FWD) {
                const float4 z = HZ[(rip * nj + q) * n + p];
                X[u] = c ? fixf_pair(z.z, z.w, f) : fixf_pair(z.x, z.y, f);
              } else {
                double2 v;
                if (REAL) {
                  if (p <= h) {
                    v = gval(i3, rip, jn[q], p);
                  } else {   // x_{p} = conj G_{n-p, -n} (the job's own n = 0 column for the n = 0 job)
                    v = gval(i3, rip, jp[q] >= 0 ? jp[q] : jn[q], n - p);
                    v.y = -v.y;
                  }
                } else {
                  v = gval(i3, rip, jn[q], (p <= h ? p : p - n) - a.mlo);
                }
                X[u] = fix47(c ? v.y : v.x, f);
              }
            }
          }
        }
        slice_store(col, kg, X);
      }
      tc::fence_proxy_async();   // the slices (generic-proxy writes) are read by the MMAs
      if (i + 1 < my) rings_of_pass(i + 1);
      pbar();
      // forward: pull the next pass's pixel rows (Ng rows of n samples per ring) into L2 while
      // this pass's MMAs and the TMEM warps run
      if (FWD && i + 1 < my && pt < rpp * Ng) {
        const int rip = pt / Ng, g = pt - rip * Ng, bb = rbb_s[(i + 1) % kPSlots][rip];
        if (bb >= 0) {
          const size_t es = REAL ? sizeof(double) : sizeof(double2);
          const char* row = (const char*)a.pix_in +
                            ((int64_t)bb * a.pix_sb + g * ringlen + (int64_t)rt_s[(i + 1) % kPSlots][rip] * n) * es;
          // bulk L2 prefetch: 16-byte aligned start, size a multiple of 16 (whole 16-byte blocks)
          const uintptr_t a0 = (uintptr_t)row & ~(uintptr_t)15, a1 = ((uintptr_t)row + n * es + 15) & ~(uintptr_t)15;
          asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(a0), "r"((uint32_t)(a1 - a0)) : "memory");
        }
      }
      if (pt == 0) tc::mbar_arrive(&b_full);
      // the columns of pass i are no longer read: fetch those of pass i + 1 while pass i - 1 is
      // synthesised
      if (!FWD && a.gstage && i + 1 < my) fetch_cols(i + 1);
      if (!FWD && i > 0 && !synth(i - 1)) break;
    }
    if (!FWD && !p_abort && my > 0) synth(my - 1);
    // after an abort with column copies in flight: let them land before the CTA exits (bounded)
    if (!FWD && a.gstage && pt == 0 && g_pending >= 0) tc::mbar_wait(&g_full, (uint32_t)(g_pending & 1), kPWait);
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == kPMmaWarp) {
    __syncwarp();
    tc::tmem_dealloc(tmem, 512);
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

// dynamic shared memory: table, data slices, gamma / Z staging (+ staged columns, inverse)
size_t smem_bytes(int n, int n1, int nj, size_t gs_bytes = 0) {
  const int n2 = n / n1, Rs = ((n2 + 1 + 7) / 8) * 8, nkc = (n2 + 15) / 16;
  const int S = kPN / slot_width(n1), rpp = S / nj;
  const size_t abytes = (size_t)nkc * kSl * Rs * 32, boff = (abytes + 1023) & ~(size_t)1023;
  return boff + (size_t)nkc * kSl * kPBTile * 2 + (size_t)rpp * nj * n * sizeof(float4) + gs_bytes;
}

// Launches k_dftp<FWD, REAL, n1>; smem = the dynamic shared memory without the staged columns,
// gs = their bytes (inverse): they are staged only where the kernel's static shared memory leaves
// room for them under the per-block limit.
template <bool FWD, bool REAL>
cudaError_t launch_p(int n1, dim3 grid, size_t smem, size_t gs, cudaStream_t st, PArgs a) {
  auto go = [&](auto kern) -> cudaError_t {
    cudaFuncAttributes fa{};
    cudaError_t e = cudaFuncGetAttributes(&fa, kern);
    if (e != cudaSuccess) return e;
    int dev = 0, optin = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev)) != cudaSuccess) return e;
    const size_t room = (size_t)optin - fa.sharedSizeBytes;
    if (smem > room) return cudaErrorInvalidConfiguration;
    a.gstage = (!FWD && gs > 0 && smem + gs <= room) ? 1 : 0;
    const size_t dyn = smem + (a.gstage ? gs : 0);
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
    if (e != cudaSuccess) return e;
    kern<<<grid, kPT, dyn, st>>>(a);
    return cudaGetLastError();
  };
  switch (n1) {
    case 1: return go(k_dftp<FWD, REAL, 1>);
    case 3: return go(k_dftp<FWD, REAL, 3>);
    case 5: return go(k_dftp<FWD, REAL, 5>);
    case 7: return go(k_dftp<FWD, REAL, 7>);
    default: return cudaErrorInvalidValue;
  }
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

PArgs make_pargs(const GridTables& g, const TransformSpec& t, const DftpTable& tab, ColumnArgs c, bool real,
                 int* err) {
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
  a.rpp = (kPN / slot_width(tab.n1)) / nj;
  a.npass = (c.B * c.nr + a.rpp - 1) / a.rpp;
  a.hz_bytes = a.rpp * nj * g.n * (int)sizeof(float4);
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
  a.err = err;
  return a;
}

}  // namespace

// Factorisation n = 2L - 1 = n1 n2 for the prime-factor tensor-core DFTs: the smallest n1 in
// {1, 3, 5, 7} with gcd(n1, n2) = 1, n2 + 1 <= 128 table rows and the kernel's shared memory
// within the limit for the transform's job count; false if none fits (or the jobs do not: at most
// four jobs, the gamma DFT's pass width, and every carried n != 0 with its -n partner for real
// maps).
bool dftp_shape(const TransformSpec& t, bool real, int* n1_out, int* n2_out) {
  const int nj = jobs_of_p(t, real);
  if (nj < 1 || t.L < 2 || 2 * t.N - 1 > kPMaxNg) return false;
  if (real)
    for (int v : t.nvals_h)
      if (v != 0 && std::find(t.nvals_h.begin(), t.nvals_h.end(), -v) == t.nvals_h.end()) return false;
  const int n = 2 * t.L - 1;
  for (int n1 : {1, 3, 5, 7}) {
    if (n % n1 != 0) continue;
    const int n2 = n / n1;
    if (gcd_i(n1, n2) != 1 || n2 + 1 > 128 || n2 < 2) continue;
    if (nj > kJobChunk || nj > kPN / slot_width(n1) || (kPN / slot_width(n1)) / nj > kPMaxRpp) continue;
    if (smem_bytes(n, n1, nj) > (size_t)kPMaxSmem) continue;
    *n1_out = n1;
    *n2_out = n2;
    return true;
  }
  return false;
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
  PArgs a = make_pargs(g, t, tab, c, real, P->err_word);
  a.pix_in = pix;
  a.pix_sb = pix_sb;
  a.Gout = c.G;
  const size_t smem = smem_bytes(g.n, tab.n1, jobs_of_p(t, real));
  const dim3 grid(std::min(a.npass, num_sms()));
  return real ? launch_p<true, true>(tab.n1, grid, smem, 0, st, a) : launch_p<true, false>(tab.n1, grid, smem, 0, st, a);
}

cudaError_t launch_dftp_inverse(const s2w_plan* P, const GridTables& g, const TransformSpec& t, ColumnArgs c,
                                void* pix, int64_t pix_sb, bool real, cudaStream_t st) {
  const DftpTable& tab = *t.dftp_inv;
  PArgs a = make_pargs(g, t, tab, c, real, P->err_word);
  a.Gin = c.G;
  a.pix_out = pix;
  a.pix_sb = pix_sb;
  // the pass's columns are staged in shared memory where they fit (16-byte rows by construction)
  const size_t gs = (size_t)a.rpp * t.nact * c.Mc * sizeof(double2);
  const size_t smem = smem_bytes(g.n, tab.n1, jobs_of_p(t, real));
  const dim3 grid(std::min(a.npass, num_sms()));
  return real ? launch_p<false, true>(tab.n1, grid, smem, gs, st, a) : launch_p<false, false>(tab.n1, grid, smem, gs, st, a);
}

}  // namespace s2w

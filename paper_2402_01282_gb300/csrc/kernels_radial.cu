// Fourier-Laguerre radial transform on the device (Sec. 2.3, Eqs. 7-8): for every angular
// coefficient column c, out[b][p][c] = sum_i R[p][i] in[b][i][c] with a dense real P x P
// matrix R (forward: omega_i K_p(r_i); inverse: K_i(r_p) transposed).  The columns are the
// complex harmonic coefficients of every radial node.  One thread owns one complex column
// and a strip of kRows output rows; R is staged through shared memory in 32-column chunks.
// C32 accumulates in compensated float32 pairs (comp32.cuh), otherwise in native float64.
#include "comp32.cuh"
#include "s2w_internal.h"

namespace s2w {
namespace {

constexpr int kRows = 16;
constexpr int kChunk = 32;
constexpr int kThreads = 128;

template <bool C32>
__global__ void __launch_bounds__(kThreads) k_radial(const double* __restrict__ R, const float2* __restrict__ R2,
                                                     const double2* __restrict__ in, double2* __restrict__ out,
                                                     int P, int64_t ncol) {
  __shared__ double Rs[kRows * kChunk];
  const int64_t c = (int64_t)blockIdx.x * kThreads + threadIdx.x;
  const int p0 = blockIdx.y * kRows;
  const int b = blockIdx.z;
  const double2* inb = in + (int64_t)b * P * ncol;
  double2* outb = out + (int64_t)b * P * ncol;
  Acc ar[C32 ? kRows : 1], ai[C32 ? kRows : 1];
  double2 acc[C32 ? 1 : kRows];
#pragma unroll
  for (int k = 0; k < kRows; ++k) {
    if (C32) ar[k] = ai[k] = Acc{0.f, 0.f};
    else acc[C32 ? 0 : k] = make_double2(0.0, 0.0);
  }
  float2* Rs2 = reinterpret_cast<float2*>(Rs);
  for (int i0 = 0; i0 < P; i0 += kChunk) {
    const int cnt = min(kChunk, P - i0);
    __syncthreads();
    for (int idx = threadIdx.x; idx < kRows * kChunk; idx += kThreads) {
      const int r = idx / kChunk, i = idx - r * kChunk, p = p0 + r;
      const bool ok = p < P && i < cnt;
      if (C32) Rs2[idx] = ok ? R2[(int64_t)p * P + i0 + i] : make_float2(0.f, 0.f);
      else Rs[idx] = ok ? R[(int64_t)p * P + i0 + i] : 0.0;
    }
    __syncthreads();
    if (c < ncol) {
      for (int i = 0; i < cnt; ++i) {
        const double2 v = inb[(int64_t)(i0 + i) * ncol + c];
        if (C32) {
          const float4 x = split(v);
#pragma unroll
          for (int k = 0; k < kRows; ++k) {
            const float2 w = Rs2[k * kChunk + i];
            acc_add(ar[k], x.x, x.y, w.x, w.y);
            acc_add(ai[k], x.z, x.w, w.x, w.y);
          }
        } else {
#pragma unroll
          for (int k = 0; k < (C32 ? 1 : kRows); ++k) {
            const double w = Rs[k * kChunk + i];
            acc[k].x = fma(w, v.x, acc[k].x);
            acc[k].y = fma(w, v.y, acc[k].y);
          }
        }
      }
    }
  }
  if (c < ncol) {
#pragma unroll
    for (int k = 0; k < kRows; ++k) {
      const int p = p0 + k;
      if (p >= P) break;
      outb[(int64_t)p * ncol + c] = C32 ? make_double2(to_double(ar[k]), to_double(ai[k])) : acc[C32 ? 0 : k];
    }
  }
}

// General radial map for the ball wavelet transforms: out[b][o][c] (+)= wo[o][l] sum_q R[o][q]
// wi[q][l] in[b][q][c] with R of Pout x Pin, c = l Mc + m, optional weights wi, wo ([rows][L])
// and accumulation into out.  Compensated accumulation as above.
__global__ void __launch_bounds__(kThreads) k_radial_gen(const float2* __restrict__ R2, const double2* __restrict__ in,
                                                         double2* __restrict__ out, int Pout, int Pin, int64_t ncol,
                                                         int Mc, int L, const double* __restrict__ wi,
                                                         const double* __restrict__ wo, int accumulate) {
  __shared__ float2 Rs2[kRows * kChunk];
  const int64_t c = (int64_t)blockIdx.x * kThreads + threadIdx.x;
  const int p0 = blockIdx.y * kRows;
  const int b = blockIdx.z;
  const int l = (int)(c / Mc);
  const double2* inb = in + (int64_t)b * Pin * ncol;
  double2* outb = out + (int64_t)b * Pout * ncol;
  Acc ar[kRows], ai[kRows];
#pragma unroll
  for (int k = 0; k < kRows; ++k) ar[k] = ai[k] = Acc{0.f, 0.f};
  for (int i0 = 0; i0 < Pin; i0 += kChunk) {
    const int cnt = min(kChunk, Pin - i0);
    __syncthreads();
    for (int idx = threadIdx.x; idx < kRows * kChunk; idx += kThreads) {
      const int r = idx / kChunk, i = idx - r * kChunk, p = p0 + r;
      Rs2[idx] = (p < Pout && i < cnt) ? R2[(int64_t)p * Pin + i0 + i] : make_float2(0.f, 0.f);
    }
    __syncthreads();
    if (c < ncol) {
      for (int i = 0; i < cnt; ++i) {
        double2 v = inb[(int64_t)(i0 + i) * ncol + c];
        if (wi != nullptr) {
          const double w = wi[(int64_t)(i0 + i) * L + l];
          v = make_double2(v.x * w, v.y * w);
        }
        const float4 x = split(v);
#pragma unroll
        for (int k = 0; k < kRows; ++k) {
          const float2 w = Rs2[k * kChunk + i];
          acc_add(ar[k], x.x, x.y, w.x, w.y);
          acc_add(ai[k], x.z, x.w, w.x, w.y);
        }
      }
    }
  }
  if (c < ncol) {
#pragma unroll
    for (int k = 0; k < kRows; ++k) {
      const int p = p0 + k;
      if (p >= Pout) break;
      double2 r = make_double2(to_double(ar[k]), to_double(ai[k]));
      if (wo != nullptr) {
        const double w = wo[(int64_t)p * L + l];
        r = make_double2(r.x * w, r.y * w);
      }
      double2* o = outb + (int64_t)p * ncol + c;
      if (accumulate) r = make_double2(o->x + r.x, o->y + r.y);
      *o = r;
    }
  }
}

}  // namespace

cudaError_t launch_radial_gen(const float2* R2, const double2* in, double2* out, int B, int Pout, int Pin, int L,
                              int Mc, const double* wi, const double* wo, bool accumulate, cudaStream_t st) {
  const int64_t ncol = (int64_t)L * Mc;
  dim3 grid((unsigned)((ncol + kThreads - 1) / kThreads), (Pout + kRows - 1) / kRows, B);
  k_radial_gen<<<grid, kThreads, 0, st>>>(R2, in, out, Pout, Pin, ncol, Mc, L, wi, wo, accumulate ? 1 : 0);
  return cudaGetLastError();
}

cudaError_t launch_radial(const double* R, const float2* R2, const double2* in, double2* out, int B, int P,
                          int64_t ncol, bool c32, cudaStream_t st) {
  dim3 grid((unsigned)((ncol + kThreads - 1) / kThreads), (P + kRows - 1) / kRows, B);
  if (c32) k_radial<true><<<grid, kThreads, 0, st>>>(R, R2, in, out, P, ncol);
  else k_radial<false><<<grid, kThreads, 0, st>>>(R, R2, in, out, P, ncol);
  return cudaGetLastError();
}

}  // namespace s2w

// FMA throughput probe (peak denominators for the roofline): many independent chains per thread, fixed trip count.
#include <cstdio>
#include <cuda_runtime.h>
template <class T>
__global__ void k(T* out, int iters, T a, T b) {
  T x0 = threadIdx.x * (T)1e-3, x1 = x0 + 1, x2 = x0 + 2, x3 = x0 + 3, x4 = x0 + 4, x5 = x0 + 5, x6 = x0 + 6, x7 = x0 + 7;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      x0 = fma(x0, a, b); x1 = fma(x1, a, b); x2 = fma(x2, a, b); x3 = fma(x3, a, b);
      x4 = fma(x4, a, b); x5 = fma(x5, a, b); x6 = fma(x6, a, b); x7 = fma(x7, a, b);
    }
  }
  out[blockIdx.x * blockDim.x + threadIdx.x] = x0 + x1 + x2 + x3 + x4 + x5 + x6 + x7;
}
template <class T> double run(const char* name, int iters) {
  int sms; cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, 0);
  int blocks = sms * 8, threads = 256;
  T* out; cudaMalloc(&out, sizeof(T) * blocks * threads);
  k<T><<<blocks, threads>>>(out, 10, (T)0.999, (T)0.001);
  cudaEvent_t e0, e1; cudaEventCreate(&e0); cudaEventCreate(&e1);
  float best = 1e30f;
  for (int r = 0; r < 5; ++r) {
    cudaEventRecord(e0); k<T><<<blocks, threads>>>(out, iters, (T)0.999, (T)0.001); cudaEventRecord(e1);
    cudaEventSynchronize(e1); float ms; cudaEventElapsedTime(&ms, e0, e1); if (ms < best) best = ms;
  }
  double flops = 2.0 * 64 * (double)iters * blocks * threads;
  double tf = flops / (best * 1e-3) / 1e12;
  printf("%s: %.3f TFLOP/s (%.3f ms, sms=%d)\n", name, tf, best, sms);
  cudaFree(out);
  return tf;
}
int main() {
  cudaError_t e = cudaSetDevice(0); if (e) { printf("no device\n"); return 1; }
  run<double>("fp64 fma", 4000);
  run<float>("fp32 fma", 40000);
  run<double>("fp64 fma", 4000);
  e = cudaDeviceSynchronize(); printf("status %s\n", cudaGetErrorString(e));
  return e != cudaSuccess;
}

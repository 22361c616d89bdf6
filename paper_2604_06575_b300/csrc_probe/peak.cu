// ALU peak probe used to state roofline denominators for the ALU-bound
// kernels: long chains of independent fused multiply-adds in registers.
#include <cuda_runtime.h>
#include <stdint.h>

template <typename T>
__global__ void __launch_bounds__(256) fma_chains(T* out, int64_t iters, T a, T b) {
  T x[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) x[i] = T(threadIdx.x + i) * T(1e-3);
  for (int64_t it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < 8; ++i) x[i] = x[i] * a + b;
  }
  T s = 0;
#pragma unroll
  for (int i = 0; i < 8; ++i) s += x[i];
  if (s == T(12345.678)) out[threadIdx.x] = s;  // keeps the chains live
}

extern "C" {
// kind 0: FP32 FMA, kind 1: FP64 FMA.  Runs `reps` launches of
// blocks_per_sm * SMs CTAs x 256 threads x iters x 8 FMAs and returns the best
// rate in TFLOP/s (2 flops per FMA) in *tflops.  Returns 0 on success.
int polylab_probe_alu(int kind, int64_t iters, int blocks_per_sm, int reps, double* tflops) {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 1;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  void* out = nullptr;
  if (cudaMalloc(&out, 256 * sizeof(double)) != cudaSuccess) return 2;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  const int grid = sms * blocks_per_sm;
  double best = 0.0;
  for (int r = 0; r < reps; ++r) {
    cudaEventRecord(e0);
    if (kind == 0) fma_chains<float><<<grid, 256>>>((float*)out, iters, 0.999f, 1e-4f);
    else fma_chains<double><<<grid, 256>>>((double*)out, iters, 0.999, 1e-4);
    cudaEventRecord(e1);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    const double flops = 2.0 * 8.0 * (double)iters * 256.0 * grid;
    const double t = flops / (ms * 1e-3) / 1e12;
    if (t > best) best = t;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(out);
  *tflops = best;
  return cudaGetLastError() == cudaSuccess ? 0 : 3;
}
}

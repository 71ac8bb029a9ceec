// FP32 arithmetic peak of the current GPU, measured: the denominator of the
// push kernel's ALU roofline. Every thread runs eight independent chains of
// fused multiply-adds (scalar FMA, or the packed two-lane FMA of sm_100 and
// later), long enough that the launch cost is negligible; the grid covers
// every SM several times over. FLOPs = 2 per lane per FMA.
#include <cuda_runtime.h>

#include "../../include/pic.h"

namespace {

constexpr int kChains = 8;
constexpr int kThreads = 256;

__global__ void __launch_bounds__(kThreads) k_fma_scalar(float* out, int iters, float m, float c) {
  float a[kChains];
#pragma unroll
  for (int j = 0; j < kChains; j++) a[j] = (float)(threadIdx.x + j) * 1e-3f;
  for (int i = 0; i < iters; i++) {
#pragma unroll
    for (int r = 0; r < 16; r++) {
#pragma unroll
      for (int j = 0; j < kChains; j++) a[j] = fmaf(a[j], m, c);
    }
  }
  float s = 0.0f;
#pragma unroll
  for (int j = 0; j < kChains; j++) s += a[j];
  if (s == 12345.678f) out[blockIdx.x * blockDim.x + threadIdx.x] = s;   // keeps the chains live
}

__global__ void __launch_bounds__(kThreads) k_fma_packed(float* out, int iters, float m, float c) {
  float2 a[kChains];
#pragma unroll
  for (int j = 0; j < kChains; j++) a[j] = make_float2((float)(threadIdx.x + j) * 1e-3f, (float)j * 1e-3f);
  const float2 m2 = make_float2(m, m), c2 = make_float2(c, c);
  for (int i = 0; i < iters; i++) {
#pragma unroll
    for (int r = 0; r < 16; r++) {
#pragma unroll
      for (int j = 0; j < kChains; j++) a[j] = __ffma2_rn(a[j], m2, c2);
    }
  }
  float s = 0.0f;
#pragma unroll
  for (int j = 0; j < kChains; j++) s += a[j].x + a[j].y;
  if (s == 12345.678f) out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// best of `reps` timed launches, TFLOP/s
template <class K>
double time_kernel(K kern, float* out, int blocks, int iters, double flops_per_thread, int reps) {
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  kern<<<blocks, kThreads>>>(out, iters, 0.9999999f, 1e-7f);   // warm-up: clocks up
  double best = 0.0;
  for (int r = 0; r < reps; r++) {
    cudaEventRecord(e0);
    kern<<<blocks, kThreads>>>(out, iters, 0.9999999f, 1e-7f);
    cudaEventRecord(e1);
    cudaEventSynchronize(e1);
    float ms = 0.0f;
    cudaEventElapsedTime(&ms, e0, e1);
    const double tf = flops_per_thread * (double)blocks * kThreads / (ms * 1e-3) / 1e12;
    if (tf > best) best = tf;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return best;
}

}  // namespace

extern "C" int pic_measure_fp32_peak(double* scalar_tflops, double* packed_tflops) {
  if (!scalar_tflops || !packed_tflops) return PIC_EINVAL;
  int dev = 0, nsm = 0, per_sm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return PIC_ECUDA;
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fma_scalar, kThreads, 0);
  const int blocks = nsm * (per_sm > 0 ? per_sm : 1) * 4;
  const int iters = 4096;
  const double fma_per_thread = (double)iters * 16 * kChains;
  // one slot per thread for the (practically never taken) store that keeps the chains live
  float* out = nullptr;
  if (cudaMalloc(&out, sizeof(float) * (size_t)blocks * kThreads) != cudaSuccess) return PIC_ENOMEM;
  *scalar_tflops = time_kernel(k_fma_scalar, out, blocks, iters, 2.0 * fma_per_thread, 5);
  *packed_tflops = time_kernel(k_fma_packed, out, blocks, iters, 4.0 * fma_per_thread, 5);
  cudaFree(out);
  return cudaGetLastError() == cudaSuccess ? PIC_OK : PIC_ECUDA;
}

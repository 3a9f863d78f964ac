// peaks.cu — measured issue rates of the arithmetic units the retrieval's
// kernels are bound by (FP32 FMA, the SFU's ex2, FP64 FMA), for the
// roofline denominators: independent chains per thread, every SM loaded,
// timed with CUDA events. fire_measure_peak (include/firert.h).
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/firert.h"

namespace {

constexpr int kChains = 8;       // independent dependency chains per thread
constexpr int kThreads = 512;

// 8 chains of FP32 FMA; each loop trip is 8 x 8 FMAs
__global__ void __launch_bounds__(kThreads) fma32_kernel(long long trips, float seed, float *sink) {
  float a[kChains];
#pragma unroll
  for (int c = 0; c < kChains; c++) a[c] = seed + (float)(threadIdx.x + c);
  const float m = 0.999999f, k = 1e-7f;
  for (long long t = 0; t < trips; t++) {
#pragma unroll
    for (int r = 0; r < 8; r++)
#pragma unroll
      for (int c = 0; c < kChains; c++) a[c] = fmaf(a[c], m, k);
  }
  float s = 0.f;
#pragma unroll
  for (int c = 0; c < kChains; c++) s += a[c];
  if (s == 12345.f) sink[threadIdx.x] = s;   // keeps the chains live
}

// the same with the packed two-lane FP32 FMA (two FMAs per instruction)
__global__ void __launch_bounds__(kThreads) fma32x2_kernel(long long trips, float seed, float *sink) {
  float2 a[kChains];
#pragma unroll
  for (int c = 0; c < kChains; c++) a[c] = make_float2(seed + c, seed - c);
  const float2 m = make_float2(0.999999f, 0.999999f), k = make_float2(1e-7f, 1e-7f);
  for (long long t = 0; t < trips; t++) {
#pragma unroll
    for (int r = 0; r < 8; r++)
#pragma unroll
      for (int c = 0; c < kChains; c++) a[c] = __ffma2_rn(a[c], m, k);
  }
  float s = 0.f;
#pragma unroll
  for (int c = 0; c < kChains; c++) s += a[c].x + a[c].y;
  if (s == 12345.f) sink[threadIdx.x] = s;
}

// 8 chains of the SFU's base-2 exponential (ex2.approx); the argument stays
// in (-1, 0) so no chain under- or overflows
__global__ void __launch_bounds__(kThreads) ex2_kernel(long long trips, float seed, float *sink) {
  float a[kChains];
#pragma unroll
  for (int c = 0; c < kChains; c++) a[c] = -0.5f - 0.01f * (float)c - 1e-6f * seed;
  for (long long t = 0; t < trips; t++) {
#pragma unroll
    for (int r = 0; r < 8; r++)
#pragma unroll
      for (int c = 0; c < kChains; c++) {
        float y;
        asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(a[c]));
        a[c] = -y;   // ex2 of a value in (-1, 0) is in (0.5, 1): the next argument is in (-1, -0.5)
      }
  }
  float s = 0.f;
#pragma unroll
  for (int c = 0; c < kChains; c++) s += a[c];
  if (s == 12345.f) sink[threadIdx.x] = s;
}

__global__ void __launch_bounds__(kThreads) fma64_kernel(long long trips, double seed, double *sink) {
  double a[kChains];
#pragma unroll
  for (int c = 0; c < kChains; c++) a[c] = seed + (double)(threadIdx.x + c);
  const double m = 0.999999999, k = 1e-12;
  for (long long t = 0; t < trips; t++) {
#pragma unroll
    for (int r = 0; r < 8; r++)
#pragma unroll
      for (int c = 0; c < kChains; c++) a[c] = fma(a[c], m, k);
  }
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < kChains; c++) s += a[c];
  if (s == 12345.0) sink[threadIdx.x] = s;
}

}  // namespace

extern "C" fire_status_t fire_measure_peak(int32_t kind, double *rate, double *seconds,
                                           fire_stream_t stream) {
  if (!rate || kind < 0 || kind > 3) return FIRE_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return FIRE_ERR_CUDA;
  void *sink = nullptr;
  if (cudaMalloc(&sink, kThreads * sizeof(double)) != cudaSuccess) return FIRE_ERR_NOMEM;
  const int blocks = sms * 4;          // 4 x 512 threads: 64 warps, every scheduler full
  // operations per loop trip and thread: 8 x 8 instructions
  const double per_trip = kind == 1 ? 2.0 * 64 : 64.0;
  long long trips = kind == 3 ? 2000 : 20000;   // FP64 runs at a small fraction of FP32
  cudaEvent_t a, b;
  cudaEventCreate(&a);
  cudaEventCreate(&b);
  auto run = [&](long long n) {
    switch (kind) {
      case 0: fma32_kernel<<<blocks, kThreads, 0, st>>>(n, 1.f, (float *)sink); break;
      case 1: fma32x2_kernel<<<blocks, kThreads, 0, st>>>(n, 1.f, (float *)sink); break;
      case 2: ex2_kernel<<<blocks, kThreads, 0, st>>>(n, 1.f, (float *)sink); break;
      default: fma64_kernel<<<blocks, kThreads, 0, st>>>(n, 1.0, (double *)sink); break;
    }
  };
  run(trips / 10);                     // warm-up
  cudaEventRecord(a, st);
  run(trips);
  cudaEventRecord(b, st);
  cudaError_t e = cudaEventSynchronize(b);
  float ms = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  cudaFree(sink);
  if (e != cudaSuccess || !(ms > 0.f)) return FIRE_ERR_CUDA;
  const double ops = per_trip * (double)trips * (double)blocks * kThreads;
  // FMA counts two flops; ex2 one operation
  *rate = (kind == 2 ? 1.0 : 2.0) * ops / (ms * 1e-3);
  if (seconds) *seconds = ms * 1e-3;
  return FIRE_OK;
}

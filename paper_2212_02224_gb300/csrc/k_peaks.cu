// Arithmetic throughput probe: independent dependency chains of float32 FMA,
// packed float32x2 FMA, float64 FMA and MUFU reciprocal square root over a
// grid of 8 CTAs x 256 threads per SM, timed with CUDA events on the caller's
// stream.  It measures the ceilings the fused kernel's roofline refers to; it
// is not a step of the planning method.
#include "internal.cuh"

namespace plan {
namespace {

constexpr int kChains = 8;

__global__ void __launch_bounds__(256) ffma_kernel(float* out, int iters, float b, float c) {
  float a[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) a[k] = 1e-3f * float(threadIdx.x + k);
  for (int i = 0; i < iters; ++i)
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = __fmaf_rn(a[k], b, c);
  float s = 0.f;
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += a[k];
  if (s == 12345.f) out[blockIdx.x] = s;   // keeps the chains alive
}

__global__ void __launch_bounds__(256) ffma2_kernel(float* out, int iters, float b, float c) {
  float2 a[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) a[k] = make_float2(1e-3f * float(threadIdx.x + k), 2e-3f * float(k));
  const float2 bb = make_float2(b, b), cc = make_float2(c, c);
  for (int i = 0; i < iters; ++i)
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = __ffma2_rn(a[k], bb, cc);
  float s = 0.f;
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += a[k].x + a[k].y;
  if (s == 12345.f) out[blockIdx.x] = s;
}

__global__ void __launch_bounds__(256) dfma_kernel(float* out, int iters, double b, double c) {
  double a[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) a[k] = 1e-3 * double(threadIdx.x + k);
  for (int i = 0; i < iters; ++i)
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = __fma_rn(a[k], b, c);
  double s = 0.0;
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += a[k];
  if (s == 12345.0) out[blockIdx.x] = float(s);
}

__global__ void __launch_bounds__(256) rsqrt_kernel(float* out, int iters, float c) {
  float a[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) a[k] = 1.f + 1e-3f * float(threadIdx.x + k);
  for (int i = 0; i < iters; ++i)
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = rsqrtf(a[k]) + c;
  float s = 0.f;
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += a[k];
  if (s == 12345.f) out[blockIdx.x] = s;
}

template <class F>
int time_best(F launch, cudaStream_t s, float* ms_out) {
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return -1;
  float best = 1e30f;
  launch();   // warm-up
  for (int r = 0; r < 3; ++r) {
    cudaEventRecord(e0, s);
    launch();
    cudaEventRecord(e1, s);
    if (cudaEventSynchronize(e1) != cudaSuccess) break;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    best = ms < best ? ms : best;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  *ms_out = best;
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

}  // namespace

int probe_alu(double* out, cudaStream_t s) {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return -1;
  float* sink = nullptr;
  const int blocks = sms * 8, threads = 256;
  if (cudaMallocAsync(&sink, sizeof(float) * blocks, s) != cudaSuccess) return -1;
  const double lanes = double(blocks) * threads;
  const int it32 = 16384, it64 = 512, itmu = 4096;
  float ms = 0.f;
  int st = 0;
  st |= time_best([&] { ffma_kernel<<<blocks, threads, 0, s>>>(sink, it32, 0.999f, 1e-3f); }, s, &ms);
  out[0] = lanes * it32 * kChains * 2.0 / (ms * 1e-3) / 1e12;            // TFLOP/s
  st |= time_best([&] { ffma2_kernel<<<blocks, threads, 0, s>>>(sink, it32, 0.999f, 1e-3f); }, s, &ms);
  out[1] = lanes * it32 * kChains * 4.0 / (ms * 1e-3) / 1e12;            // TFLOP/s
  st |= time_best([&] { dfma_kernel<<<blocks, threads, 0, s>>>(sink, it64, 0.999, 1e-3); }, s, &ms);
  out[2] = lanes * it64 * kChains * 2.0 / (ms * 1e-3) / 1e12;            // TFLOP/s
  st |= time_best([&] { rsqrt_kernel<<<blocks, threads, 0, s>>>(sink, itmu, 1e-3f); }, s, &ms);
  out[3] = lanes * itmu * kChains / (ms * 1e-3) / 1e12;                  // T rsqrt / s
  out[4] = double(sms);
  cudaFreeAsync(sink, s);
  return st;
}

}  // namespace plan

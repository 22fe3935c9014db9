// FP32 throughput ceiling of the device (ps_fp32_peak): the second roofline of the
// interpolation and wavelet kernels, which run FP32 FMAs (packed FP32x2 where they can).
// Each thread runs independent FMA chains long enough that issue, not latency, limits
// them; the grid fills every SM with 8 CTAs of 256 threads.
#include <cuda_runtime.h>

#include <algorithm>
#include <string>

#include "internal.h"
#include "packed.cuh"

namespace ps {

constexpr int kPeakChains = 8;

template <bool PACKED>
__global__ void __launch_bounds__(256) k_fma_peak(int iters, float seed, float* __restrict__ sink) {
  const float s0 = seed + 1e-3f * (float)threadIdx.x;
  float total = 0.f;
  if (PACKED) {
    u64 a[kPeakChains];
#pragma unroll
    for (int k = 0; k < kPeakChains; ++k) a[k] = f2pack(s0 + k, s0 - k);
    const u64 m = f2pack(0.9999999f, 1.0000001f), c = f2pack(1e-7f, -1e-7f);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
      for (int k = 0; k < kPeakChains; ++k) a[k] = ffma2(a[k], m, c);
    }
#pragma unroll
    for (int k = 0; k < kPeakChains; ++k) {
      float x, y;
      f2unpack(a[k], x, y);
      total += x + y;
    }
  } else {
    float a[2 * kPeakChains];
#pragma unroll
    for (int k = 0; k < 2 * kPeakChains; ++k) a[k] = s0 + k;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
      for (int k = 0; k < 2 * kPeakChains; ++k) a[k] = fmaf(a[k], 0.9999999f, 1e-7f);
    }
#pragma unroll
    for (int k = 0; k < 2 * kPeakChains; ++k) total += a[k];
  }
  if (total == 1234.5f) sink[0] = total;   // keeps the chains live; never true for these inputs
}

}  // namespace ps

#pragma GCC visibility push(default)
extern "C" ps_status ps_fp32_peak(int32_t packed, double* flops_per_s) {
  using namespace ps;
  if (!flops_per_s) return PS_EINVAL;
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  float* sink = nullptr;
  cudaStream_t st = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (e == cudaSuccess) e = cudaMalloc((void**)&sink, sizeof(float));
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  const int iters = 8192, ctas = 8 * std::max(1, sms);
  float best = 0.f;
  for (int rep = 0; rep < 4 && e == cudaSuccess; ++rep) {
    if (packed) k_fma_peak<true><<<ctas, 256, 0, st>>>(iters, 0.5f, sink);
    else k_fma_peak<false><<<ctas, 256, 0, st>>>(iters, 0.5f, sink);
    e = cudaEventRecord(e0, st);
    if (packed) k_fma_peak<true><<<ctas, 256, 0, st>>>(iters, 0.5f, sink);
    else k_fma_peak<false><<<ctas, 256, 0, st>>>(iters, 0.5f, sink);
    if (e == cudaSuccess) e = cudaEventRecord(e1, st);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e == cudaSuccess && (best == 0.f || ms < best)) best = ms;
  }
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e1) cudaEventDestroy(e1);
  if (e0) cudaEventDestroy(e0);
  if (st) cudaStreamDestroy(st);
  if (sink) cudaFree(sink);
  if (e != cudaSuccess || !(best > 0.f)) {
    set_global_error(std::string("fp32_peak: ") + cudaGetErrorString(e));
    return PS_ECUDA;
  }
  // 2 FLOPs per FMA; a packed FMA is two.
  const double fmas = (double)ctas * 256.0 * iters * 2.0 * kPeakChains;
  *flops_per_s = 2.0 * fmas / (best * 1e-3);
  return PS_OK;
}
#pragma GCC visibility pop

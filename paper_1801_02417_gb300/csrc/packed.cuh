// Packed FP32x2 arithmetic for the CUDA kernels (sm_100 family and later): two
// FP32 lanes in one 64-bit register pair, one fma.rn.f32x2 for both. Each lane is
// rounded exactly like a separate fmaf.
#pragma once

#include <cuda_runtime.h>

namespace ps {

typedef unsigned long long u64;
__device__ __forceinline__ u64 f2pack(float a, float b) {
  u64 r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
  return r;
}
__device__ __forceinline__ void f2unpack(u64 v, float& a, float& b) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(v));
}
__device__ __forceinline__ u64 ffma2(u64 a, u64 b, u64 c) {
  u64 d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}
__device__ __forceinline__ u64 fdup(float a) { return f2pack(a, a); }
// Ordering of generic-proxy shared-memory accesses before later bulk (async-proxy) copies.
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

}  // namespace ps

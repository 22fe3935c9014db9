// Device helpers shared by the CUDA kernels (sm_100 family and later).
// Packed FP32x2 arithmetic: two FP32 lanes in one 64-bit register pair, one
// fma.rn.f32x2 for both; each lane is rounded exactly like a separate fmaf.
// Bulk copies (cp.async.bulk, global to shared) completing on mbarriers, with
// bounded waits.
#pragma once

#include <cstdint>

#include <cuda.h>
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

// ---- bulk-copy (TMA) and mbarrier helpers (inline PTX, sm_90+).
__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}
// 2D tensor-map copy (TMA) of one box into shared memory (128-byte aligned destination), completing
// on `bar`. The map lives in kernel-parameter space (a __grid_constant__ argument). x is the
// innermost coordinate in elements (x * 4 bytes a multiple of 16 for float data); parts of the
// box outside the tensor are filled with zeros and still count toward the transaction bytes.
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
          smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}

// Poll budget of the bounded waits. c_wait_polls (one copy per translation unit,
// set by set_wait_polls_here) bounds the first wait on a barrier phase; a CTA
// whose wait gave up drains its copies still in flight with the full budget
// (mbar_drain) before it returns, so no copy lands after it has exited.
constexpr uint32_t kWaitPolls = 1u << 22;
static __constant__ uint32_t c_wait_polls = kWaitPolls;

__device__ __forceinline__ bool mbar_poll(uint64_t* bar, uint32_t parity, uint32_t polls) {
  const uint32_t a = smem_u32(bar);
  for (uint32_t i = 0; i < polls; ++i) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(a), "r"(parity)
        : "memory");
    if (ok) return true;
  }
  return false;
}
// Bounded wait on phase `parity`: false (and the caller raises the error flag) if it never completes.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) { return mbar_poll(bar, parity, c_wait_polls); }
// Second wait of a CTA that gave up: the copies it issued get the full budget to land.
__device__ __forceinline__ bool mbar_drain(uint64_t* bar, uint32_t parity) { return mbar_poll(bar, parity, kWaitPolls); }

// Host side: sets this translation unit's c_wait_polls (polls < 0: the default).
static inline cudaError_t set_wait_polls_here(int polls) {
  const uint32_t v = polls < 0 ? kWaitPolls : (uint32_t)polls;
  return cudaMemcpyToSymbol(c_wait_polls, &v, sizeof(v));
}
}  // namespace ps

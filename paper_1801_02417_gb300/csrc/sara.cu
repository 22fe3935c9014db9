// SARA dictionary (Section 4.1) on the GPU: Dirac + Daubechies db1..db8, periodic
// orthonormal 2D Mallat transforms, concatenation scaled by 1/3.
//
// Analysis Psi^dagger runs one launch per level for all 8 Daubechies bases and 4
// maps (grid.y = basis, grid.z = map). Each CTA computes one TO x TO tile of the
// four subbands from a (2 TO + 14)^2 input tile held in shared memory (rows
// filtered first, then columns; indices modulo the level size, i.e. periodic).
// The detail coefficients are consumed in the epilogue instead of being stored:
//   SARA_DUAL      A = clamp(A + rho1/3 * coef, -gamma W, +gamma W)   (Alg. 1 steps 5-6)
//   SARA_APPLY     A = coef / 3                                       (operator)
//   SARA_REWEIGHT  gamma W = gamma delta / (delta + |coef / 3|)       (Eq. weights)
// Only the approximation goes to scratch for the next level.
//
// Synthesis Psi runs one launch per level from coarse to fine; the finest level
// sums the eight bases and the Dirac part in registers and writes Psi A once.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <mutex>
#include <string>

#include "internal.h"
#include "packed.cuh"

namespace ps {

__constant__ __align__(16) float c_h[kDb][kMaxTaps];
__constant__ __align__(16) float c_g[kDb][kMaxTaps];
// The same taps duplicated in both halves of a 64-bit word, the operand of packed
// FP32x2 FMAs that apply one tap to two neighbouring samples.
__constant__ __align__(16) float2 c_hd[kDb][kMaxTaps];
__constant__ __align__(16) float2 c_gd[kDb][kMaxTaps];

cudaError_t upload_filters(const double h[kDb][kMaxTaps], cudaStream_t stream) {
  float hf[kDb][kMaxTaps], gf[kDb][kMaxTaps];
  for (int b = 0; b < kDb; ++b) {
    const int Lf = 2 * (b + 1);
    for (int j = 0; j < kMaxTaps; ++j) {
      hf[b][j] = j < Lf ? (float)h[b][j] : 0.f;
      gf[b][j] = j < Lf ? (float)(((j & 1) ? -1.0 : 1.0) * h[b][Lf - 1 - j]) : 0.f;
    }
  }
  float2 hd[kDb][kMaxTaps], gd[kDb][kMaxTaps];
  for (int b = 0; b < kDb; ++b)
    for (int j = 0; j < kMaxTaps; ++j) {
      hd[b][j] = make_float2(hf[b][j], hf[b][j]);
      gd[b][j] = make_float2(gf[b][j], gf[b][j]);
    }
  // On the caller's stream and waited for: kernels launched on non-blocking streams are
  // not ordered after the legacy stream's copies.
  cudaError_t e = cudaMemcpyToSymbolAsync(c_h, hf, sizeof(hf), 0, cudaMemcpyHostToDevice, stream);
  if (e == cudaSuccess) e = cudaMemcpyToSymbolAsync(c_g, gf, sizeof(gf), 0, cudaMemcpyHostToDevice, stream);
  if (e == cudaSuccess) e = cudaMemcpyToSymbolAsync(c_hd, hd, sizeof(hd), 0, cudaMemcpyHostToDevice, stream);
  if (e == cudaSuccess) e = cudaMemcpyToSymbolAsync(c_gd, gd, sizeof(gd), 0, cudaMemcpyHostToDevice, stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
  return e;
}

// A tap pair as one 64-bit FMA operand: {c[j], c[j+1]} (j even) or a duplicated tap.
__device__ __forceinline__ u64 cpair(const float* c) { return *reinterpret_cast<const u64*>(c); }
__device__ __forceinline__ u64 cdup(const float2& c) { return *reinterpret_cast<const u64*>(&c); }

// Calls CALL(LF) with the compile-time filter length of basis bi (db1..db8).
#define PS_SWITCH_LF(bi, CALL)    \
  switch (bi) {                   \
    case 0: CALL(2); break;       \
    case 1: CALL(4); break;       \
    case 2: CALL(6); break;       \
    case 3: CALL(8); break;       \
    case 4: CALL(10); break;      \
    case 5: CALL(12); break;      \
    case 6: CALL(14); break;      \
    default: CALL(16); break;     \
  }

__device__ __forceinline__ void sara_epilogue(int mode, float val, size_t idx, float* coef, float* thr, float scale,
                                              float gamma, float delta) {
  if (mode == SARA_DUAL) {
    const float t = thr[idx];
    const float a = fmaf(scale, val, coef[idx]);
    coef[idx] = fminf(fmaxf(a, -t), t);
  } else if (mode == SARA_APPLY) {
    coef[idx] = scale * val;
  } else {
    thr[idx] = gamma * delta / (delta + fabsf(scale * val));
  }
}

// One synthesis level: coefficients at level l (approximation from `approx_in`
// or, at the coarsest level, from coef; details from coef) -> approximation at
// level l-1 (m x m) into approx_out, or at level 1 the summed image
// out = (A_dirac + sum_b synth_b) / 3.
__global__ void __launch_bounds__(256) k_synthesis(const float* __restrict__ coef, const float* __restrict__ approx_in,
                                                   int coarsest, int m, int TI, int n, int finest,
                                                   float* __restrict__ approx_out, float* __restrict__ out) {
  extern __shared__ float sm[];
  const int map = blockIdx.z;
  const int hm = m >> 1;
  const int tilesx = m / TI;
  const int oy0 = (blockIdx.x / tilesx) * TI, ox0 = (blockIdx.x % tilesx) * TI;
  const int CI = TI / 2 + kMaxTaps / 2 - 1;      // coefficient tile side (sized for db8)
  float* s_ll = sm;
  float* s_lh = s_ll + CI * CI;
  float* s_hl = s_lh + CI * CI;
  float* s_hh = s_hl + CI * CI;
  float* s_lo = s_hh + CI * CI;                   // TI x CI
  float* s_hi = s_lo + TI * CI;
  constexpr int kOut = 8;                         // outputs per thread (TI^2 <= 8 * 256)
  float accv[kOut];
#pragma unroll
  for (int t = 0; t < kOut; ++t) accv[t] = 0.f;
  const int b_begin = finest ? 0 : blockIdx.y, b_end = finest ? kDb : blockIdx.y + 1;
  for (int bi = b_begin; bi < b_end; ++bi) {
    const int Lf = 2 * (bi + 1);
    const int half = Lf / 2 - 1;
    const int ky0 = oy0 / 2 - half, kx0 = ox0 / 2 - half;
    const int CIb = TI / 2 + half;                 // rows/cols actually used by this basis
    const size_t base = ((size_t)map * kBases + (bi + 1)) * (size_t)n * n;
    const float* apx = coarsest ? nullptr : approx_in + ((size_t)map * kDb + bi) * (size_t)hm * hm;
    for (int i = threadIdx.x; i < CIb * CIb; i += blockDim.x) {
      const int r = i / CIb, c = i - r * CIb;
      const int Yk = ((ky0 + r) % hm + hm) % hm, Xk = ((kx0 + c) % hm + hm) % hm;
      s_ll[r * CI + c] = coarsest ? coef[base + (size_t)Yk * n + Xk] : apx[(size_t)Yk * hm + Xk];
      s_hl[r * CI + c] = coef[base + (size_t)Yk * n + hm + Xk];
      s_lh[r * CI + c] = coef[base + (size_t)(hm + Yk) * n + Xk];
      s_hh[r * CI + c] = coef[base + (size_t)(hm + Yk) * n + hm + Xk];
    }
    __syncthreads();
    const float* h = c_h[bi];
    const float* g = c_g[bi];
    // Along y: lo[r][c] = sum_j h[j] ll[kl][c] + g[j] lh[kl][c], kl = (r - j)/2 + half, j = r mod 2.
    for (int i = threadIdx.x; i < TI * CIb; i += blockDim.x) {
      const int r = i / CIb, c = i - r * CIb;
      float lo = 0.f, hi = 0.f;
      for (int j = (r & 1); j < Lf; j += 2) {
        const int kl = ((r - j) >> 1) + half;
        lo = fmaf(h[j], s_ll[kl * CI + c], fmaf(g[j], s_lh[kl * CI + c], lo));
        hi = fmaf(h[j], s_hl[kl * CI + c], fmaf(g[j], s_hh[kl * CI + c], hi));
      }
      s_lo[r * CI + c] = lo;
      s_hi[r * CI + c] = hi;
    }
    __syncthreads();
    // Along x.
#pragma unroll
    for (int t = 0; t < kOut; ++t) {
      const int i = threadIdx.x + t * blockDim.x;
      if (i < TI * TI) {
        const int r = i / TI, c = i - r * TI;
        float v = 0.f;
        for (int j = (c & 1); j < Lf; j += 2) {
          const int kl = ((c - j) >> 1) + half;
          v = fmaf(h[j], s_lo[r * CI + kl], fmaf(g[j], s_hi[r * CI + kl], v));
        }
        accv[t] += v;
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int t = 0; t < kOut; ++t) {
    const int i = threadIdx.x + t * blockDim.x;
    if (i < TI * TI) {
      const int r = i / TI, c = i - r * TI;
      const int y = oy0 + r, x = ox0 + c;
      if (finest) {
        const size_t dirac = (size_t)map * kBases * (size_t)n * n + (size_t)y * n + x;
        out[(size_t)map * n * n + (size_t)y * n + x] = (coef[dirac] + accv[t]) * (1.0f / 3.0f);
      } else {
        approx_out[((size_t)map * kDb + blockIdx.y) * (size_t)m * m + (size_t)y * m + x] = accv[t];
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Fast path for levels whose half size is >= 32: 32 x 32 output tiles, filter
// length and tile shape known at compile time, each thread producing a strip of
// four outputs from registers (inputs read once from shared memory per strip).
constexpr int kTO = 32;                          // analysis output tile (per subband)
constexpr int kRSmax = 2 * kTO + kMaxTaps - 2;   // 78: input tile side for db8
constexpr int kA2Cols = 2 * kTO + 16;            // 80 staged input columns (covers 2 TO + 14 for db8)
constexpr int kA2Pitch = kA2Cols + 4;            // 84 = 20 mod 32 banks: row-parallel 16-byte reads conflict-free
constexpr int kA2In = kRSmax * kA2Pitch;         // input tile
constexpr int kPlo = kTO + 4;                    // row-filtered tiles (16-byte aligned rows)
constexpr int kTI = 32;                          // synthesis output tile
constexpr int kCImax = kTI / 2 + kMaxTaps / 2 - 1;   // 23
constexpr int kPs = kCImax + 2;                  // 25

__device__ __forceinline__ int wrap1(int v, int m) { return v < 0 ? v + m : (v >= m ? v - m : v); }

// 4-byte asynchronous global->shared copies (cp.async), grouped and awaited per group.
__device__ __forceinline__ void cp_async4(float* dst, const float* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// Rows: lo/hi[r][k] = sum_j h/g[j] in[r][2k + j], k in [0, TO). Each thread makes
// four outputs of one row from 16-byte reads; the taps go in pairs,
// {c[2p], c[2p+1]} x {in[2k+2p], in[2k+2p+1]}, and the two halves are added at the end.
template <int LF>
__device__ __forceinline__ void ana_rows(const float* __restrict__ in_s, float* __restrict__ lo_s,
                                         float* __restrict__ hi_s) {
  constexpr int RS = 2 * kTO + LF - 2;
  constexpr int b = LF / 2 - 1;
  constexpr int NP = LF / 2 + 3;            // sample pairs feeding four outputs
  constexpr int NV = (NP + 1) / 2;          // 16-byte reads
  for (int u = threadIdx.x; u < RS * (kTO / 4); u += blockDim.x) {
    const int r = u % RS, k0 = (u / RS) * 4;
    const float* row = in_s + r * kA2Pitch + 2 * k0;
    u64 x[2 * NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      const ulonglong2 q = *reinterpret_cast<const ulonglong2*>(row + 4 * v);
      x[2 * v] = q.x;
      x[2 * v + 1] = q.y;
    }
    float lo[4], hi[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      u64 a = 0ull, c = 0ull;
#pragma unroll
      for (int p = 0; p < LF / 2; ++p) {
        a = ffma2(cpair(&c_h[b][2 * p]), x[q + p], a);
        c = ffma2(cpair(&c_g[b][2 * p]), x[q + p], c);
      }
      float a0, a1, c0, c1;
      f2unpack(a, a0, a1);
      f2unpack(c, c0, c1);
      lo[q] = a0 + a1;
      hi[q] = c0 + c1;
    }
    *reinterpret_cast<float4*>(lo_s + r * kPlo + k0) = make_float4(lo[0], lo[1], lo[2], lo[3]);
    *reinterpret_cast<float4*>(hi_s + r * kPlo + k0) = make_float4(hi[0], hi[1], hi[2], hi[3]);
  }
}

__device__ __forceinline__ float4 f4fma(float a, float4 x, float4 y) {
  return make_float4(fmaf(a, x.x, y.x), fmaf(a, x.y, y.y), fmaf(a, x.z, y.z), fmaf(a, x.w, y.w));
}
__device__ __forceinline__ float4 f4clamp(float4 a, float4 t) {
  return make_float4(fminf(fmaxf(a.x, -t.x), t.x), fminf(fmaxf(a.y, -t.y), t.y), fminf(fmaxf(a.z, -t.z), t.z),
                     fminf(fmaxf(a.w, -t.w), t.w));
}
__device__ __forceinline__ float4 f4of(u64 a, u64 b) {
  float4 r;
  f2unpack(a, r.x, r.y);
  f2unpack(b, r.z, r.w);
  return r;
}

// Epilogue on four consecutive coefficients (16-byte aligned).
__device__ __forceinline__ void sara_epilogue4(int mode, float4 v, size_t idx, float4 a_old, float4 t_old,
                                               float* coef, float* thr, float scale, float gamma, float delta) {
  if (mode == SARA_DUAL) {
    *reinterpret_cast<float4*>(coef + idx) = f4clamp(f4fma(scale, v, a_old), t_old);
  } else if (mode == SARA_APPLY) {
    *reinterpret_cast<float4*>(coef + idx) = make_float4(scale * v.x, scale * v.y, scale * v.z, scale * v.w);
  } else {
    const float gd = gamma * delta;
    *reinterpret_cast<float4*>(thr + idx) =
        make_float4(gd / (delta + fabsf(scale * v.x)), gd / (delta + fabsf(scale * v.y)),
                    gd / (delta + fabsf(scale * v.z)), gd / (delta + fabsf(scale * v.w)));
  }
}

// Columns + epilogue for one basis: four subbands of a TO x TO tile. Each thread
// owns four consecutive columns of one output row (two packed pairs per subband),
// so the epilogue reads and writes A and gamma W as float4 (staged before the filtering).
template <int LF>
__device__ __forceinline__ void ana_cols(const float* __restrict__ lo_s, const float* __restrict__ hi_s, int bi,
                                         int map, int n, int hm, int oy0, int ox0, int last, float* __restrict__ coef,
                                         float* __restrict__ thr, float* __restrict__ approx_out, int mode,
                                         float scale, float gamma, float delta, const float* __restrict__ st_a,
                                         const float* __restrict__ st_t) {
  constexpr int b = LF / 2 - 1;
  const size_t base = ((size_t)map * kBases + (bi + 1)) * (size_t)n * n;
  for (int u = threadIdx.x; u < kTO * kTO / 4; u += blockDim.x) {
    const int kx0 = (u % (kTO / 4)) * 4, ky = u / (kTO / 4);
    const int Y = oy0 + ky, X = ox0 + kx0;
    const size_t i_hl = base + (size_t)Y * n + (hm + X);
    const size_t i_lh = base + (size_t)(hm + Y) * n + X;
    const size_t i_hh = base + (size_t)(hm + Y) * n + (hm + X);
    const size_t i_ll = base + (size_t)Y * n + X;
    u64 ll0 = 0ull, ll1 = 0ull, lh0 = 0ull, lh1 = 0ull, hl0 = 0ull, hl1 = 0ull, hh0 = 0ull, hh1 = 0ull;
#pragma unroll
    for (int j = 0; j < LF; ++j) {
      const ulonglong2 a = *reinterpret_cast<const ulonglong2*>(lo_s + (2 * ky + j) * kPlo + kx0);
      const ulonglong2 c = *reinterpret_cast<const ulonglong2*>(hi_s + (2 * ky + j) * kPlo + kx0);
      const u64 ph = cdup(c_hd[b][j]), pg = cdup(c_gd[b][j]);
      ll0 = ffma2(ph, a.x, ll0);
      ll1 = ffma2(ph, a.y, ll1);
      lh0 = ffma2(pg, a.x, lh0);
      lh1 = ffma2(pg, a.y, lh1);
      hl0 = ffma2(ph, c.x, hl0);
      hl1 = ffma2(ph, c.y, hl1);
      hh0 = ffma2(pg, c.x, hh0);
      hh1 = ffma2(pg, c.y, hh1);
    }
    const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
    float4 a_hl = z, a_lh = z, a_hh = z, a_ll = z, t_hl = z, t_lh = z, t_hh = z, t_ll = z;
    if (mode == SARA_DUAL) {
      // Staged by the bulk-copy engine: [subband][row][32].
      const int so = ky * kTO + kx0;
      a_hl = *reinterpret_cast<const float4*>(st_a + so);
      a_lh = *reinterpret_cast<const float4*>(st_a + kTO * kTO + so);
      a_hh = *reinterpret_cast<const float4*>(st_a + 2 * kTO * kTO + so);
      t_hl = *reinterpret_cast<const float4*>(st_t + so);
      t_lh = *reinterpret_cast<const float4*>(st_t + kTO * kTO + so);
      t_hh = *reinterpret_cast<const float4*>(st_t + 2 * kTO * kTO + so);
      if (last) {
        a_ll = *reinterpret_cast<const float4*>(coef + i_ll);
        t_ll = *reinterpret_cast<const float4*>(thr + i_ll);
      }
    }
    sara_epilogue4(mode, f4of(hl0, hl1), i_hl, a_hl, t_hl, coef, thr, scale, gamma, delta);   // x-high, y-low
    sara_epilogue4(mode, f4of(lh0, lh1), i_lh, a_lh, t_lh, coef, thr, scale, gamma, delta);   // x-low, y-high
    sara_epilogue4(mode, f4of(hh0, hh1), i_hh, a_hh, t_hh, coef, thr, scale, gamma, delta);
    if (last) sara_epilogue4(mode, f4of(ll0, ll1), i_ll, a_ll, t_ll, coef, thr, scale, gamma, delta);
    else
      *reinterpret_cast<float4*>(approx_out + ((size_t)map * kDb + bi) * (size_t)hm * hm + (size_t)Y * hm + X) =
          f4of(ll0, ll1);
  }
}

// 2D tensor maps (TMA) of the arrays whose tiles the tiled SARA kernels stage, one box
// each, with the box's row pitch equal to the shared-memory pitch of the staged tile:
//   in    analysis input planes, width m, box kA2Pitch x kRSmax (the whole input tile)
//   coef  analysis: coefficients, width n, box kTO x kTO (one subband tile of A)
//   thr   analysis: thresholds gamma W, same box (one subband tile of gamma W)
//   scoef synthesis: coefficients, width n, box kC2Pitch x kC2Rows (one subband tile)
//   apx   synthesis: approximations of the level, width hm, same box
// A use_* flag is 0 when its map was not made (then the per-row bulk copies run).
// Tiles whose rows or columns wrap around the periodic edges always take the per-row copies.
struct SaraTma {
  CUtensorMap in, coef, thr, scoef, apx;
  int use_in, use_stage, use_scoef, use_apx;
};

// Input tile of one analysis CTA: RS rows from row 2 oy0 and the 80 columns from
// column 2 ox0 (both modulo m), one bulk copy per row, two where the row wraps
// around the periodic right edge (then the first piece is 64 columns).
__device__ __forceinline__ void ana_issue_input(const float* __restrict__ src, int m, int oy0, int ox0, int RS,
                                                float* __restrict__ in_s, uint64_t* bar) {
  const int x0 = 2 * ox0;
  const int first = min(kA2Cols, m - x0);
  if (threadIdx.x == 0) mbar_expect_tx(bar, (uint32_t)(RS * kA2Cols * sizeof(float)));
  for (int r = threadIdx.x; r < RS; r += blockDim.x) {
    int y = 2 * oy0 + r;
    if (y >= m) y -= m;
    const float* row = src + (size_t)y * m;
    float* dst = in_s + r * kA2Pitch;
    fence_proxy_async();
    bulk_g2s(dst, row + x0, first * sizeof(float), bar);
    if (first < kA2Cols) bulk_g2s(dst + first, row, (kA2Cols - first) * sizeof(float), bar);
  }
}

// The input tile by one tensor-map copy when it does not wrap (kRSmax rows of kA2Pitch
// columns; the rows past RS and columns past kA2Cols are not read), else by rows.
// `in_row0` is the row of the plane's first row in the input map.
__device__ __forceinline__ void ana_issue_input_t(const SaraTma& tm, int in_row0, const float* __restrict__ src,
                                                  int m, int oy0, int ox0, int RS, float* __restrict__ in_s,
                                                  uint64_t* bar) {
  if (tm.use_in && 2 * ox0 + kA2Cols <= m && 2 * oy0 + kRSmax <= m) {
    if (threadIdx.x == 0) {
      mbar_expect_tx(bar, (uint32_t)(kRSmax * kA2Pitch * sizeof(float)));
      fence_proxy_async();
      tma_load_2d(in_s, &tm.in, 2 * ox0, in_row0 + 2 * oy0, bar);
    }
  } else {
    ana_issue_input(src, m, oy0, ox0, RS, in_s, bar);
  }
}

// Shared-memory layout of the fast analysis kernels (floats): input tile, row-filtered
// low/high tiles, the staged A and gamma W rows of the three detail subbands, and two
// mbarriers (input tile, staged epilogue operands).
constexpr int kStage = 3 * kTO * kTO;
// Staged epilogue operands start on a 128-byte boundary (tensor-map copy destinations).
constexpr int kAnaPre = (kA2In + 2 * kRSmax * kPlo + 31) / 32 * 32;
constexpr int kAnaFloats = kAnaPre + 2 * kStage;
static_assert(kA2In % 4 == 0 && (kRSmax * kPlo) % 4 == 0 && kStage % 32 == 0, "aligned stage buffers");

// The first 3 * 32 * 2 threads each start one bulk copy of this tile's A and gamma W
// detail rows (3 subbands x 32 rows x 128 B) so they arrive while the rows are
// filtered; thread 0 sets the expected byte count (the barrier's transaction count
// may run ahead of it).
__device__ __forceinline__ void stage_epilogue(const float* coef, const float* thr, size_t base, int n, int hm,
                                               int oy0, int ox0, float* st_a, float* st_t, uint64_t* bar) {
  if (threadIdx.x == 0) mbar_expect_tx(bar, 2u * kStage * sizeof(float));
  const int k = threadIdx.x;
  if (k < 2 * 3 * kTO) {
    const int arr = k / (3 * kTO), kk = k - arr * (3 * kTO);
    const int sb = kk / kTO, r = kk - sb * kTO;
    const int Y = oy0 + r;
    const size_t off = sb == 0 ? base + (size_t)Y * n + hm + ox0
                               : (sb == 1 ? base + (size_t)(hm + Y) * n + ox0 : base + (size_t)(hm + Y) * n + hm + ox0);
    float* dst = (arr ? st_t : st_a) + sb * kTO * kTO + r * kTO;
    fence_proxy_async();   // the persistent form refills buffers its threads have read
    bulk_g2s(dst, (arr ? thr : coef) + off, kTO * sizeof(float), bar);
  }
}

// The same operands as six tensor-map copies (three subband tiles of A and of gamma W) by
// one thread, when the maps were made; `prow` is the row of the basis plane in the maps.
__device__ __forceinline__ void stage_epilogue_t(const SaraTma& tm, const float* coef, const float* thr, size_t base,
                                                 int prow, int n, int hm, int oy0, int ox0, float* st_a, float* st_t,
                                                 uint64_t* bar) {
  if (!tm.use_stage) {
    stage_epilogue(coef, thr, base, n, hm, oy0, ox0, st_a, st_t, bar);
    return;
  }
  if (threadIdx.x == 0) {
    mbar_expect_tx(bar, 2u * kStage * sizeof(float));
    fence_proxy_async();   // the persistent and multi-basis forms refill buffers their threads have read
    const int xs[3] = {hm + ox0, ox0, hm + ox0}, ys[3] = {prow + oy0, prow + hm + oy0, prow + hm + oy0};
#pragma unroll
    for (int sb = 0; sb < 3; ++sb) {
      tma_load_2d(st_a + sb * kTO * kTO, &tm.coef, xs[sb], ys[sb], bar);
      tma_load_2d(st_t + sb * kTO * kTO, &tm.thr, xs[sb], ys[sb], bar);
    }
  }
}

struct AnaSmem {
  float *in_s, *lo_s, *hi_s, *st_a, *st_t;
  uint64_t* bar;   // [0] input tile, [1] staged epilogue operands
};
__device__ __forceinline__ AnaSmem ana_smem(float4* sma) {
  AnaSmem a;
  a.in_s = reinterpret_cast<float*>(sma);
  a.lo_s = a.in_s + kA2In;
  a.hi_s = a.lo_s + kRSmax * kPlo;
  a.st_a = a.in_s + kAnaPre;
  a.st_t = a.st_a + kStage;
  a.bar = reinterpret_cast<uint64_t*>(a.st_t + kStage);
  return a;
}

// A bounded wait gave up: raise the flag, give the copies in flight a second bounded
// wait so none lands after the CTA has gone, and let the caller return.
__device__ __forceinline__ void ana_abort(const AnaSmem& S, int staged, int* err) {
  if (threadIdx.x == 0) {
    atomicExch(err, 1);
    (void)mbar_drain(&S.bar[0], 0);
    if (staged) (void)mbar_drain(&S.bar[1], 0);
  }
}

// One basis of one tile: input copies (issued first), staged epilogue operands (dual
// mode), rows, columns + epilogue.
template <int LF>
__device__ __forceinline__ void ana_basis(const SaraTma& tm, int in_row0, const float* src, int m, const AnaSmem& S,
                                          int bi, int map, int n, int hm, int oy0, int ox0, int last, float* coef,
                                          float* thr, float* approx_out, int mode, float scale, float gamma,
                                          float delta, int* err) {
  ana_issue_input_t(tm, in_row0, src, m, oy0, ox0, 2 * kTO + LF - 2, S.in_s, &S.bar[0]);
  if (mode == SARA_DUAL)
    stage_epilogue_t(tm, coef, thr, ((size_t)map * kBases + bi + 1) * (size_t)n * n, (map * kBases + bi + 1) * n, n,
                     hm, oy0, ox0, S.st_a, S.st_t, &S.bar[1]);
  const bool ok = mbar_wait(&S.bar[0], 0);
  if (__syncthreads_or(!ok)) {
    ana_abort(S, mode == SARA_DUAL, err);
    return;   // this tile is left unchanged (the host reports PS_ETIMEOUT)
  }
  ana_rows<LF>(S.in_s, S.lo_s, S.hi_s);
  __syncthreads();
  if (mode == SARA_DUAL && !mbar_wait(&S.bar[1], 0)) {
    atomicExch(err, 1);
    (void)mbar_drain(&S.bar[1], 0);
    return;
  }
  ana_cols<LF>(S.lo_s, S.hi_s, bi, map, n, hm, oy0, ox0, last, coef, thr, approx_out, mode, scale, gamma, delta,
               S.st_a, S.st_t);
}

__device__ __forceinline__ void ana_dispatch(const SaraTma& tm, int in_row0, int bi, const float* src, int m,
                                             const AnaSmem& S, int map, int n, int hm, int oy0, int ox0, int last,
                                             float* coef, float* thr, float* approx_out, int mode, float scale,
                                             float gamma, float delta, int* err) {
#define PS_ANA(LFv)                                                                                              \
  ana_basis<LFv>(tm, in_row0, src, m, S, bi, map, n, hm, oy0, ox0, last, coef, thr, approx_out, mode, scale, gamma, \
                 delta, err)
  PS_SWITCH_LF(bi, PS_ANA)
#undef PS_ANA
}

// Level-1 analysis: input is the map itself; one basis per CTA (grid.y).
__global__ void __launch_bounds__(256, 3) k_ana_l1(const float* __restrict__ X, int n, int last, float* __restrict__ coef,
                                                   float* __restrict__ thr, float* __restrict__ approx_out, int mode,
                                                   float scale, float gamma, float delta, int* err,
                                                   const __grid_constant__ SaraTma tm) {
  extern __shared__ __align__(128) float4 sma[];
  const AnaSmem S = ana_smem(sma);
  const int bi = blockIdx.y, map = blockIdx.z;
  const int hm = n >> 1, tilesx = hm / kTO;
  const int oy0 = (blockIdx.x / tilesx) * kTO, ox0 = (blockIdx.x % tilesx) * kTO;
  if (threadIdx.x == 0) {
    mbar_init(&S.bar[0], 1);
    mbar_init(&S.bar[1], 1);
  }
  __syncthreads();
  ana_dispatch(tm, map * n, bi, X + (size_t)map * n * n, n, S, map, n, hm, oy0, ox0, last, coef, thr, approx_out, mode,
               scale, gamma, delta, err);
}

// Levels >= 2 with half size >= 32: one basis per CTA (grid.y). (A basis-slowest grid, which
// keeps the co-resident CTAs on one filter's code, measured 5 us slower at 1024^2.)
__global__ void __launch_bounds__(256, 3) k_ana_lv(const float* __restrict__ approx_in, int m, int n, int last,
                                                   float* __restrict__ coef, float* __restrict__ thr,
                                                   float* __restrict__ approx_out, int mode, float scale, float gamma,
                                                   float delta, int* err, const __grid_constant__ SaraTma tm) {
  extern __shared__ __align__(128) float4 sma[];
  const AnaSmem S = ana_smem(sma);
  const int bi = blockIdx.y, map = blockIdx.z;
  const int hm = m >> 1, tilesx = hm / kTO;
  const int oy0 = (blockIdx.x / tilesx) * kTO, ox0 = (blockIdx.x % tilesx) * kTO;
  if (threadIdx.x == 0) {
    mbar_init(&S.bar[0], 1);
    mbar_init(&S.bar[1], 1);
  }
  __syncthreads();
  ana_dispatch(tm, (map * kDb + bi) * m, bi, approx_in + ((size_t)map * kDb + bi) * (size_t)m * m, m, S, map, n, hm,
               oy0, ox0, last, coef, thr, approx_out, mode, scale, gamma, delta, err);
}

// Columns + epilogue for one basis with two columns per thread (the 512-thread form): each
// thread owns two consecutive columns of one output row (one packed pair per subband).
template <int LF>
__device__ __forceinline__ void ana_cols2(const float* __restrict__ lo_s, const float* __restrict__ hi_s, int bi,
                                          int map, int n, int hm, int oy0, int ox0, int last, float* __restrict__ coef,
                                          float* __restrict__ thr, float* __restrict__ approx_out, int mode,
                                          float scale, float gamma, float delta, const float* __restrict__ st_a,
                                          const float* __restrict__ st_t) {
  constexpr int b = LF / 2 - 1;
  const size_t base = ((size_t)map * kBases + (bi + 1)) * (size_t)n * n;
  for (int u = threadIdx.x; u < kTO * kTO / 2; u += blockDim.x) {
    const int kx0 = (u % (kTO / 2)) * 2, ky = u / (kTO / 2);
    const int Y = oy0 + ky, X = ox0 + kx0;
    const size_t idx[4] = {base + (size_t)Y * n + (hm + X), base + (size_t)(hm + Y) * n + X,
                           base + (size_t)(hm + Y) * n + (hm + X), base + (size_t)Y * n + X};   // HL, LH, HH, LL
    u64 ll = 0ull, lh = 0ull, hl = 0ull, hh = 0ull;
#pragma unroll
    for (int j = 0; j < LF; ++j) {
      const u64 a = *reinterpret_cast<const u64*>(lo_s + (2 * ky + j) * kPlo + kx0);
      const u64 c = *reinterpret_cast<const u64*>(hi_s + (2 * ky + j) * kPlo + kx0);
      const u64 ph = cdup(c_hd[b][j]), pg = cdup(c_gd[b][j]);
      ll = ffma2(ph, a, ll);
      lh = ffma2(pg, a, lh);
      hl = ffma2(ph, c, hl);
      hh = ffma2(pg, c, hh);
    }
    const u64 v[4] = {hl, lh, hh, ll};
    const int nsb = last ? 4 : 3;
    for (int sb = 0; sb < nsb; ++sb) {
      float v0, v1;
      f2unpack(v[sb], v0, v1);
      float2* dst = reinterpret_cast<float2*>(coef + idx[sb]);
      if (mode == SARA_DUAL) {
        float2 a2, t2;
        if (sb < 3) {
          a2 = *reinterpret_cast<const float2*>(st_a + sb * kTO * kTO + ky * kTO + kx0);
          t2 = *reinterpret_cast<const float2*>(st_t + sb * kTO * kTO + ky * kTO + kx0);
        } else {
          a2 = *reinterpret_cast<const float2*>(coef + idx[sb]);
          t2 = *reinterpret_cast<const float2*>(thr + idx[sb]);
        }
        *dst = make_float2(fminf(fmaxf(fmaf(scale, v0, a2.x), -t2.x), t2.x),
                           fminf(fmaxf(fmaf(scale, v1, a2.y), -t2.y), t2.y));
      } else if (mode == SARA_APPLY) {
        *dst = make_float2(scale * v0, scale * v1);
      } else {
        const float gd = gamma * delta;
        *reinterpret_cast<float2*>(thr + idx[sb]) =
            make_float2(gd / (delta + fabsf(scale * v0)), gd / (delta + fabsf(scale * v1)));
      }
    }
    if (!last) {
      float a0, a1;
      f2unpack(ll, a0, a1);
      *reinterpret_cast<float2*>(approx_out + ((size_t)map * kDb + bi) * (size_t)hm * hm + (size_t)Y * hm + X) =
          make_float2(a0, a1);
    }
  }
}

// Level-1 analysis with the input tile shared by NB bases: one CTA per (tile, group of NB
// bases, map). The 2 TO + 14 rows the db8 filter needs cover every shorter filter (same
// origin), so the map's tile is copied once and each basis filters it from shared memory.
// NSET = 2: the staged A and gamma W rows of basis i + 1 (dual mode) are copied into the
// second of two staging sets while basis i is filtered (2 CTAs/SM). NSET = 1: one staging
// set, refilled for basis i + 1 once basis i's columns have read it, so the copy overlaps the
// next basis' row pass; the smaller footprint fits 3 CTAs/SM (256 threads).
constexpr int kAnaMFloats = kAnaPre + 4 * kStage;
static size_t multi_analysis_smem(int nset = 2) {
  return (size_t)(kAnaPre + 2 * nset * kStage) * sizeof(float) + 32;
}

template <int NB, int THREADS, int NSET = 2>
__global__ void __launch_bounds__(THREADS, NSET == 1 ? 3 : 2) k_ana_l1m(const float* __restrict__ X, int n, int last,
                                                    float* __restrict__ coef, float* __restrict__ thr,
                                                    float* __restrict__ approx_out, int mode, float scale,
                                                    float gamma, float delta, int* err,
                                                    const __grid_constant__ SaraTma tm) {
  extern __shared__ __align__(128) float4 smm[];
  float* in_s = reinterpret_cast<float*>(smm);
  float* lo_s = in_s + kA2In;
  float* hi_s = lo_s + kRSmax * kPlo;
  float* st = in_s + kAnaPre;                                          // set s: A at st + 2 s kStage, gamma W after it
  uint64_t* bar = reinterpret_cast<uint64_t*>(st + 2 * NSET * kStage);    // [0] input tile, [1 + s] stage set s
  const int map = blockIdx.z, b0 = blockIdx.y * NB;
  const int hm = n >> 1, tilesx = hm / kTO;
  const int oy0 = (blockIdx.x / tilesx) * kTO, ox0 = (blockIdx.x % tilesx) * kTO;
  const bool staged = mode == SARA_DUAL;
  auto plane = [&](int bi) { return ((size_t)map * kBases + bi + 1) * (size_t)n * n; };
  auto prow = [&](int bi) { return (map * kBases + bi + 1) * n; };
  auto set_a = [&](int s) { return st + 2 * s * kStage; };
  auto set_t = [&](int s) { return st + (2 * s + 1) * kStage; };
  if (threadIdx.x == 0)
    for (int q = 0; q < 1 + NSET; ++q) mbar_init(&bar[q], 1);
  __syncthreads();
  ana_issue_input_t(tm, map * n, X + (size_t)map * n * n, n, oy0, ox0, kRSmax, in_s, &bar[0]);
  if (staged) stage_epilogue_t(tm, coef, thr, plane(b0), prow(b0), n, hm, oy0, ox0, set_a(0), set_t(0), &bar[1]);
  const bool ok = mbar_wait(&bar[0], 0);
  if (__syncthreads_or(!ok)) {
    if (threadIdx.x == 0) {
      atomicExch(err, 1);
      (void)mbar_drain(&bar[0], 0);
      if (staged) (void)mbar_drain(&bar[1], 0);
    }
    return;   // the CTA's tiles are left unchanged (the host reports PS_ETIMEOUT)
  }
  for (int i = 0; i < NB; ++i) {
    const int bi = b0 + i, s = NSET == 2 ? (i & 1) : 0;
    // Phase of set s's barrier for basis i (each use completes one phase).
    const uint32_t par = NSET == 2 ? (uint32_t)((i >> 1) & 1) : (uint32_t)(i & 1);
    // NSET = 2: set s ^ 1 was last read by basis i - 1, which ended at a barrier: refill it
    // for basis i + 1.
    if (NSET == 2 && staged && i + 1 < NB)
      stage_epilogue_t(tm, coef, thr, plane(bi + 1), prow(bi + 1), n, hm, oy0, ox0, set_a(s ^ 1), set_t(s ^ 1),
                       &bar[1 + (s ^ 1)]);
#define PS_MR(LFv) ana_rows<LFv>(in_s, lo_s, hi_s)
    PS_SWITCH_LF(bi, PS_MR)
#undef PS_MR
    if (staged) {
      const bool ok2 = mbar_wait(&bar[1 + s], par);
      if (__syncthreads_or(!ok2)) {
        if (threadIdx.x == 0) {
          atomicExch(err, 1);
          (void)mbar_drain(&bar[1 + s], par);
          if (NSET == 2 && i + 1 < NB) (void)mbar_drain(&bar[1 + (s ^ 1)], (uint32_t)(((i + 1) >> 1) & 1));
        }
        return;
      }
    } else {
      __syncthreads();
    }
#define PS_MC(LFv)                                                                                           \
  if (THREADS == 512)                                                                                        \
    ana_cols2<LFv>(lo_s, hi_s, bi, map, n, hm, oy0, ox0, last, coef, thr, approx_out, mode, scale, gamma, delta, \
                   set_a(s), set_t(s));                                                                      \
  else                                                                                                       \
    ana_cols<LFv>(lo_s, hi_s, bi, map, n, hm, oy0, ox0, last, coef, thr, approx_out, mode, scale, gamma, delta,  \
                  set_a(s), set_t(s))
    PS_SWITCH_LF(bi, PS_MC)
#undef PS_MC
    __syncthreads();   // lo/hi and stage set s consumed before the next basis
    // NSET = 1: the single set is free now: refill it for basis i + 1 (its rows run meanwhile).
    if (NSET == 1 && staged && i + 1 < NB)
      stage_epilogue_t(tm, coef, thr, plane(bi + 1), prow(bi + 1), n, hm, oy0, ox0, set_a(0), set_t(0), &bar[1]);
  }
}

// Persistent form of the tiled analysis levels: 2 CTAs per SM loop over the units
// (tile, basis, map) of a level, tile fastest. A unit's input rows are copied while
// the previous unit's columns are filtered, and its staged A and gamma W rows
// (double-buffered) while the whole previous unit runs, so the copy latency that the
// one-unit-per-CTA form exposes once per CTA is hidden behind compute.
constexpr int kAnaPFloats = kAnaPre + 4 * kStage;
static size_t pers_analysis_smem() { return (size_t)kAnaPFloats * sizeof(float) + 32; }

__global__ void __launch_bounds__(256, 2) k_ana_pers(const float* __restrict__ in, size_t in_map, size_t in_basis, int m,
                                                     int n, int last, float* __restrict__ coef,
                                                     float* __restrict__ thr, float* __restrict__ approx_out,
                                                     int mode, float scale, float gamma, float delta, int* err,
                                                     int nmaps, const __grid_constant__ SaraTma tm) {
  extern __shared__ __align__(128) float4 smp[];
  float* in_s = reinterpret_cast<float*>(smp);
  float* lo_s = in_s + kA2In;
  float* hi_s = lo_s + kRSmax * kPlo;
  float* st = in_s + kAnaPre;                                        // set s: A at st + 2 s kStage, gamma W after it
  uint64_t* bar = reinterpret_cast<uint64_t*>(st + 4 * kStage);     // [0] input rows, [1 + s] stage set s
  const int hm = m >> 1, tilesx = hm / kTO, tiles = tilesx * tilesx;
  const int units = tiles * kDb * nmaps;
  const bool staged = mode == SARA_DUAL;
  if (threadIdx.x == 0)
    for (int q = 0; q < 3; ++q) mbar_init(&bar[q], 1);
  __syncthreads();
  int issued_in = 0, issued_st[2] = {0, 0};
  auto decode = [&](int u, int& bi, int& map, int& oy0, int& ox0) {
    const int t = u % tiles, r = u / tiles;
    bi = r % kDb;
    map = r / kDb;
    oy0 = (t / tilesx) * kTO;
    ox0 = (t % tilesx) * kTO;
  };
  auto issue = [&](int u, int s) {
    int bi, map, oy0, ox0;
    decode(u, bi, map, oy0, ox0);
    const size_t in_off = (size_t)map * in_map + (size_t)bi * in_basis;
    ana_issue_input_t(tm, (int)(in_off / (size_t)m), in + in_off, m, oy0, ox0, 2 * kTO + 2 * (bi + 1) - 2, in_s,
                      &bar[0]);
    ++issued_in;
    if (staged) {
      stage_epilogue_t(tm, coef, thr, ((size_t)map * kBases + bi + 1) * (size_t)n * n, (map * kBases + bi + 1) * n, n,
                       hm, oy0, ox0, st + 2 * s * kStage, st + (2 * s + 1) * kStage, &bar[1 + s]);
      ++issued_st[s];
    }
  };
  auto abort_all = [&]() {
    if (threadIdx.x == 0) {
      atomicExch(err, 1);
      if (issued_in) (void)mbar_drain(&bar[0], (issued_in - 1) & 1);
      for (int q = 0; q < 2; ++q)
        if (issued_st[q]) (void)mbar_drain(&bar[1 + q], (issued_st[q] - 1) & 1);
    }
  };
  int u = blockIdx.x;
  if (u < units) issue(u, 0);
  for (int i = 0; u < units; ++i, u += gridDim.x) {
    const int s = i & 1;
    int bi, map, oy0, ox0;
    decode(u, bi, map, oy0, ox0);
    const bool ok = mbar_wait(&bar[0], i & 1);
    if (__syncthreads_or(!ok)) {
      abort_all();
      return;
    }
#define PS_PR(LFv) ana_rows<LFv>(in_s, lo_s, hi_s)
    PS_SWITCH_LF(bi, PS_PR)
#undef PS_PR
    // The input tile is consumed and every thread is past the previous unit's columns,
    // so the input buffer and stage set s ^ 1 can be refilled for the next unit.
    __syncthreads();
    if (u + (int)gridDim.x < units) issue(u + gridDim.x, s ^ 1);
    if (staged) {
      const bool ok2 = mbar_wait(&bar[1 + s], (i >> 1) & 1);
      if (__syncthreads_or(!ok2)) {
        abort_all();
        return;
      }
    }
#define PS_PC(LFv)                                                                                                 \
  ana_cols<LFv>(lo_s, hi_s, bi, map, n, hm, oy0, ox0, last, coef, thr, approx_out, mode, scale, gamma, delta,      \
                st + 2 * s * kStage, st + (2 * s + 1) * kStage)
    PS_SWITCH_LF(bi, PS_PC)
#undef PS_PC
    __syncthreads();   // lo/hi consumed before the next unit's rows
  }
}

// Synthesis of one basis on a TI x TI output tile, split in two steps so the
// next basis' coefficients can be in flight (cp.async) while this one is filtered:
//   syn_load     copies the four subband tiles (with the filter halo, periodic wrap);
//   syn_compute  filters along y then x and adds to acc[4], this thread's outputs
//                out[r][c0 .. c0+3] with r = tid % 32, c0 = 4 (tid / 32).
// Each subband tile is loaded as rows of 32 floats starting 8 columns left of the
// tile's coefficient origin (16-byte aligned), covering every halo width.
constexpr int kSRow = 36;                         // floats per staged row (16-byte aligned pitch)
constexpr int kSTile = kCImax * kSRow;            // one subband tile
constexpr int kS4 = 4 * kSTile;                   // one set of four subband tiles
__device__ __forceinline__ void cp_async16(float* dst, const float* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}

template <int LF>
__device__ __forceinline__ void syn_load(const float* __restrict__ cb, const float* __restrict__ apx, int n, int m,
                                         int oy0, int ox0, float* __restrict__ s4) {
  constexpr int half = LF / 2 - 1;
  constexpr int CI = kTI / 2 + half;
  const int hm = m >> 1;
  const int ky0 = oy0 / 2 - half, kxa = ox0 / 2 - 8;     // kxa: 16-byte aligned start column
  // CI rows x 8 chunks of 4 floats, for each of the four subbands (chunks never straddle the wrap).
  for (int i = threadIdx.x; i < 4 * CI * 8; i += blockDim.x) {
    const int sb = i / (CI * 8), rc = i - sb * (CI * 8);
    const int r = rc >> 3, k = rc & 7;
    const int Yk = wrap1(ky0 + r, hm), Xk = wrap1(kxa + 4 * k, hm);
    const float* src;
    if (sb == 0) src = apx ? apx + (size_t)Yk * hm + Xk : cb + (size_t)Yk * n + Xk;   // LL
    else if (sb == 1) src = cb + (size_t)(hm + Yk) * n + Xk;                         // LH (x-low, y-high)
    else if (sb == 2) src = cb + (size_t)Yk * n + hm + Xk;                           // HL (x-high, y-low)
    else src = cb + (size_t)(hm + Yk) * n + hm + Xk;                                 // HH
    cp_async16(s4 + sb * kSTile + r * kSRow + 4 * k, src);
  }
}

template <int LF>
__device__ __forceinline__ void syn_compute(const float* __restrict__ s4, float* __restrict__ s_lo,
                                            float* __restrict__ s_hi, float acc[4]) {
  constexpr int half = LF / 2 - 1;
  constexpr int CI = kTI / 2 + half;
  constexpr int b = LF / 2 - 1;
  const float* s_ll = s4 + (8 - half);             // column c of the halo tile = staged column c + 8 - half
  const float* s_lh = s4 + kSTile + (8 - half);
  const float* s_hl = s4 + 2 * kSTile + (8 - half);
  const float* s_hh = s4 + 3 * kSTile + (8 - half);
  // Along y: lo[r][c] = sum_{j = r mod 2} h[j] ll[(r - j)/2 + half][c] + g[j] lh[...]; coefficient
  // row r0/2 + i feeds output row r0 + t through tap j = t - 2 (i - half).
  for (int u = threadIdx.x; u < CI * (kTI / 4); u += blockDim.x) {
    const int c = u % CI, r0 = (u / CI) * 4;
    float lo[4] = {0.f, 0.f, 0.f, 0.f}, hi[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int i = 0; i < half + 2; ++i) {
      const int o = (r0 / 2 + i) * kSRow + c;
      const float vll = s_ll[o], vlh = s_lh[o], vhl = s_hl[o], vhh = s_hh[o];
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        const int j = t - 2 * (i - half);
        if (j >= 0 && j < LF) {
          lo[t] = fmaf(c_h[b][j], vll, fmaf(c_g[b][j], vlh, lo[t]));
          hi[t] = fmaf(c_h[b][j], vhl, fmaf(c_g[b][j], vhh, hi[t]));
        }
      }
    }
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      s_lo[(r0 + t) * kPs + c] = lo[t];
      s_hi[(r0 + t) * kPs + c] = hi[t];
    }
  }
  __syncthreads();
  // Along x: warp w owns output columns 4w .. 4w+3 of all 32 rows (row = lane), so the
  // 32 lanes read 32 different rows at an odd pitch (no bank conflicts).
  const int r = threadIdx.x & 31, c0 = (threadIdx.x >> 5) * 4;
#pragma unroll
  for (int i = 0; i < half + 2; ++i) {
    const float vlo = s_lo[r * kPs + c0 / 2 + i], vhi = s_hi[r * kPs + c0 / 2 + i];
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      const int j = t - 2 * (i - half);
      if (j >= 0 && j < LF) acc[t] = fmaf(c_h[b][j], vlo, fmaf(c_g[b][j], vhi, acc[t]));
    }
  }
}


__device__ __forceinline__ void syn_load_dispatch(int bi, const float* cb, const float* apx, int n, int m, int oy0,
                                                  int ox0, float* s4) {
#define PS_L(LFv) syn_load<LFv>(cb, apx, n, m, oy0, ox0, s4)
  PS_SWITCH_LF(bi, PS_L)
#undef PS_L
}
__device__ __forceinline__ void syn_compute_dispatch(int bi, const float* s4, float* s_lo, float* s_hi, float acc[4]) {
#define PS_C(LFv) syn_compute<LFv>(s4, s_lo, s_hi, acc)
  PS_SWITCH_LF(bi, PS_C)
#undef PS_C
}

constexpr int kSynSmemFloats = 2 * kS4 + 2 * kTI * kPs;

// Finest level (m = n): all eight bases plus Dirac summed in registers -> Psi A.
// Basis bi+1's tiles are copied asynchronously while basis bi is filtered.
__global__ void __launch_bounds__(256, 3) k_syn_fine(const float* __restrict__ coef, const float* __restrict__ approx_in,
                                                     int coarsest, int n, float* __restrict__ out) {
  __shared__ __align__(16) float sm_s[kSynSmemFloats];
  float* s4b[2] = {sm_s, sm_s + kS4};
  float* s_lo = sm_s + 2 * kS4;
  float* s_hi = s_lo + kTI * kPs;
  const int map = blockIdx.z;
  const int tilesx = n / kTI;
  const int oy0 = (blockIdx.x / tilesx) * kTI, ox0 = (blockIdx.x % tilesx) * kTI;
  const int hm = n >> 1;
  auto cbp = [&](int bi) { return coef + ((size_t)map * kBases + bi + 1) * (size_t)n * n; };
  auto apxp = [&](int bi) {
    return coarsest ? (const float*)nullptr : approx_in + ((size_t)map * kDb + bi) * (size_t)hm * hm;
  };
  float acc[4] = {0.f, 0.f, 0.f, 0.f};
  syn_load_dispatch(0, cbp(0), apxp(0), n, n, oy0, ox0, s4b[0]);
  cp_async_commit();
  for (int bi = 0; bi < kDb; ++bi) {
    if (bi + 1 < kDb) {
      syn_load_dispatch(bi + 1, cbp(bi + 1), apxp(bi + 1), n, n, oy0, ox0, s4b[(bi + 1) & 1]);
      cp_async_commit();
      cp_async_wait<1>();
    } else {
      cp_async_wait<0>();
    }
    __syncthreads();
    syn_compute_dispatch(bi, s4b[bi & 1], s_lo, s_hi, acc);
    __syncthreads();
  }
  const int r = threadIdx.x & 31, c0 = (threadIdx.x >> 5) * 4;
  const size_t o = (size_t)(oy0 + r) * n + ox0 + c0;
  const float4 d = *reinterpret_cast<const float4*>(coef + (size_t)map * kBases * n * n + o);
  const float k = 1.0f / 3.0f;
  *reinterpret_cast<float4*>(out + (size_t)map * n * n + o) =
      make_float4((d.x + acc[0]) * k, (d.y + acc[1]) * k, (d.z + acc[2]) * k, (d.w + acc[3]) * k);
}


// ---------------------------------------------------------------------------
// Synthesis for levels with output side m >= 64: 64 x 64 output tiles.
//   * The four subband tiles of one basis (rows of 40 coefficients starting 8
//     columns left of the tile's coefficient origin, with the filter halo) are
//     staged by bulk copies, one per row (two where the row wraps around the
//     periodic left edge), completing on an mbarrier; the finest-level kernel
//     double-buffers them so basis b+1 is in flight while basis b is filtered.
//   * Along y, each thread computes two adjacent columns x four rows of the
//     low/high row-filtered tiles with packed FP32x2 FMAs and stores them
//     column-major ([column][row]).
//   * Along x, each thread owns a 4 x 4 output block; the column-major
//     intermediates give it two rows per 64-bit operand, so the taps are again
//     packed FP32x2 FMAs with the coefficient duplicated in both halves.
constexpr int kT2 = 64;                                  // output tile side
constexpr int kC2Rows = kT2 / 2 + kMaxTaps / 2 - 1;      // 39 coefficient rows (db8 halo)
constexpr int kC2Cols = kT2 / 2 + 8;                     // 40 staged columns: [ox0/2 - 8, ox0/2 + 32)
constexpr int kC2Pitch = 40;                             // staged row pitch: the 40 staged columns
constexpr int kC2Sub = (kC2Rows * kC2Pitch + 31) / 32 * 32;   // one subband tile, 128-byte aligned
constexpr int kC2Set = 4 * kC2Sub;                       // LL, LH, HL, HH
constexpr int kLoPitch = kT2 + 4;                        // column-major intermediates: [column][row]
constexpr int kLoSize = kC2Cols * kLoPitch;
static_assert(kC2Sub % 32 == 0 && kLoSize % 4 == 0, "aligned synthesis buffers");

// Issue the bulk copies of basis `half` (db(half+1)) for the tile at (oy0, ox0):
// subband sb row r <- coefficient row (oy0/2 - half + r) mod hm, columns
// [ox0/2 - 8, ox0/2 + 32) mod hm. Thread 0 posts the byte count; any thread may
// start copies before or after it (the barrier's transaction count may run ahead).
__device__ __forceinline__ void syn2_issue(int half, const float* __restrict__ cb, const float* __restrict__ apx,
                                           int n, int hm, int oy0, int ox0, float* __restrict__ s4, uint64_t* bar) {
  const int CI = kT2 / 2 + half;
  const int ky0 = oy0 / 2 - half, kxa = ox0 / 2 - 8;
  if (threadIdx.x == 0) mbar_expect_tx(bar, (uint32_t)(4 * CI * kC2Cols * sizeof(float)));
  for (int k = threadIdx.x; k < 4 * CI; k += blockDim.x) {
    const int sb = k / CI, r = k - sb * CI;
    const int Yk = wrap1(ky0 + r, hm);
    const float* row;
    if (sb == 0) row = apx ? apx + (size_t)Yk * hm : cb + (size_t)Yk * n;   // LL
    else if (sb == 1) row = cb + (size_t)(hm + Yk) * n;                     // LH (x-low, y-high)
    else if (sb == 2) row = cb + (size_t)Yk * n + hm;                       // HL (x-high, y-low)
    else row = cb + (size_t)(hm + Yk) * n + hm;                             // HH
    float* dst = s4 + sb * kC2Sub + r * kC2Pitch;
    fence_proxy_async();
    if (kxa >= 0) {
      bulk_g2s(dst, row + kxa, kC2Cols * sizeof(float), bar);
    } else {   // left edge: columns hm-8 .. hm-1, then 0 .. 31
      bulk_g2s(dst, row + hm - 8, 8 * sizeof(float), bar);
      bulk_g2s(dst + 8, row, (kC2Cols - 8) * sizeof(float), bar);
    }
  }
}

// The four subband tiles by four tensor-map copies from one thread when the tile does not
// wrap (ox0, oy0 > 0) and the maps were made, else by rows. Each box is kC2Rows x kC2Pitch
// (rows past CI and columns past kC2Cols are not read). `prow` is the row of the basis plane
// in the coefficient map, `aprow` the row of the (map, basis) approximation in the
// approximation map (apx non-null).
__device__ __forceinline__ void syn2_issue_t(const SaraTma& tm, int prow, int aprow, int half,
                                             const float* __restrict__ cb, const float* __restrict__ apx, int n, int hm,
                                             int oy0, int ox0, float* __restrict__ s4, uint64_t* bar) {
  if (!(tm.use_scoef && ox0 > 0 && oy0 > 0 && (apx == nullptr || tm.use_apx))) {
    syn2_issue(half, cb, apx, n, hm, oy0, ox0, s4, bar);
    return;
  }
  if (threadIdx.x == 0) {
    const int ky0 = oy0 / 2 - half, kxa = ox0 / 2 - 8;
    mbar_expect_tx(bar, (uint32_t)(4 * kC2Rows * kC2Pitch * sizeof(float)));
    fence_proxy_async();
    if (apx) tma_load_2d(s4, &tm.apx, kxa, aprow + ky0, bar);               // LL from the approximations
    else tma_load_2d(s4, &tm.scoef, kxa, prow + ky0, bar);                  // LL (coarsest level)
    tma_load_2d(s4 + kC2Sub, &tm.scoef, kxa, prow + hm + ky0, bar);         // LH (x-low, y-high)
    tma_load_2d(s4 + 2 * kC2Sub, &tm.scoef, hm + kxa, prow + ky0, bar);     // HL (x-high, y-low)
    tma_load_2d(s4 + 3 * kC2Sub, &tm.scoef, hm + kxa, prow + hm + ky0, bar);  // HH
  }
}

// Along y for basis LF: lo/hi at output rows 4 rg + t (t = 0..3) and staged columns
// c, c + 1, from coefficient rows 2 rg + i (i = 0 .. half + 1) through tap
// j = t - 2 (i - half). Columns start at the even column at or left of 8 - half.
template <int LF>
__device__ __forceinline__ void syn2_ypass(const float* __restrict__ s4, float* __restrict__ loT,
                                           float* __restrict__ hiT) {
  constexpr int half = LF / 2 - 1;
  constexpr int cs = (8 - half) & ~1;
  constexpr int NCP = (kC2Cols - cs) / 2;
  for (int u = threadIdx.x; u < NCP * (kT2 / 4); u += blockDim.x) {
    const int cp = u % NCP, rg = u / NCP;
    const int c = cs + 2 * cp;
    u64 lo[4], hi[4];
#pragma unroll
    for (int t = 0; t < 4; ++t) lo[t] = hi[t] = 0ull;
#pragma unroll
    for (int i = 0; i < half + 2; ++i) {
      const int o = (2 * rg + i) * kC2Pitch + c;
      const u64 vll = *reinterpret_cast<const u64*>(s4 + o);
      const u64 vlh = *reinterpret_cast<const u64*>(s4 + kC2Sub + o);
      const u64 vhl = *reinterpret_cast<const u64*>(s4 + 2 * kC2Sub + o);
      const u64 vhh = *reinterpret_cast<const u64*>(s4 + 3 * kC2Sub + o);
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        const int j = t - 2 * (i - half);
        if (j >= 0 && j < LF) {
          const u64 ph = cdup(c_hd[half][j]), pg = cdup(c_gd[half][j]);
          lo[t] = ffma2(ph, vll, ffma2(pg, vlh, lo[t]));
          hi[t] = ffma2(ph, vhl, ffma2(pg, vhh, hi[t]));
        }
      }
    }
    float l0[4], l1[4], h0[4], h1[4];
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      f2unpack(lo[t], l0[t], l1[t]);
      f2unpack(hi[t], h0[t], h1[t]);
    }
    *reinterpret_cast<float4*>(loT + c * kLoPitch + 4 * rg) = make_float4(l0[0], l0[1], l0[2], l0[3]);
    *reinterpret_cast<float4*>(loT + (c + 1) * kLoPitch + 4 * rg) = make_float4(l1[0], l1[1], l1[2], l1[3]);
    *reinterpret_cast<float4*>(hiT + c * kLoPitch + 4 * rg) = make_float4(h0[0], h0[1], h0[2], h0[3]);
    *reinterpret_cast<float4*>(hiT + (c + 1) * kLoPitch + 4 * rg) = make_float4(h1[0], h1[1], h1[2], h1[3]);
  }
}

// Along x for basis LF, accumulated into this thread's 4 x 4 block: rows 4 rq .. 4 rq + 3,
// columns 4 cg + t; acc[2t] holds rows (4rq, 4rq+1), acc[2t+1] rows (4rq+2, 4rq+3).
// Output column 4 cg + t reads staged column 8 - half + 2 cg + i through tap t - 2 (i - half).
template <int LF>
__device__ __forceinline__ void syn2_xpass(const float* __restrict__ loT, const float* __restrict__ hiT,
                                           u64 acc[8]) {
  constexpr int half = LF / 2 - 1;
  const int rq = threadIdx.x & 15, cg = threadIdx.x >> 4;
#pragma unroll
  for (int i = 0; i < half + 2; ++i) {
    const int col = 2 * cg + (8 - half) + i;
    const ulonglong2 vlo = *reinterpret_cast<const ulonglong2*>(loT + col * kLoPitch + 4 * rq);
    const ulonglong2 vhi = *reinterpret_cast<const ulonglong2*>(hiT + col * kLoPitch + 4 * rq);
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      const int j = t - 2 * (i - half);
      if (j >= 0 && j < LF) {
        const u64 ph = cdup(c_hd[half][j]), pg = cdup(c_gd[half][j]);
        acc[2 * t] = ffma2(ph, vlo.x, ffma2(pg, vhi.x, acc[2 * t]));
        acc[2 * t + 1] = ffma2(ph, vlo.y, ffma2(pg, vhi.y, acc[2 * t + 1]));
      }
    }
  }
}

__device__ __forceinline__ void syn2_ypass_dispatch(int bi, const float* s4, float* loT, float* hiT) {
#define PS_Y(LFv) syn2_ypass<LFv>(s4, loT, hiT)
  PS_SWITCH_LF(bi, PS_Y)
#undef PS_Y
}
__device__ __forceinline__ void syn2_xpass_dispatch(int bi, const float* loT, const float* hiT, u64 acc[8]) {
#define PS_X(LFv) syn2_xpass<LFv>(loT, hiT, acc)
  PS_SWITCH_LF(bi, PS_X)
#undef PS_X
}

// Row rr (0..3) of this thread's 4 x 4 block.
__device__ __forceinline__ float4 syn2_row(const u64 acc[8], int rr) {
  float v[4];
#pragma unroll
  for (int t = 0; t < 4; ++t) {
    float a, b;
    f2unpack(acc[2 * t + (rr >> 1)], a, b);
    v[t] = (rr & 1) ? b : a;
  }
  return make_float4(v[0], v[1], v[2], v[3]);
}

static size_t syn2_smem(int sets) { return (size_t)(sets * kC2Set + 2 * kLoSize) * sizeof(float) + 16; }

// After a bounded wait gave up somewhere in the CTA: raise the flag (when given),
// give the copies still in flight a bounded chance to land, and let the caller return.
__device__ __forceinline__ void syn2_abort(uint64_t* b0, uint32_t p0, uint64_t* b1, uint32_t p1, int* err) {
  if (threadIdx.x == 0) {
    if (err) atomicExch(err, 1);
    (void)mbar_drain(b0, p0);
    if (b1) (void)mbar_drain(b1, p1);
  }
  __syncthreads();
}

// Finest level (m = n >= 64): the eight bases plus the Dirac part summed in registers -> Psi A.
// NBUF = 2: two staging sets, basis b+1 copied while basis b is filtered (3 CTAs per SM).
// NBUF = 1: one staging set, refilled with basis b+1 as soon as the y-pass of basis b
// has read it, so the copy overlaps the x-pass (4 CTAs per SM hide the rest).
template <int NBUF>
__global__ void __launch_bounds__(256, NBUF == 1 ? 4 : 3)
    k_syn2_fine(const float* __restrict__ coef, const float* __restrict__ approx_in, int coarsest, int n,
                float* __restrict__ out, int* err, const __grid_constant__ SaraTma tm) {
  extern __shared__ __align__(128) float4 sm2[];
  float* const s4 = reinterpret_cast<float*>(sm2);   // staging set(s): basis b in set b % NBUF
  float* loT = s4 + NBUF * kC2Set;
  float* hiT = loT + kLoSize;
  uint64_t* bar = reinterpret_cast<uint64_t*>(hiT + kLoSize);
  const int map = blockIdx.z, tilesx = n / kT2;
  const int oy0 = (blockIdx.x / tilesx) * kT2, ox0 = (blockIdx.x % tilesx) * kT2;
  const int hm = n >> 1;
  const float* cmap = coef + (size_t)map * kBases * n * n;
  auto cbp = [&](int bi) { return cmap + (size_t)(bi + 1) * n * n; };
  auto apxp = [&](int bi) {
    return coarsest ? (const float*)nullptr : approx_in + ((size_t)map * kDb + bi) * (size_t)hm * hm;
  };
  auto set = [&](int bi) { return s4 + (bi % NBUF) * kC2Set; };
  auto issue = [&](int bi) {
    syn2_issue_t(tm, (map * kBases + bi + 1) * n, (map * kDb + bi) * hm, bi, cbp(bi), apxp(bi), n, hm, oy0, ox0, set(bi),
                 &bar[bi % NBUF]);
  };
  // Barrier of basis bi and the parity of its phase (each barrier completes once per use).
  auto bar_of = [&](int bi) { return &bar[bi % NBUF]; };
  auto par_of = [&](int bi) { return (uint32_t)((bi / NBUF) & 1); };
  if (threadIdx.x == 0)
    for (int q = 0; q < NBUF; ++q) mbar_init(&bar[q], 1);
  __syncthreads();
  issue(0);
  u64 acc[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) acc[q] = 0ull;
  for (int bi = 0; bi < kDb; ++bi) {
    // NBUF = 2: set (bi+1)&1 last fed the y-pass of basis bi-1, which ended at a barrier.
    if (NBUF == 2 && bi + 1 < kDb) issue(bi + 1);
    const bool ok = mbar_wait(bar_of(bi), par_of(bi));
    // Also orders the previous x-pass' reads of loT/hiT before this y-pass writes them.
    if (__syncthreads_or(!ok)) {
      const bool next = NBUF == 2 && bi + 1 < kDb;
      syn2_abort(bar_of(bi), par_of(bi), next ? bar_of(bi + 1) : nullptr, next ? par_of(bi + 1) : 0u, err);
      return;
    }
    syn2_ypass_dispatch(bi, set(bi), loT, hiT);
    __syncthreads();
    // NBUF = 1: the set is free once every y-pass read of it has passed the barrier above.
    if (NBUF == 1 && bi + 1 < kDb) issue(bi + 1);
    syn2_xpass_dispatch(bi, loT, hiT, acc);
  }
  const int rq = threadIdx.x & 15, cg = threadIdx.x >> 4;
  const float k3 = 1.0f / 3.0f;
#pragma unroll
  for (int rr = 0; rr < 4; ++rr) {
    const size_t o = (size_t)(oy0 + 4 * rq + rr) * n + ox0 + 4 * cg;
    const float4 d = *reinterpret_cast<const float4*>(cmap + o);
    const float4 s = syn2_row(acc, rr);
    *reinterpret_cast<float4*>(out + (size_t)map * n * n + o) =
        make_float4((d.x + s.x) * k3, (d.y + s.y) * k3, (d.z + s.z) * k3, (d.w + s.w) * k3);
  }
}

// Persistent form of the finest level: the CTAs (4 per SM) loop over the (tile, map) units,
// and the single staging set runs on across units: the copies of the next unit's first
// basis go out right after the y-pass of the current unit's last basis, so neither a
// CTA's start nor the end of a unit exposes a copy's latency, and no wave runs part-full.
__global__ void __launch_bounds__(256, 4)
    k_syn2_fine_pers(const float* __restrict__ coef, const float* __restrict__ approx_in, int coarsest, int n,
                     float* __restrict__ out, int* err, int nmaps, const __grid_constant__ SaraTma tm) {
  extern __shared__ __align__(128) float4 sm2[];
  float* const s4 = reinterpret_cast<float*>(sm2);
  float* loT = s4 + kC2Set;
  float* hiT = loT + kLoSize;
  uint64_t* bar = reinterpret_cast<uint64_t*>(hiT + kLoSize);
  const int tilesx = n / kT2, units = tilesx * tilesx * nmaps;
  const int hm = n >> 1;
  auto issue = [&](int unit, int bi) {
    const int map = unit / (tilesx * tilesx), t = unit % (tilesx * tilesx);
    const int oy0 = (t / tilesx) * kT2, ox0 = (t % tilesx) * kT2;
    const float* cb = coef + ((size_t)map * kBases + bi + 1) * (size_t)n * n;
    const float* apx = coarsest ? nullptr : approx_in + ((size_t)map * kDb + bi) * (size_t)hm * hm;
    syn2_issue_t(tm, (map * kBases + bi + 1) * n, (map * kDb + bi) * hm, bi, cb, apx, n, hm, oy0, ox0, s4, bar);
  };
  if (threadIdx.x == 0) mbar_init(bar, 1);
  __syncthreads();
  uint32_t phase = 0;            // uses of the barrier so far (each copy set completes one phase)
  int unit = blockIdx.x;
  if (unit < units) issue(unit, 0);
  for (; unit < units; unit += gridDim.x) {
    const int map = unit / (tilesx * tilesx), t = unit % (tilesx * tilesx);
    const int oy0 = (t / tilesx) * kT2, ox0 = (t % tilesx) * kT2;
    u64 acc[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) acc[q] = 0ull;
    for (int bi = 0; bi < kDb; ++bi, ++phase) {
      const bool ok = mbar_wait(bar, phase & 1);
      // Also orders the previous x-pass' reads of loT/hiT before this y-pass writes them.
      if (__syncthreads_or(!ok)) {
        syn2_abort(bar, phase & 1, nullptr, 0u, err);
        return;
      }
      syn2_ypass_dispatch(bi, s4, loT, hiT);
      __syncthreads();
      // The staging set is free once every y-pass read of it has passed the barrier above.
      if (bi + 1 < kDb) issue(unit, bi + 1);
      else if (unit + (int)gridDim.x < units) issue(unit + gridDim.x, 0);
      syn2_xpass_dispatch(bi, loT, hiT, acc);
    }
    const int rq = threadIdx.x & 15, cg = threadIdx.x >> 4;
    const float k3 = 1.0f / 3.0f;
    const float* cmap = coef + (size_t)map * kBases * n * n;
#pragma unroll
    for (int rr = 0; rr < 4; ++rr) {
      const size_t o = (size_t)(oy0 + 4 * rq + rr) * n + ox0 + 4 * cg;
      const float4 d = *reinterpret_cast<const float4*>(cmap + o);
      const float4 sv = syn2_row(acc, rr);
      *reinterpret_cast<float4*>(out + (size_t)map * n * n + o) =
          make_float4((d.x + sv.x) * k3, (d.y + sv.y) * k3, (d.z + sv.z) * k3, (d.w + sv.w) * k3);
    }
  }
}

// Coarser levels with output side m >= 64: one basis per CTA (grid.z, basis slowest), output to
// approximation scratch.
__global__ void __launch_bounds__(256, 3) k_syn2_lv(const float* __restrict__ coef, const float* __restrict__ approx_in,
                                                    int coarsest, int m, int n, float* __restrict__ approx_out,
                                                    int* err, const __grid_constant__ SaraTma tm) {
  extern __shared__ __align__(128) float4 sm2[];
  float* s4 = reinterpret_cast<float*>(sm2);
  float* loT = s4 + kC2Set;
  float* hiT = loT + kLoSize;
  uint64_t* bar = reinterpret_cast<uint64_t*>(hiT + kLoSize);
  const int bi = blockIdx.z, map = blockIdx.y, tilesx = m / kT2;   // basis slowest, as k_ana_lv
  const int oy0 = (blockIdx.x / tilesx) * kT2, ox0 = (blockIdx.x % tilesx) * kT2;
  const int hm = m >> 1;
  const float* cb = coef + ((size_t)map * kBases + bi + 1) * (size_t)n * n;
  const float* apx = coarsest ? nullptr : approx_in + ((size_t)map * kDb + bi) * (size_t)hm * hm;
  if (threadIdx.x == 0) mbar_init(bar, 1);
  __syncthreads();
  syn2_issue_t(tm, (map * kBases + bi + 1) * n, (map * kDb + bi) * hm, bi, cb, apx, n, hm, oy0, ox0, s4, bar);
  const bool ok = mbar_wait(bar, 0);
  if (__syncthreads_or(!ok)) {
    syn2_abort(bar, 0, nullptr, 0, err);
    return;
  }
  syn2_ypass_dispatch(bi, s4, loT, hiT);
  __syncthreads();
  u64 acc[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) acc[q] = 0ull;
  syn2_xpass_dispatch(bi, loT, hiT, acc);
  const int rq = threadIdx.x & 15, cg = threadIdx.x >> 4;
  float* dst = approx_out + ((size_t)map * kDb + bi) * (size_t)m * m;
#pragma unroll
  for (int rr = 0; rr < 4; ++rr)
    *reinterpret_cast<float4*>(dst + (size_t)(oy0 + 4 * rq + rr) * m + ox0 + 4 * cg) = syn2_row(acc, rr);
}

static size_t fast_analysis_smem() { return (size_t)kAnaFloats * sizeof(float) + 16; }

static size_t synthesis_smem(int TI) {
  const int CI = TI / 2 + kMaxTaps / 2 - 1;
  return (size_t)(4 * CI * CI + 2 * TI * CI) * sizeof(float);
}

// ---------------------------------------------------------------------------
// Coarse levels in one launch. The analysis levels whose input side is at most
// kTail (all levels for images of at most kTail), and the synthesis levels whose
// output side is at most kTailSyn (from the coarsest up to level 2), each take a few
// microseconds of work but cost one dependent launch each when tiled. Here one CTA
// per (basis, map) keeps a whole level in shared memory and runs the levels back to
// back; periodic boundaries are indices modulo the level side (a power of two).
constexpr int kTail = 64;      // analysis: fused levels have input side <= kTail
constexpr int kTailSyn = 32;   // synthesis: fused levels have output side <= kTailSyn (tiled is faster above)
constexpr int kTailThreads = 512;

// One analysis level of side m held in img (m x m, row-major): rows then columns,
// epilogue on the three detail subbands (and on LL at the last level, else LL
// replaces img as the next level's input, side m/2).
template <int LF>
__device__ __forceinline__ void tail_ana_level(float* img, float* lo, float* hi, int m, int bi, int map, int n,
                                               int last, float* coef, float* thr, int mode, float scale, float gamma,
                                               float delta) {
  constexpr int b = LF / 2 - 1;
  const int hm = m >> 1, mask = m - 1;
  for (int u = threadIdx.x; u < m * hm; u += blockDim.x) {      // lo/hi[r][k] = sum_j h/g[j] img[r][2k + j]
    const int r = u / hm, k = u - r * hm;
    const float* row = img + r * m;
    float a = 0.f, c = 0.f;
#pragma unroll
    for (int j = 0; j < LF; ++j) {
      const float v = row[(2 * k + j) & mask];
      a = fmaf(c_h[b][j], v, a);
      c = fmaf(c_g[b][j], v, c);
    }
    lo[u] = a;
    hi[u] = c;
  }
  __syncthreads();
  const size_t base = ((size_t)map * kBases + (bi + 1)) * (size_t)n * n;
  for (int u = threadIdx.x; u < hm * hm; u += blockDim.x) {     // columns: rows 2 ky + j of lo/hi
    const int ky = u / hm, kx = u - ky * hm;
    float ll = 0.f, lh = 0.f, hl = 0.f, hh = 0.f;
#pragma unroll
    for (int j = 0; j < LF; ++j) {
      const int y = (2 * ky + j) & mask;
      const float a = lo[y * hm + kx], c = hi[y * hm + kx];
      ll = fmaf(c_h[b][j], a, ll);
      lh = fmaf(c_g[b][j], a, lh);
      hl = fmaf(c_h[b][j], c, hl);
      hh = fmaf(c_g[b][j], c, hh);
    }
    sara_epilogue(mode, hl, base + (size_t)ky * n + (hm + kx), coef, thr, scale, gamma, delta);         // x-high, y-low
    sara_epilogue(mode, lh, base + (size_t)(hm + ky) * n + kx, coef, thr, scale, gamma, delta);         // x-low, y-high
    sara_epilogue(mode, hh, base + (size_t)(hm + ky) * n + (hm + kx), coef, thr, scale, gamma, delta);
    if (last) sara_epilogue(mode, ll, base + (size_t)ky * n + kx, coef, thr, scale, gamma, delta);
    else img[u] = ll;   // img was fully consumed by the row pass before the barrier above
  }
  __syncthreads();
}

// Analysis levels l0..L in one CTA per (basis, map) = (blockIdx.x, blockIdx.y). The
// input of level l0 (side m0 <= kTail) is X (l0 = 1) or that level's approximation
// scratch (layout [map][basis][m0][m0]).
__global__ void __launch_bounds__(kTailThreads) k_ana_tail(const float* __restrict__ in, int l0, int L, int n,
                                                           float* __restrict__ coef, float* __restrict__ thr, int mode,
                                                           float scale, float gamma, float delta) {
  extern __shared__ float4 smt[];
  float* img = reinterpret_cast<float*>(smt);
  const int bi = blockIdx.x, map = blockIdx.y;
  const int m0 = n >> (l0 - 1);
  float* lo = img + m0 * m0;
  float* hi = lo + m0 * (m0 >> 1);
  const float* src = l0 == 1 ? in + (size_t)map * n * n : in + ((size_t)map * kDb + bi) * (size_t)m0 * m0;
  for (int i = threadIdx.x; i < m0 * m0 / 4; i += blockDim.x)
    reinterpret_cast<float4*>(img)[i] = reinterpret_cast<const float4*>(src)[i];
  __syncthreads();
  for (int l = l0, m = m0; l <= L; ++l, m >>= 1) {
#define PS_TA(LFv) tail_ana_level<LFv>(img, lo, hi, m, bi, map, n, l == L, coef, thr, mode, scale, gamma, delta)
    PS_SWITCH_LF(bi, PS_TA)
#undef PS_TA
  }
}

// One synthesis level to output side m: LL (hm x hm) in shared memory; the level's
// detail subbands are first copied from the coefficient plane cb into det
// (LH, HL, HH, each hm x hm); output into out (m x m).
template <int LF>
__device__ __forceinline__ void tail_syn_level(const float* LLs, const float* __restrict__ cb, int n, int m,
                                               float* det, float* lo, float* hi, float* out) {
  constexpr int b = LF / 2 - 1;
  const int hm = m >> 1, hmask = hm - 1, hh2 = hm * hm;
  for (int i = threadIdx.x; i < 3 * hh2; i += blockDim.x) {
    const int sb = i / hh2, k = i - sb * hh2, r = k / hm, c = k - r * hm;
    det[i] = sb == 0 ? cb[(size_t)(hm + r) * n + c] : (sb == 1 ? cb[(size_t)r * n + hm + c]
                                                             : cb[(size_t)(hm + r) * n + hm + c]);
  }
  __syncthreads();
  // Along y: output row R takes coefficient rows (R - j)/2 (mod hm) through taps j = R mod 2.
  for (int u = threadIdx.x; u < m * hm; u += blockDim.x) {
    const int R = u / hm, c = u - R * hm;
    float a = 0.f, d = 0.f;
#pragma unroll
    for (int j = 0; j < LF; ++j) {
      if ((j & 1) != (R & 1)) continue;
      const int kr = ((R - j) >> 1) & hmask;
      const float vll = LLs[kr * hm + c];
      const float vlh = det[kr * hm + c];
      const float vhl = det[hh2 + kr * hm + c];
      const float vhh = det[2 * hh2 + kr * hm + c];
      a = fmaf(c_h[b][j], vll, fmaf(c_g[b][j], vlh, a));
      d = fmaf(c_h[b][j], vhl, fmaf(c_g[b][j], vhh, d));
    }
    lo[u] = a;
    hi[u] = d;
  }
  __syncthreads();
  // Along x.
  for (int u = threadIdx.x; u < m * m; u += blockDim.x) {
    const int R = u / m, X = u - R * m;
    float v = 0.f;
#pragma unroll
    for (int j = 0; j < LF; ++j) {
      if ((j & 1) != (X & 1)) continue;
      const int kc = ((X - j) >> 1) & hmask;
      v = fmaf(c_h[b][j], lo[R * hm + kc], fmaf(c_g[b][j], hi[R * hm + kc], v));
    }
    out[u] = v;
  }
  __syncthreads();
}

// Synthesis levels L..l1 (l1 >= 2, output side of level l1 <= kTail) in one CTA per
// (basis, map); the level-l1 output goes to approx_out ([map][basis][m][m]).
__global__ void __launch_bounds__(kTailThreads) k_syn_tail(const float* __restrict__ coef, int L, int l1, int n,
                                                           float* __restrict__ approx_out) {
  extern __shared__ float4 smt[];
  const int bi = blockIdx.x, map = blockIdx.y;
  const int mmax = n >> (l1 - 1);
  float* bufA = reinterpret_cast<float*>(smt);          // mmax^2
  float* bufB = bufA + mmax * mmax;                     // mmax^2 / 4
  float* lo = bufB + mmax * mmax / 4;                   // mmax x mmax/2
  float* hi = lo + mmax * (mmax >> 1);
  float* det = hi + mmax * (mmax >> 1);                 // 3 x (mmax/2)^2
  const float* cb = coef + ((size_t)map * kBases + bi + 1) * (size_t)n * n;
  const int s0 = n >> L;                                // coarsest approximation side
  // Level l writes bufA when l - l1 is even (the last level, the largest output, lands in
  // bufA), so the coarsest approximation starts in the other buffer.
  float* cur = (((L - l1) & 1) == 0) ? bufB : bufA;
  for (int i = threadIdx.x; i < s0 * s0; i += blockDim.x) cur[i] = cb[(size_t)(i / s0) * n + (i % s0)];
  __syncthreads();
  for (int l = L; l >= l1; --l) {
    const int m = n >> (l - 1);
    float* nxt = (cur == bufA) ? bufB : bufA;
#define PS_TS(LFv) tail_syn_level<LFv>(cur, cb, n, m, det, lo, hi, nxt)
    PS_SWITCH_LF(bi, PS_TS)
#undef PS_TS
    cur = nxt;
  }
  float* dst = approx_out + ((size_t)map * kDb + bi) * (size_t)mmax * mmax;
  for (int i = threadIdx.x; i < mmax * mmax / 4; i += blockDim.x)
    reinterpret_cast<float4*>(dst)[i] = reinterpret_cast<const float4*>(cur)[i];
}

static size_t ana_tail_smem(int m0) { return (size_t)2 * m0 * m0 * sizeof(float); }
static size_t syn_tail_smem(int mmax) {
  return (size_t)(mmax * mmax + mmax * mmax / 4 + mmax * mmax + 3 * (mmax / 2) * (mmax / 2)) * sizeof(float);
}

// ---- tensor maps (host side). cuTensorMapEncodeTiled comes from the driver through the
// runtime's entry-point query, so the library links against the runtime alone; without it
// (or when an encode fails) the kernels take the per-row bulk copies.
static PFN_cuTensorMapEncodeTiled_v12000 g_encode_tiled = nullptr;
static std::once_flag g_encode_once;

static bool tensor_maps_available() {
  std::call_once(g_encode_once, [] {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q{};
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      g_encode_tiled = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    else
      cudaGetLastError();
  });
  return g_encode_tiled != nullptr;
}

// Map of a row-major float array of `height` rows of `width` floats, box bw x bh (zero fill
// outside). Returns 1 when made. The base must be 16-byte aligned and width * 4 a multiple of
// 16 (every array here: n, m, hm >= 16).
static int make_map(CUtensorMap* map, const float* base, uint64_t width, uint64_t height, uint32_t bw, uint32_t bh) {
  std::memset(map, 0, sizeof(*map));
  if (!base || !tensor_maps_available() || ((uintptr_t)base & 15u) || (width * 4) % 16 != 0 || bw > 256 || bh > 256 ||
      bw > width || bh > height)
    return 0;
  const cuuint64_t dims[2] = {width, height};
  const cuuint64_t strides[1] = {width * sizeof(float)};
  const cuuint32_t box[2] = {bw, bh};
  const cuuint32_t estr[2] = {1, 1};
  const CUresult r = g_encode_tiled(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(base), dims, strides,
                                    box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                                    CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? 1 : 0;
}

// Maps of one tiled analysis level: input planes of side m (`planes` of them), and the
// coefficient and threshold arrays (36 n x n) for the staged epilogue operands.
static SaraTma analysis_maps(const float* in, int m, int planes, const float* coef, const float* thr, int n, int nmaps,
                             int mode) {
  SaraTma t;
  std::memset(&t, 0, sizeof(t));
  t.use_in = make_map(&t.in, in, (uint64_t)m, (uint64_t)planes * m, kA2Pitch, kRSmax);
  if (mode == SARA_DUAL)
    t.use_stage = make_map(&t.coef, coef, (uint64_t)n, (uint64_t)kBases * nmaps * n, kTO, kTO) &
                  make_map(&t.thr, thr, (uint64_t)n, (uint64_t)kBases * nmaps * n, kTO, kTO);
  return t;
}

// Maps of one tiled synthesis level of output side m: coefficients and, below the coarsest
// level, the 32 (map, basis) approximations of side m / 2.
static SaraTma synthesis_maps(const float* coef, const float* approx_in, int m, int n, int nmaps) {
  SaraTma t;
  std::memset(&t, 0, sizeof(t));
  t.use_scoef = make_map(&t.scoef, coef, (uint64_t)n, (uint64_t)kBases * nmaps * n, kC2Pitch, kC2Rows);
  if (approx_in)
    t.use_apx = make_map(&t.apx, approx_in, (uint64_t)(m / 2), (uint64_t)kDb * nmaps * (m / 2), kC2Pitch, kC2Rows);
  return t;
}

cudaError_t configure_nufft_kernels();

cudaError_t configure_kernels() {
  cudaError_t e = cudaFuncSetAttribute((const void*)k_synthesis, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)synthesis_smem(32));
  if (e != cudaSuccess) return e;
  for (const void* f : {(const void*)k_ana_l1, (const void*)k_ana_lv}) {
    e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fast_analysis_smem());
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(f, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
    if (e != cudaSuccess) return e;
  }
  e = cudaFuncSetAttribute((const void*)k_syn2_fine<2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)syn2_smem(2));
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute((const void*)k_syn2_fine<1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)syn2_smem(1));
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute((const void*)k_syn2_lv, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)syn2_smem(1));
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute((const void*)k_syn2_fine_pers, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)syn2_smem(1));
  if (e != cudaSuccess) return e;
  for (const void* f : {(const void*)k_syn2_fine<2>, (const void*)k_syn2_fine<1>, (const void*)k_syn2_lv,
                        (const void*)k_syn2_fine_pers}) {
    e = cudaFuncSetAttribute(f, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
    if (e != cudaSuccess) return e;
  }
  for (const void* f : {(const void*)k_ana_l1m<8, 256>, (const void*)k_ana_l1m<4, 256>,
                        (const void*)k_ana_l1m<4, 512>, (const void*)k_ana_l1m<4, 256, 1>}) {
    e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)multi_analysis_smem());
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(f, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
    if (e != cudaSuccess) return e;
  }
  e = cudaFuncSetAttribute((const void*)k_ana_pers, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)pers_analysis_smem());
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute((const void*)k_ana_pers, cudaFuncAttributePreferredSharedMemoryCarveout,
                           cudaSharedmemCarveoutMaxShared);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute((const void*)k_ana_tail, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)ana_tail_smem(kTail));
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute((const void*)k_syn_tail, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)syn_tail_smem(kTailSyn));
  if (e != cudaSuccess) return e;
  return configure_nufft_kernels();
}

cudaError_t sara_analysis(Handle* h, const float* X, float* coef, float* thr, int mode, float scale, float gamma,
                          float delta, cudaEvent_t fine_done) {
  const int n = h->n, L = h->L;
  const int nmaps = h->nmaps;
  float* buf[2] = {h->approx, h->approx2};
  int lt = L + 1;                                   // first level of the fused tail
  for (int l = 1; l <= L; ++l)
    if ((n >> (l - 1)) <= kTail) {
      lt = l;
      break;
    }
  // Levels with input side > kTail: tiled, one launch per level (half side >= 128).
  for (int l = 1; l < lt; ++l) {
    const int m = n >> (l - 1), hm = m / 2;
    const dim3 grid((hm / kTO) * (hm / kTO), kDb, nmaps);
    if (l == 1 && h->tune[PS_TUNE_ANALYSIS] >= 2) {
      const int choice = h->tune[PS_TUNE_ANALYSIS], nb = choice == 2 ? 8 : 4;
      const dim3 gm((hm / kTO) * (hm / kTO), kDb / nb, nmaps);
      const SaraTma tm = analysis_maps(X, n, nmaps, coef, thr, n, nmaps, mode);
      if (choice == 2)
        k_ana_l1m<8, 256><<<gm, 256, multi_analysis_smem(), h->stream>>>(X, n, l == L, coef, thr, buf[0], mode,
                                                                         scale, gamma, delta, h->dev_flags, tm);
      else if (choice == 3)
        k_ana_l1m<4, 256><<<gm, 256, multi_analysis_smem(), h->stream>>>(X, n, l == L, coef, thr, buf[0], mode,
                                                                         scale, gamma, delta, h->dev_flags, tm);
      else if (choice == 4)
        k_ana_l1m<4, 512><<<gm, 512, multi_analysis_smem(), h->stream>>>(X, n, l == L, coef, thr, buf[0], mode,
                                                                         scale, gamma, delta, h->dev_flags, tm);
      else
        k_ana_l1m<4, 256, 1><<<gm, 256, multi_analysis_smem(1), h->stream>>>(X, n, l == L, coef, thr, buf[0], mode,
                                                                            scale, gamma, delta, h->dev_flags, tm);
      if (fine_done) {
        const cudaError_t e = cudaEventRecord(fine_done, h->stream);
        if (e != cudaSuccess) return e;
      }
    } else if (h->tune[PS_TUNE_ANALYSIS] == 1) {
      const int units = (int)(grid.x * grid.y * grid.z);
      const int ctas = std::min(units, 2 * std::max(1, h->num_sms));
      const float* in = l == 1 ? X : buf[(l - 2) & 1];
      const size_t in_map = l == 1 ? (size_t)n * n : (size_t)kDb * m * m, in_basis = l == 1 ? 0 : (size_t)m * m;
      const SaraTma tm = analysis_maps(in, m, l == 1 ? nmaps : kDb * nmaps, coef, thr, n, nmaps, mode);
      k_ana_pers<<<ctas, 256, pers_analysis_smem(), h->stream>>>(in, in_map, in_basis, m, n, l == L, coef, thr,
                                                                 buf[(l - 1) & 1], mode, scale, gamma, delta,
                                                                 h->dev_flags, nmaps, tm);
      if (l == 1 && fine_done) {
        const cudaError_t e = cudaEventRecord(fine_done, h->stream);
        if (e != cudaSuccess) return e;
      }
    } else if (l == 1) {
      const SaraTma tm = analysis_maps(X, n, nmaps, coef, thr, n, nmaps, mode);
      k_ana_l1<<<grid, 256, fast_analysis_smem(), h->stream>>>(X, n, l == L, coef, thr, buf[(l - 1) & 1], mode, scale,
                                                              gamma, delta, h->dev_flags, tm);
      if (fine_done) {
        const cudaError_t e = cudaEventRecord(fine_done, h->stream);
        if (e != cudaSuccess) return e;
      }
    } else {
      const SaraTma tm = analysis_maps(buf[(l - 2) & 1], m, kDb * nmaps, coef, thr, n, nmaps, mode);
      k_ana_lv<<<grid, 256, fast_analysis_smem(), h->stream>>>(buf[(l - 2) & 1], m, n, l == L, coef, thr,
                                                              buf[(l - 1) & 1], mode, scale, gamma, delta,
                                                              h->dev_flags, tm);
    }
  }
  if (lt <= L) {
    const float* in = lt == 1 ? X : buf[(lt - 2) & 1];
    k_ana_tail<<<dim3(kDb, nmaps), kTailThreads, ana_tail_smem(n >> (lt - 1)), h->stream>>>(in, lt, L, n, coef, thr,
                                                                                         mode, scale, gamma, delta);
    if (lt == 1 && fine_done) {
      const cudaError_t e = cudaEventRecord(fine_done, h->stream);
      if (e != cudaSuccess) return e;
    }
  }
  return cudaGetLastError();
}

// Psi A on `stream` with `approx` as the per-level approximation scratch
// (2 x 32 x (n/2)^2 floats); `err` (may be null) receives the bounded-wait flag;
// `variant` is the PS_TUNE_SYNTHESIS choice of the finest level.
static cudaError_t synthesis_levels(cudaStream_t stream, int n, int L, const float* coef, float* out, float* approx0,
                                    float* approx1, int nmaps, int* err, int variant,
                                    cudaEvent_t fine_start = nullptr) {
  float* buf[2] = {approx0, approx1};
  int lt = 0;                                       // lowest level of the fused tail (>= 2), 0: none
  for (int l = 2; l <= L; ++l)
    if ((n >> (l - 1)) <= kTailSyn) {
      lt = l;
      break;
    }
  if (lt)
    k_syn_tail<<<dim3(kDb, nmaps), kTailThreads, syn_tail_smem(n >> (lt - 1)), stream>>>(coef, L, lt, n,
                                                                                      buf[(lt - 1) & 1]);
  for (int l = lt ? lt - 1 : L; l >= 1; --l) {
    const int m = n >> (l - 1);
    const int TI = m < 32 ? m : 32;
    const int tiles = (m / TI) * (m / TI);
    const float* ain = (l == L) ? nullptr : buf[l & 1];
    float* aout = (l == 1) ? nullptr : buf[(l - 1) & 1];
    if (l == 1 && fine_start) {
      const cudaError_t e = cudaEventRecord(fine_start, stream);
      if (e != cudaSuccess) return e;
    }
    const SaraTma tm = m >= kT2 ? synthesis_maps(coef, ain, m, n, nmaps) : SaraTma{};
    if (m >= kT2 && l == 1) {
      const dim3 grid((m / kT2) * (m / kT2), 1, nmaps);
      if (variant == 2) {
        int dev = 0, sms = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        const int units = (int)(grid.x * grid.z);
        k_syn2_fine_pers<<<std::min(units, 4 * std::max(1, sms)), 256, syn2_smem(1), stream>>>(coef, ain, l == L, n,
                                                                                              out, err, nmaps, tm);
      } else if (variant == 1) k_syn2_fine<1><<<grid, 256, syn2_smem(1), stream>>>(coef, ain, l == L, n, out, err, tm);
      else k_syn2_fine<2><<<grid, 256, syn2_smem(2), stream>>>(coef, ain, l == L, n, out, err, tm);
    } else if (m >= kT2) {
      k_syn2_lv<<<dim3((m / kT2) * (m / kT2), nmaps, kDb), 256, syn2_smem(1), stream>>>(coef, ain, l == L, m, n, aout,
                                                                                     err, tm);
    } else if (m >= kTI && l == 1) {
      k_syn_fine<<<dim3(tiles, 1, nmaps), 256, 0, stream>>>(coef, ain, l == L, n, out);
    } else {
      dim3 grid(tiles, l == 1 ? 1 : kDb, nmaps);
      k_synthesis<<<grid, 256, synthesis_smem(TI), stream>>>(coef, ain, l == L, m, TI, n, l == 1, aout, out);
    }
  }
  return cudaGetLastError();
}

cudaError_t sara_synthesis(Handle* h, const float* coef, float* out, cudaEvent_t fine_start) {
  return synthesis_levels(h->stream, h->n, h->L, coef, out, h->approx, h->approx2, h->nmaps, h->dev_flags,
                          h->tune[PS_TUNE_SYNTHESIS],
                          fine_start);
}

// ---------------------------------------------------------------------------
// Allocation-free synthesis (ps_apply_psi_static). Its level scratch lives in
// this file-scope device array, sized for images up to kStaticMaxN; every GPU
// that loads the library holds it until the process exits.
constexpr int kStaticMaxN = 256;
constexpr size_t kStaticScratchFloats = 2ull * kDb * 4 * (kStaticMaxN / 2) * (kStaticMaxN / 2);   // 4 MiB
static __device__ __align__(256) float g_static_scratch[kStaticScratchFloats];
// Raised by a kernel of ps_apply_psi_static whose bounded wait gave up (cleared by each call).
static __device__ int g_static_err;

constexpr int kMaxDevices = 64;
static std::mutex g_static_mu;
static float* g_static_ptr[kMaxDevices] = {};    // device address of g_static_scratch, per device
static int* g_static_err_ptr[kMaxDevices] = {};  // device address of g_static_err, per device

// Sets this file's bounded-wait poll budget (ps_debug_set_wait_polls).
cudaError_t set_wait_polls_sara(int polls) { return set_wait_polls_here(polls); }

// A caller pointer of ps_apply_psi_static must be device or managed memory of the current device.
static bool device_pointer_here(const void* p, int dev) {
  cudaPointerAttributes a{};
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  if (a.type == cudaMemoryTypeManaged) return true;
  return a.type == cudaMemoryTypeDevice && a.device == dev;
}

}  // namespace ps

#pragma GCC visibility push(default)
extern "C" ps_status ps_apply_psi_static(const float* A, float* S, int32_t n, int32_t levels, void* cuda_stream) {
  using namespace ps;
  auto bad = [](const std::string& m) {
    set_global_error("apply_psi_static: " + m);
    return PS_EINVAL;
  };
  if (n < 16 || n > kStaticMaxN || (n & (n - 1)) != 0)
    return bad("n must be a power of two in [16, " + std::to_string(kStaticMaxN) + "] (static scratch limit)");
  if (levels < 1 || (n % (1 << levels)) != 0) return bad("levels must satisfy n divisible by 2^levels");
  if (!A || !S || ((uintptr_t)A & 15u) || ((uintptr_t)S & 15u))
    return bad("A and S must be non-null, 16-byte aligned device pointers");
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    set_global_error(std::string("apply_psi_static: no usable current device: ") + cudaGetErrorString(e));
    return PS_ECUDA;
  }
  if (!device_pointer_here(A, dev) || !device_pointer_here(S, dev))
    return bad("A and S must point to device (or managed) memory of the current device");
  float* scratch = nullptr;
  int* flag = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_static_mu);
    if (!g_static_ptr[dev]) {
      // Set-up on this device, once: the device addresses of the scratch and the error
      // flag, and the filter taps.
      void* p = nullptr;
      void* q = nullptr;
      e = cudaGetSymbolAddress(&p, g_static_scratch);
      if (e == cudaSuccess) e = cudaGetSymbolAddress(&q, g_static_err);
      if (e != cudaSuccess) {
        set_global_error(std::string("apply_psi_static: cudaGetSymbolAddress: ") + cudaGetErrorString(e));
        return PS_ECUDA;
      }
      g_static_err_ptr[dev] = static_cast<int*>(q);
      double filt[kDb][kMaxTaps];
      daubechies_filters(filt);
      e = upload_filters(filt, (cudaStream_t)cuda_stream);
      if (e != cudaSuccess) {
        set_global_error(std::string("apply_psi_static: filter upload: ") + cudaGetErrorString(e));
        return PS_ECUDA;
      }
      e = configure_kernels();   // shared-memory limits of the kernels (function attributes, no allocation)
      if (e != cudaSuccess) {
        set_global_error(std::string("apply_psi_static: kernel attributes: ") + cudaGetErrorString(e));
        return PS_ECUDA;
      }
      g_static_ptr[dev] = static_cast<float*>(p);
    }
    scratch = g_static_ptr[dev];
    flag = g_static_err_ptr[dev];
  }
  e = cudaMemsetAsync(flag, 0, sizeof(int), (cudaStream_t)cuda_stream);
  if (e == cudaSuccess)
    e = synthesis_levels((cudaStream_t)cuda_stream, n, levels, A, S, scratch, scratch + kStaticScratchFloats / 2, 4, flag,
                         0);
  if (e != cudaSuccess) {
    set_global_error(std::string("apply_psi_static: launch: ") + cudaGetErrorString(e));
    return PS_ECUDA;
  }
  return PS_OK;
}

extern "C" ps_status ps_static_status(void* cuda_stream) {
  using namespace ps;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    set_global_error(std::string("static_status: no usable current device: ") + cudaGetErrorString(e));
    return PS_ECUDA;
  }
  int* flag = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_static_mu);
    flag = g_static_err_ptr[dev];
  }
  e = cudaStreamSynchronize((cudaStream_t)cuda_stream);
  if (e != cudaSuccess) {
    set_global_error(std::string("static_status: ") + cudaGetErrorString(e));
    return PS_ECUDA;
  }
  if (!flag) return PS_OK;   // ps_apply_psi_static has not run on this device
  int v = 0;
  e = cudaMemcpy(&v, flag, sizeof(int), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) {
    set_global_error(std::string("static_status: ") + cudaGetErrorString(e));
    return PS_ECUDA;
  }
  if (v) {
    set_global_error("apply_psi_static: a bounded device wait (bulk-copy barrier) gave up; S is incomplete");
    return PS_ETIMEOUT;
  }
  return PS_OK;
}
#pragma GCC visibility pop

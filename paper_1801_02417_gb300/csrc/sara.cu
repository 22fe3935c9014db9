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
#include <cuda_runtime.h>

#include "internal.h"

namespace ps {

__constant__ float c_h[kDb][kMaxTaps];
__constant__ float c_g[kDb][kMaxTaps];

cudaError_t upload_filters(const double h[kDb][kMaxTaps]) {
  float hf[kDb][kMaxTaps], gf[kDb][kMaxTaps];
  for (int b = 0; b < kDb; ++b) {
    const int Lf = 2 * (b + 1);
    for (int j = 0; j < kMaxTaps; ++j) {
      hf[b][j] = j < Lf ? (float)h[b][j] : 0.f;
      gf[b][j] = j < Lf ? (float)(((j & 1) ? -1.0 : 1.0) * h[b][Lf - 1 - j]) : 0.f;
    }
  }
  cudaError_t e = cudaMemcpyToSymbol(c_h, hf, sizeof(hf));
  if (e != cudaSuccess) return e;
  return cudaMemcpyToSymbol(c_g, gf, sizeof(gf));
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

// One analysis level. Input arrays: in + map*in_map + basis*in_basis, m x m.
__global__ void __launch_bounds__(256) k_analysis(const float* __restrict__ in, size_t in_map, size_t in_basis, int m,
                                                  int TO, int n, int last, float* __restrict__ coef,
                                                  float* __restrict__ thr, float* __restrict__ approx_out,
                                                  int mode, float scale, float gamma, float delta) {
  extern __shared__ float sm[];
  const int bi = blockIdx.y;  // 0..7 -> db1..db8
  const int map = blockIdx.z;
  const int Lf = 2 * (bi + 1);
  const int hm = m >> 1;
  const int tilesx = hm / TO;
  const int oy0 = (blockIdx.x / tilesx) * TO, ox0 = (blockIdx.x % tilesx) * TO;
  const int RS = 2 * TO + Lf - 2;               // input tile side
  float* in_s = sm;                              // RS x RS
  float* lo_s = sm + RS * RS;                    // RS x TO
  float* hi_s = lo_s + RS * TO;                  // RS x TO
  const float* src = in + (size_t)map * in_map + (size_t)bi * in_basis;
  for (int i = threadIdx.x; i < RS * RS; i += blockDim.x) {
    const int r = i / RS, c = i - r * RS;
    const int y = (2 * oy0 + r) % m, x = (2 * ox0 + c) % m;
    in_s[i] = src[(size_t)y * m + x];
  }
  __syncthreads();
  const float* h = c_h[bi];
  const float* g = c_g[bi];
  for (int i = threadIdx.x; i < RS * TO; i += blockDim.x) {
    const int r = i / TO, k = i - r * TO;
    const float* row = in_s + r * RS + 2 * k;
    float lo = 0.f, hi = 0.f;
    for (int j = 0; j < Lf; ++j) {
      const float v = row[j];
      lo = fmaf(h[j], v, lo);
      hi = fmaf(g[j], v, hi);
    }
    lo_s[i] = lo;
    hi_s[i] = hi;
  }
  __syncthreads();
  const size_t base = ((size_t)map * kBases + (bi + 1)) * (size_t)n * n;
  for (int i = threadIdx.x; i < TO * TO; i += blockDim.x) {
    const int ky = i / TO, kx = i - ky * TO;
    float ll = 0.f, lh = 0.f, hl = 0.f, hh = 0.f;
    for (int j = 0; j < Lf; ++j) {
      const float a = lo_s[(2 * ky + j) * TO + kx];
      const float b = hi_s[(2 * ky + j) * TO + kx];
      ll = fmaf(h[j], a, ll);
      lh = fmaf(g[j], a, lh);
      hl = fmaf(h[j], b, hl);
      hh = fmaf(g[j], b, hh);
    }
    const int Y = oy0 + ky, X = ox0 + kx;
    sara_epilogue(mode, hl, base + (size_t)Y * n + (hm + X), coef, thr, scale, gamma, delta);        // x-high, y-low
    sara_epilogue(mode, lh, base + (size_t)(hm + Y) * n + X, coef, thr, scale, gamma, delta);        // x-low, y-high
    sara_epilogue(mode, hh, base + (size_t)(hm + Y) * n + (hm + X), coef, thr, scale, gamma, delta);
    if (last) {
      sara_epilogue(mode, ll, base + (size_t)Y * n + X, coef, thr, scale, gamma, delta);
    } else {
      approx_out[((size_t)map * kDb + bi) * (size_t)hm * hm + (size_t)Y * hm + X] = ll;
    }
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
constexpr int kPin = kRSmax | 1;                 // odd pitch: conflict-free row reads
constexpr int kPlo = kTO + 4;                    // row-filtered tiles (16-byte aligned rows)
constexpr int kInSize = (kRSmax * kPin + 3) / 4 * 4;   // input tile, padded so lo_s starts 16-byte aligned
constexpr int kTI = 32;                          // synthesis output tile
constexpr int kCImax = kTI / 2 + kMaxTaps / 2 - 1;   // 23
constexpr int kPc = kCImax | 1;                  // 23 (odd)
constexpr int kPs = kCImax + 2;                  // 25

__device__ __forceinline__ int wrap1(int v, int m) { return v < 0 ? v + m : (v >= m ? v - m : v); }

// Rows: lo/hi[r][k] = sum_j h/g[j] in[r][2k + j], k in [0, TO).
template <int LF>
__device__ __forceinline__ void ana_rows(const float* __restrict__ in_s, float* __restrict__ lo_s,
                                         float* __restrict__ hi_s) {
  constexpr int RS = 2 * kTO + LF - 2;
  constexpr int b = LF / 2 - 1;
  for (int u = threadIdx.x; u < RS * (kTO / 4); u += blockDim.x) {
    const int r = u % RS, k0 = (u / RS) * 4;
    const float* row = in_s + r * kPin + 2 * k0;
    float x[LF + 6];
#pragma unroll
    for (int j = 0; j < LF + 6; ++j) x[j] = row[j];
    float lo[4], hi[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      float a = 0.f, c = 0.f;
#pragma unroll
      for (int j = 0; j < LF; ++j) {
        a = fmaf(c_h[b][j], x[2 * q + j], a);
        c = fmaf(c_g[b][j], x[2 * q + j], c);
      }
      lo[q] = a;
      hi[q] = c;
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
// owns four consecutive columns of one output row, so the epilogue reads and
// writes A and gamma W as float4 (prefetched before the filtering).
template <int LF>
__device__ __forceinline__ void ana_cols(const float* __restrict__ lo_s, const float* __restrict__ hi_s, int bi,
                                         int map, int n, int hm, int oy0, int ox0, int last, float* __restrict__ coef,
                                         float* __restrict__ thr, float* __restrict__ approx_out, int mode,
                                         float scale, float gamma, float delta) {
  constexpr int b = LF / 2 - 1;
  const size_t base = ((size_t)map * kBases + (bi + 1)) * (size_t)n * n;
  for (int u = threadIdx.x; u < kTO * kTO / 4; u += blockDim.x) {
    const int kx0 = (u % (kTO / 4)) * 4, ky = u / (kTO / 4);
    const int Y = oy0 + ky, X = ox0 + kx0;
    const size_t i_hl = base + (size_t)Y * n + (hm + X);
    const size_t i_lh = base + (size_t)(hm + Y) * n + X;
    const size_t i_hh = base + (size_t)(hm + Y) * n + (hm + X);
    const size_t i_ll = base + (size_t)Y * n + X;
    const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
    float4 a_hl = z, a_lh = z, a_hh = z, a_ll = z, t_hl = z, t_lh = z, t_hh = z, t_ll = z;
    if (mode == SARA_DUAL) {
      a_hl = *reinterpret_cast<const float4*>(coef + i_hl);
      a_lh = *reinterpret_cast<const float4*>(coef + i_lh);
      a_hh = *reinterpret_cast<const float4*>(coef + i_hh);
      t_hl = *reinterpret_cast<const float4*>(thr + i_hl);
      t_lh = *reinterpret_cast<const float4*>(thr + i_lh);
      t_hh = *reinterpret_cast<const float4*>(thr + i_hh);
      if (last) {
        a_ll = *reinterpret_cast<const float4*>(coef + i_ll);
        t_ll = *reinterpret_cast<const float4*>(thr + i_ll);
      }
    }
    float4 ll = z, lh = z, hl = z, hh = z;
#pragma unroll
    for (int j = 0; j < LF; ++j) {
      const float4 a = *reinterpret_cast<const float4*>(lo_s + (2 * ky + j) * kPlo + kx0);
      const float4 c = *reinterpret_cast<const float4*>(hi_s + (2 * ky + j) * kPlo + kx0);
      ll = f4fma(c_h[b][j], a, ll);
      lh = f4fma(c_g[b][j], a, lh);
      hl = f4fma(c_h[b][j], c, hl);
      hh = f4fma(c_g[b][j], c, hh);
    }
    sara_epilogue4(mode, hl, i_hl, a_hl, t_hl, coef, thr, scale, gamma, delta);   // x-high, y-low
    sara_epilogue4(mode, lh, i_lh, a_lh, t_lh, coef, thr, scale, gamma, delta);   // x-low, y-high
    sara_epilogue4(mode, hh, i_hh, a_hh, t_hh, coef, thr, scale, gamma, delta);
    if (last) sara_epilogue4(mode, ll, i_ll, a_ll, t_ll, coef, thr, scale, gamma, delta);
    else *reinterpret_cast<float4*>(approx_out + ((size_t)map * kDb + bi) * (size_t)hm * hm + (size_t)Y * hm + X) = ll;
  }
}

template <int LF>
__device__ __forceinline__ void ana_basis(const float* in_s, float* lo_s, float* hi_s, int bi, int map, int n, int hm,
                                          int oy0, int ox0, int last, float* coef, float* thr, float* approx_out,
                                          int mode, float scale, float gamma, float delta) {
  ana_rows<LF>(in_s, lo_s, hi_s);
  __syncthreads();
  ana_cols<LF>(lo_s, hi_s, bi, map, n, hm, oy0, ox0, last, coef, thr, approx_out, mode, scale, gamma, delta);
  __syncthreads();
}

__device__ __forceinline__ void ana_dispatch(int bi, const float* in_s, float* lo_s, float* hi_s, int map, int n,
                                             int hm, int oy0, int ox0, int last, float* coef, float* thr,
                                             float* approx_out, int mode, float scale, float gamma, float delta) {
#define PS_ANA(LFv) ana_basis<LFv>(in_s, lo_s, hi_s, bi, map, n, hm, oy0, ox0, last, coef, thr, approx_out, mode, \
                                   scale, gamma, delta)
  switch (bi) {
    case 0: PS_ANA(2); break;
    case 1: PS_ANA(4); break;
    case 2: PS_ANA(6); break;
    case 3: PS_ANA(8); break;
    case 4: PS_ANA(10); break;
    case 5: PS_ANA(12); break;
    case 6: PS_ANA(14); break;
    default: PS_ANA(16); break;
  }
#undef PS_ANA
}

__device__ __forceinline__ void load_in_tile(const float* __restrict__ src, int m, int oy0, int ox0, int RS,
                                             float* __restrict__ in_s) {
  for (int i = threadIdx.x; i < RS * RS; i += blockDim.x) {
    const int r = i / RS, c = i - r * RS;
    int y = 2 * oy0 + r, x = 2 * ox0 + c;
    if (y >= m) y -= m;
    if (x >= m) x -= m;
    in_s[r * kPin + c] = src[(size_t)y * m + x];
  }
}

// Level-1 analysis: input is the map itself; one basis per CTA (grid.y).
__global__ void __launch_bounds__(256, 3) k_ana_l1(const float* __restrict__ X, int n, int last, float* __restrict__ coef,
                                                float* __restrict__ thr, float* __restrict__ approx_out, int mode,
                                                float scale, float gamma, float delta) {
  extern __shared__ float4 sma[];
  float* in_s = reinterpret_cast<float*>(sma);
  float* lo_s = in_s + kInSize;
  float* hi_s = lo_s + kRSmax * kPlo;
  const int bi = blockIdx.y, map = blockIdx.z;
  const int hm = n >> 1, tilesx = hm / kTO;
  const int oy0 = (blockIdx.x / tilesx) * kTO, ox0 = (blockIdx.x % tilesx) * kTO;
  load_in_tile(X + (size_t)map * n * n, n, oy0, ox0, 2 * kTO + 2 * bi, in_s);
  __syncthreads();
  ana_dispatch(bi, in_s, lo_s, hi_s, map, n, hm, oy0, ox0, last, coef, thr, approx_out, mode, scale, gamma, delta);
}

// Levels >= 2 with half size >= 32: one basis per CTA (grid.y).
__global__ void __launch_bounds__(256, 3) k_ana_lv(const float* __restrict__ approx_in, int m, int n, int last,
                                                float* __restrict__ coef, float* __restrict__ thr,
                                                float* __restrict__ approx_out, int mode, float scale, float gamma,
                                                float delta) {
  extern __shared__ float4 sma[];
  float* in_s = reinterpret_cast<float*>(sma);
  float* lo_s = in_s + kInSize;
  float* hi_s = lo_s + kRSmax * kPlo;
  const int bi = blockIdx.y, map = blockIdx.z;
  const int hm = m >> 1, tilesx = hm / kTO;
  const int oy0 = (blockIdx.x / tilesx) * kTO, ox0 = (blockIdx.x % tilesx) * kTO;
  load_in_tile(approx_in + ((size_t)map * kDb + bi) * (size_t)m * m, m, oy0, ox0, 2 * kTO + 2 * bi, in_s);
  __syncthreads();
  ana_dispatch(bi, in_s, lo_s, hi_s, map, n, hm, oy0, ox0, last, coef, thr, approx_out, mode, scale, gamma, delta);
}

// Synthesis of one basis on a TI x TI output tile: loads the four subband tiles
// (with the filter halo), filters along y then x, adds the result to acc[4]
// (this thread's four outputs out[r][c0 .. c0+3], r = tid / 8, c0 = 4 (tid % 8)).
template <int LF>
__device__ __forceinline__ void syn_basis(const float* __restrict__ cb, const float* __restrict__ apx, int n, int m,
                                          int oy0, int ox0, float* __restrict__ s4, float* __restrict__ s_lo,
                                          float* __restrict__ s_hi, float acc[4]) {
  constexpr int half = LF / 2 - 1;
  constexpr int CI = kTI / 2 + half;
  constexpr int b = LF / 2 - 1;
  const int hm = m >> 1;
  float* s_ll = s4;
  float* s_lh = s4 + kCImax * kPc;
  float* s_hl = s_lh + kCImax * kPc;
  float* s_hh = s_hl + kCImax * kPc;
  const int ky0 = oy0 / 2 - half, kx0 = ox0 / 2 - half;
  for (int i = threadIdx.x; i < CI * CI; i += blockDim.x) {
    const int r = i / CI, c = i - r * CI;
    const int Yk = wrap1(ky0 + r, hm), Xk = wrap1(kx0 + c, hm);
    s_ll[r * kPc + c] = apx ? apx[(size_t)Yk * hm + Xk] : cb[(size_t)Yk * n + Xk];
    s_hl[r * kPc + c] = cb[(size_t)Yk * n + hm + Xk];
    s_lh[r * kPc + c] = cb[(size_t)(hm + Yk) * n + Xk];
    s_hh[r * kPc + c] = cb[(size_t)(hm + Yk) * n + hm + Xk];
  }
  __syncthreads();
  // Along y: lo[r][c] = sum_{j = r mod 2} h[j] ll[(r - j)/2 + half][c] + g[j] lh[...]; coefficient
  // row r0/2 + i feeds output row r0 + t through tap j = t - 2 (i - half).
  for (int u = threadIdx.x; u < CI * (kTI / 4); u += blockDim.x) {
    const int c = u % CI, r0 = (u / CI) * 4;
    float lo[4] = {0.f, 0.f, 0.f, 0.f}, hi[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int i = 0; i < half + 2; ++i) {
      const int o = (r0 / 2 + i) * kPc + c;
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
  {
    const int r = threadIdx.x >> 3, c0 = (threadIdx.x & 7) * 4;
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
  __syncthreads();
}

__device__ __forceinline__ void syn_dispatch(int bi, const float* cb, const float* apx, int n, int m, int oy0,
                                             int ox0, float* s4, float* s_lo, float* s_hi, float acc[4]) {
#define PS_SYN(LFv) syn_basis<LFv>(cb, apx, n, m, oy0, ox0, s4, s_lo, s_hi, acc)
  switch (bi) {
    case 0: PS_SYN(2); break;
    case 1: PS_SYN(4); break;
    case 2: PS_SYN(6); break;
    case 3: PS_SYN(8); break;
    case 4: PS_SYN(10); break;
    case 5: PS_SYN(12); break;
    case 6: PS_SYN(14); break;
    default: PS_SYN(16); break;
  }
#undef PS_SYN
}

constexpr int kSynSmemFloats = 4 * kCImax * kPc + 2 * kTI * kPs;

// Finest level (m = n): all eight bases plus Dirac summed in registers -> Psi A.
__global__ void __launch_bounds__(256, 3) k_syn_fine(const float* __restrict__ coef, const float* __restrict__ approx_in,
                                                  int coarsest, int n, float* __restrict__ out) {
  __shared__ __align__(16) float sm_s[kSynSmemFloats];
  float* s4 = sm_s;
  float* s_lo = sm_s + 4 * kCImax * kPc;
  float* s_hi = s_lo + kTI * kPs;
  const int map = blockIdx.z;
  const int tilesx = n / kTI;
  const int oy0 = (blockIdx.x / tilesx) * kTI, ox0 = (blockIdx.x % tilesx) * kTI;
  const int hm = n >> 1;
  float acc[4] = {0.f, 0.f, 0.f, 0.f};
  for (int bi = 0; bi < kDb; ++bi) {
    const float* cb = coef + ((size_t)map * kBases + bi + 1) * (size_t)n * n;
    const float* apx = coarsest ? nullptr : approx_in + ((size_t)map * kDb + bi) * (size_t)hm * hm;
    syn_dispatch(bi, cb, apx, n, n, oy0, ox0, s4, s_lo, s_hi, acc);
  }
  const int r = threadIdx.x >> 3, c0 = (threadIdx.x & 7) * 4;
  const size_t o = (size_t)(oy0 + r) * n + ox0 + c0;
  const float4 d = *reinterpret_cast<const float4*>(coef + (size_t)map * kBases * n * n + o);
  const float k = 1.0f / 3.0f;
  *reinterpret_cast<float4*>(out + (size_t)map * n * n + o) =
      make_float4((d.x + acc[0]) * k, (d.y + acc[1]) * k, (d.z + acc[2]) * k, (d.w + acc[3]) * k);
}

// Coarser levels with output side m >= 32: one basis per CTA (grid.y), output to approximation scratch.
__global__ void __launch_bounds__(256, 4) k_syn_lv(const float* __restrict__ coef, const float* __restrict__ approx_in,
                                                int coarsest, int m, int n, float* __restrict__ approx_out) {
  __shared__ __align__(16) float sm_s[kSynSmemFloats];
  float* s4 = sm_s;
  float* s_lo = sm_s + 4 * kCImax * kPc;
  float* s_hi = s_lo + kTI * kPs;
  const int bi = blockIdx.y, map = blockIdx.z;
  const int tilesx = m / kTI;
  const int oy0 = (blockIdx.x / tilesx) * kTI, ox0 = (blockIdx.x % tilesx) * kTI;
  const int hm = m >> 1;
  float acc[4] = {0.f, 0.f, 0.f, 0.f};
  const float* cb = coef + ((size_t)map * kBases + bi + 1) * (size_t)n * n;
  const float* apx = coarsest ? nullptr : approx_in + ((size_t)map * kDb + bi) * (size_t)hm * hm;
  syn_dispatch(bi, cb, apx, n, m, oy0, ox0, s4, s_lo, s_hi, acc);
  const int r = threadIdx.x >> 3, c0 = (threadIdx.x & 7) * 4;
  *reinterpret_cast<float4*>(approx_out + ((size_t)map * kDb + bi) * (size_t)m * m + (size_t)(oy0 + r) * m + ox0 + c0) =
      make_float4(acc[0], acc[1], acc[2], acc[3]);
}

static_assert(kInSize % 4 == 0 && (kRSmax * kPlo) % 4 == 0 && kPlo % 4 == 0, "float4 rows of lo_s/hi_s");
static size_t fast_analysis_smem() { return (size_t)(kInSize + 2 * kRSmax * kPlo) * sizeof(float); }

static size_t analysis_smem(int TO) {
  const int RS = 2 * TO + kMaxTaps - 2;
  return (size_t)(RS * RS + 2 * RS * TO) * sizeof(float);
}
static size_t synthesis_smem(int TI) {
  const int CI = TI / 2 + kMaxTaps / 2 - 1;
  return (size_t)(4 * CI * CI + 2 * TI * CI) * sizeof(float);
}

cudaError_t configure_nufft_kernels();

cudaError_t configure_kernels() {
  cudaError_t e = cudaFuncSetAttribute((const void*)k_analysis, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)analysis_smem(32));
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute((const void*)k_synthesis, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)synthesis_smem(32));
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute((const void*)k_ana_l1, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)fast_analysis_smem());
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute((const void*)k_ana_lv, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)fast_analysis_smem());
  if (e != cudaSuccess) return e;
  return configure_nufft_kernels();
}

cudaError_t sara_analysis(Handle* h, const float* X, float* coef, float* thr, int mode, float scale, float gamma,
                          float delta) {
  const int n = h->n, L = h->L;
  const size_t quarter = (size_t)kDb * 4 * (n / 2) * (n / 2);
  float* buf[2] = {h->approx, h->approx + quarter};
  for (int l = 1; l <= L; ++l) {
    const int m = n >> (l - 1), hm = m / 2;
    const int TO = hm < 32 ? hm : 32;
    const float* in;
    size_t in_map, in_basis;
    if (l == 1) {
      in = X;
      in_map = (size_t)n * n;
      in_basis = 0;
    } else {
      in = buf[(l - 2) & 1];
      in_map = (size_t)kDb * m * m;
      in_basis = (size_t)m * m;
    }
    if (hm >= kTO && l == 1) {
      dim3 grid((hm / kTO) * (hm / kTO), kDb, 4);
      k_ana_l1<<<grid, 256, fast_analysis_smem(), h->stream>>>(X, n, l == L, coef, thr, buf[(l - 1) & 1], mode, scale,
                                                              gamma, delta);
    } else if (hm >= kTO) {
      dim3 grid((hm / kTO) * (hm / kTO), kDb, 4);
      k_ana_lv<<<grid, 256, fast_analysis_smem(), h->stream>>>(in, m, n, l == L, coef, thr, buf[(l - 1) & 1], mode,
                                                              scale, gamma, delta);
    } else {
      dim3 grid((hm / TO) * (hm / TO), kDb, 4);
      k_analysis<<<grid, 256, analysis_smem(TO), h->stream>>>(in, in_map, in_basis, m, TO, n, l == L, coef, thr,
                                                              buf[(l - 1) & 1], mode, scale, gamma, delta);
    }
  }
  return cudaGetLastError();
}

cudaError_t sara_synthesis(Handle* h, const float* coef, float* out) {
  const int n = h->n, L = h->L;
  const size_t quarter = (size_t)kDb * 4 * (n / 2) * (n / 2);
  float* buf[2] = {h->approx, h->approx + quarter};
  for (int l = L; l >= 1; --l) {
    const int m = n >> (l - 1);
    const int TI = m < 32 ? m : 32;
    const int tiles = (m / TI) * (m / TI);
    const float* ain = (l == L) ? nullptr : buf[l & 1];
    float* aout = (l == 1) ? nullptr : buf[(l - 1) & 1];
    if (m >= kTI && l == 1) {
      k_syn_fine<<<dim3(tiles, 1, 4), 256, 0, h->stream>>>(coef, ain, l == L, n, out);
    } else if (m >= kTI) {
      k_syn_lv<<<dim3(tiles, kDb, 4), 256, 0, h->stream>>>(coef, ain, l == L, m, n, aout);
    } else {
      dim3 grid(tiles, l == 1 ? 1 : kDb, 4);
      k_synthesis<<<grid, 256, synthesis_smem(TI), h->stream>>>(coef, ain, l == L, m, TI, n, l == 1, aout, out);
    }
  }
  return cudaGetLastError();
}

}  // namespace ps

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
    dim3 grid((hm / TO) * (hm / TO), kDb, 4);
    k_analysis<<<grid, 256, analysis_smem(TO), h->stream>>>(in, in_map, in_basis, m, TO, n, l == L, coef, thr,
                                                            buf[(l - 1) & 1], mode, scale, gamma, delta);
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
    dim3 grid(tiles, l == 1 ? 1 : kDb, 4);
    k_synthesis<<<grid, 256, synthesis_smem(TI), h->stream>>>(coef, ain, l == L, m, TI, n, l == 1, aout, out);
  }
  return cudaGetLastError();
}

}  // namespace ps

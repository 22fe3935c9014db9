// Per-pixel steps of Algorithm 1 and the reductions of the stopping rules.
//
// k_primal fuses, per pixel, Algorithm 1 steps 3-4 (primal S and Z with P_U or
// P_U' and P_V), the extrapolations 2 S^(k+1) - S^(k), 2 Z^(k+1) - Z^(k), steps
// 9-12 (epigraph duals C, D through P_E1 and P_E2, Eqs. proj_e1 and
// proj_e2_def) and the Dirac part of steps 5-6 (A_dirac = clamp(A + rho1 Xb/3,
// +-gamma W)). In PS_SOC mode the epigraph steps are replaced by the direct
// cone dual C = C~ - rho3 P_P(C~ / rho3) (Z and D are not touched). In the TV modes
// (Algorithm 3) the same sweep takes the data gradient -phi^dagger(Y - phi S) / 2 in place
// of phi^dagger B, Psi A = grad^T A from k_tv_adj, and skips the SARA Dirac part. It also writes per-CTA FP64 partials of ||S^(k+1) - S^(k)||^2 and
// ||S^(k)||^2 per map for the relative-change rule (Eq. stop_crit).
#include <cuda_runtime.h>

#include "internal.h"

namespace ps {

constexpr int kSweepThreads = 256;
constexpr int kSweepPix = 4;   // pixels per thread

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// P_E1 of Eq. proj_e1 on (c, d).
__device__ __forceinline__ void proj_e1(float c, float d, float& pc, float& pd) {
  if (c + d >= 0.f) {
    pc = c;
    pd = d;
  } else {
    pc = 0.5f * (c - d);
    pd = 0.5f * (d - c);
  }
}

// P_E2 of Eq. proj_e2_def on (r1, r2, r3, d).
__device__ __forceinline__ void proj_e2(float r1, float r2, float r3, float d, float& p1, float& p2, float& p3,
                                        float& pd) {
  const float nr = sqrtf(r1 * r1 + r2 * r2 + r3 * r3);
  if (nr < -d || (nr == 0.f && d <= 0.f)) {
    p1 = p2 = p3 = pd = 0.f;
  } else if (nr < d) {
    p1 = r1;
    p2 = r2;
    p3 = r3;
    pd = d;
  } else {
    const float a = 0.5f * (1.0f + d / nr);
    p1 = a * r1;
    p2 = a * r2;
    p3 = a * r3;
    pd = a * nr;
  }
}

__device__ __forceinline__ float4 ld4(const float* p) { return *reinterpret_cast<const float4*>(p); }
__device__ __forceinline__ void st4(float* p, float4 v) { *reinterpret_cast<float4*>(p) = v; }
__device__ __forceinline__ float comp(const float4& v, int k) { return k == 0 ? v.x : (k == 1 ? v.y : (k == 2 ? v.z : v.w)); }
__device__ __forceinline__ void setc(float4& v, int k, float x) {
  if (k == 0) v.x = x;
  else if (k == 1) v.y = x;
  else if (k == 2) v.z = x;
  else v.w = x;
}

// One thread = four consecutive pixels (float4 on every plane). grid.y indexes the problems
// of a batch's size class, whose arrays follow one another (S, C, Xb, PsiA, Adj: 4 N floats
// each; Z, D: 2 N; A, T: 4 cstride; partials: part_stride doubles); one problem: grid.y = 1.
__global__ void __launch_bounds__(kSweepThreads, 3) k_primal(
    int N, int mode, float tau, float rho1, float rho3, float* __restrict__ S, float* __restrict__ Z,
    float* __restrict__ C, float* __restrict__ D, const float* __restrict__ PsiA, const float* __restrict__ Adj,
    float* __restrict__ Xb, float* __restrict__ A, const float* __restrict__ T, size_t cstride,
    double* __restrict__ part, size_t part_stride) {
  __shared__ double sh[kSweepThreads / 32][8];
  if (blockIdx.y) {
    const size_t p = blockIdx.y, n4 = 4 * (size_t)N, n2 = 2 * (size_t)N;
    S += p * n4;
    C += p * n4;
    Xb += p * n4;
    PsiA += p * n4;
    Adj += p * n4;
    Z += p * n2;
    D += p * n2;
    A += p * 4 * cstride;
    T += p * 4 * cstride;
    part += p * part_stride;
  }
  float dss[4] = {0.f, 0.f, 0.f, 0.f}, ss[4] = {0.f, 0.f, 0.f, 0.f};
  const int i = 4 * (blockIdx.x * kSweepThreads + threadIdx.x);
  const float inv_r3 = 1.0f / rho3;
  const float r1_3 = rho1 * (1.0f / 3.0f);
  if (i < N) {
    float4 xb[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const size_t o = (size_t)c * N + i;
      float4 g = ld4(Adj + o);
      // TV modes (Algorithm 3 step 3): Adj holds phi^dagger(Y - phi(S)), so the data
      // gradient 1/2 phi^dagger(phi(S) - Y) is -Adj / 2.
      if (tv_mode(mode)) g = make_float4(-0.5f * g.x, -0.5f * g.y, -0.5f * g.z, -0.5f * g.w);
      if (mode != PS_NNLS) {
        const float4 p = ld4(PsiA + o);
        g = make_float4(g.x + p.x, g.y + p.y, g.z + p.z, g.w + p.w);
      }
      if (constrained_mode(mode)) {
        const float4 q = ld4(C + o);
        g = make_float4(g.x + q.x, g.y + q.y, g.z + q.z, g.w + q.w);
      }
      const float4 so = ld4(S + o);
      float4 sn = make_float4(so.x - tau * g.x, so.y - tau * g.y, so.z - tau * g.z, so.w - tau * g.w);   // step 3
      if (!constrained_mode(mode) && c == 0)                                                          // P_U'
        sn = make_float4(fmaxf(sn.x, 0.f), fmaxf(sn.y, 0.f), fmaxf(sn.z, 0.f), fmaxf(sn.w, 0.f));
      xb[c] = make_float4(2.f * sn.x - so.x, 2.f * sn.y - so.y, 2.f * sn.z - so.z, 2.f * sn.w - so.w);
      dss[c] += (sn.x - so.x) * (sn.x - so.x) + (sn.y - so.y) * (sn.y - so.y) + (sn.z - so.z) * (sn.z - so.z) +
                (sn.w - so.w) * (sn.w - so.w);
      ss[c] += so.x * so.x + so.y * so.y + so.z * so.z + so.w * so.w;
      st4(S + o, sn);
      st4(Xb + o, xb[c]);
      if (mode != PS_NNLS && !tv_mode(mode)) {                          // Dirac part of steps 5-6
        const size_t ao = (size_t)c * cstride + i;
        const float4 t = ld4(T + ao), a = ld4(A + ao);
        st4(A + ao, make_float4(fminf(fmaxf(fmaf(r1_3, xb[c].x, a.x), -t.x), t.x),
                                fminf(fmaxf(fmaf(r1_3, xb[c].y, a.y), -t.y), t.y),
                                fminf(fmaxf(fmaf(r1_3, xb[c].z, a.z), -t.z), t.z),
                                fminf(fmaxf(fmaf(r1_3, xb[c].w, a.w), -t.w), t.w)));
      }
    }
    if (mode == PS_POLARIZED || mode == PS_TV || mode == PS_L1TV) {   // epigraph split (Alg. 1 / Alg. 3)
      const float4 z1o = ld4(Z + i), z2o = ld4(Z + (size_t)N + i);
      const float4 d1o = ld4(D + i), d2o = ld4(D + (size_t)N + i);
      float4 c0 = ld4(C + i), c1 = ld4(C + (size_t)N + i), c2 = ld4(C + 2 * (size_t)N + i),
             c3 = ld4(C + 3 * (size_t)N + i);
      float4 z1n, z2n, d1n, d2n;
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        // Step 4: Z = P_V(Z - tau D).
        const float za = comp(z1o, k), zb = comp(z2o, k);
        float z1 = za - tau * comp(d1o, k), z2 = zb - tau * comp(d2o, k);
        if (z1 + z2 > 0.f) {
          const float a = 0.5f * (z1 - z2);
          z2 = 0.5f * (z2 - z1);
          z1 = a;
        }
        setc(z1n, k, z1);
        setc(z2n, k, z2);
        const float zb1 = 2.f * z1 - za, zb2 = 2.f * z2 - zb;
        // Steps 9-12.
        const float ct0 = comp(c0, k) + rho3 * comp(xb[0], k), ct1 = comp(c1, k) + rho3 * comp(xb[1], k);
        const float ct2 = comp(c2, k) + rho3 * comp(xb[2], k), ct3 = comp(c3, k) + rho3 * comp(xb[3], k);
        const float dt1 = comp(d1o, k) + rho3 * zb1, dt2 = comp(d2o, k) + rho3 * zb2;
        float pc, pd;
        proj_e1(ct0 * inv_r3, dt1 * inv_r3, pc, pd);
        setc(c0, k, ct0 - rho3 * pc);
        setc(d1n, k, dt1 - rho3 * pd);
        float p1, p2, p3, pd2;
        proj_e2(ct1 * inv_r3, ct2 * inv_r3, ct3 * inv_r3, dt2 * inv_r3, p1, p2, p3, pd2);
        setc(c1, k, ct1 - rho3 * p1);
        setc(c2, k, ct2 - rho3 * p2);
        setc(c3, k, ct3 - rho3 * p3);
        setc(d2n, k, dt2 - rho3 * pd2);
      }
      st4(Z + i, z1n);
      st4(Z + (size_t)N + i, z2n);
      st4(D + i, d1n);
      st4(D + (size_t)N + i, d2n);
      st4(C + i, c0);
      st4(C + (size_t)N + i, c1);
      st4(C + 2 * (size_t)N + i, c2);
      st4(C + 3 * (size_t)N + i, c3);
    } else if (mode == PS_SOC) {
      // Direct cone dual: C = C~ - rho3 P_P(C~ / rho3), P_P = P_E2 with (r, d) = ((Q, U, V), I).
      float4 c0 = ld4(C + i), c1 = ld4(C + (size_t)N + i), c2 = ld4(C + 2 * (size_t)N + i),
             c3 = ld4(C + 3 * (size_t)N + i);
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const float ct0 = comp(c0, k) + rho3 * comp(xb[0], k), ct1 = comp(c1, k) + rho3 * comp(xb[1], k);
        const float ct2 = comp(c2, k) + rho3 * comp(xb[2], k), ct3 = comp(c3, k) + rho3 * comp(xb[3], k);
        float p1, p2, p3, p0;
        proj_e2(ct1 * inv_r3, ct2 * inv_r3, ct3 * inv_r3, ct0 * inv_r3, p1, p2, p3, p0);
        setc(c0, k, ct0 - rho3 * p0);
        setc(c1, k, ct1 - rho3 * p1);
        setc(c2, k, ct2 - rho3 * p2);
        setc(c3, k, ct3 - rho3 * p3);
      }
      st4(C + i, c0);
      st4(C + (size_t)N + i, c1);
      st4(C + 2 * (size_t)N + i, c2);
      st4(C + 3 * (size_t)N + i, c3);
    }
  }
  // Partials for the relative-change statistic: FP32 within a warp (at most 128
  // terms), FP64 across warps and CTAs.
  double v[8];
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    v[c] = (double)warp_sum(dss[c]);
    v[4 + c] = (double)warp_sum(ss[c]);
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0)
#pragma unroll
    for (int c = 0; c < 8; ++c) sh[wid][c] = v[c];
  __syncthreads();
  if (threadIdx.x < 8) {
    double s = 0.0;
    for (int w = 0; w < kSweepThreads / 32; ++w) s += sh[w][threadIdx.x];
    part[(size_t)blockIdx.x * 8 + threadIdx.x] = s;
  }
}

int sweep_blocks(int N) { return (N + kSweepThreads * kSweepPix - 1) / (kSweepThreads * kSweepPix); }

cudaError_t primal_sweep(Handle* h) {
  const dim3 grid(sweep_blocks(h->N), h->problems);
  k_primal<<<grid, kSweepThreads, 0, h->stream>>>(h->N, h->mode, (float)h->tau, (float)h->rho1, (float)h->rho3, h->S,
                                                  h->Z, h->C, h->D, h->PsiA, h->Adj, h->Xb, h->A, h->T,
                                                  (size_t)kBases * h->N, h->red, (size_t)h->red_cap);
  return cudaGetLastError();
}

// Dirac part of Psi^dagger for the APPLY and REWEIGHT modes.
__global__ void k_dirac(int N, const float* __restrict__ X, float* __restrict__ coef, float* __restrict__ thr,
                        size_t cstride, int mode, float scale, float gamma, float delta) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int c = blockIdx.y;
  if (i >= N) return;
  const float v = X[(size_t)c * N + i];
  const size_t o = (size_t)c * cstride + i;
  if (mode == SARA_APPLY) coef[o] = scale * v;
  else thr[o] = gamma * delta / (delta + fabsf(scale * v));
}

cudaError_t dirac_apply(Handle* h, const float* X, float* coef, float* thr, int mode, float scale, float gamma,
                        float delta) {
  dim3 grid((h->N + 255) / 256, h->nmaps);
  k_dirac<<<grid, 256, 0, h->stream>>>(h->N, X, coef, thr, (size_t)kBases * h->N, mode, scale, gamma, delta);
  return cudaGetLastError();
}

// Deterministic two-stage FP64 reductions: per-CTA partials then one CTA.
__global__ void k_dot_partial(const float* __restrict__ a, const float* __restrict__ b, size_t len,
                              double* __restrict__ part) {
  __shared__ double sh[32];
  double s = 0.0;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < len; i += (size_t)gridDim.x * blockDim.x)
    s += (double)a[i] * (double)b[i];
  s = warp_sum(s);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sh[w];
    part[blockIdx.x] = t;
  }
}

__global__ void k_sum_partials(const double* __restrict__ part, int np, double* __restrict__ out) {
  __shared__ double sh[32];
  double s = 0.0;
  for (int i = threadIdx.x; i < np; i += blockDim.x) s += part[i];
  s = warp_sum(s);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sh[w];
    *out = t;
  }
}

// Column sums of the per-CTA relative-change partials that k_primal writes (8 per CTA: the
// squared changes of the four maps, then their squared norms), in FP64 and a fixed order,
// written with the device error flags (as ints after the 8 sums) straight into `out`, which
// may be mapped host memory.
__global__ void k_relc_sums(const double* __restrict__ part, int nb, const int* __restrict__ flags,
                            double* __restrict__ out) {
  __shared__ double sh[8][8];   // [warp][column]
  const int c = threadIdx.x & 7;
  double s = 0.0;
  for (int b = threadIdx.x >> 3; b < nb; b += blockDim.x >> 3) s += part[8 * (size_t)b + c];
  s += __shfl_xor_sync(0xffffffffu, s, 8);    // lanes c, c + 8, c + 16, c + 24 hold column c
  s += __shfl_xor_sync(0xffffffffu, s, 16);
  if ((threadIdx.x & 31) < 8) sh[threadIdx.x >> 5][c] = s;
  __syncthreads();
  if (threadIdx.x < 8) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sh[w][threadIdx.x];
    out[threadIdx.x] = t;
  } else if (threadIdx.x < 12) {
    reinterpret_cast<int*>(out + 8)[threadIdx.x - 8] = flags[threadIdx.x - 8];
  }
  __threadfence_system();
}

cudaError_t relc_sums(Handle* h, int nb, double* out) {
  k_relc_sums<<<1, 256, 0, h->stream>>>(h->red, nb, h->dev_flags, out);
  return cudaGetLastError();
}

static constexpr int kRedBlocks = 256;

cudaError_t reduce_dot(Handle* h, const float* a, const float* b, size_t len, double* dev_out) {
  double* part = h->red + (size_t)h->red_cap - 2 * kRedBlocks;
  k_dot_partial<<<kRedBlocks, 256, 0, h->stream>>>(a, b, len, part);
  k_sum_partials<<<1, 256, 0, h->stream>>>(part, kRedBlocks, dev_out);
  return cudaGetLastError();
}

__global__ void k_violations(int N, const float* __restrict__ S, double zeta, double* __restrict__ part) {
  __shared__ double sh[2][32];
  double c0 = 0.0, c1 = 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
    const double I = S[i], Q = S[(size_t)N + i], U = S[2 * (size_t)N + i], V = S[3 * (size_t)N + i];
    const double p = -I + sqrt(Q * Q + U * U + V * V);
    c0 += (p > zeta) ? 1.0 : 0.0;
    c1 += (p > 0.0) ? 1.0 : 0.0;
  }
  c0 = warp_sum(c0);
  c1 = warp_sum(c1);
  if ((threadIdx.x & 31) == 0) {
    sh[0][threadIdx.x >> 5] = c0;
    sh[1][threadIdx.x >> 5] = c1;
  }
  __syncthreads();
  if (threadIdx.x < 2) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sh[threadIdx.x][w];
    part[2 * blockIdx.x + threadIdx.x] = t;
  }
}

__global__ void k_sum_pairs(const double* __restrict__ part, int np, double* __restrict__ out) {
  if (threadIdx.x < 2) {
    double s = 0.0;
    for (int i = 0; i < np; ++i) s += part[2 * i + threadIdx.x];
    out[threadIdx.x] = s;
  }
}

cudaError_t violation_count(Handle* h, const float* S, double zeta, double* dev_out) {
  double* part = h->red + (size_t)h->red_cap - 2 * kRedBlocks;
  k_violations<<<kRedBlocks / 2, 256, 0, h->stream>>>(h->N, S, zeta, part);
  k_sum_pairs<<<1, 32, 0, h->stream>>>(part, kRedBlocks / 2, dev_out);
  return cudaGetLastError();
}

__global__ void k_wl1_partial(const float* __restrict__ c, const float* __restrict__ t, size_t len,
                              double* __restrict__ part) {
  __shared__ double sh[32];
  double s = 0.0;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < len; i += (size_t)gridDim.x * blockDim.x)
    s += (double)t[i] * fabs((double)c[i]);
  s = warp_sum(s);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double r = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) r += sh[w];
    part[blockIdx.x] = r;
  }
}

cudaError_t weighted_l1(Handle* h, const float* coef, const float* thr, double* dev_out) {
  double* part = h->red + (size_t)h->red_cap - 2 * kRedBlocks;
  k_wl1_partial<<<kRedBlocks, 256, 0, h->stream>>>(coef, thr, (size_t)36 * h->N, part);
  k_sum_partials<<<1, 256, 0, h->stream>>>(part, kRedBlocks, dev_out);
  return cudaGetLastError();
}

__global__ void k_maxabs_partial(const float* __restrict__ c, size_t len, float* __restrict__ part) {
  __shared__ float sh[32];
  float m = 0.f;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < len; i += (size_t)gridDim.x * blockDim.x)
    m = fmaxf(m, fabsf(c[i]));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    float r = 0.f;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) r = fmaxf(r, sh[w]);
    part[blockIdx.x] = r;
  }
}

__global__ void k_max_partials(const float* __restrict__ part, int np, double* __restrict__ out) {
  if (threadIdx.x == 0) {
    float r = 0.f;
    for (int i = 0; i < np; ++i) r = fmaxf(r, part[i]);
    *out = (double)r;
  }
}

cudaError_t max_abs(Handle* h, const float* c, size_t len, double* dev_out) {
  float* part = reinterpret_cast<float*>(h->red + (size_t)h->red_cap - 2 * kRedBlocks);
  k_maxabs_partial<<<kRedBlocks, 256, 0, h->stream>>>(c, len, part);
  k_max_partials<<<1, 32, 0, h->stream>>>(part, kRedBlocks, dev_out);
  return cudaGetLastError();
}

__global__ void k_scale_copy(const float* __restrict__ x, float* __restrict__ y, size_t len, double s) {
  const float sf = (float)s;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < len; i += (size_t)gridDim.x * blockDim.x)
    y[i] = x[i] * sf;
}

cudaError_t scale_copy(Handle* h, const float* x, float* y, size_t len, double s) {
  k_scale_copy<<<1024, 256, 0, h->stream>>>(x, y, len, s);
  return cudaGetLastError();
}

// Lanczos three-term recurrence: w = w - alpha v - beta u (FP32 vectors, FP64 coefficients).
__global__ void k_lanczos_update(float* __restrict__ w, const float* __restrict__ v, const float* __restrict__ u,
                                 size_t len, double alpha, double beta) {
  const float a = (float)alpha, b = (float)beta;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < len; i += (size_t)gridDim.x * blockDim.x)
    w[i] = fmaf(-b, u[i], fmaf(-a, v[i], w[i]));
}

cudaError_t lanczos_update(Handle* h, float* w, const float* v, const float* u, size_t len, double alpha,
                           double beta) {
  k_lanczos_update<<<1024, 256, 0, h->stream>>>(w, v, u, len, alpha, beta);
  return cudaGetLastError();
}

// Visibility order changes: sorted row m holds caller row perm[m].
__global__ void k_gather_vis(int M, const int32_t* __restrict__ perm, const float4* __restrict__ user,
                             float4* __restrict__ sorted) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= M) return;
  const size_t u = (size_t)perm[m];
  sorted[2 * (size_t)m] = user[2 * u];
  sorted[2 * (size_t)m + 1] = user[2 * u + 1];
}

__global__ void k_scatter_vis(int M, const int32_t* __restrict__ perm, const float4* __restrict__ sorted,
                              float4* __restrict__ user) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= M) return;
  const size_t u = (size_t)perm[m];
  user[2 * u] = sorted[2 * (size_t)m];
  user[2 * u + 1] = sorted[2 * (size_t)m + 1];
}

cudaError_t gather_vis(Handle* h, const float2* user, float2* sorted) {
  if (h->M == 0) return cudaSuccess;
  k_gather_vis<<<(h->M + 255) / 256, 256, 0, h->stream>>>(h->M, h->perm, reinterpret_cast<const float4*>(user),
                                                          reinterpret_cast<float4*>(sorted));
  return cudaGetLastError();
}

cudaError_t scatter_vis(Handle* h, const float2* sorted, float2* user) {
  if (h->M == 0) return cudaSuccess;
  k_scatter_vis<<<(h->M + 255) / 256, 256, 0, h->stream>>>(h->M, h->perm, reinterpret_cast<const float4*>(sorted),
                                                           reinterpret_cast<float4*>(user));
  return cudaGetLastError();
}

__global__ void k_scale_vis(int M, const uint16_t* __restrict__ vblk, const float* __restrict__ cb,
                            float4* __restrict__ v) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= M) return;
  const float s = cb[vblk[m]];
  const float4 a = v[2 * (size_t)m], b = v[2 * (size_t)m + 1];
  v[2 * (size_t)m] = make_float4(a.x * s, a.y * s, a.z * s, a.w * s);
  v[2 * (size_t)m + 1] = make_float4(b.x * s, b.y * s, b.z * s, b.w * s);
}

cudaError_t scale_vis(Handle* h, float2* v) {
  if (h->M == 0) return cudaSuccess;
  k_scale_vis<<<(h->M + 255) / 256, 256, 0, h->stream>>>(h->M, h->vblk, h->cb, reinterpret_cast<float4*>(v));
  return cudaGetLastError();
}

}  // namespace ps

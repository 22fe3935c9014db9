// Kernels of the TV and l1 + TV problems (Algorithm 3, Section 4.4): the dictionary
// Psi = grad (periodic forward differences, Eq. TV) or [Id, grad].
//
//   k_tv_dual   steps 5-6: A_tv = A~ - rho1 prox_{(mu/rho1)||.||_{2,1}}(A~ / rho1),
//               A~ = A_tv + rho1 grad(2 S^(k+1) - S^(k)); by the Moreau identity this is
//               the projection of A~ onto the disc of radius mu per pixel and map. With
//               the l1 term, A_l1 = clamp(A_l1 + rho1 (2 S^(k+1) - S^(k)), +-nu).
//   k_tv_adj    Psi A = grad^T A_tv (+ A_l1) for the next primal step.
//
// A_tv of map c sits in planes 0 (x) and 1 (y) of map c's nine coefficient planes
// (the SARA coefficient buffer, A + c * 9N), A_l1 in plane 2. One thread per pixel;
// neighbours wrap around the image edges (periodic boundaries).
#include <cuda_runtime.h>

#include "internal.h"

namespace ps {

constexpr int kTvThreads = 256;

__global__ void __launch_bounds__(kTvThreads) k_tv_dual(int n, const float* __restrict__ Xb, float* __restrict__ A,
                                                        size_t cstride, float rho1, float4 mu, float4 nu, int l1) {
  const int N = n * n;
  const int i = blockIdx.x * kTvThreads + threadIdx.x;
  const int c = blockIdx.y;
  if (i >= N) return;
  const int p = i / n, q = i - (i / n) * n;
  const float* x = Xb + (size_t)c * N;
  const float xc = x[i];
  const float gx = x[p * n + (q + 1 == n ? 0 : q + 1)] - xc;      // X[p, q+1] - X[p, q]
  const float gy = x[(p + 1 == n ? 0 : p + 1) * n + q] - xc;      // X[p+1, q] - X[p, q]
  float* a = A + (size_t)c * cstride;
  const float m = c == 0 ? mu.x : (c == 1 ? mu.y : (c == 2 ? mu.z : mu.w));
  const float ax = fmaf(rho1, gx, a[i]), ay = fmaf(rho1, gy, a[(size_t)N + i]);
  const float r = sqrtf(ax * ax + ay * ay);
  const float k = r > m ? m / r : 1.0f;
  a[i] = ax * k;
  a[(size_t)N + i] = ay * k;
  if (l1) {
    const float v = c == 0 ? nu.x : (c == 1 ? nu.y : (c == 2 ? nu.z : nu.w));
    a[2 * (size_t)N + i] = fminf(fmaxf(fmaf(rho1, xc, a[2 * (size_t)N + i]), -v), v);
  }
}

__global__ void __launch_bounds__(kTvThreads) k_tv_adj(int n, const float* __restrict__ A, size_t cstride,
                                                       float* __restrict__ PsiA, int l1) {
  const int N = n * n;
  const int i = blockIdx.x * kTvThreads + threadIdx.x;
  const int c = blockIdx.y;
  if (i >= N) return;
  const int p = i / n, q = i - (i / n) * n;
  const float* ax = A + (size_t)c * cstride;
  const float* ay = ax + N;
  // grad^T (a_x, a_y)[p, q] = a_x[p, q-1] - a_x[p, q] + a_y[p-1, q] - a_y[p, q].
  float v = (ax[p * n + (q == 0 ? n - 1 : q - 1)] - ax[i]) + (ay[(p == 0 ? n - 1 : p - 1) * n + q] - ay[i]);
  if (l1) v += ax[2 * (size_t)N + i];
  PsiA[(size_t)c * N + i] = v;
}

cudaError_t tv_dual(Handle* h) {
  const int N = h->N;
  const dim3 grid((N + kTvThreads - 1) / kTvThreads, 4);
  const float4 mu = make_float4((float)h->tv_mu[0], (float)h->tv_mu[1], (float)h->tv_mu[2], (float)h->tv_mu[3]);
  const float4 nu = make_float4((float)h->l1_mu[0], (float)h->l1_mu[1], (float)h->l1_mu[2], (float)h->l1_mu[3]);
  k_tv_dual<<<grid, kTvThreads, 0, h->stream>>>(h->n, h->Xb, h->A, (size_t)kBases * N, (float)h->rho1, mu, nu,
                                                h->mode == PS_L1TV || h->mode == PS_L1TV_NC);
  return cudaGetLastError();
}

cudaError_t tv_adjoint(Handle* h) {
  const int N = h->N;
  const dim3 grid((N + kTvThreads - 1) / kTvThreads, 4);
  k_tv_adj<<<grid, kTvThreads, 0, h->stream>>>(h->n, h->A, (size_t)kBases * N, h->PsiA,
                                               h->mode == PS_L1TV || h->mode == PS_L1TV_NC);
  return cudaGetLastError();
}

}  // namespace ps

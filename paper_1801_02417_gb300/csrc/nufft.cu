// Measurement operator phi = Phi S L and its adjoint (Section 5.1, Eq. meas_op;
// Algorithm 1 steps 3 and 7), as a non-uniform FFT on the GPU.
//
// Phi = G F Z: Z de-apodises and zero-pads each map to the K = 2n grid, F is the
// K x K FFT, G interpolates the spectrum at each sampled frequency with a W x W
// "exponential of semicircle" kernel. The four real Stokes maps travel as two
// complex images, I + iQ and U + iV, so two complex FFTs serve four maps; the
// correlations are recovered from the spectrum at +u and -u (Hermitian
// symmetry of real maps) and mixed by L of Section 2.1 inside the degridding
// kernel. The spectrum is stored only on the window of frequencies the
// interpolation touches ([-R, R]^2), which prunes the column FFTs and the grid.
//
// Kernels (one launch each):
//   k_fwd_rows    row FFTs of the de-apodised, zero-padded rows     (n CTAs)
//   k_fwd_cols    column FFTs, kept on the window                    (Wd CTAs)
//   k_degrid      interpolation + Stokes->correlation mixing + dual update of B
//                 and per-chunk FP64 partial of ||B~/rho2 - Y||^2     (1 CTA / chunk)
//   k_block_scale per-block l2-ball projection factor (FP64)
//   k_grid        mixing by conj(L) + tile-privatised gridding in shared memory
//   k_adj_cols    Hermitian symmetrisation + inverse column FFTs     (R+1 CTAs)
//   k_adj_rows    inverse row FFTs + crop + de-apodisation -> phi^dagger planes
#include <cuda_runtime.h>

#include "internal.h"
#include "packed.cuh"

namespace ps {

// Sets this file's bounded-wait poll budget (ps_debug_set_wait_polls).
cudaError_t set_wait_polls_nufft(int polls) { return set_wait_polls_here(polls); }

__device__ __forceinline__ float4 f4add(float4 a, float4 b) {
  return make_float4(a.x + b.x, a.y + b.y, a.z + b.z, a.w + b.w);
}
__device__ __forceinline__ float4 f4sub(float4 a, float4 b) {
  return make_float4(a.x - b.x, a.y - b.y, a.z - b.z, a.w - b.w);
}
__device__ __forceinline__ float4 f4scale(float4 a, float s) {
  return make_float4(a.x * s, a.y * s, a.z * s, a.w * s);
}
__device__ __forceinline__ float4 f4fma(float s, float4 a, float4 acc) {
  return make_float4(fmaf(s, a.x, acc.x), fmaf(s, a.y, acc.y), fmaf(s, a.z, acc.z), fmaf(s, a.w, acc.w));
}
// Multiply both complex numbers held in a float4 by w.
__device__ __forceinline__ float4 cmul2(float4 a, float2 w) {
  return make_float4(a.x * w.x - a.y * w.y, a.x * w.y + a.y * w.x,
                     a.z * w.x - a.w * w.y, a.z * w.y + a.w * w.x);
}
__device__ __forceinline__ int bitrev(int i, int logK) { return (int)(__brev((unsigned)i) >> (32 - logK)); }

// Bank-group swizzle of float4 indices in the FFT buffers. Bits 0-2 of an index
// pick one of the eight 16-byte bank groups of a 128-byte row; they are XORed with
// a linear (GF(2)) function of the higher bits chosen so that the eight lanes of a
// quarter-warp hit eight different groups in every access pattern of the
// transforms: the bit-reversed scatter (lanes differ in the top three index bits),
// the radix-4 passes of stages (0,1) and (2,3) (lanes differ in bits 2-4, resp. 0,
// 1 and 4), the later passes and the natural-order reads (bits 0-2). Being linear,
// fsw(a ^ d) = fsw(a) ^ fsw(d).
__device__ __forceinline__ int fsw(int i) {
  const int h = i >> 5;
  const int r = (h ^ (h >> 3) ^ (h >> 6)) & 7;   // bit t: XOR of index bits 5+t, 8+t, 11+t
  return i ^ ((i >> 3) & 1) ^ (((i >> 4) & 1) * 6) ^ ((r & 1) << 1) ^ ((r & 2) << 1) ^ ((r >> 2) & 1);
}

// Twiddle p of radix-2 stage t (span 2^(t+1)): tw[2^t - 1 + p] = exp(-2 pi i p / 2^(t+1));
// each stage's twiddles are contiguous, so the lanes of a pass read consecutive words.
template <bool INV>
__device__ __forceinline__ float2 twid(const float2* __restrict__ tw, int idx) {
  float2 w = __ldg(tw + idx);
  if (INV) w.y = -w.y;
  return w;
}

// In-place decimation-in-time FFT of K = 2^logK float4 (two complex sequences) held
// in shared memory (swizzled by fsw) in bit-reversed order; output in natural
// order. INV selects exp(+2 pi i jk/K) (no 1/K normalisation). Radix-2 stages s
// and s+1 are done together by one thread on the four elements a, a+h, a+2h, a+3h
// (h = 2^s, bits s and s+1 of a clear), so there is one shared-memory pass and one
// barrier per two stages; an odd stage count ends with a plain radix-2 stage.
// Stages below s0 are taken as done (the caller wrote their output); stages from
// s_end on are left to the caller (fft_out).
template <bool INV>
__device__ void fft_smem(float4* buf, const float2* __restrict__ tw, int logK, int s0 = 0, int s_end = -1) {
  const int K = 1 << logK;
  if (s_end < 0) s_end = logK;
  int s = s0;
  for (; s + 1 < s_end; s += 2) {
    const int hs = 1 << s;
    const int c1 = fsw(hs), c2 = fsw(2 * hs);
    for (int g = threadIdx.x; g < (K >> 2); g += blockDim.x) {
      const int pos = g & (hs - 1);
      const int a = fsw(((g >> s) << (s + 2)) + pos);
      const float2 w0 = twid<INV>(tw, hs - 1 + pos);          // stage s
      const float2 w1 = twid<INV>(tw, 2 * hs - 1 + pos);      // stage s+1, pair (a, a+2h)
      const float2 w2 = twid<INV>(tw, 3 * hs - 1 + pos);      // stage s+1, pair (a+h, a+3h)
      const float4 x0 = buf[a], x1 = buf[a ^ c1], x2 = buf[a ^ c2], x3 = buf[a ^ c1 ^ c2];
      const float4 t1 = cmul2(x1, w0), t3 = cmul2(x3, w0);
      const float4 y0 = f4add(x0, t1), y1 = f4sub(x0, t1), y2 = f4add(x2, t3), y3 = f4sub(x2, t3);
      const float4 u2 = cmul2(y2, w1), u3 = cmul2(y3, w2);
      buf[a] = f4add(y0, u2);
      buf[a ^ c2] = f4sub(y0, u2);
      buf[a ^ c1] = f4add(y1, u3);
      buf[a ^ c1 ^ c2] = f4sub(y1, u3);
    }
    __syncthreads();
  }
  if (s < s_end) {
    const int hs = 1 << s;
    const int c1 = fsw(hs);
    for (int b = threadIdx.x; b < (K >> 1); b += blockDim.x) {
      const int pos = b & (hs - 1);
      const int i0 = fsw(((b >> s) << (s + 1)) + pos);
      const float2 w = twid<INV>(tw, hs - 1 + pos);
      const float4 u = buf[i0];
      const float4 v = cmul2(buf[i0 ^ c1], w);
      buf[i0] = f4add(u, v);
      buf[i0 ^ c1] = f4sub(u, v);
    }
    __syncthreads();
  }
}

// Input of a K-point transform whose nonzero samples fill exactly one of each pair of
// natural indices (x, x + K/2), i.e. the bit-reversed neighbours (r, r ^ 1) that the
// first radix-2 stage combines (twiddle 1): that stage is folded into the scatter.
// Sample v at natural index idx writes both outputs of its pair, v at the even slot
// and +v or -v (idx < K/2 or not) at the odd one; fft_smem then starts at stage 1.
// Every slot is written, so the buffer needs no clearing.
__device__ __forceinline__ void scatter_stage0(float4* buf, int idx, int logK, float4 v) {
  const int r = bitrev(idx, logK);
  buf[fsw(r & ~1)] = v;
  buf[fsw(r | 1)] = (idx < (1 << (logK - 1))) ? v : make_float4(-v.x, -v.y, -v.z, -v.w);
}

// First stage fft_out finishes when the passes start at s0: the last radix-4 pass, or
// the last radix-2 stage when the stage count from s0 is odd.
__device__ __forceinline__ int fft_tail_start(int logK, int s0) {
  return ((logK - s0) & 1) ? logK - 1 : logK - 2;
}

// Natural-order output k of the transform whose stages below s_last are done in buf;
// its remaining one (s_last = logK - 1) or two (s_last = logK - 2) stages are applied
// here for this output alone (the same arithmetic as the last pass of fft_smem), so
// a caller that needs few outputs skips that pass, its barrier and a buffer rewrite.
template <bool INV>
__device__ __forceinline__ float4 fft_out(const float4* buf, const float2* __restrict__ tw, int logK, int s_last,
                                          int k) {
  const int hs = 1 << s_last;
  const int g = k & (hs - 1);
  if (s_last == logK - 2) {
    const float2 w0 = twid<INV>(tw, hs - 1 + g), w1 = twid<INV>(tw, 2 * hs - 1 + g), w2 = twid<INV>(tw, 3 * hs - 1 + g);
    const float4 x0 = buf[fsw(g)], x1 = buf[fsw(g + hs)], x2 = buf[fsw(g + 2 * hs)], x3 = buf[fsw(g + 3 * hs)];
    const float4 t1 = cmul2(x1, w0), t3 = cmul2(x3, w0);
    const int j = k >> s_last;
    if (j == 0) return f4add(f4add(x0, t1), cmul2(f4add(x2, t3), w1));
    if (j == 2) return f4sub(f4add(x0, t1), cmul2(f4add(x2, t3), w1));
    if (j == 1) return f4add(f4sub(x0, t1), cmul2(f4sub(x2, t3), w2));
    return f4sub(f4sub(x0, t1), cmul2(f4sub(x2, t3), w2));
  }
  const float2 w = twid<INV>(tw, hs - 1 + g);
  const float4 u = buf[fsw(g)], v = cmul2(buf[fsw(g + hs)], w);
  return k < hs ? f4add(u, v) : f4sub(u, v);
}

__device__ __forceinline__ int gidx(int k, int off, int full, int K) {
  return full ? (k & (K - 1)) : (k + off);
}

// ---------------------------------------------------------------- forward
__global__ void k_fwd_rows(const float* __restrict__ X, int n, int N, const float* __restrict__ corr,
                           const float2* __restrict__ tw, int K, int logK, float4* __restrict__ T1,
                           int Wd, int off, int full) {
  extern __shared__ float4 sm[];
  float4* buf = sm;
  const int p = blockIdx.x;
  const float cy = corr[p];
  const size_t row = (size_t)p * n;
  // The n samples sit at natural indices [0, n/2) and [K - n/2, K) of K = 2n: one per pair.
  for (int q = threadIdx.x; q < n; q += blockDim.x) {
    const int idx = (q - n / 2 + K) & (K - 1);
    const float c = cy * corr[q];
    const size_t o = row + q;
    scatter_stage0(buf, idx, logK, make_float4(X[o] * c, X[N + o] * c, X[2 * (size_t)N + o] * c,
                                               X[3 * (size_t)N + o] * c));
  }
  __syncthreads();
  const int st = fft_tail_start(logK, 1);
  fft_smem<false>(buf, tw, logK, 1, st);
  for (int gx = threadIdx.x; gx < Wd; gx += blockDim.x) {
    const int k = full ? gx : gx - off;
    T1[(size_t)p * Wd + gx] = fft_out<false>(buf, tw, logK, st, (k + K) & (K - 1));
  }
}

__global__ void k_fwd_cols(const float4* __restrict__ T1, int n, const float2* __restrict__ tw, int K,
                           int logK, float4* __restrict__ G, int Wd, int off, int full) {
  extern __shared__ float4 sm[];
  float4* buf = sm;
  const int gx = blockIdx.x;
  for (int p = threadIdx.x; p < n; p += blockDim.x) {
    const int idx = (p - n / 2 + K) & (K - 1);
    scatter_stage0(buf, idx, logK, T1[(size_t)p * Wd + gx]);
  }
  __syncthreads();
  const int st = fft_tail_start(logK, 1);
  fft_smem<false>(buf, tw, logK, 1, st);
  for (int gy = threadIdx.x; gy < Wd; gy += blockDim.x) {
    const int k = full ? gy : gy - off;
    G[(size_t)gy * Wd + gx] = fft_out<false>(buf, tw, logK, st, (k + K) & (K - 1));
  }
}

template <int W>
__device__ __forceinline__ void es_weights(float f, float beta, float* wt) {
  // wt[j] = phi(f + hw - j), tap j at frequency c - hw + j.
  constexpr int hw = W / 2;
  const float inv = 2.0f / W;
#pragma unroll
  for (int j = 0; j < W; ++j) {
    const float z = (f + (float)(hw - j)) * inv;
    const float s = 1.0f - z * z;
    wt[j] = s > 0.f ? __expf(beta * (s * rsqrtf(s) - 1.0f)) : 0.f;
  }
}

__device__ __forceinline__ void unpack_rec(float4 r, float& fx, float& fy, float& w, int& cx, int& cy) {
  fx = r.x;
  fy = r.y;
  w = r.z;
  const int pk = __float_as_int(r.w);
  cx = (int)(short)(pk & 0xFFFF);
  cy = pk >> 16;
}

template <typename T>
__device__ __forceinline__ T block_sum(T v, T* sh) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  T r = 0;
  if (threadIdx.x < 32) {
    r = (threadIdx.x < (blockDim.x >> 5)) ? sh[threadIdx.x] : (T)0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) r += __shfl_xor_sync(0xffffffffu, r, o);
  }
  return r;  // valid in thread 0
}

// FP32 -> TF32 hi part (round to nearest, ties away) and the TF32 rounding of the
// remainder; hi + lo carries the operand to about 2^-21 of its value.
__device__ __forceinline__ void tf32_split(float a, uint32_t& hi, uint32_t& lo) {
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(hi) : "f"(a));
  const float r = a - __uint_as_float(hi);
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(lo) : "f"(r));
}
// The same split with integer rounding of the hi part (round half up on the magnitude) and
// the remainder left for the tensor core to truncate to TF32: |a - hi - lo_tf32| <= 2^-21 |a|.
__device__ __forceinline__ void tf32_split_fast(float a, uint32_t& hi, uint32_t& lo) {
  hi = (__float_as_uint(a) + 0x1000u) & 0xFFFFE000u;
  lo = __float_as_uint(a - __uint_as_float(hi));
}
// d += A B for one m16n8k8 TF32 tile: A (16 x 8) fragment a[4], B (8 x 8) fragment b[2].
__device__ __forceinline__ void mma_tf32(float (&d)[4], const uint32_t (&a)[4], const uint32_t (&b)[2]) {
  asm("mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
      "{%0, %1, %2, %3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// Second half of a degridding row m (all 32 lanes of the warp call it together: the
// block-sum combination is warp-collective; inactive lanes add nothing): from the
// interpolated packed spectra sp (at +u) and sn (at -u) to the row's visibilities
// (or residuals), and its term of the per-block sums.
__device__ __forceinline__ void degrid_finish(int m, bool active, float w, float4 sp, float4 sn, int mode,
                                              float2* __restrict__ R, const float2* __restrict__ Yv,
                                              const float* __restrict__ cb, float inv_rho2,
                                              const uint16_t* __restrict__ vblk, bool reduce, bool private_bins,
                                              double* bsum, float2* __restrict__ out) {
  float4* R4 = reinterpret_cast<float4*>(R);
  const float4* Y4 = reinterpret_cast<const float4*>(Yv);
  int blk = -1;
  float e2 = 0.f;
  if (active) {
    // G1 = F(I + iQ), G2 = F(U + iV); F(I) = (G1(u) + conj G1(-u))/2, F(Q) = (G1(u) - conj G1(-u))/(2i).
    const float FIr = 0.5f * (sp.x + sn.x), FIi = 0.5f * (sp.y - sn.y);
    const float FQr = 0.5f * (sp.y + sn.y), FQi = -0.5f * (sp.x - sn.x);
    float4 v01 = make_float4(w * (FIr + FQr), w * (FIi + FQi), w * sp.z, w * sp.w);   // RR, RL = G2(u)
    float4 v23 = make_float4(w * sn.z, -w * sn.w, w * (FIr - FQr), w * (FIi - FQi));  // LR = conj G2(-u), LL
    if (mode == DEG_APPLY) {
      float4* o4 = reinterpret_cast<float4*>(out);
      o4[2 * (size_t)m] = v01;
      o4[2 * (size_t)m + 1] = v23;
    } else {
      blk = vblk[m];
      const float4 y0 = Y4[2 * (size_t)m], y1 = Y4[2 * (size_t)m + 1];
      if (mode == DEG_DUAL) {
        const float cs = cb[blk] * inv_rho2;
        const float4 r0 = R4[2 * (size_t)m], r1 = R4[2 * (size_t)m + 1];
        v01 = f4sub(f4fma(cs, r0, v01), y0);
        v23 = f4sub(f4fma(cs, r1, v23), y1);
        R4[2 * (size_t)m] = v01;
        R4[2 * (size_t)m + 1] = v23;
      } else {
        v01 = f4sub(y0, v01);
        v23 = f4sub(y1, v23);
        if (out) {
          float4* o4 = reinterpret_cast<float4*>(out);
          o4[2 * (size_t)m] = v01;
          o4[2 * (size_t)m + 1] = v23;
        }
      }
      e2 = (v01.x * v01.x + v01.y * v01.y + v01.z * v01.z + v01.w * v01.w) +
           (v23.x * v23.x + v23.y * v23.y + v23.z * v23.z + v23.w * v23.w);
    }
  }
  if (reduce) {
    // Lanes holding the same block add their terms (FP32, at most 32 of them); the
    // lowest such lane adds the group's sum in FP64 to this warp's bin of the block
    // (private bins: no other lane or warp writes it) or, with many blocks, to the
    // CTA's shared bin by an atomic.
    const unsigned peers = __match_any_sync(0xffffffffu, blk);
    float sum = 0.f;
    for (unsigned p = peers; p; p &= p - 1) sum += __shfl_sync(peers, e2, __ffs(p) - 1);
    if (blk >= 0 && (threadIdx.x & 31) == __ffs(peers) - 1) {
      if (private_bins) bsum[(threadIdx.x >> 5) * kWarpBins + blk] += (double)sum;
      else atomicAdd(&bsum[blk], (double)sum);
    }
    __syncwarp();   // the next row's leader of this block may be another lane
  }
}

// Ask L1 for the row's inputs of degrid_finish (R, Y: one 32-byte sector each) before the
// interpolation, so that their latency overlaps it instead of following it.
__device__ __forceinline__ void degrid_prefetch(int m, int mode, const float2* R, const float2* Yv) {
  if (mode == DEG_APPLY) return;
  asm volatile("prefetch.global.L1 [%0];" ::"l"(Yv + 4 * (size_t)m));
  if (mode == DEG_DUAL) asm volatile("prefetch.global.L1 [%0];" ::"l"(R + 4 * (size_t)m));
}

// One row of a degridding work item on the CUDA cores: the 2 W^2 taps read from the
// staged spectrum cells, then degrid_finish (warp-collective, like it).
template <int W>
__device__ __forceinline__ void degrid_row(int m, bool active, const GridItem& it, const float4* __restrict__ rec,
                                           const float4* Gp, const float4* Gn, int off, int full, int K, float beta,
                                           int mode, float2* __restrict__ R, const float2* __restrict__ Yv,
                                           const float* __restrict__ cb, float inv_rho2,
                                           const uint16_t* __restrict__ vblk, bool reduce, bool private_bins,
                                           double* bsum,
                                           float2* __restrict__ out) {
  constexpr int TS = kGridTile;
  constexpr int SS = TS + W - 1;
  float4 sp = make_float4(0.f, 0.f, 0.f, 0.f), sn = sp;
  float w = 0.f;
  if (active) {
    degrid_prefetch(m, mode, R, Yv);
    float fx, fy;
    int cx, cy;
    unpack_rec(rec[m], fx, fy, w, cx, cy);
    float wx[W], wy[W];
    es_weights<W>(fx, beta, wx);
    es_weights<W>(fy, beta, wy);
    // Local centre within the tile (tap j of +u at local j + lc; of -u at local (TS-1-lc) + j).
    const int lcy = gidx(cy, off, full, K) - it.ty * TS, lcx = gidx(cx, off, full, K) - it.tx * TS;
    const float4* gp = Gp + lcy * SS + lcx;
    const float4* gn = Gn + (TS - 1 - lcy) * SS + (TS - 1 - lcx);
    // Packed FP32x2: channels (x, y) and (z, w) of each float4 cell in one FMA each.
    u64 sp0 = 0ull, sp1 = 0ull, sn0 = 0ull, sn1 = 0ull;
#pragma unroll
    for (int jy = 0; jy < W; ++jy) {
      u64 ap0 = 0ull, ap1 = 0ull, an0 = 0ull, an1 = 0ull;
#pragma unroll
      for (int jx = 0; jx < W; ++jx) {
        const ulonglong2 vp = *reinterpret_cast<const ulonglong2*>(gp + jy * SS + jx);
        const ulonglong2 vn = *reinterpret_cast<const ulonglong2*>(gn + jy * SS + jx);
        const u64 kp = fdup(wx[jx]), kn = fdup(wx[W - 1 - jx]);
        ap0 = ffma2(kp, vp.x, ap0);
        ap1 = ffma2(kp, vp.y, ap1);
        an0 = ffma2(kn, vn.x, an0);
        an1 = ffma2(kn, vn.y, an1);
      }
      const u64 ky = fdup(wy[jy]), kny = fdup(wy[W - 1 - jy]);
      sp0 = ffma2(ky, ap0, sp0);
      sp1 = ffma2(ky, ap1, sp1);
      sn0 = ffma2(kny, an0, sn0);
      sn1 = ffma2(kny, an1, sn1);
    }
    f2unpack(sp0, sp.x, sp.y);
    f2unpack(sp1, sp.z, sp.w);
    f2unpack(sn0, sn.x, sn.y);
    f2unpack(sn1, sn.z, sn.w);
  }
  degrid_finish(m, active, w, sp, sn, mode, R, Yv, cb, inv_rho2, vblk, reduce, private_bins, bsum, out);
}

// Interpolate the packed spectra at +u and -u, unpack the four Stokes spectra,
// mix into RR, RL, LR, LL (Section 2.1) and weight by w_m. One CTA per gridding
// work item (rows whose tap centres lie in one kGridTile^2 tile): the spectrum
// cells every tap of the item can touch at +u, and the mirrored cells at -u, are
// staged in shared memory once; each thread then interpolates one row with taps at
// fixed offsets from its centre. Per-block sums of ||B~/rho2 - Y||^2 (DUAL) or
// ||Y - phi X||^2 (RESID): per row and per warp group of same-block lanes in FP32,
// then in FP64 through per-warp shared bins (up to kWarpBins blocks; shared FP64
// atomics beyond) and one global FP64 atomic per block and CTA (block_sum, cleared
// by the caller).
// FORM 0: one row per thread over the item; 1: one same-cell chunk per warp (broadcast
// stencil reads); 2: as 0 with registers capped for 6 CTAs per SM at W = 7 (40 instead of
// 51, so more rows are in flight per SM; other widths would spill under a cap and run as 0).
template <int W, int FORM>
__global__ void __launch_bounds__(256, (FORM == 2 && W == 7) ? 6 : 0) k_degrid(
    const GridItem* __restrict__ items, const int32_t* __restrict__ chunks, const float4* __restrict__ rec, const float4* __restrict__ G, int Wd,
    int off, int full, int K, float beta, int mode, float2* __restrict__ R, const float2* __restrict__ Yv,
    const float* __restrict__ cb, float inv_rho2, const uint16_t* __restrict__ vblk, int nblocks,
    double* __restrict__ block_sum, float2* __restrict__ out) {
  constexpr int TS = kGridTile;
  constexpr int SS = TS + W - 1;
  constexpr int hw = W / 2;
  extern __shared__ float4 smd[];
  float4* Gp = smd;                 // +u cells: grid rows/cols ty*TS - hw + [0, SS)
  float4* Gn = smd + SS * SS;       // -u cells: mirrored rows/cols -(ty*TS + TS-1) - hw + [0, SS)
  double* bsum = reinterpret_cast<double*>(smd + 2 * SS * SS);
  const GridItem it = items[blockIdx.x];
  const bool reduce = (mode != DEG_APPLY);
  const bool private_bins = nblocks <= kWarpBins;   // per-warp bins: kWarpBins x 8 warps doubles
  const int nbins = private_bins ? kWarpBins * (blockDim.x >> 5) : nblocks;
  if (reduce)
    for (int b = threadIdx.x; b < nbins; b += blockDim.x) bsum[b] = 0.0;
  // Grid frequency (k) of local row 0: +u region starts at tile origin - hw; the -u region
  // holds frequencies -(centre) - hw + j for every centre of the tile.
  const int ky0 = it.ty * TS - hw - (full ? 0 : off), kx0 = it.tx * TS - hw - (full ? 0 : off);
  const int nky0 = -(it.ty * TS + TS - 1 - (full ? 0 : off)) - hw, nkx0 = -(it.tx * TS + TS - 1 - (full ? 0 : off)) - hw;
  for (int i = threadIdx.x; i < SS * SS; i += blockDim.x) {
    const int ly = i / SS, lx = i - (i / SS) * SS;
    int py = ky0 + ly, px = kx0 + lx, ny = nky0 + ly, nx = nkx0 + lx;
    float4 vp = make_float4(0.f, 0.f, 0.f, 0.f), vn = vp;
    if (full) {
      vp = G[(size_t)(py & (K - 1)) * Wd + (px & (K - 1))];
      vn = G[(size_t)(ny & (K - 1)) * Wd + (nx & (K - 1))];
    } else {
      py += off; px += off; ny += off; nx += off;
      if (py >= 0 && py < Wd && px >= 0 && px < Wd) vp = G[(size_t)py * Wd + px];
      if (ny >= 0 && ny < Wd && nx >= 0 && nx < Wd) vn = G[(size_t)ny * Wd + nx];
    }
    Gp[i] = vp;
    Gn[i] = vn;
  }
  __syncthreads();
  if (FORM == 1) {
    // One same-cell chunk (<= 32 rows) per warp: every lane reads the same stencil
    // cells, so the shared-memory gathers are broadcasts.
    const int lane = threadIdx.x & 31, nwarps = blockDim.x >> 5;
    for (int c = threadIdx.x >> 5; c < it.cend - it.cstart; c += nwarps) {
      const int pk = chunks[it.cstart + c];
      const int v0 = pk & 1023, cnt = (pk >> 10) & 63;
      degrid_row<W>(it.vstart + v0 + lane, lane < cnt, it, rec, Gp, Gn, off, full, K, beta, mode, R, Yv, cb, inv_rho2,
                    vblk, reduce, private_bins, bsum, out);
    }
  } else {
    for (int base = it.vstart; base < it.vend; base += blockDim.x) {
      const int m = base + threadIdx.x;
      degrid_row<W>(m, m < it.vend, it, rec, Gp, Gn, off, full, K, beta, mode, R, Yv, cb, inv_rho2, vblk, reduce,
                    private_bins, bsum, out);
    }
  }
  if (reduce) {
    __syncthreads();
    for (int b = threadIdx.x; b < nblocks; b += blockDim.x) {
      double t = 0.0;
      if (private_bins)
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += bsum[w * kWarpBins + b];
      else
        t = bsum[b];
      if (t != 0.0) atomicAdd(&block_sum[b], t);
    }
  }
}

template <int W>
static constexpr size_t degrid_smem_tiles() {
  return (size_t)2 * (kGridTile + W - 1) * (kGridTile + W - 1) * sizeof(float4);
}

// Per-block factor c_b of B = c_b R after the l2-ball step (Algorithm 1 step 8):
// with r = ||B~/rho2 - Y||_b, c_b = rho2 (1 - min(1, radius / r)).
__global__ void k_block_scale(const double* __restrict__ block_sum, const double* __restrict__ eps, int nblocks,
                              double rho2, int literal, float* __restrict__ cb) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nblocks) return;
  const double r = sqrt(block_sum[b]);
  const double radius = literal ? eps[b] / rho2 : eps[b];
  const double keep = (r > radius) ? radius / r : 1.0;
  cb[b] = (float)(rho2 * (1.0 - keep));
}

// Gridding (adjoint of the interpolation), Alg. 1 step 3's phi^dagger.
// Rows are stored sorted by tap-centre cell. One CTA owns a work item:
// up to kGridItemG visibilities whose centres lie in one kGridTileG^2 tile.
//  1. Each thread stages one visibility in shared memory: the conj(L)-mixed
//     values x_I = RR + LL, x_Q = RR - LL, x_U = RL + LR, x_V = i (LR - RL)
//     scaled by c_b w_m (two float4), and its W x and W y kernel weights (planes
//     with an odd stride, so lanes reading different taps hit different banks).
//  2. Visibilities sharing a centre cell (a chunk of <= 32) touch the same W x W
//     cells. One warp takes one chunk; lane l owns kernel cells l, l+32, ... and
//     accumulates their 8 channels over the chunk in registers (two rows per
//     step, channel values read as broadcasts), then adds them once to a
//     channel-planar shared-memory tile.
//  3. The tile (with halo) is added to the global accumulator.
// Channels are gridded at +u only; k_adj_cols forms the -u half by Hermitian
// symmetrisation.
// Stride of the staged per-row weight planes: tap j of row v sits in bank (2 j + v) mod 32, so
// the lanes of a warp (one row, or two rows v, v+1 in the half-warp form) reading their
// cells' taps never share a bank.
constexpr int kGridV = kGridItemG + 2;

// Work split of a same-cell chunk (one warp per chunk in every form):
// FORM 0: lane l owns kernel cells l, l + 32, all 8 channels.
// FORM 1: the two half-warps take alternate rows of the chunk, lane l owns cells
//   (l & 15) + 16 q; each 16-byte broadcast read of a row's channels then serves 16 lanes
//   (two rows per instruction), and the halves' sums are combined by shuffles before the
//   shared-memory flush.
// FORM 2 (W <= 8): lane l < 4 W owns stencil row jy = l / 4 and channel pair cp = l % 4,
//   i.e. the W cells (jy, 0..W-1) of two channels: per row it reads w_y[jy], its channel
//   pair and the W x-weights (broadcasts), forms t = w_y x once and applies W packed FMAs.
// FORM 3 (W <= 8): the chunk's block as a product of two small matrices on the tensor
//   cores (mma.m16n8k8, TF32 with hi/lo operand splitting for FP32 accuracy); lanes load
//   distinct words of the rows instead of broadcasts.
// Stride of the 8 channel planes of a gridding tile: its (kGridTileG + W - 1)^2 cells plus
// one, odd modulo 32, so lanes adding to the same cell of different planes spread over banks.
template <int W>
__host__ __device__ constexpr int grid_plane() {
  return (kGridTileG + W - 1) * (kGridTileG + W - 1) + 1;
}

// FORM 3 keeps 8 y-weights and 8 x-weights per row for kGridItemG rows plus 8 spare
// rows (its last k-step of a chunk may read, and then discard, up to 7 rows past it).
constexpr int kGridRows3 = kGridItemG + 8;
// Floats of staged weights per work item (a multiple of 4: the tile planes after them stay 16-byte aligned).
template <int W, int FORM>
__host__ __device__ constexpr int grid_wts_floats() {
  return FORM >= 3 ? 16 * kGridRows3 : (2 * W * kGridV + 3) / 4 * 4;
}

// Step 1 for one visibility j of a work item: row record r (fx, fy, w), its correlations
// b0 = (RR, RL), b1 = (LR, LL) and its block scale. FORM 0-2 evaluate its weights into
// wts as W x-planes then W y-planes of stride kGridV; FORM 3 copies them instead (8
// y-weights per row for kGridRows3 rows, then 8 x-weights per row, zero past W).
template <int W, int FORM>
__device__ __forceinline__ void grid_stage_row(int j, float4 r, float4 b0, float4 b1, float blk_scale, float beta,
                                               float4* __restrict__ x4, float* __restrict__ wts) {
  float fx, fy, w;
  int cx, cy;
  unpack_rec(r, fx, fy, w, cx, cy);
  const float sc = blk_scale * w;
  // x_I = RR + LL, x_Q = RR - LL, x_U = RL + LR, x_V = i (LR - RL).
  x4[2 * j] = make_float4(sc * (b0.x + b1.z), sc * (b0.y + b1.w), sc * (b0.x - b1.z), sc * (b0.y - b1.w));
  x4[2 * j + 1] = make_float4(sc * (b0.z + b1.x), sc * (b0.w + b1.y), -sc * (b1.y - b0.w), sc * (b1.x - b0.z));
  if (FORM == 3) {
    // Weights arrive by bulk copies from the per-row table (k_row_weights).
  } else if (FORM == 4) {
    // The layout of FORM 3, evaluated here instead of copied from the table.
    float wx[W], wy[W];
    es_weights<W>(fx, beta, wx);
    es_weights<W>(fy, beta, wy);
    float t[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) t[k] = k < W ? wy[k] : 0.f;
    float4* py = reinterpret_cast<float4*>(wts) + 2 * j;
    py[0] = make_float4(t[0], t[1], t[2], t[3]);
    py[1] = make_float4(t[4], t[5], t[6], t[7]);
#pragma unroll
    for (int k = 0; k < 8; ++k) t[k] = k < W ? wx[k] : 0.f;
    float4* px = reinterpret_cast<float4*>(wts + 8 * kGridRows3) + 2 * j;
    px[0] = make_float4(t[0], t[1], t[2], t[3]);
    px[1] = make_float4(t[4], t[5], t[6], t[7]);
  } else {
    float wx[W], wy[W];
    es_weights<W>(fx, beta, wx);
    es_weights<W>(fy, beta, wy);
    float* wxs = wts;
    float* wys = wts + W * kGridV;
#pragma unroll
    for (int k = 0; k < W; ++k) {
      wxs[k * kGridV + j] = wx[k];
      wys[k * kGridV + j] = wy[k];
    }
  }
}

// Step 2: every same-cell chunk of the work item, one warp per chunk (FORM as above),
// added to the channel-planar tile acc (8 planes of grid_plane<W>() floats).
template <int W, int FORM>
__device__ __forceinline__ void grid_chunks(const int32_t* __restrict__ chunks, int nc, const float4* __restrict__ x4,
                                            const float* __restrict__ wts, float* __restrict__ acc) {
  const float* wxs = wts;
  const float* wys = wts + W * kGridV;
  constexpr int TS = kGridTileG;
  constexpr int SS = TS + W - 1;
  constexpr int NP = grid_plane<W>();
  constexpr bool HALF = FORM == 1;
  constexpr int LPR = HALF ? 16 : 32;            // lanes per row in flight
  constexpr int CPL = (W * W + LPR - 1) / LPR;   // kernel cells per lane
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  const int sub = HALF ? (lane >> 4) : 0, sl = HALF ? (lane & 15) : lane;
  int wxo[CPL], wyo[CPL], coff[CPL];
#pragma unroll
  for (int q = 0; q < CPL; ++q) {
    const int cell = sl + LPR * q;
    const int jy = cell < W * W ? cell / W : 0, jx = cell < W * W ? cell - (cell / W) * W : 0;
    wxo[q] = jx * kGridV;
    wyo[q] = jy * kGridV;
    coff[q] = jy * SS + jx;
  }
  const ulonglong2* xv = reinterpret_cast<const ulonglong2*>(x4);
  for (int c = warp; c < nc; c += nwarps) {
    const int pk = chunks[c];
    const int v0 = pk & 1023, cnt = (pk >> 10) & 63, ly = (pk >> 16) & 255, lx = (pk >> 24) & 255;
    if constexpr (FORM >= 3) {
      // Tensor cores: the chunk's W x W x 8 block is the product G = P^T Y over its rows,
      // P[v][(jx, c)] = w_x[v][jx] x_c[v] (64 rows (jx, c) in MT m-tiles of 16) and
      // Y[v][jy] = w_y[v][jy] (8 columns), k = 8 rows per mma.m16n8k8 (TF32). Each FP32
      // operand is split into TF32 hi + lo parts and the three products hi hi, hi lo,
      // lo hi are accumulated in FP32 (the lo lo term is below FP32 rounding). Rows of
      // the last k-step past the chunk enter as zeros.
      constexpr int MT = (W + 1) / 2;
      const int g = lane >> 2, tig = lane & 3;
      const float* xs = reinterpret_cast<const float*>(x4);
      const float* wyb = wts;
      const float* wxb = wts + 8 * kGridRows3;
      float d[MT][4];
#pragma unroll
      for (int t = 0; t < MT; ++t) d[t][0] = d[t][1] = d[t][2] = d[t][3] = 0.f;
      const int vend = v0 + cnt;
      for (int k0 = v0; k0 < vend; k0 += 8) {
        const int va = k0 + tig, vb = va + 4;
        // Rows past the chunk (the next chunk's, or the zeroed spare rows after the
        // item) keep their finite P entries; their Y entries are zeroed.
        const float xa = xs[8 * va + g], xb = xs[8 * vb + g];
        uint32_t bh[2], bl[2];
        tf32_split(va < vend ? wyb[8 * va + g] : 0.f, bh[0], bl[0]);
        tf32_split(vb < vend ? wyb[8 * vb + g] : 0.f, bh[1], bl[1]);
        const float4* wa = reinterpret_cast<const float4*>(wxb + 8 * va);
        const float4* wb = reinterpret_cast<const float4*>(wxb + 8 * vb);
        const float4 wa0 = wa[0], wa1 = wa[1], wb0 = wb[0], wb1 = wb[1];
        const float pa[8] = {wa0.x, wa0.y, wa0.z, wa0.w, wa1.x, wa1.y, wa1.z, wa1.w};
        const float pb[8] = {wb0.x, wb0.y, wb0.z, wb0.w, wb1.x, wb1.y, wb1.z, wb1.w};
        uint32_t ah[MT][4], al[MT][4];
#pragma unroll
        for (int t = 0; t < MT; ++t) {
          tf32_split_fast(pa[2 * t] * xa, ah[t][0], al[t][0]);
          tf32_split_fast(pb[2 * t] * xb, ah[t][2], al[t][2]);
          if (2 * t + 1 < W) {
            tf32_split_fast(pa[2 * t + 1] * xa, ah[t][1], al[t][1]);
            tf32_split_fast(pb[2 * t + 1] * xb, ah[t][3], al[t][3]);
          } else {
            ah[t][1] = al[t][1] = ah[t][3] = al[t][3] = 0u;
          }
        }
        // Small terms first; consecutive products go to different tiles (independent).
#pragma unroll
        for (int t = 0; t < MT; ++t) mma_tf32(d[t], al[t], bh);
#pragma unroll
        for (int t = 0; t < MT; ++t) mma_tf32(d[t], ah[t], bl);
#pragma unroll
        for (int t = 0; t < MT; ++t) mma_tf32(d[t], ah[t], bh);
      }
      // d[t][i]: cell (jy = 2 tig + (i & 1), jx = 2 t + (i >> 1)), channel g.
      const int base = g * NP + ly * SS + lx;
#pragma unroll
      for (int t = 0; t < MT; ++t)
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const int jy = 2 * tig + (i & 1), jx = 2 * t + (i >> 1);
          if (jy < W && jx < W) atomicAdd(acc + base + jy * SS + jx, d[t][i]);
        }
    } else if constexpr (FORM == 2) {
      static_assert(FORM != 2 || 4 * W <= 32, "row-channel lanes need 4 W <= 32");
      const int jy = lane >> 2, cp = lane & 3;
      if (lane < 4 * W) {
        const u64* xp = reinterpret_cast<const u64*>(x4);   // row v, channel pair cp at 4 v + cp
        const float* wyr = wys + jy * kGridV;
        u64 acc2[W];
#pragma unroll
        for (int k = 0; k < W; ++k) acc2[k] = 0ull;
        for (int v = v0; v < v0 + cnt; ++v) {
          const u64 t = ffma2(fdup(wyr[v]), xp[4 * v + cp], 0ull);
#pragma unroll
          for (int k = 0; k < W; ++k) acc2[k] = ffma2(fdup(wxs[k * kGridV + v]), t, acc2[k]);
        }
        const int cell0 = (ly + jy) * SS + lx;
#pragma unroll
        for (int k = 0; k < W; ++k) {
          float lo, hi;
          f2unpack(acc2[k], lo, hi);
          atomicAdd(acc + (2 * cp) * NP + cell0 + k, lo);
          atomicAdd(acc + (2 * cp + 1) * NP + cell0 + k, hi);
        }
      }
    } else {
      // a2[q][p] holds channels (2p, 2p+1) of kernel cell q: packed FP32x2 accumulation.
      u64 a2[CPL][4];
#pragma unroll
      for (int q = 0; q < CPL; ++q)
#pragma unroll
        for (int p = 0; p < 4; ++p) a2[q][p] = 0ull;
      if (HALF) {
        for (int v = v0 + sub; v < v0 + cnt; v += 2) {
          const ulonglong2 x0 = xv[2 * v], x1 = xv[2 * v + 1];
#pragma unroll
          for (int q = 0; q < CPL; ++q) {
            const u64 k0 = fdup(wxs[wxo[q] + v] * wys[wyo[q] + v]);
            a2[q][0] = ffma2(k0, x0.x, a2[q][0]);
            a2[q][1] = ffma2(k0, x0.y, a2[q][1]);
            a2[q][2] = ffma2(k0, x1.x, a2[q][2]);
            a2[q][3] = ffma2(k0, x1.y, a2[q][3]);
          }
        }
#pragma unroll
        for (int q = 0; q < CPL; ++q)
#pragma unroll
          for (int p = 0; p < 4; ++p) {
            float lo, hi;
            f2unpack(a2[q][p], lo, hi);
            lo += __shfl_xor_sync(0xffffffffu, lo, 16);
            hi += __shfl_xor_sync(0xffffffffu, hi, 16);
            a2[q][p] = f2pack(lo, hi);
          }
      } else {
        int v = v0;
        for (; v + 1 < v0 + cnt; v += 2) {
          const ulonglong2 x0 = xv[2 * v], x1 = xv[2 * v + 1], y0 = xv[2 * v + 2], y1 = xv[2 * v + 3];
#pragma unroll
          for (int q = 0; q < CPL; ++q) {
            const u64 k0 = fdup(wxs[wxo[q] + v] * wys[wyo[q] + v]);
            const u64 k1 = fdup(wxs[wxo[q] + v + 1] * wys[wyo[q] + v + 1]);
            a2[q][0] = ffma2(k1, y0.x, ffma2(k0, x0.x, a2[q][0]));
            a2[q][1] = ffma2(k1, y0.y, ffma2(k0, x0.y, a2[q][1]));
            a2[q][2] = ffma2(k1, y1.x, ffma2(k0, x1.x, a2[q][2]));
            a2[q][3] = ffma2(k1, y1.y, ffma2(k0, x1.y, a2[q][3]));
          }
        }
        if (v < v0 + cnt) {
          const ulonglong2 x0 = xv[2 * v], x1 = xv[2 * v + 1];
#pragma unroll
          for (int q = 0; q < CPL; ++q) {
            const u64 k0 = fdup(wxs[wxo[q] + v] * wys[wyo[q] + v]);
            a2[q][0] = ffma2(k0, x0.x, a2[q][0]);
            a2[q][1] = ffma2(k0, x0.y, a2[q][1]);
            a2[q][2] = ffma2(k0, x1.x, a2[q][2]);
            a2[q][3] = ffma2(k0, x1.y, a2[q][3]);
          }
        }
      }
      const int cbase = ly * SS + lx;
#pragma unroll
      for (int q = 0; q < CPL; ++q) {
        if (sub == 0 && sl + LPR * q < W * W) {
#pragma unroll
          for (int p = 0; p < 4; ++p) {
            float lo, hi;
            f2unpack(a2[q][p], lo, hi);
            atomicAdd(acc + (2 * p) * NP + cbase + coff[q], lo);
            atomicAdd(acc + (2 * p + 1) * NP + cbase + coff[q], hi);
          }
        }
      }
    }
  }
}

// Step 3: the tile with its halo added to the global accumulator.
template <int W>
__device__ __forceinline__ void grid_flush(const float* __restrict__ acc, int ty, int tx, int Wd, int full, int K,
                                           float4* __restrict__ Acc) {
  constexpr int TS = kGridTileG;
  constexpr int SS = TS + W - 1;
  constexpr int NC = SS * SS;
  constexpr int NP = grid_plane<W>();
  constexpr int hw = W / 2;
  for (int c = threadIdx.x; c < NC; c += blockDim.x) {
    const int ly = c / SS, lx = c - (c / SS) * SS;
    int gy = ty * TS - hw + ly, gx = tx * TS - hw + lx;
    if (full) {
      gy &= (K - 1);
      gx &= (K - 1);
    } else if (gy < 0 || gy >= Wd || gx < 0 || gx >= Wd) {
      continue;
    }
    const float4 lo = make_float4(acc[0 * NP + c], acc[1 * NP + c], acc[2 * NP + c], acc[3 * NP + c]);
    const float4 hi = make_float4(acc[4 * NP + c], acc[5 * NP + c], acc[6 * NP + c], acc[7 * NP + c]);
    float4* dst = Acc + 2 * ((size_t)gy * Wd + gx);
    if (lo.x != 0.f || lo.y != 0.f || lo.z != 0.f || lo.w != 0.f) atomicAdd(dst, lo);
    if (hi.x != 0.f || hi.y != 0.f || hi.z != 0.f || hi.w != 0.f) atomicAdd(dst + 1, hi);
  }
}

constexpr int kGridThreads = 256;   // threads of a gridding CTA

template <int W, int FORM>
__global__ void __launch_bounds__(kGridThreads) k_grid(
    const GridItem* __restrict__ items, const int32_t* __restrict__ chunks, const uint16_t* __restrict__ vblk,
    const float4* __restrict__ rec, const float2* __restrict__ vin, const float* __restrict__ cb, int use_scale,
    int Wd, int full, int K, float beta, const float* __restrict__ wrow, int M, float4* __restrict__ Acc,
    int* __restrict__ err) {
  constexpr int NP = grid_plane<W>();
  __shared__ uint64_t wbar;                      // FORM 3: completion of the weight copies
  extern __shared__ float4 smg[];
  float4* x4 = smg;                              // kGridItemG x 2: mixed, scaled channels of each row
  float* wts = reinterpret_cast<float*>(smg + 2 * kGridItemG);  // weights (layout by FORM)
  float* acc = wts + grid_wts_floats<W, FORM>(); // 8 planes of NP floats
  const GridItem it = items[blockIdx.x];
  for (int i = threadIdx.x; i < 8 * NP; i += blockDim.x) acc[i] = 0.f;
  const int nv = it.vend - it.vstart;
  if (FORM == 3 && threadIdx.x == 0) {
    mbar_init(&wbar, 1);
    mbar_expect_tx(&wbar, (uint32_t)nv * 64u);
    bulk_g2s(wts, wrow + 8 * (size_t)it.vstart, (uint32_t)nv * 32u, &wbar);
    bulk_g2s(wts + 8 * kGridRows3, wrow + 8 * ((size_t)M + it.vstart), (uint32_t)nv * 32u, &wbar);
  }
  const float4* v4 = reinterpret_cast<const float4*>(vin);
  // Every global load of this thread's rows is issued before the first is used.
  constexpr int RPT = (kGridItemG + kGridThreads - 1) / kGridThreads;   // rows per thread
  float4 r[RPT], b0[RPT], b1[RPT];
  int blk[RPT];
#pragma unroll
  for (int q = 0; q < RPT; ++q) {
    const int j = threadIdx.x + q * kGridThreads;
    const size_t idx = (size_t)it.vstart + (j < nv ? j : 0);
    r[q] = rec[idx];
    b0[q] = v4[2 * idx];
    b1[q] = v4[2 * idx + 1];
    blk[q] = use_scale ? vblk[idx] : 0;
  }
#pragma unroll
  for (int q = 0; q < RPT; ++q) {
    const int j = threadIdx.x + q * kGridThreads;
    if (j < nv) grid_stage_row<W, FORM>(j, r[q], b0[q], b1[q], use_scale ? cb[blk[q]] : 1.0f, beta, x4, wts);
  }
  if (FORM >= 3 && threadIdx.x < 8) {
    // Spare rows after the item: finite (zero) operands for the last k-step of its last chunk.
    const int j = nv + threadIdx.x;
    const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
    if (j < kGridItemG) x4[2 * j] = x4[2 * j + 1] = z;
    float4* yb = reinterpret_cast<float4*>(wts) + 2 * j;
    float4* xb = reinterpret_cast<float4*>(wts + 8 * kGridRows3) + 2 * j;
    yb[0] = yb[1] = xb[0] = xb[1] = z;
  }
  __syncthreads();
  if (FORM == 3) {
    const bool ok = mbar_wait(&wbar, 0);
    if (__syncthreads_or(!ok)) {
      if (threadIdx.x == 0) {
        atomicExch(err, 1);
        (void)mbar_drain(&wbar, 0);
      }
      return;
    }
  }
  grid_chunks<W, FORM>(chunks + it.cstart, it.cend - it.cstart, x4, wts, acc);
  __syncthreads();
  grid_flush<W>(acc, it.ty, it.tx, Wd, full, K, Acc);
}

template <int W, int FORM>
static constexpr size_t grid_smem() {
  return (size_t)2 * kGridItemG * sizeof(float4) +
         (size_t)(grid_wts_floats<W, FORM>() + 8 * grid_plane<W>()) * sizeof(float);
}

// Hermitian symmetrisation + inverse column FFTs for the column pair (kx, -kx).
// H1(k) = P1(k) + i Q1(k), P1(k) = aI(k) + conj aI(-k), Q1(k) = aQ(k) + conj aQ(-k);
// H2 likewise from aU, aV. H(-k) = conj P(k) + i conj Q(k).
__global__ void k_adj_cols(const float4* __restrict__ Acc, int n, const float2* __restrict__ tw, int K,
                           int logK, float4* __restrict__ T2, int Wd, int off, int full) {
  extern __shared__ float4 sm[];
  float4* bp = sm;
  float4* bm = sm + K;
  const int kx = blockIdx.x;
  const int self = (kx == 0) || (full && kx == K / 2);
  const int gxp = gidx(kx, off, full, K), gxm = gidx(-kx, off, full, K);
  // H(ky) of this column pair: hp for +kx (slot ky of bp), hm for -kx (slot -ky of bm).
  auto hpm = [&](int ky, float4& hp, float4& hm) {
    const int gy = gidx(ky, off, full, K), gym = gidx(-ky, off, full, K);
    const float4 a0 = Acc[2 * ((size_t)gy * Wd + gxp)], a1 = Acc[2 * ((size_t)gy * Wd + gxp) + 1];
    const float4 b0 = Acc[2 * ((size_t)gym * Wd + gxm)], b1 = Acc[2 * ((size_t)gym * Wd + gxm) + 1];
    const float P1r = a0.x + b0.x, P1i = a0.y - b0.y, Q1r = a0.z + b0.z, Q1i = a0.w - b0.w;
    const float P2r = a1.x + b1.x, P2i = a1.y - b1.y, Q2r = a1.z + b1.z, Q2i = a1.w - b1.w;
    hp = make_float4(P1r - Q1i, P1i + Q1r, P2r - Q2i, P2i + Q2r);
    hm = make_float4(P1r + Q1i, -P1i + Q1r, P2r + Q2i, -P2i + Q2r);
  };
  int st;
  if (!full && 8 * off < K) {
    // As in k_adj_rows: the window [-R, R] with R < K/8 puts at most one sample in each
    // block of natural indices x + j K/4, so the first two inverse stages are written
    // directly (v (i^{j t})_t, j = 0 or 3) and fft_smem starts at stage 2.
    const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
    auto put4 = [&](float4* b, int r0, int j, float4 v) {
      if (j == 0) {
        b[fsw(r0)] = b[fsw(r0 + 1)] = b[fsw(r0 + 2)] = b[fsw(r0 + 3)] = v;
      } else if (j == 3) {
        b[fsw(r0)] = v;
        b[fsw(r0 + 1)] = make_float4(v.y, -v.x, v.w, -v.z);
        b[fsw(r0 + 2)] = make_float4(-v.x, -v.y, -v.z, -v.w);
        b[fsw(r0 + 3)] = make_float4(-v.y, v.x, -v.w, v.z);
      } else {
        b[fsw(r0)] = b[fsw(r0 + 1)] = b[fsw(r0 + 2)] = b[fsw(r0 + 3)] = z;
      }
    };
    for (int x = threadIdx.x; x < (K >> 2); x += blockDim.x) {
      const int r0 = bitrev(x, logK);
      const int j = x <= off ? 0 : (x >= (K >> 2) - off ? 3 : -1);
      const int k = j == 0 ? x : x - (K >> 2);    // the block's sample index (when j >= 0)
      float4 hp = z, hm = z, unused;
      if (j >= 0) {
        hpm(k, hp, unused);                       // bp[k] = hp(k)
        if (!self) hpm(-k, unused, hm);           // bm[k] = hm(-k)
      }
      put4(bp, r0, j, hp);
      if (!self) put4(bm, r0, j, hm);
    }
    __syncthreads();
    st = fft_tail_start(logK, 2);
    fft_smem<true>(bp, tw, logK, 2, st);
    if (!self) fft_smem<true>(bm, tw, logK, 2, st);
  } else {
    for (int i = threadIdx.x; i < 2 * K; i += blockDim.x) sm[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    __syncthreads();
    for (int gy = threadIdx.x; gy < Wd; gy += blockDim.x) {
      const int ky = full ? (gy <= K / 2 ? gy : gy - K) : gy - off;
      const int gym = gidx(-ky, off, full, K);
      const float4 a0 = Acc[2 * ((size_t)gy * Wd + gxp)], a1 = Acc[2 * ((size_t)gy * Wd + gxp) + 1];
      const float4 b0 = Acc[2 * ((size_t)gym * Wd + gxm)], b1 = Acc[2 * ((size_t)gym * Wd + gxm) + 1];
      const float P1r = a0.x + b0.x, P1i = a0.y - b0.y, Q1r = a0.z + b0.z, Q1i = a0.w - b0.w;
      const float P2r = a1.x + b1.x, P2i = a1.y - b1.y, Q2r = a1.z + b1.z, Q2i = a1.w - b1.w;
      const float4 hp = make_float4(P1r - Q1i, P1i + Q1r, P2r - Q2i, P2i + Q2r);
      bp[fsw(bitrev((ky + K) & (K - 1), logK))] = hp;
      if (!self) {
        const float4 hm = make_float4(P1r + Q1i, -P1i + Q1r, P2r + Q2i, -P2i + Q2r);
        bm[fsw(bitrev((-ky + K) & (K - 1), logK))] = hm;
      }
    }
    __syncthreads();
    st = fft_tail_start(logK, 0);
    fft_smem<true>(bp, tw, logK, 0, st);
    if (!self) fft_smem<true>(bm, tw, logK, 0, st);
  }
  for (int p = threadIdx.x; p < n; p += blockDim.x) {
    const int k = (p - n / 2 + K) & (K - 1);
    T2[(size_t)p * Wd + gxp] = fft_out<true>(bp, tw, logK, st, k);
    if (!self) T2[(size_t)p * Wd + gxm] = fft_out<true>(bm, tw, logK, st, k);
  }
}

__global__ void k_adj_rows(const float4* __restrict__ T2, int n, int N, const float* __restrict__ corr,
                           const float2* __restrict__ tw, int K, int logK, int Wd, int off, int full,
                           float* __restrict__ out) {
  extern __shared__ float4 sm[];
  float4* buf = sm;
  const int p = blockIdx.x;
  int st;
  if (!full && 8 * off < K) {
    // Window [-R, R] with R < K/8: of the natural indices x + j K/4 (j = 0..3) at most
    // one holds a sample (j = 0: k = x <= R; j = 3: k = x - K/4 >= -R), so the first two
    // radix-2 stages reduce to the 4-point inverse DFT of one sample, v (i^{j t})_t,
    // written straight to the four slots 4B + t of its block (x = bitrev(4B)); blocks
    // without a sample get zeros, and fft_smem starts at stage 2.
    const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int x = threadIdx.x; x < (K >> 2); x += blockDim.x) {
      const int r0 = bitrev(x, logK);
      float4 v0 = z, v1 = z, v2 = z, v3 = z;
      if (x <= off) {
        v0 = v1 = v2 = v3 = T2[(size_t)p * Wd + x + off];
      } else if (x >= (K >> 2) - off) {
        const float4 v = T2[(size_t)p * Wd + x - (K >> 2) + off];
        v0 = v;
        v1 = make_float4(v.y, -v.x, v.w, -v.z);    // -i v
        v2 = make_float4(-v.x, -v.y, -v.z, -v.w);  // -v
        v3 = make_float4(-v.y, v.x, -v.w, v.z);    // +i v
      }
      buf[fsw(r0)] = v0;
      buf[fsw(r0 + 1)] = v1;
      buf[fsw(r0 + 2)] = v2;
      buf[fsw(r0 + 3)] = v3;
    }
    __syncthreads();
    st = fft_tail_start(logK, 2);
    fft_smem<true>(buf, tw, logK, 2, st);
  } else {
    for (int i = threadIdx.x; i < K; i += blockDim.x) buf[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    __syncthreads();
    for (int gx = threadIdx.x; gx < Wd; gx += blockDim.x) {
      const int k = full ? gx : gx - off;
      buf[fsw(bitrev((k + K) & (K - 1), logK))] = T2[(size_t)p * Wd + gx];
    }
    __syncthreads();
    st = fft_tail_start(logK, 0);
    fft_smem<true>(buf, tw, logK, 0, st);
  }
  const float cy = 0.5f * corr[p];
  for (int q = threadIdx.x; q < n; q += blockDim.x) {
    const float4 v = fft_out<true>(buf, tw, logK, st, (q - n / 2 + K) & (K - 1));
    const float c = cy * corr[q];
    const size_t o = (size_t)p * n + q;
    out[o] = v.x * c;
    out[(size_t)N + o] = v.y * c;
    out[2 * (size_t)N + o] = v.z * c;
    out[3 * (size_t)N + o] = v.w * c;
  }
}

static size_t fft_smem_bytes(int K, int nbuf) { return (size_t)nbuf * K * sizeof(float4); }

static cudaError_t set_smem(const void* fn, size_t bytes) {
  return cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

cudaError_t configure_nufft_kernels() {
  // Largest grid: n = 2048, K = 4096.
  const size_t sm1 = fft_smem_bytes(4096, 1), sm2 = fft_smem_bytes(4096, 2);
  cudaError_t e;
  if ((e = set_smem((const void*)k_fwd_rows, sm1)) != cudaSuccess) return e;
  if ((e = set_smem((const void*)k_fwd_cols, sm1)) != cudaSuccess) return e;
  if ((e = set_smem((const void*)k_adj_rows, sm1)) != cudaSuccess) return e;
  const void* grids[] = {(const void*)k_grid<5, 0>, (const void*)k_grid<7, 0>, (const void*)k_grid<9, 0>,
                         (const void*)k_grid<5, 1>, (const void*)k_grid<7, 1>, (const void*)k_grid<9, 1>,
                         (const void*)k_grid<5, 2>, (const void*)k_grid<7, 2>, (const void*)k_grid<5, 3>,
                         (const void*)k_grid<7, 3>, (const void*)k_grid<5, 4>, (const void*)k_grid<7, 4>};
  const size_t grid_bytes[] = {grid_smem<5, 0>(), grid_smem<7, 0>(), grid_smem<9, 0>(), grid_smem<5, 1>(),
                               grid_smem<7, 1>(), grid_smem<9, 1>(), grid_smem<5, 2>(), grid_smem<7, 2>(),
                               grid_smem<5, 3>(), grid_smem<7, 3>(), grid_smem<5, 4>(), grid_smem<7, 4>()};
  for (int i = 0; i < 12; ++i)
    if ((e = set_smem(grids[i], grid_bytes[i])) != cudaSuccess) return e;
  // Per-block FP64 accumulators of the degridding kernels (up to 2047 blocks).
  const void* degrids[] = {(const void*)k_degrid<5, 0>, (const void*)k_degrid<7, 0>, (const void*)k_degrid<9, 0>,
                           (const void*)k_degrid<5, 1>, (const void*)k_degrid<7, 1>, (const void*)k_degrid<9, 1>,
                           (const void*)k_degrid<5, 2>, (const void*)k_degrid<7, 2>, (const void*)k_degrid<9, 2>};
  const size_t degrid_smem[] = {degrid_smem_tiles<5>(), degrid_smem_tiles<7>(), degrid_smem_tiles<9>()};
  for (int i = 0; i < 9; ++i)
    if ((e = set_smem(degrids[i], degrid_smem[i % 3] + 2048 * sizeof(double))) != cudaSuccess) return e;
  return set_smem((const void*)k_adj_cols, sm2);
}

cudaError_t nufft_forward_grid(Handle* h, const float* X) {
  const GridGeom& g = h->g;
  const size_t sm1 = fft_smem_bytes(g.K, 1);
  k_fwd_rows<<<h->n, 256, sm1, h->stream>>>(X, h->n, h->N, h->corr, h->tw, g.K, g.logK, h->T1, g.Wd, g.off, g.full);
  k_fwd_cols<<<g.Wd, 512, sm1, h->stream>>>(h->T1, h->n, h->tw, g.K, g.logK, h->G, g.Wd, g.off, g.full);
  return cudaGetLastError();
}

template <int W>
static void launch_degrid(Handle* h, int mode, float2* out) {
  const GridGeom& g = h->g;
  const int nbins = h->nblocks <= kWarpBins ? kWarpBins * 8 : h->nblocks;   // 8 warps of 256 threads
  const size_t sm = degrid_smem_tiles<W>() + (size_t)nbins * sizeof(double);
  const int form = h->tune[PS_TUNE_DEGRID];
  auto kern = form == 1 ? k_degrid<W, 1> : (form == 2 ? k_degrid<W, 2> : k_degrid<W, 0>);
  kern<<<h->nitems, 256, sm, h->stream>>>(h->items, h->gchunks, h->rec, h->G, g.Wd, g.off, g.full, g.K, g.beta, mode,
                                          h->R, h->Y, h->cb, (float)(1.0 / h->rho2), h->vblk, h->nblocks,
                                          h->block_sum, out);
}

cudaError_t nufft_degrid(Handle* h, int mode, float2* out) {
  if (h->M == 0) return cudaSuccess;
  if (mode != DEG_APPLY) {
    cudaError_t e = cudaMemsetAsync(h->block_sum, 0, (size_t)h->nblocks * sizeof(double), h->stream);
    if (e != cudaSuccess) return e;
  }
  switch (h->g.W) {
    case 5: launch_degrid<5>(h, mode, out); break;
    case 9: launch_degrid<9>(h, mode, out); break;
    default: launch_degrid<7>(h, mode, out); break;
  }
  return cudaGetLastError();
}

cudaError_t block_scales(Handle* h) {
  if (h->nblocks == 0) return cudaSuccess;
  k_block_scale<<<(h->nblocks + 127) / 128, 128, 0, h->stream>>>(h->block_sum, h->eps, h->nblocks, h->rho2,
                                                                 h->cfg.literal_ball, h->cb);
  return cudaGetLastError();
}

// Kernel weights of every stored row, computed once per set of measurements (the rows'
// fractional offsets do not change): y-taps in the first M x 8 floats, x-taps after.
template <int W>
__global__ void k_row_weights(const float4* __restrict__ rec, int M, float beta, float* __restrict__ wrow) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= M) return;
  float fx, fy, w;
  int cx, cy;
  unpack_rec(rec[m], fx, fy, w, cx, cy);
  float wx[W], wy[W], t[8];
  es_weights<W>(fx, beta, wx);
  es_weights<W>(fy, beta, wy);
  float4* py = reinterpret_cast<float4*>(wrow) + 2 * (size_t)m;
  float4* px = reinterpret_cast<float4*>(wrow + 8 * (size_t)M) + 2 * (size_t)m;
#pragma unroll
  for (int k = 0; k < 8; ++k) t[k] = k < W ? wy[k] : 0.f;
  py[0] = make_float4(t[0], t[1], t[2], t[3]);
  py[1] = make_float4(t[4], t[5], t[6], t[7]);
#pragma unroll
  for (int k = 0; k < 8; ++k) t[k] = k < W ? wx[k] : 0.f;
  px[0] = make_float4(t[0], t[1], t[2], t[3]);
  px[1] = make_float4(t[4], t[5], t[6], t[7]);
}

cudaError_t nufft_row_weights(Handle* h) {
  if (!h->wrow || h->M == 0) return cudaSuccess;
  const int blocks = (h->M + 255) / 256;
  if (h->g.W == 5)
    k_row_weights<5><<<blocks, 256, 0, h->stream>>>(h->rec, h->M, h->g.beta, h->wrow);
  else
    k_row_weights<7><<<blocks, 256, 0, h->stream>>>(h->rec, h->M, h->g.beta, h->wrow);
  return cudaGetLastError();
}

template <int W, int FORM>
static void launch_grid_form(Handle* h, const float2* in, int use_scale) {
  const GridGeom& g = h->g;
  k_grid<W, FORM><<<h->nitems_g, kGridThreads, grid_smem<W, FORM>(), h->stream>>>(
      h->items_g, h->gchunks_g, h->vblk, h->rec, in, h->cb, use_scale, g.Wd, g.full, g.K, g.beta, h->wrow, h->M, h->Acc,
      h->dev_flags);
}

template <int W>
static void launch_grid(Handle* h, const float2* in, int use_scale) {
  // FORM 2 needs 4 W <= 32 lanes and FORMs 3-4 8 taps per row: W = 9 runs FORM 0 for them.
  constexpr bool narrow = W <= 8;
  switch (h->tune[PS_TUNE_GRID]) {
    case 1: launch_grid_form<W, 1>(h, in, use_scale); break;
    case 2: launch_grid_form<W, narrow ? 2 : 0>(h, in, use_scale); break;
    case 3: launch_grid_form<W, narrow ? 3 : 0>(h, in, use_scale); break;
    case 4: launch_grid_form<W, narrow ? 4 : 0>(h, in, use_scale); break;
    default: launch_grid_form<W, 0>(h, in, use_scale); break;
  }
}

cudaError_t nufft_grid(Handle* h, const float2* in, int use_scale) {
  const GridGeom& g = h->g;
  cudaError_t e = cudaMemsetAsync(h->Acc, 0, (size_t)g.Wd * g.Wd * 2 * sizeof(float4), h->stream);
  if (e != cudaSuccess || h->nitems_g == 0) return e;
  switch (g.W) {
    case 5: launch_grid<5>(h, in, use_scale); break;
    case 9: launch_grid<9>(h, in, use_scale); break;
    default: launch_grid<7>(h, in, use_scale); break;
  }
  return cudaGetLastError();
}

cudaError_t nufft_adjoint_image(Handle* h, float* out) {
  const GridGeom& g = h->g;
  const size_t sm2 = fft_smem_bytes(g.K, 2), sm1 = fft_smem_bytes(g.K, 1);
  const int ncols = g.full ? (g.K / 2 + 1) : (g.R + 1);
  k_adj_cols<<<ncols, 512, sm2, h->stream>>>(h->Acc, h->n, h->tw, g.K, g.logK, h->T2, g.Wd, g.off, g.full);
  k_adj_rows<<<h->n, 256, sm1, h->stream>>>(h->T2, h->n, h->N, h->corr, h->tw, g.K, g.logK, g.Wd, g.off, g.full, out);
  return cudaGetLastError();
}

}  // namespace ps

// Internal declarations of the Polarized SARA CUDA library (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "polsara.h"

namespace ps {

constexpr int kBases = 9;        // Dirac + db1..db8
constexpr int kDb = 8;           // Daubechies bases
constexpr int kMaxTaps = 16;     // db8 filter length
constexpr int kGridTile = 16;    // degridding tile side (cells)
constexpr int kGridTileG = 8;    // gridding tile side (cells): a quarter of a degridding tile
static_assert(kGridTile % kGridTileG == 0, "gridding tiles subdivide degridding tiles");
constexpr int kChunk = 1024;     // visibilities per reduction chunk
constexpr int kGridItem = 768;   // visibilities per degridding work item
constexpr int kGridItemG = 384;  // visibilities per gridding work item (smaller: 4 CTAs per SM)
static_assert(kGridItem <= 1024 && kGridItemG <= 1024, "a chunk's start is a 10-bit offset in its item");
constexpr int kBinChunk = 32;    // visibilities per same-cell accumulation chunk
constexpr int kWarpBins = 64;    // l2 blocks up to which degridding keeps per-warp FP64 block sums
constexpr int kGraphIters = 8;   // iterations per launch of the multi-iteration graph

// Analysis / synthesis kernel modes.
enum { SARA_DUAL = 0, SARA_APPLY = 1, SARA_REWEIGHT = 2 };
// Degridding modes.
enum { DEG_DUAL = 0, DEG_APPLY = 1, DEG_RESID = 2 };

struct GridItem {      // one gridding CTA: gridding-order rows [vstart, vend), centres in tile (ty, tx),
  int32_t ty, tx;      // same-cell chunks [cstart, cend)
  int32_t vstart, vend, cstart, cend;
  int32_t pad0, pad1;
};

// Geometry of the NUFFT grid: the K x K oversampled spectrum is kept only on a
// window of frequencies [-R, R]^2 covering every interpolation tap (window
// mode), or whole (full mode, indices modulo K).
struct GridGeom {
  int K = 0, logK = 0;   // oversampled FFT length (2n)
  int W = 7;             // interpolation kernel width
  int R = 0;             // window half-width (cells)
  int Wd = 0;            // stored grid side: 2R+1 (window) or K (full)
  int full = 0;          // 1: full grid, indices wrap modulo K
  int off = 0;           // grid index of frequency k: (k + off) [& (K-1) if full]
  int tilesX = 0;        // gridding tiles per side
  float beta = 0.f;      // ES kernel shape
};

struct Handle {
  ps_config cfg{};
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  cudaStream_t aux = nullptr;       // second stream: SARA chain runs beside the NUFFT chain in graphs
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  std::string err;
  int n = 0, N = 0, L = 0, mode = PS_POLARIZED;
  double tau = 0, rho1 = 1, rho2 = 1, rho3 = 1, opnorm_sq = 0, gamma = 1;
  double gamma_default = 0;       // cfg.gamma, else 1e-3 max|Psi^dagger phi^dagger Y| / ||phi||^2
  double tv_mu[4] = {0, 0, 0, 0}, l1_mu[4] = {0, 0, 0, 0};   // TV and l1 weights (Algorithm 3)
  bool have_meas = false;
  bool derived_valid = false;     // PsiA and Adj hold Psi A and phi^dagger B of the current state
  int64_t iterations = 0;
  int64_t bytes = 0;

  // Image-domain state (float32 planes).
  float *S = nullptr, *Z = nullptr, *C = nullptr, *D = nullptr;
  float *Xb = nullptr;        // 2 S^(k+1) - S^(k)
  float *PsiA = nullptr;      // Psi A
  float *Adj = nullptr;       // phi^dagger B
  float *tmp4 = nullptr;      // 4N scratch for operators
  float *A = nullptr, *T = nullptr;   // 36N coefficients and thresholds gamma W
  float *approx = nullptr;    // ping-pong buffers of 32 * (N/4) approximations: approx and approx2
  float *approx2 = nullptr;
  int nmaps = 4;              // maps the SARA and primal launches cover (4 P for a batch's size class)
  int problems = 1;           // problems of a batched primal launch (the per-problem arrays are consecutive)
  bool in_slab = false;       // state arrays are slices of a batch's class slabs (not freed by ps_destroy)
  double *red = nullptr;      // reduction partials
  int red_cap = 0;
  double *red_host = nullptr; // pinned
  double *relc_host = nullptr; // pinned, mapped: relative-change sums (8) and the device flags of the last request
  double *relc_dev = nullptr;  // the device's address of relc_host
  cudaEvent_t relc_ev = nullptr;
  bool relc_pending = false;
  int *dev_flags = nullptr;   // device error flags: [0] a bounded wait gave up

  // Visibility-domain state, rows stored in tap-centre-cell order (tile-major).
  int M = 0, nblocks = 0;
  float2 *R = nullptr;        // residual form of B: B = c_b R  (M x 4)
  float2 *Y = nullptr;        // measurements (M x 4)
  float4 *rec = nullptr;      // (fx, fy, w, packed (cx, cy))
  int32_t *perm = nullptr;    // sorted row -> caller row
  float2 *vtmp = nullptr;     // M x 4 scratch
  double *eps = nullptr;      // per block radius (device)
  float *cb = nullptr;        // per block scale c_b (device)
  double *block_sum = nullptr;     // nblocks FP64 sums filled by the degridding kernel
  int nitems = 0, ngchunks = 0;
  GridItem *items = nullptr;       // degridding work items (<= kGridItem rows)
  int32_t *gchunks = nullptr;      // packed (start, count, ly, lx) of their same-cell chunks
  int nitems_g = 0, ngchunks_g = 0;
  GridItem *items_g = nullptr;     // gridding work items (<= kGridItemG rows) and their chunks
  int32_t *gchunks_g = nullptr;
  uint16_t *vblk = nullptr;        // l2 block of each stored row
  float *wrow = nullptr;           // W <= 8: kernel weights of each stored row, 8 y-taps (M x 8)
                                   // then 8 x-taps (M x 8), zero past W
  std::vector<double> eps_host;
  double psf_peak = 0.0;      // 2 sum w_m^2: peak of the Stokes-I PSF
  float *tmp36 = nullptr;     // 36N scratch for operator calls (allocated on first use)
  std::vector<int64_t> offsets_host;

  // NUFFT buffers.
  GridGeom g;
  float4 *T1 = nullptr;       // n x Wd row spectra (forward)
  float4 *G = nullptr;        // Wd x Wd packed spectra (I+iQ, U+iV)
  float4 *Acc = nullptr;      // Wd x Wd x 2 gridding accumulators (xI, xQ | xU, xV)
  float4 *T2 = nullptr;       // n x Wd column-transformed adjoint
  float2 *tw = nullptr;       // K per-stage twiddles: stage t at [2^t - 1, 2^(t+1) - 1)
  float *corr = nullptr;      // n de-apodisation factors 1 / phihat(2 pi x / K)

  // Launch choices (PS_TUNE_* slots) and the device's SM count (persistent grids).
  int32_t tune[PS_TUNE_COUNT] = {};
  int num_sms = 0;

  // CUDA graph of one iteration.
  cudaGraphExec_t graph = nullptr;
  cudaGraphExec_t graph_multi = nullptr;   // kGraphIters iterations back to back (same mode as graph)
  int graph_mode = -1;
  uint64_t version = 1;       // bumped when mode, state or measurements change (batch graphs rebuild)
};

// Bounded-wait poll budget of each translation unit with bulk-copy waits (polls < 0: default).
cudaError_t set_wait_polls_sara(int polls);
cudaError_t set_wait_polls_nufft(int polls);

// Message returned by ps_last_error(NULL) (calls without a handle).
void set_global_error(const std::string& msg);

// Host-side constants.
void daubechies_filters(double h[kDb][kMaxTaps]);          // db1..db8 scaling filters
double es_beta(int W);
double es_kernel(double t, int W, double beta);            // ES kernel value at offset t (cells)
double es_fourier(double xi, int W, double beta);          // its Fourier transform at xi

// Kernel launchers (return cudaGetLastError()).
cudaError_t upload_filters(const double h[kDb][kMaxTaps], cudaStream_t stream);

// NUFFT pieces (nufft.cu).
cudaError_t nufft_forward_grid(Handle* h, const float* X);                 // X (4 planes) -> G
cudaError_t nufft_degrid(Handle* h, int mode, float2* out);                // G -> visibilities
cudaError_t nufft_grid(Handle* h, const float2* in, int use_block_scale);  // visibilities -> Acc
cudaError_t nufft_row_weights(Handle* h);                                   // rec -> wrow (W <= 8)
cudaError_t tv_dual(Handle* h);      // Algorithm 3 steps 5-6 on Xb -> A (TV layout)
cudaError_t tv_adjoint(Handle* h);   // Psi A = grad^T A_tv (+ A_l1) -> PsiA
__host__ __device__ inline bool tv_mode(int m) { return m >= PS_TV && m <= PS_L1TV_NC; }
__host__ __device__ inline bool constrained_mode(int m) { return m == PS_POLARIZED || m == PS_SOC || m == PS_TV || m == PS_L1TV; }
cudaError_t nufft_adjoint_image(Handle* h, float* out);                    // Acc -> 4 planes
cudaError_t block_scales(Handle* h);                                        // chunk partials -> c_b

// SARA pieces (sara.cu).
// `fine_done` (may be null) is recorded on h->stream after the level-1 analysis launch;
// `fine_start` (may be null) before the finest synthesis level (stage profiling).
cudaError_t sara_analysis(Handle* h, const float* X, float* coef, float* thr, int mode,
                          float scale, float gamma, float delta, cudaEvent_t fine_done = nullptr);
cudaError_t sara_synthesis(Handle* h, const float* coef, float* out, cudaEvent_t fine_start = nullptr);

// Elementwise / reductions (prox.cu).
cudaError_t primal_sweep(Handle* h);
cudaError_t dirac_apply(Handle* h, const float* X, float* coef, float* thr, int mode,
                        float scale, float gamma, float delta);
cudaError_t reduce_dot(Handle* h, const float* a, const float* b, size_t len, double* dev_out);
cudaError_t relc_sums(Handle* h, int nb, double* out);   // 8 column sums of k_primal's partials + the flags
cudaError_t violation_count(Handle* h, const float* S, double zeta, double* dev_out);
cudaError_t weighted_l1(Handle* h, const float* coef, const float* thr, double* dev_out);
cudaError_t max_abs(Handle* h, const float* c, size_t len, double* dev_out);
cudaError_t scale_copy(Handle* h, const float* x, float* y, size_t len, double s);
cudaError_t lanczos_update(Handle* h, float* w, const float* v, const float* u, size_t len, double alpha,
                           double beta);                                    // w -= alpha v + beta u
cudaError_t gather_vis(Handle* h, const float2* user, float2* sorted);
cudaError_t scatter_vis(Handle* h, const float2* sorted, float2* user);
cudaError_t scale_vis(Handle* h, float2* v);   // v = c_b v per block (state readout)

}  // namespace ps

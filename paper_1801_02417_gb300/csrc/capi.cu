// C ABI of the Polarized SARA imager (declared in include/polsara.h).
//
// One handle = one imaging problem resident on the device. ps_pd_iterate replays
// a CUDA graph of one iteration of Algorithm 1:
//   k_primal                    steps 3, 4, 9-12 and the Dirac part of 5-6
//   k_analysis x levels         steps 5-6 (Psi^dagger of 2S'-S, soft-threshold dual)
//   k_synthesis x levels        Psi A^(k+1) for the next step 3
//   k_fwd_rows, k_fwd_cols      F Z of phi(2S'-S)                  (step 7)
//   k_degrid                    G, mixing by L, B~ and ||B~/rho2 - Y||^2 partials
//   k_block_scale               step 8 (l2-ball factor per block)
//   k_grid, k_adj_cols, k_adj_rows   phi^dagger B^(k+1) for the next step 3
// B is kept as R = B~/rho2 - Y with a per-block factor: B = c_b R, c_b =
// rho2 (1 - min(1, eps_b / ||R_b||)), which is the step-8 result written out.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <numeric>
#include <string>
#include <thread>
#include <vector>

#include "internal.h"

using ps::Handle;

struct ps_handle : public Handle {};

namespace ps {
cudaError_t configure_kernels();
}

static std::string g_create_error;

namespace ps {
void set_global_error(const std::string& msg) { g_create_error = msg; }
}  // namespace ps

static ps_status fail(Handle* h, ps_status st, const std::string& msg) {
  if (h) h->err = msg;
  else g_create_error = msg;
  return st;
}

#define CK(h, x)                                                                               \
  do {                                                                                         \
    cudaError_t _e = (x);                                                                      \
    if (_e != cudaSuccess)                                                                     \
      return fail((h), _e == cudaErrorMemoryAllocation ? PS_ENOMEM : PS_ECUDA,                 \
                  std::string(#x) + ": " + cudaGetErrorString(_e));                          \
  } while (0)

template <typename T>
static cudaError_t dalloc(Handle* h, T** p, size_t count) {
  *p = nullptr;
  if (count == 0) return cudaSuccess;
  cudaError_t e = cudaMalloc((void**)p, count * sizeof(T));
  if (e == cudaSuccess) h->bytes += (int64_t)(count * sizeof(T));
  return e;
}

template <typename T>
static void dfree(Handle* h, T*& p, size_t count) {
  if (p) {
    cudaFree(p);
    h->bytes -= (int64_t)(count * sizeof(T));
  }
  p = nullptr;
}

static bool is_pow2(int v) { return v > 0 && (v & (v - 1)) == 0; }

// Host-side row preparation on several threads: f(t, begin, end) over contiguous parts
// [begin, end) of [0, n), part t on thread t (part 0 on the caller). The partition
// depends only on n and `parts`, so results that are combined part by part in order
// do not depend on the machine.
template <typename F>
static void parallel_parts(int64_t n, int parts, F f) {
  std::vector<std::thread> th;
  for (int t = 1; t < parts; ++t) {
    try {
      th.emplace_back([&, t] { f(t, n * t / parts, n * (t + 1) / parts); });
    } catch (...) {   // no thread to be had: this part runs on the caller
      f(t, n * t / parts, n * (t + 1) / parts);
    }
  }
  f(0, 0, n / parts);
  for (auto& x : th) x.join();
}
static int host_parts(int64_t n) {
  const unsigned hc = std::thread::hardware_concurrency();
  const int64_t by_size = std::max<int64_t>(1, n / 65536);
  return (int)std::max<int64_t>(1, std::min<int64_t>({(int64_t)(hc ? hc : 1), 16, by_size}));
}

// Stable counting sort of idx by key(i) in [0, nb) (parallel: per-part counts, then
// each part scatters its rows in order after the rows of the earlier parts).
template <typename K>
static void counting_sort(const std::vector<int32_t>& idx, std::vector<int32_t>& out, int64_t nb, int parts, K key) {
  const int64_t n = (int64_t)idx.size();
  std::vector<std::vector<int64_t>> cnt(parts, std::vector<int64_t>(nb, 0));
  parallel_parts(n, parts, [&](int t, int64_t b, int64_t e) {
    for (int64_t i = b; i < e; ++i) ++cnt[t][key(idx[i])];
  });
  int64_t run = 0;
  for (int64_t k = 0; k < nb; ++k)
    for (int t = 0; t < parts; ++t) {
      const int64_t c = cnt[t][k];
      cnt[t][k] = run;
      run += c;
    }
  parallel_parts(n, parts, [&](int t, int64_t b, int64_t e) {
    for (int64_t i = b; i < e; ++i) out[cnt[t][key(idx[i])]++] = idx[i];
  });
}

// Device arrays are read and written as float4: caller device pointers must be 16-byte aligned.
static bool misaligned(const void* p, int device_ptrs) { return device_ptrs && p && ((uintptr_t)p & 15u) != 0; }
#define CHECK_ALIGN(h, p, dp, what)                                                               \
  do {                                                                                            \
    if (misaligned((p), (dp))) return fail((h), PS_EINVAL, std::string(what) + ": device pointer not 16-byte aligned"); \
  } while (0)

static int sweep_blocks_host(int N) { return (N + 1023) / 1024; }

static void free_vis(Handle* h) {
  const size_t M = h->M;
  dfree(h, h->R, 4 * M);
  dfree(h, h->Y, 4 * M);
  dfree(h, h->vtmp, 4 * M);
  dfree(h, h->rec, M);
  dfree(h, h->perm, M);
  dfree(h, h->eps, (size_t)h->nblocks);
  dfree(h, h->cb, (size_t)h->nblocks);
  dfree(h, h->block_sum, (size_t)h->nblocks);
  dfree(h, h->items, (size_t)h->nitems);
  dfree(h, h->gchunks, (size_t)h->ngchunks);
  dfree(h, h->items_g, (size_t)h->nitems_g);
  dfree(h, h->gchunks_g, (size_t)h->ngchunks_g);
  dfree(h, h->vblk, M);
  dfree(h, h->wrow, 16 * M);
  const size_t Wd = h->g.Wd;
  dfree(h, h->T1, (size_t)h->n * Wd);
  dfree(h, h->G, Wd * Wd);
  dfree(h, h->Acc, 2 * Wd * Wd);
  dfree(h, h->T2, (size_t)h->n * Wd);
  dfree(h, h->tw, (size_t)h->g.K);
  dfree(h, h->corr, (size_t)h->n);
  h->M = h->nblocks = h->nitems = h->ngchunks = h->nitems_g = h->ngchunks_g = 0;
  h->g = ps::GridGeom{};
}

static void drop_graph(Handle* h) {
  if (h->graph) cudaGraphExecDestroy(h->graph);
  if (h->graph_multi) cudaGraphExecDestroy(h->graph_multi);
  h->graph = h->graph_multi = nullptr;
  h->graph_mode = -1;
}

static void set_default_steps(Handle* h) {
  const ps_config& c = h->cfg;
  h->rho1 = c.rho1 > 0 ? c.rho1 : 1.0;
  h->rho3 = c.rho3 > 0 ? c.rho3 : 1.0;
  const double on = h->opnorm_sq > 0 ? h->opnorm_sq : 0.0;
  h->rho2 = c.rho2 > 0 ? c.rho2 : (on > 0 ? 1.0 / on : 1.0);
  double denom = h->rho2 * on;
  if (h->mode != PS_NNLS) denom += h->rho1;
  if (h->mode == PS_POLARIZED || h->mode == PS_SOC) denom += h->rho3;
  if (ps::tv_mode(h->mode)) {
    // Algorithm 3: the data gradient is Lipschitz with beta = ||phi||^2 / 2 (phi~ = phi L^-1,
    // L L^H = 2 I); 1/tau - rho1 ||Psi||^2 - rho3 >= beta / 2, ||grad||^2 = 8, ||[Id; grad]||^2 = 9.
    // Default dual steps balanced against beta: rho1 ||Psi||^2 = rho3 = beta / 2.
    const double beta = on / 2.0, npsi = (h->mode == PS_L1TV || h->mode == PS_L1TV_NC) ? 9.0 : 8.0;
    if (!(c.rho1 > 0) && beta > 0) h->rho1 = beta / (2.0 * npsi);
    if (!(c.rho3 > 0) && beta > 0) h->rho3 = beta / 2.0;
    denom = beta / 2.0 + h->rho1 * npsi;
    if (ps::constrained_mode(h->mode)) denom += h->rho3;
  }
  h->tau = c.tau > 0 ? c.tau : (denom > 0 ? 0.99 / denom : 0.99);
}

static ps_status reset_state(Handle* h) {
  const size_t N = h->N;
  CK(h, cudaMemsetAsync(h->S, 0, 4 * N * sizeof(float), h->stream));
  CK(h, cudaMemsetAsync(h->Z, 0, 2 * N * sizeof(float), h->stream));
  CK(h, cudaMemsetAsync(h->C, 0, 4 * N * sizeof(float), h->stream));
  CK(h, cudaMemsetAsync(h->D, 0, 2 * N * sizeof(float), h->stream));
  CK(h, cudaMemsetAsync(h->A, 0, 36 * N * sizeof(float), h->stream));
  CK(h, cudaMemsetAsync(h->PsiA, 0, 4 * N * sizeof(float), h->stream));
  CK(h, cudaMemsetAsync(h->Adj, 0, 4 * N * sizeof(float), h->stream));
  CK(h, cudaMemsetAsync(h->Xb, 0, 4 * N * sizeof(float), h->stream));
  CK(h, cudaMemsetAsync(h->red, 0, (size_t)h->red_cap * sizeof(double), h->stream));
  CK(h, cudaMemsetAsync(h->dev_flags, 0, 4 * sizeof(int), h->stream));
  if (h->M > 0) {
    CK(h, cudaMemsetAsync(h->R, 0, 4 * (size_t)h->M * sizeof(float2), h->stream));
    CK(h, cudaMemsetAsync(h->cb, 0, (size_t)h->nblocks * sizeof(float), h->stream));
  }
  h->derived_valid = true;   // Psi 0 = 0, phi^dagger 0 = 0
  h->iterations = 0;
  ++h->version;
  return PS_OK;
}

// Psi A and phi^dagger(c_b R) of the current state.
static cudaError_t nufft_gradient_chain(Handle* h, cudaEvent_t* ev);
static ps_status compute_derived(Handle* h) {
  if (ps::tv_mode(h->mode)) {   // Psi A = grad^T A (+ A_l1) and phi^dagger(Y - phi S) of the current state
    CK(h, ps::tv_adjoint(h));
    if (h->M > 0) {
      CK(h, nufft_gradient_chain(h, nullptr));
    } else {
      CK(h, cudaMemsetAsync(h->Adj, 0, 4 * (size_t)h->N * sizeof(float), h->stream));
    }
    h->derived_valid = true;
    return PS_OK;
  }
  CK(h, ps::sara_synthesis(h, h->A, h->PsiA));
  if (h->M > 0) {
    CK(h, ps::nufft_grid(h, h->R, 1));
    CK(h, ps::nufft_adjoint_image(h, h->Adj));
  } else {
    CK(h, cudaMemsetAsync(h->Adj, 0, 4 * (size_t)h->N * sizeof(float), h->stream));
  }
  h->derived_valid = true;
  return PS_OK;
}

// One iteration of Algorithm 1. With `ev` (PS_NSTAGES + 1 events) the stage
// boundaries are recorded on the stream for ps_profile_stages (stages run in order).
// Without it, after the per-pixel sweep the SARA chain (steps 5-6 and the next
// Psi A) runs on the handle's second stream beside the NUFFT chain (steps 7-8 and
// the next phi^dagger B): both only read 2S'-S and write disjoint buffers, and the
// two join before the iteration ends.
static cudaError_t sara_chain(Handle* h) {
  cudaError_t e = ps::sara_analysis(h, h->Xb, h->A, h->T, ps::SARA_DUAL, (float)(h->rho1 / 3.0), 0.f, 0.f);
  if (e != cudaSuccess) return e;
  return ps::sara_synthesis(h, h->A, h->PsiA);
}

static cudaError_t nufft_chain(Handle* h, cudaEvent_t* ev) {
  auto mark = [&](int i) { return ev ? cudaEventRecord(ev[i], h->stream) : cudaSuccess; };
  cudaError_t e;
  if ((e = mark(PS_STAGE_FWD_FFT)) != cudaSuccess) return e;
  if (h->M > 0 && (e = ps::nufft_forward_grid(h, h->Xb)) != cudaSuccess) return e;
  if ((e = mark(PS_STAGE_DEGRID)) != cudaSuccess) return e;
  if (h->M > 0 && (e = ps::nufft_degrid(h, ps::DEG_DUAL, nullptr)) != cudaSuccess) return e;
  if ((e = mark(PS_STAGE_BALL)) != cudaSuccess) return e;
  if (h->M > 0 && (e = ps::block_scales(h)) != cudaSuccess) return e;
  if ((e = mark(PS_STAGE_GRID)) != cudaSuccess) return e;
  if (h->M > 0 && (e = ps::nufft_grid(h, h->R, 1)) != cudaSuccess) return e;
  if ((e = mark(PS_STAGE_ADJ_FFT)) != cudaSuccess) return e;
  if (h->M > 0 && (e = ps::nufft_adjoint_image(h, h->Adj)) != cudaSuccess) return e;
  return mark(PS_NSTAGES);
}

// Algorithm 3: the data-term gradient of the next primal step, at the new S:
// Adj = phi^dagger(Y - phi(S)) (k_primal takes -Adj / 2). Stage events as in nufft_chain
// (the ball stage is empty).
static cudaError_t nufft_gradient_chain(Handle* h, cudaEvent_t* ev) {
  auto mark = [&](int i) { return ev ? cudaEventRecord(ev[i], h->stream) : cudaSuccess; };
  cudaError_t e;
  if ((e = mark(PS_STAGE_FWD_FFT)) != cudaSuccess) return e;
  if (h->M > 0 && (e = ps::nufft_forward_grid(h, h->S)) != cudaSuccess) return e;
  if ((e = mark(PS_STAGE_DEGRID)) != cudaSuccess) return e;
  if (h->M > 0 && (e = ps::nufft_degrid(h, ps::DEG_RESID, h->vtmp)) != cudaSuccess) return e;
  if ((e = mark(PS_STAGE_BALL)) != cudaSuccess) return e;
  if ((e = mark(PS_STAGE_GRID)) != cudaSuccess) return e;
  if (h->M > 0 && (e = ps::nufft_grid(h, h->vtmp, 0)) != cudaSuccess) return e;
  if ((e = mark(PS_STAGE_ADJ_FFT)) != cudaSuccess) return e;
  if (h->M > 0 && (e = ps::nufft_adjoint_image(h, h->Adj)) != cudaSuccess) return e;
  return mark(PS_NSTAGES);
}

// Algorithm 3 steps 5-6 and the next Psi A.
static cudaError_t tv_chain(Handle* h) {
  cudaError_t e = ps::tv_dual(h);
  if (e != cudaSuccess) return e;
  return ps::tv_adjoint(h);
}

static cudaError_t one_iteration(Handle* h, cudaEvent_t* ev = nullptr) {
  auto mark = [&](int i) { return ev ? cudaEventRecord(ev[i], h->stream) : cudaSuccess; };
  cudaError_t e;
  if ((e = mark(PS_STAGE_PRIMAL)) != cudaSuccess) return e;
  if ((e = ps::primal_sweep(h)) != cudaSuccess) return e;
  if (ps::tv_mode(h->mode)) {
    // The TV chain (sparsity duals, next Psi A) and the data-gradient chain (on the new S)
    // read disjoint inputs and write disjoint buffers: concurrent branches as in Alg. 1.
    if (ev || h->M == 0 || !h->aux) {
      if ((e = mark(PS_STAGE_ANALYSIS)) != cudaSuccess) return e;
      if ((e = ps::tv_dual(h)) != cudaSuccess) return e;
      if ((e = mark(PS_STAGE_ANALYSIS_COARSE)) != cudaSuccess) return e;
      if ((e = mark(PS_STAGE_SYNTHESIS_COARSE)) != cudaSuccess) return e;
      if ((e = mark(PS_STAGE_SYNTHESIS)) != cudaSuccess) return e;
      if ((e = ps::tv_adjoint(h)) != cudaSuccess) return e;
      return nufft_gradient_chain(h, ev);
    }
    if ((e = cudaEventRecord(h->ev_fork, h->stream)) != cudaSuccess) return e;
    if ((e = cudaStreamWaitEvent(h->aux, h->ev_fork, 0)) != cudaSuccess) return e;
    cudaStream_t main = h->stream;
    h->stream = h->aux;
    e = tv_chain(h);
    cudaError_t e2 = cudaEventRecord(h->ev_join, h->aux);
    h->stream = main;
    if (e != cudaSuccess) return e;
    if (e2 != cudaSuccess) return e2;
    if ((e = nufft_gradient_chain(h, nullptr)) != cudaSuccess) return e;
    return cudaStreamWaitEvent(h->stream, h->ev_join, 0);
  }
  const bool sara = (h->mode != PS_NNLS);
  if (ev || !sara || h->M == 0 || !h->aux) {
    if ((e = mark(PS_STAGE_ANALYSIS)) != cudaSuccess) return e;
    if (sara && (e = ps::sara_analysis(h, h->Xb, h->A, h->T, ps::SARA_DUAL, (float)(h->rho1 / 3.0), 0.f, 0.f,
                                       ev ? ev[PS_STAGE_ANALYSIS_COARSE] : nullptr)) != cudaSuccess)
      return e;
    if (!sara && (e = mark(PS_STAGE_ANALYSIS_COARSE)) != cudaSuccess) return e;
    if ((e = mark(PS_STAGE_SYNTHESIS_COARSE)) != cudaSuccess) return e;
    if (sara && (e = ps::sara_synthesis(h, h->A, h->PsiA, ev ? ev[PS_STAGE_SYNTHESIS] : nullptr)) != cudaSuccess)
      return e;
    if (!sara && (e = mark(PS_STAGE_SYNTHESIS)) != cudaSuccess) return e;
    return nufft_chain(h, ev);
  }
  if ((e = cudaEventRecord(h->ev_fork, h->stream)) != cudaSuccess) return e;
  if ((e = cudaStreamWaitEvent(h->aux, h->ev_fork, 0)) != cudaSuccess) return e;
  cudaStream_t main = h->stream;
  h->stream = h->aux;                     // the SARA launchers use h->stream
  e = sara_chain(h);
  cudaError_t e2 = cudaEventRecord(h->ev_join, h->aux);
  h->stream = main;
  if (e != cudaSuccess) return e;
  if (e2 != cudaSuccess) return e2;
  if ((e = nufft_chain(h, nullptr)) != cudaSuccess) return e;
  return cudaStreamWaitEvent(h->stream, h->ev_join, 0);
}

// Graph of `iters` iterations back to back (their launches in order on the handle's streams).
static ps_status capture_iterations(Handle* h, int iters, cudaGraphExec_t* exec) {
  cudaGraph_t graph = nullptr;
  CK(h, cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
  cudaError_t e = cudaSuccess;
  for (int i = 0; i < iters && e == cudaSuccess; ++i) e = one_iteration(h);
  cudaError_t e2 = cudaStreamEndCapture(h->stream, &graph);
  if (e != cudaSuccess || e2 != cudaSuccess) {
    if (graph) cudaGraphDestroy(graph);
    return fail(h, PS_ECUDA, std::string("graph capture: ") + cudaGetErrorString(e != cudaSuccess ? e : e2));
  }
  e = cudaGraphInstantiate(exec, graph, cudaGraphInstantiateFlagUseNodePriority);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) return fail(h, PS_ECUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
  return PS_OK;
}

// The one-iteration graph, and the kGraphIters-iteration one that ps_pd_iterate launches for
// runs of that many iterations: one launch instead of kGraphIters, which matters where an
// iteration is a few microseconds of work (small images).
static ps_status build_graph(Handle* h) {
  drop_graph(h);
  ps_status st = capture_iterations(h, 1, &h->graph);
  if (st == PS_OK) st = capture_iterations(h, ps::kGraphIters, &h->graph_multi);
  if (st != PS_OK) {
    drop_graph(h);
    return st;
  }
  h->graph_mode = h->mode;
  return PS_OK;
}

#pragma GCC visibility push(default)
extern "C" {

const char* ps_last_error(const ps_handle* h) { return h ? h->err.c_str() : g_create_error.c_str(); }

int64_t ps_estimate_bytes(int32_t n, int32_t levels, int64_t M) {
  if (n < 16 || n > 2048 || !is_pow2(n) || levels < 1 || (n % (1 << levels)) != 0 || M < 0) return 0;
  const int64_t N = (int64_t)n * n, K = 2 * (int64_t)n;
  const int64_t img = (28 + 72 + 16) * N * 4 + (8 * (int64_t)sweep_blocks_host((int)N) + 1024) * 8;
  const int64_t vis = M * (3 * 32 + 16 + 4 + 64) + (M / ps::kChunk + 64) * 24 + M / 2;   // + item and chunk lists
  const int64_t grid = 2 * (int64_t)n * K * 16 + 48 * K * K + K * 12 + (int64_t)n * 4;
  return img + vis + grid;
}

int64_t ps_device_bytes(const ps_handle* h) { return h ? h->bytes : 0; }

ps_status ps_create(const ps_config* cfg, void* cuda_stream, ps_handle** out) {
  if (!cfg || !out) return fail(nullptr, PS_EINVAL, "ps_create: null argument");
  *out = nullptr;
  const int n = cfg->n, L = cfg->levels;
  if (n < 16 || n > 2048 || !is_pow2(n))
    return fail(nullptr, PS_EINVAL, "ps_create: n must be a power of two in [16, 2048]");
  if (L < 1 || (n % (1 << L)) != 0 || (n >> L) < 1)
    return fail(nullptr, PS_EINVAL, "ps_create: levels must satisfy 1 <= levels and n divisible by 2^levels");
  if (cfg->mode < PS_POLARIZED || cfg->mode > PS_L1TV_NC) return fail(nullptr, PS_EINVAL, "ps_create: bad mode");
  const int W = cfg->kernel_width == 0 ? 7 : cfg->kernel_width;
  if (W != 5 && W != 7 && W != 9) return fail(nullptr, PS_EINVAL, "ps_create: kernel_width must be 5, 7 or 9");
  if (cfg->tau < 0 || cfg->rho1 < 0 || cfg->rho2 < 0 || cfg->rho3 < 0)
    return fail(nullptr, PS_EINVAL, "ps_create: step sizes must be >= 0");
  if (cfg->stop_maps != 0 && cfg->stop_maps != 3 && cfg->stop_maps != 4)
    return fail(nullptr, PS_EINVAL, "ps_create: stop_maps must be 0, 3 or 4");
  if (!(cfg->alpha == 0.0 || cfg->alpha == 2.0))
    return fail(nullptr, PS_EINVAL, "ps_create: alpha (NUFFT oversampling) must be 0 or 2");
  for (double v : {cfg->gamma, cfg->noise_sigma, cfg->rel_tol, cfg->resid_tol, cfg->np_tol, cfg->zeta_sigma})
    if (!(v >= 0) || !std::isfinite(v))
      return fail(nullptr, PS_EINVAL, "ps_create: gamma, noise_sigma and the stopping tolerances must be finite and >= 0");
  int dev_count = 0;
  if (cudaGetDeviceCount(&dev_count) != cudaSuccess || dev_count == 0)
    return fail(nullptr, PS_ECUDA, "ps_create: no CUDA device");

  ps_handle* h = new ps_handle();
  h->cfg = *cfg;
  h->cfg.kernel_width = W;
  // Defaults of Section 5.5 (rel_tol = epsilon, resid_tol = vartheta, np_tol = varrho in
  // percent) and Section 5.2 (zeta = 3 rms), and the oversampling 2.
  h->cfg.alpha = 2.0;
  if (h->cfg.stop_maps == 0) h->cfg.stop_maps = 4;
  if (!(h->cfg.rel_tol > 0)) h->cfg.rel_tol = 1e-5;
  if (!(h->cfg.resid_tol > 0)) h->cfg.resid_tol = 5e-3;
  if (!(h->cfg.np_tol > 0)) h->cfg.np_tol = 0.5;
  if (!(h->cfg.zeta_sigma > 0)) h->cfg.zeta_sigma = 3.0;
  h->gamma_default = cfg->gamma > 0 ? cfg->gamma : 1.0;
  h->n = n;
  h->N = n * n;
  h->L = L;
  h->mode = cfg->mode;
  auto bail = [&](ps_status st) {
    g_create_error = h->err;
    ps_destroy(h);
    return st;
  };
  if (cuda_stream) {
    h->stream = (cudaStream_t)cuda_stream;
  } else {
    if (cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking) != cudaSuccess) {
      h->err = "ps_create: cudaStreamCreate failed";
      return bail(PS_ECUDA);
    }
    h->own_stream = true;
  }
  // The SARA branch of the iteration graph runs at the highest stream priority (graph
  // nodes keep their capture stream's priority): measured slightly faster at 1024^2 than
  // equal priorities, and faster than prioritising the NUFFT branch.
  int prio_lo = 0, prio_hi = 0;
  cudaDeviceGetStreamPriorityRange(&prio_lo, &prio_hi);
  if (cudaStreamCreateWithPriority(&h->aux, cudaStreamNonBlocking, prio_hi) != cudaSuccess ||
      cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&h->ev_join, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&h->relc_ev, cudaEventDisableTiming) != cudaSuccess) {
    h->err = "ps_create: auxiliary stream/events";
    return bail(PS_ECUDA);
  }
  cudaError_t e = ps::configure_kernels();
  if (e != cudaSuccess) {
    h->err = std::string("configure kernels: ") + cudaGetErrorString(e);
    return bail(PS_ECUDA);
  }
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    h->err = "ps_create: device attributes";
    return bail(PS_ECUDA);
  }
  double filt[ps::kDb][ps::kMaxTaps];
  ps::daubechies_filters(filt);
  if ((e = ps::upload_filters(filt, h->stream)) != cudaSuccess) {
    h->err = std::string("upload filters: ") + cudaGetErrorString(e);
    return bail(PS_ECUDA);
  }
  const size_t N = h->N;
  h->red_cap = 8 * sweep_blocks_host((int)N) + 1024;
  bool ok = dalloc(h, &h->S, 4 * N) == cudaSuccess && dalloc(h, &h->Z, 2 * N) == cudaSuccess &&
            dalloc(h, &h->C, 4 * N) == cudaSuccess && dalloc(h, &h->D, 2 * N) == cudaSuccess &&
            dalloc(h, &h->Xb, 4 * N) == cudaSuccess && dalloc(h, &h->PsiA, 4 * N) == cudaSuccess &&
            dalloc(h, &h->Adj, 4 * N) == cudaSuccess && dalloc(h, &h->tmp4, 4 * N) == cudaSuccess &&
            dalloc(h, &h->A, 36 * N) == cudaSuccess && dalloc(h, &h->T, 36 * N) == cudaSuccess &&
            dalloc(h, &h->approx, 16 * N) == cudaSuccess && dalloc(h, &h->red, (size_t)h->red_cap) == cudaSuccess &&
            dalloc(h, &h->dev_flags, 4) == cudaSuccess &&
            cudaMallocHost((void**)&h->red_host, 1024 * sizeof(double)) == cudaSuccess &&
            cudaHostAlloc((void**)&h->relc_host, 16 * sizeof(double), cudaHostAllocMapped) == cudaSuccess &&
            cudaHostGetDevicePointer((void**)&h->relc_dev, h->relc_host, 0) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    h->err = "ps_create: device allocation failed";
    return bail(PS_ENOMEM);
  }
  h->approx2 = h->approx + 8 * N;
  if (reset_state(h) != PS_OK) return bail(PS_ECUDA);
  // Thresholds default to 1 (gamma = 1, W = 1).
  std::vector<float> ones(36 * N, 1.0f);
  if (cudaMemcpyAsync(h->T, ones.data(), ones.size() * sizeof(float), cudaMemcpyHostToDevice, h->stream) !=
          cudaSuccess ||
      cudaStreamSynchronize(h->stream) != cudaSuccess) {
    h->err = "ps_create: initialisation failed";
    return bail(PS_ECUDA);
  }
  set_default_steps(h);
  *out = h;
  return PS_OK;
}

void ps_destroy(ps_handle* h) {
  if (!h) return;
  if (h->stream) cudaStreamSynchronize(h->stream);
  drop_graph(h);
  free_vis(h);
  const size_t N = h->N;
  if (h->in_slab) {   // these arrays belong to a batch's class slabs
    h->S = h->Z = h->C = h->D = h->Xb = h->PsiA = h->Adj = h->A = h->T = h->approx = h->approx2 = nullptr;
    h->red = nullptr;
  }
  dfree(h, h->S, 4 * N);
  dfree(h, h->Z, 2 * N);
  dfree(h, h->C, 4 * N);
  dfree(h, h->D, 2 * N);
  dfree(h, h->Xb, 4 * N);
  dfree(h, h->PsiA, 4 * N);
  dfree(h, h->Adj, 4 * N);
  dfree(h, h->tmp4, 4 * N);
  dfree(h, h->tmp36, 36 * N);
  dfree(h, h->A, 36 * N);
  dfree(h, h->T, 36 * N);
  dfree(h, h->approx, 16 * N);
  dfree(h, h->red, (size_t)h->red_cap);
  dfree(h, h->dev_flags, 4);
  if (h->red_host) cudaFreeHost(h->red_host);
  if (h->relc_host) cudaFreeHost(h->relc_host);
  if (h->relc_ev) cudaEventDestroy(h->relc_ev);
  if (h->aux) cudaStreamDestroy(h->aux);
  if (h->ev_fork) cudaEventDestroy(h->ev_fork);
  if (h->ev_join) cudaEventDestroy(h->ev_join);
  if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
  delete h;
}

// Reads the device error flags after a synchronisation: a bounded in-kernel wait
// that gave up is reported as PS_ETIMEOUT (the flag is then cleared).
static ps_status check_flags(Handle* h) {
  int f[4] = {0, 0, 0, 0};
  CK(h, cudaMemcpyAsync(f, h->dev_flags, sizeof(f), cudaMemcpyDeviceToHost, h->stream));
  CK(h, cudaStreamSynchronize(h->stream));
  if (f[0]) {
    CK(h, cudaMemsetAsync(h->dev_flags, 0, sizeof(f), h->stream));
    return fail(h, PS_ETIMEOUT, "a bounded device wait (bulk-copy barrier) gave up; results of that launch are invalid");
  }
  return PS_OK;
}

ps_status ps_synchronize(ps_handle* h) {
  if (!h) return PS_EINVAL;
  CK(h, cudaStreamSynchronize(h->stream));
  CK(h, cudaGetLastError());
  return check_flags(h);
}

// Copy `bytes` from a caller pointer into device memory `dst` (or alias when on device).
static ps_status stage_in(Handle* h, const void* src, size_t bytes, int device_ptrs, void* dst) {
  CK(h, cudaMemcpyAsync(dst, src, bytes, device_ptrs ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, h->stream));
  return PS_OK;
}

static ps_status opnorm_lanczos(Handle* h);
static ps_status default_gamma(Handle* h);
}  // extern "C"

static __global__ void k_fill(float* p, int n, float v) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) p[i] = v;
}

// p[0 .. len) = v, grid-stride, float4 stores (p 16-byte aligned, len a multiple of 4).
static __global__ void k_fill4(float4* p, size_t len4, float v) {
  const float4 q = make_float4(v, v, v, v);
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < len4; i += (size_t)gridDim.x * blockDim.x)
    p[i] = q;
}

extern "C" {

ps_status ps_set_measurements(ps_handle* h, int64_t M64, const double* uv, const float* vis, const float* weights,
                              int32_t nblocks, const int64_t* block_offsets, const double* eps, int32_t device_ptrs) {
  if (!h) return PS_EINVAL;
  if (M64 < 0 || M64 > (int64_t)1 << 30) return fail(h, PS_EINVAL, "set_measurements: M out of range");
  const int M = (int)M64;
  CHECK_ALIGN(h, uv, device_ptrs, "set_measurements");
  CHECK_ALIGN(h, vis, device_ptrs, "set_measurements");
  CHECK_ALIGN(h, weights, device_ptrs, "set_measurements");
  if (M > 0 && (!uv || !vis || !block_offsets || nblocks < 1 || nblocks > 2047))
    return fail(h, PS_EINVAL, "set_measurements: need uv, vis, block_offsets and 1 <= nblocks <= 2047");
  std::vector<double> eps_chi2;
  if (M > 0) {
    if (block_offsets[0] != 0 || block_offsets[nblocks] != M64)
      return fail(h, PS_EINVAL, "set_measurements: block_offsets must start at 0 and end at M");
    for (int b = 0; b < nblocks; ++b)
      if (block_offsets[b + 1] < block_offsets[b]) return fail(h, PS_EINVAL, "set_measurements: offsets decrease");
    if (!eps) {
      // Section 5.1: ||E_b||^2 / (sigma^2 / 2) is chi^2 with 8 M_b degrees of freedom; the radius
      // sits two standard deviations above the mean, eps_b^2 = (8 M_b + 2 sqrt(16 M_b)) sigma^2 / 2.
      const double sig = h->cfg.noise_sigma;
      if (!(sig > 0)) return fail(h, PS_EINVAL, "set_measurements: eps = NULL needs cfg.noise_sigma > 0");
      eps_chi2.resize(nblocks);
      for (int b = 0; b < nblocks; ++b) {
        const double dof = 8.0 * (double)(block_offsets[b + 1] - block_offsets[b]);
        eps_chi2[b] = std::sqrt((dof + 2.0 * std::sqrt(2.0 * dof)) * sig * sig / 2.0);
      }
      eps = eps_chi2.data();
    }
    for (int b = 0; b < nblocks; ++b)
      if (!(eps[b] > 0) || !std::isfinite(eps[b])) return fail(h, PS_EINVAL, "set_measurements: eps must be > 0");
  }
  CK(h, cudaStreamSynchronize(h->stream));
  drop_graph(h);
  free_vis(h);
  h->have_meas = false;

  // Host views of the measurement rows: caller host arrays are read in place, caller
  // device arrays are copied on the handle's stream (its order, not the legacy stream's).
  const int parts = host_parts(M);
  std::vector<double> uv_copy;
  std::vector<float> w_copy;
  const double* uvh = uv;
  const float* wsrc = weights;
  if (M > 0 && device_ptrs) {
    uv_copy.resize(2 * (size_t)M);
    CK(h, cudaMemcpyAsync(uv_copy.data(), uv, uv_copy.size() * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    uvh = uv_copy.data();
    if (weights) {
      w_copy.resize(M);
      CK(h, cudaMemcpyAsync(w_copy.data(), weights, w_copy.size() * sizeof(float), cudaMemcpyDeviceToHost, h->stream));
      wsrc = w_copy.data();
    }
    CK(h, cudaStreamSynchronize(h->stream));
  }
  auto wrow_of = [&](int64_t m) { return wsrc ? wsrc[m] : 1.0f; };

  // Grid geometry: tap centres c = floor(u + 1/2), u = omega K / (2 pi); rows checked.
  ps::GridGeom& g = h->g;
  g.K = 2 * h->n;
  g.logK = 0;
  while ((1 << g.logK) < g.K) ++g.logK;
  g.W = h->cfg.kernel_width;
  g.beta = (float)ps::es_beta(g.W);
  const int hw = g.W / 2;
  std::vector<int> cx(M), cy(M);
  std::vector<float> fx(M), fy(M);
  std::vector<int> part_cmax(parts, 0), part_bad(parts, 0);
  parallel_parts(M, parts, [&](int t, int64_t b, int64_t e) {
    int cm = 0, bad = 0;
    for (int64_t m = b; m < e; ++m) {
      const double ou = uvh[2 * m], ov = uvh[2 * m + 1];
      const float wm = wrow_of(m);
      if (!std::isfinite(ou) || !std::isfinite(ov) || std::fabs(ou) >= M_PI || std::fabs(ov) >= M_PI) {
        bad |= 1;
        continue;
      }
      if (!(wm >= 0.f) || !std::isfinite(wm)) bad |= 2;
      const double u = ou * g.K / (2.0 * M_PI), v = ov * g.K / (2.0 * M_PI);
      const double cu = std::floor(u + 0.5), cv = std::floor(v + 0.5);
      cx[m] = (int)cu;
      cy[m] = (int)cv;
      fx[m] = (float)(u - cu);
      fy[m] = (float)(v - cv);
      cm = std::max(cm, std::max(std::abs(cx[m]), std::abs(cy[m])));
    }
    part_cmax[t] = cm;
    part_bad[t] = bad;
  });
  int cmax = 0, bad = 0;
  for (int t = 0; t < parts; ++t) {
    cmax = std::max(cmax, part_cmax[t]);
    bad |= part_bad[t];
  }
  if (bad) h->g = ps::GridGeom{};
  if (bad & 1) return fail(h, PS_EINVAL, "set_measurements: |omega| must be < pi (radians per pixel)");
  if (bad & 2) return fail(h, PS_EINVAL, "set_measurements: weights must be >= 0");
  g.R = cmax + hw;
  if (2 * g.R + 1 <= g.K) {
    g.full = 0;
    g.Wd = 2 * g.R + 1;
    g.off = g.R;
  } else {
    g.full = 1;
    g.Wd = g.K;
    g.off = 0;
  }
  g.tilesX = (g.Wd + ps::kGridTile - 1) / ps::kGridTile;
  auto gi = [&](int k) { return g.full ? (k & (g.K - 1)) : k + g.off; };

  // Storage order: rows sorted by degridding tile (TS x TS cells), then by gridding tile
  // within it (TG x TG), then by tap-centre cell (row-major in the gridding tile), rows of
  // one cell in the caller's order: three stable counting-sort passes, least significant
  // first. The rows of every degridding tile, of every gridding tile and of every cell are
  // then contiguous.
  const int TS = ps::kGridTile, TG = ps::kGridTileG, NS = TS / TG;
  auto tile_of = [&](int32_t m) { return (int64_t)(gi(cy[m]) / TS) * g.tilesX + gi(cx[m]) / TS; };
  auto sub_of = [&](int32_t m) { return (int64_t)(((gi(cy[m]) % TS) / TG) * NS + (gi(cx[m]) % TS) / TG); };
  auto cell_of = [&](int32_t m) { return (int64_t)((gi(cy[m]) % TG) * TG + gi(cx[m]) % TG); };
  std::vector<int32_t> perm(M), tmp(M);
  std::iota(tmp.begin(), tmp.end(), 0);
  counting_sort(tmp, perm, (int64_t)TG * TG, parts, cell_of);
  tmp.swap(perm);
  counting_sort(tmp, perm, (int64_t)NS * NS, parts, sub_of);
  tmp.swap(perm);
  counting_sort(tmp, perm, (int64_t)g.tilesX * g.tilesX, parts, tile_of);
  std::vector<int32_t> sgy(M), sgx(M);   // grid cell of each row, in storage order
  parallel_parts(M, parts, [&](int, int64_t b, int64_t e) {
    for (int64_t i = b; i < e; ++i) {
      sgy[i] = gi(cy[perm[i]]);
      sgx[i] = gi(cx[perm[i]]);
    }
  });
  if (M > 0) h->offsets_host.assign(block_offsets, block_offsets + nblocks + 1);
  else h->offsets_host.assign(1, 0);
  std::vector<uint16_t> blk_user(M);
  for (int b = 0; b < (M > 0 ? nblocks : 0); ++b)
    std::fill(blk_user.begin() + block_offsets[b], blk_user.begin() + block_offsets[b + 1], (uint16_t)b);
  std::vector<uint16_t> vblk(M);
  std::vector<float4> rech(M);
  parallel_parts(M, parts, [&](int, int64_t b, int64_t e) {
    for (int64_t i = b; i < e; ++i) {
      const int m = perm[i];
      vblk[i] = blk_user[m];
      const int packed = (cx[m] & 0xFFFF) | (cy[m] << 16);
      float pf;
      std::memcpy(&pf, &packed, sizeof(pf));
      rech[i] = make_float4(fx[m], fy[m], wrow_of(m), pf);
    }
  });
  // 2 sum w_m^2 over a fixed partition (the same sum on every machine).
  constexpr int kPsfParts = 16;
  std::vector<double> part_psf(kPsfParts, 0.0);
  parallel_parts(M, kPsfParts, [&](int t, int64_t b, int64_t e) {
    double acc = 0.0;
    for (int64_t m = b; m < e; ++m) acc += 2.0 * (double)wrow_of(m) * wrow_of(m);
    part_psf[t] = acc;
  });
  h->psf_peak = std::accumulate(part_psf.begin(), part_psf.end(), 0.0);
  // Work items (<= cap rows of one tile of side tsz) and same-cell chunks (<= kBinChunk
  // rows): kGridItem rows of a TS tile per degridding item, kGridItemG rows of a TG tile per
  // gridding item; a chunk holds its cell's position in the item's tile.
  auto make_items = [&](int cap, int tsz, std::vector<ps::GridItem>& items, std::vector<int32_t>& gchunks) {
    int j0 = 0;
    while (j0 < M) {
      const int ty = sgy[j0] / tsz, tx = sgx[j0] / tsz;
      int j1 = j0;
      while (j1 < M && j1 - j0 < cap && sgy[j1] / tsz == ty && sgx[j1] / tsz == tx) ++j1;
      ps::GridItem it{};
      it.ty = ty;
      it.tx = tx;
      it.vstart = j0;
      it.vend = j1;
      it.cstart = (int32_t)gchunks.size();
      int c0 = j0;
      while (c0 < j1) {
        int c1 = c0;
        while (c1 < j1 && c1 - c0 < ps::kBinChunk && sgy[c1] == sgy[c0] && sgx[c1] == sgx[c0]) ++c1;
        const int ly = sgy[c0] - ty * tsz, lx = sgx[c0] - tx * tsz;
        gchunks.push_back((c0 - j0) | ((c1 - c0) << 10) | (ly << 16) | (lx << 24));
        c0 = c1;
      }
      it.cend = (int32_t)gchunks.size();
      items.push_back(it);
      j0 = j1;
    }
  };
  std::vector<ps::GridItem> items, items_g;
  std::vector<int32_t> gchunks, gchunks_g;
  make_items(ps::kGridItem, TS, items, gchunks);
  make_items(ps::kGridItemG, TG, items_g, gchunks_g);
  h->M = M;
  h->nblocks = M > 0 ? nblocks : 0;
  h->nitems = (int)items.size();
  h->ngchunks = (int)gchunks.size();
  h->nitems_g = (int)items_g.size();
  h->ngchunks_g = (int)gchunks_g.size();
  if (M > 0) h->eps_host.assign(eps, eps + h->nblocks);
  else h->eps_host.clear();

  // Device buffers for the visibility domain and the grid.
  const size_t Wd = g.Wd;
  bool ok = dalloc(h, &h->R, 4 * (size_t)M) == cudaSuccess && dalloc(h, &h->Y, 4 * (size_t)M) == cudaSuccess &&
            dalloc(h, &h->vtmp, 4 * (size_t)M) == cudaSuccess && dalloc(h, &h->rec, (size_t)M) == cudaSuccess &&
            dalloc(h, &h->perm, (size_t)M) == cudaSuccess && dalloc(h, &h->eps, (size_t)h->nblocks) == cudaSuccess &&
            dalloc(h, &h->cb, (size_t)h->nblocks) == cudaSuccess &&
            dalloc(h, &h->block_sum, (size_t)h->nblocks) == cudaSuccess &&
            dalloc(h, &h->items, items.size()) == cudaSuccess &&
            dalloc(h, &h->gchunks, gchunks.size()) == cudaSuccess &&
            dalloc(h, &h->items_g, items_g.size()) == cudaSuccess &&
            dalloc(h, &h->gchunks_g, gchunks_g.size()) == cudaSuccess && dalloc(h, &h->vblk, (size_t)M) == cudaSuccess &&
            dalloc(h, &h->T1, (size_t)h->n * Wd) == cudaSuccess && dalloc(h, &h->G, Wd * Wd) == cudaSuccess &&
            dalloc(h, &h->Acc, 2 * Wd * Wd) == cudaSuccess && dalloc(h, &h->T2, (size_t)h->n * Wd) == cudaSuccess &&
            dalloc(h, &h->tw, (size_t)g.K) == cudaSuccess && dalloc(h, &h->corr, (size_t)h->n) == cudaSuccess &&
            (g.W > 8 || dalloc(h, &h->wrow, 16 * (size_t)M) == cudaSuccess);
  if (!ok) {
    cudaGetLastError();
    free_vis(h);
    return fail(h, PS_ENOMEM, "set_measurements: device allocation failed");
  }
  // Twiddles of radix-2 stage t (span 2^(t+1)) at [2^t - 1, 2^(t+1) - 1): exp(-2 pi i p / 2^(t+1)).
  std::vector<float2> twh(g.K, make_float2(0.f, 0.f));
  for (int t = 0; t < g.logK; ++t)
    for (int p = 0; p < (1 << t); ++p) {
      const double a = -2.0 * M_PI * p / (double)(2 << t);
      twh[(1 << t) - 1 + p] = make_float2((float)std::cos(a), (float)std::sin(a));
    }
  std::vector<float> corrh(h->n);
  // phihat is even: q and n - q (offsets -d and +d from the centre) share a value.
  for (int q = 0; q <= h->n / 2; ++q) {
    corrh[q] = (float)(1.0 / ps::es_fourier(2.0 * M_PI * (q - h->n / 2) / g.K, g.W, g.beta));
    if (q > 0 && q < h->n / 2) corrh[h->n - q] = corrh[q];
  }
  CK(h, cudaMemcpyAsync(h->tw, twh.data(), twh.size() * sizeof(float2), cudaMemcpyHostToDevice, h->stream));
  CK(h, cudaMemcpyAsync(h->corr, corrh.data(), corrh.size() * sizeof(float), cudaMemcpyHostToDevice, h->stream));
  if (M > 0) {
    CK(h, cudaMemcpyAsync(h->rec, rech.data(), rech.size() * sizeof(float4), cudaMemcpyHostToDevice, h->stream));
    CK(h, cudaMemcpyAsync(h->perm, perm.data(), perm.size() * sizeof(int32_t), cudaMemcpyHostToDevice, h->stream));
    CK(h, cudaMemcpyAsync(h->eps, eps, h->nblocks * sizeof(double), cudaMemcpyHostToDevice, h->stream));
    CK(h, cudaMemcpyAsync(h->items, items.data(), items.size() * sizeof(ps::GridItem), cudaMemcpyHostToDevice, h->stream));
    CK(h, cudaMemcpyAsync(h->gchunks, gchunks.data(), gchunks.size() * sizeof(int32_t), cudaMemcpyHostToDevice, h->stream));
    CK(h, cudaMemcpyAsync(h->items_g, items_g.data(), items_g.size() * sizeof(ps::GridItem), cudaMemcpyHostToDevice,
                          h->stream));
    CK(h, cudaMemcpyAsync(h->gchunks_g, gchunks_g.data(), gchunks_g.size() * sizeof(int32_t), cudaMemcpyHostToDevice,
                          h->stream));
    CK(h, cudaMemcpyAsync(h->vblk, vblk.data(), vblk.size() * sizeof(uint16_t), cudaMemcpyHostToDevice, h->stream));
    CK(h, ps::nufft_row_weights(h));
    // Measurements into sorted order.
    ps_status st = stage_in(h, vis, 4 * (size_t)M * sizeof(float2), device_ptrs, h->vtmp);
    if (st != PS_OK) return st;
    CK(h, ps::gather_vis(h, h->vtmp, h->Y));
  }
  CK(h, cudaStreamSynchronize(h->stream));
  h->have_meas = true;
  ps_status st = opnorm_lanczos(h);
  if (st != PS_OK) return st;
  set_default_steps(h);
  if ((st = default_gamma(h)) != PS_OK) return st;
  return reset_state(h);
}

// Largest eigenvalue of the symmetric tridiagonal matrix with diagonal a and
// off-diagonal b (|b| = |a| - 1), by bisection on the Sturm count.
static double tridiag_max_eig(const std::vector<double>& a, const std::vector<double>& b) {
  const size_t k = a.size();
  double lo = a[0], hi = a[0];
  for (size_t i = 0; i < k; ++i) {
    const double r = (i > 0 ? std::fabs(b[i - 1]) : 0.0) + (i + 1 < k ? std::fabs(b[i]) : 0.0);
    lo = std::min(lo, a[i] - r);
    hi = std::max(hi, a[i] + r);
  }
  auto below = [&](double x) {   // number of eigenvalues < x
    int cnt = 0;
    double q = a[0] - x;
    for (size_t i = 0;; ++i) {
      if (q == 0.0) q = -1e-300;
      if (q < 0) ++cnt;
      if (i + 1 == k) break;
      q = a[i + 1] - x - b[i] * b[i] / q;
    }
    return cnt;
  };
  for (int it = 0; it < 200 && hi - lo > 1e-15 * std::max(std::fabs(hi), 1e-300); ++it) {
    const double mid = 0.5 * (lo + hi);
    if (below(mid) >= (int)k) hi = mid;
    else lo = mid;
  }
  return 0.5 * (lo + hi);
}

// ||phi||_sp^2, the step-size bound of Section 4.3.3, as the largest eigenvalue of
// phi^dagger phi by Lanczos iterations (three-term recurrence, FP32 vectors, FP64
// coefficients; the largest Ritz value rises monotonically to it). Stops when that
// value changes by <= 1e-9 relative, or the Krylov space is invariant. Scratch: tmp4,
// Xb and Adj (all cleared by the caller's reset of the state).
static ps_status opnorm_lanczos(Handle* h) {
  h->opnorm_sq = 0.0;
  if (h->M == 0) return PS_OK;
  const size_t N4 = 4 * (size_t)h->N;
  std::vector<float> x(N4);
  uint64_t s = 0x9E3779B97F4A7C15ull;
  double nrm = 0.0;
  for (size_t i = 0; i < N4; ++i) {
    s = s * 6364136223846793005ull + 1442695040888963407ull;
    x[i] = (float)((double)(s >> 11) / 9007199254740992.0 - 0.5);
    nrm += (double)x[i] * x[i];
  }
  const float inv = (float)(1.0 / std::sqrt(nrm));
  for (auto& v : x) v *= inv;
  float *v = h->tmp4, *u = h->Xb, *w = h->Adj;   // current, previous and new Lanczos vectors
  // On the handle's (non-blocking) stream, so the iterations below are ordered after the copy.
  CK(h, cudaMemcpyAsync(v, x.data(), N4 * sizeof(float), cudaMemcpyHostToDevice, h->stream));
  CK(h, cudaMemsetAsync(u, 0, N4 * sizeof(float), h->stream));
  double* dres = h->red + (size_t)h->red_cap - 600;
  std::vector<double> al, be;
  double theta = 0.0, beta = 0.0;
  for (int j = 0; j < 300; ++j) {
    CK(h, ps::nufft_forward_grid(h, v));
    CK(h, ps::nufft_degrid(h, ps::DEG_APPLY, h->vtmp));
    CK(h, ps::nufft_grid(h, h->vtmp, 0));
    CK(h, ps::nufft_adjoint_image(h, w));
    CK(h, ps::reduce_dot(h, w, v, N4, dres));
    CK(h, cudaMemcpyAsync(h->red_host, dres, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    const double alpha = h->red_host[0];
    if (!std::isfinite(alpha)) return fail(h, PS_ENONFINITE, "Lanczos: non-finite phi^dagger phi x");
    CK(h, ps::lanczos_update(h, w, v, u, N4, alpha, beta));
    CK(h, ps::reduce_dot(h, w, w, N4, dres + 1));
    CK(h, cudaMemcpyAsync(h->red_host + 1, dres + 1, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    const double beta_new = std::sqrt(h->red_host[1]);
    if (!std::isfinite(beta_new)) return fail(h, PS_ENONFINITE, "Lanczos: non-finite phi^dagger phi x");
    al.push_back(alpha);
    const double theta_new = tridiag_max_eig(al, be);
    if (!(theta_new > 0)) return fail(h, PS_ENONFINITE, "Lanczos: zero phi^dagger phi x");
    const bool done = (j >= 4 && std::fabs(theta_new - theta) <= 1e-9 * theta_new) || beta_new <= 1e-12 * theta_new;
    theta = theta_new;
    if (done) break;
    be.push_back(beta_new);
    CK(h, ps::scale_copy(h, w, u, N4, 1.0 / beta_new));   // the new vector over the previous one
    std::swap(u, v);
    beta = beta_new;
  }
  h->opnorm_sq = theta;
  return PS_OK;
}

// gamma of step 6: cfg.gamma, else 1e-3 max|Psi^dagger phi^dagger Y| / ||phi||^2 (image
// units; 1 without data); then the thresholds gamma W with W = 1. Scratch: Adj and A,
// which the caller's reset of the state clears.
static ps_status default_gamma(Handle* h) {
  if (h->cfg.gamma > 0) {
    h->gamma_default = h->cfg.gamma;
  } else if (h->M > 0 && h->opnorm_sq > 0) {
    double* dres = h->red + (size_t)h->red_cap - 600;
    CK(h, ps::nufft_grid(h, h->Y, 0));
    CK(h, ps::nufft_adjoint_image(h, h->Adj));
    CK(h, ps::dirac_apply(h, h->Adj, h->A, nullptr, ps::SARA_APPLY, 1.0f / 3.0f, 0.f, 0.f));
    CK(h, ps::sara_analysis(h, h->Adj, h->A, nullptr, ps::SARA_APPLY, 1.0f / 3.0f, 0.f, 0.f));
    CK(h, ps::max_abs(h, h->A, 36 * (size_t)h->N, dres + 8));
    CK(h, cudaMemcpyAsync(h->red_host, dres + 8, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    const double g = 1e-3 * h->red_host[0] / h->opnorm_sq;
    if (!std::isfinite(g)) return fail(h, PS_ENONFINITE, "set_measurements: non-finite phi^dagger Y");
    h->gamma_default = g > 0 ? g : 1.0;
  } else {
    h->gamma_default = 1.0;
  }
  h->gamma = h->gamma_default;
  const size_t len = 36 * (size_t)h->N;
  k_fill4<<<1024, 256, 0, h->stream>>>(reinterpret_cast<float4*>(h->T), len / 4, (float)h->gamma);
  CK(h, cudaGetLastError());
  return PS_OK;
}

ps_status ps_set_sara_weights(ps_handle* h, const float* W, double gamma, int32_t device_ptrs) {
  if (!h) return PS_EINVAL;
  CHECK_ALIGN(h, W, device_ptrs, "set_sara_weights");
  if (gamma == 0) gamma = h->gamma_default;
  if (!(gamma > 0) || !std::isfinite(gamma))
    return fail(h, PS_EINVAL, "set_sara_weights: gamma must be > 0 (or 0 for the handle's gamma)");
  const size_t len = 36 * (size_t)h->N;
  if (W) {
    ps_status st = stage_in(h, W, len * sizeof(float), device_ptrs, h->T);
    if (st != PS_OK) return st;
    CK(h, ps::scale_copy(h, h->T, h->T, len, gamma));
  } else {   // W = 1: gamma W filled on the device
    k_fill4<<<1024, 256, 0, h->stream>>>(reinterpret_cast<float4*>(h->T), len / 4, (float)gamma);
    CK(h, cudaGetLastError());
  }
  h->gamma = gamma;
  if (!device_ptrs) CK(h, cudaStreamSynchronize(h->stream));
  return PS_OK;
}

ps_status ps_set_mode(ps_handle* h, int32_t mode) {
  if (!h) return PS_EINVAL;
  if (mode < PS_POLARIZED || mode > PS_L1TV_NC) return fail(h, PS_EINVAL, "set_mode: bad mode");
  if (ps::tv_mode(mode) != ps::tv_mode(h->mode)) {   // A changes meaning: start it from zero
    CK(h, cudaMemsetAsync(h->A, 0, 36 * (size_t)h->N * sizeof(float), h->stream));
    h->derived_valid = false;
  } else if (ps::tv_mode(mode) && mode != h->mode) {
    h->derived_valid = false;                          // the l1 part of Psi A may change
  }
  h->mode = mode;
  h->cfg.mode = mode;
  set_default_steps(h);
  drop_graph(h);
  ++h->version;
  return PS_OK;
}

ps_status ps_set_tv_weights(ps_handle* h, const double* tv, const double* l1) {
  if (!h) return PS_EINVAL;
  if (!tv) return fail(h, PS_EINVAL, "set_tv_weights: null TV weights");
  for (int i = 0; i < 4; ++i) {
    if (!(tv[i] >= 0) || !std::isfinite(tv[i])) return fail(h, PS_EINVAL, "set_tv_weights: weights must be >= 0");
    if (l1 && (!(l1[i] >= 0) || !std::isfinite(l1[i])))
      return fail(h, PS_EINVAL, "set_tv_weights: weights must be >= 0");
  }
  for (int i = 0; i < 4; ++i) {
    h->tv_mu[i] = tv[i];
    h->l1_mu[i] = l1 ? l1[i] : 0.0;
  }
  drop_graph(h);   // the weights are kernel arguments of the captured iteration
  ++h->version;
  return PS_OK;
}

ps_status ps_pd_iterate(ps_handle* h, int32_t n_iter, ps_stats* stats) {
  if (!h) return PS_EINVAL;
  if (n_iter < 0) return fail(h, PS_EINVAL, "pd_iterate: n_iter < 0");
  if (!h->have_meas) return fail(h, PS_ESTATE, "pd_iterate: call ps_set_measurements first");
  if (n_iter > 0) {
    if (!h->derived_valid) {
      ps_status st = compute_derived(h);
      if (st != PS_OK) return st;
    }
    if (!h->graph || h->graph_mode != h->mode) {
      ps_status st = build_graph(h);
      if (st != PS_OK) return st;
    }
    int i = 0;
    for (; i + ps::kGraphIters <= n_iter; i += ps::kGraphIters) CK(h, cudaGraphLaunch(h->graph_multi, h->stream));
    for (; i < n_iter; ++i) CK(h, cudaGraphLaunch(h->graph, h->stream));
    h->iterations += n_iter;
  }
  return stats ? ps_compute_stats(h, 0.0, stats) : PS_OK;
}

ps_status ps_reweight(ps_handle* h, double delta) {
  if (!h) return PS_EINVAL;
  if (!(delta > 0) || !std::isfinite(delta)) return fail(h, PS_EINVAL, "reweight: delta must be > 0");
  if (ps::tv_mode(h->mode)) return fail(h, PS_ESTATE, "reweight: the TV modes have no SARA weights");
  CK(h, ps::dirac_apply(h, h->S, nullptr, h->T, ps::SARA_REWEIGHT, 1.0f / 3.0f, (float)h->gamma, (float)delta));
  CK(h, ps::sara_analysis(h, h->S, nullptr, h->T, ps::SARA_REWEIGHT, 1.0f / 3.0f, (float)h->gamma, (float)delta));
  return PS_OK;
}

static ps_status copy_out(Handle* h, const void* dsrc, void* dst, size_t bytes, int device_ptrs) {
  CK(h, cudaMemcpyAsync(dst, dsrc, bytes, device_ptrs ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, h->stream));
  if (!device_ptrs) CK(h, cudaStreamSynchronize(h->stream));
  return PS_OK;
}

ps_status ps_get_stokes(ps_handle* h, float* out, int32_t device_ptrs) {
  if (!h || !out) return h ? fail(h, PS_EINVAL, "get_stokes: null output") : PS_EINVAL;
  CHECK_ALIGN(h, out, device_ptrs, "get_stokes");
  return copy_out(h, h->S, out, 4 * (size_t)h->N * sizeof(float), device_ptrs);
}

ps_status ps_get_sara_weights(ps_handle* h, float* out, int32_t device_ptrs) {
  if (!h || !out) return h ? fail(h, PS_EINVAL, "get_sara_weights: null output") : PS_EINVAL;
  CHECK_ALIGN(h, out, device_ptrs, "get_sara_weights");
  return copy_out(h, h->T, out, 36 * (size_t)h->N * sizeof(float), device_ptrs);
}

ps_status ps_get_state(ps_handle* h, const ps_state_view* v) {
  if (!h || !v) return PS_EINVAL;
  for (const void* p : {(const void*)v->S, (const void*)v->Z, (const void*)v->A, (const void*)v->B, (const void*)v->C,
                        (const void*)v->D})
    CHECK_ALIGN(h, p, v->device_ptrs, "get_state");
  const size_t N = h->N;
  const int dp = v->device_ptrs;
  ps_status st;
  if (v->S && (st = copy_out(h, h->S, v->S, 4 * N * sizeof(float), dp)) != PS_OK) return st;
  if (v->Z && (st = copy_out(h, h->Z, v->Z, 2 * N * sizeof(float), dp)) != PS_OK) return st;
  if (v->A && (st = copy_out(h, h->A, v->A, 36 * N * sizeof(float), dp)) != PS_OK) return st;
  if (v->C && (st = copy_out(h, h->C, v->C, 4 * N * sizeof(float), dp)) != PS_OK) return st;
  if (v->D && (st = copy_out(h, h->D, v->D, 2 * N * sizeof(float), dp)) != PS_OK) return st;
  if (v->B && h->M > 0) {
    float2* tmp = nullptr;
    CK(h, dalloc(h, &tmp, 4 * (size_t)h->M));
    cudaError_t e = cudaMemcpyAsync(h->vtmp, h->R, 4 * (size_t)h->M * sizeof(float2), cudaMemcpyDeviceToDevice, h->stream);
    if (e == cudaSuccess) e = ps::scale_vis(h, h->vtmp);
    if (e == cudaSuccess) e = ps::scatter_vis(h, h->vtmp, tmp);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(v->B, tmp, 4 * (size_t)h->M * sizeof(float2),
                          dp ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    dfree(h, tmp, 4 * (size_t)h->M);
    CK(h, e);
  }
  return PS_OK;
}

ps_status ps_set_state(ps_handle* h, const ps_state_view* v) {
  if (!h || !v) return PS_EINVAL;
  for (const void* p : {(const void*)v->S, (const void*)v->Z, (const void*)v->A, (const void*)v->B, (const void*)v->C,
                        (const void*)v->D})
    CHECK_ALIGN(h, p, v->device_ptrs, "set_state");
  if (!h->have_meas) return fail(h, PS_ESTATE, "set_state: call ps_set_measurements first");
  const size_t N = h->N;
  const int dp = v->device_ptrs;
  ps_status st;
  if (v->S && (st = stage_in(h, v->S, 4 * N * sizeof(float), dp, h->S)) != PS_OK) return st;
  if (v->Z && (st = stage_in(h, v->Z, 2 * N * sizeof(float), dp, h->Z)) != PS_OK) return st;
  if (v->A && (st = stage_in(h, v->A, 36 * N * sizeof(float), dp, h->A)) != PS_OK) return st;
  if (v->C && (st = stage_in(h, v->C, 4 * N * sizeof(float), dp, h->C)) != PS_OK) return st;
  if (v->D && (st = stage_in(h, v->D, 2 * N * sizeof(float), dp, h->D)) != PS_OK) return st;
  if (v->B && h->M > 0) {
    if ((st = stage_in(h, v->B, 4 * (size_t)h->M * sizeof(float2), dp, h->vtmp)) != PS_OK) return st;
    CK(h, ps::gather_vis(h, h->vtmp, h->R));
    k_fill<<<(h->nblocks + 127) / 128, 128, 0, h->stream>>>(h->cb, h->nblocks, 1.0f);
    CK(h, cudaGetLastError());
  }
  if (!dp) CK(h, cudaStreamSynchronize(h->stream));
  h->derived_valid = false;
  ++h->version;
  return PS_OK;
}

ps_status ps_get_config(const ps_handle* h, ps_config* out) {
  if (!h || !out) return PS_EINVAL;
  *out = h->cfg;
  out->mode = h->mode;
  out->gamma = h->gamma_default;
  return PS_OK;
}

ps_status ps_get_params(ps_handle* h, double* tau, double* rho1, double* rho2, double* rho3, double* opnorm_sq) {
  if (!h) return PS_EINVAL;
  if (tau) *tau = h->tau;
  if (rho1) *rho1 = h->rho1;
  if (rho2) *rho2 = h->rho2;
  if (rho3) *rho3 = h->rho3;
  if (opnorm_sq) *opnorm_sq = h->opnorm_sq;
  return PS_OK;
}

// Relative change per map (Eq. stop_crit) from the FP64 partials k_primal wrote: 0/0 = 0
// (a map that stayed zero), x/0 = +inf. Non-finite sums mean a NaN or infinity in S.
// Enqueues on the handle's stream: one small kernel that sums the last iteration's
// relative-change partials (FP64) and writes the 8 sums and the device flags straight into the
// mapped host buffer relc_host (no copy), and the event that marks them written.
static ps_status relc_enqueue(Handle* h) {
  CK(h, ps::relc_sums(h, sweep_blocks_host(h->N), h->relc_dev));
  CK(h, cudaEventRecord(h->relc_ev, h->stream));
  h->relc_pending = true;
  return PS_OK;
}

// The relative change from the landed sums (and the flags copied with them).
static ps_status relc_finish(Handle* h, double* out4) {
  h->relc_pending = false;
  const int* f = reinterpret_cast<const int*>(h->relc_host + 8);
  if (f[0]) {
    CK(h, cudaMemsetAsync(h->dev_flags, 0, 4 * sizeof(int), h->stream));
    return fail(h, PS_ETIMEOUT, "a bounded device wait (bulk-copy barrier) gave up; results of that launch are invalid");
  }
  bool finite = true;
  for (int c = 0; c < 4; ++c) {
    const double num = h->relc_host[c], den = h->relc_host[4 + c];
    finite = finite && std::isfinite(num) && std::isfinite(den);
    out4[c] = den > 0 ? std::sqrt(num / den) : (num > 0 ? INFINITY : 0.0);
  }
  if (!finite) return fail(h, PS_ENONFINITE, "the state holds a NaN or an infinity (relative-change sums are not finite)");
  return PS_OK;
}

static ps_status ensure_tmp36(Handle* h) {
  if (!h->tmp36) CK(h, dalloc(h, &h->tmp36, 36 * (size_t)h->N));
  return PS_OK;
}

ps_status ps_compute_stats(ps_handle* h, double zeta_sigma, ps_stats* out) {
  if (!h || !out) return PS_EINVAL;
  if (!h->have_meas) return fail(h, PS_ESTATE, "compute_stats: call ps_set_measurements first");
  if (!(zeta_sigma > 0)) zeta_sigma = h->cfg.zeta_sigma;
  const size_t N = h->N;
  double* dres = h->red + (size_t)h->red_cap - 600;
  // Relative change of the last iteration (from the partials written by k_primal).
  out->stop_flags = 0;
  out->converged = 0;
  {
    ps_status st = relc_enqueue(h);
    if (st != PS_OK) return st;
    CK(h, cudaStreamSynchronize(h->stream));
    st = relc_finish(h, out->rel_change);
    if (st != PS_OK) return st;
  }
  // Residual Y - phi(S) per block, and the residual image.
  std::vector<double> bsum(h->nblocks);
  double rms = 0.0;
  if (h->M > 0) {
    CK(h, ps::nufft_forward_grid(h, h->S));
    CK(h, ps::nufft_degrid(h, ps::DEG_RESID, h->vtmp));
    CK(h, cudaMemcpyAsync(bsum.data(), h->block_sum, bsum.size() * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    CK(h, ps::nufft_grid(h, h->vtmp, 0));
    CK(h, ps::nufft_adjoint_image(h, h->tmp4));
    CK(h, ps::reduce_dot(h, h->tmp4, h->tmp4, N, dres));
    CK(h, cudaMemcpyAsync(h->red_host, dres, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    rms = std::sqrt(h->red_host[0] / (double)N);
  }
  CK(h, cudaStreamSynchronize(h->stream));
  if (out->block_residual)
    for (int b = 0; b < std::min(out->nblocks, h->nblocks); ++b) out->block_residual[b] = std::sqrt(bsum[b]);
  out->zeta = h->psf_peak > 0 ? zeta_sigma * rms / h->psf_peak : 0.0;
  CK(h, ps::violation_count(h, h->S, out->zeta, dres + 2));
  ps_status st = ensure_tmp36(h);
  if (st != PS_OK) return st;
  CK(h, ps::dirac_apply(h, h->S, h->tmp36, nullptr, ps::SARA_APPLY, 1.0f / 3.0f, 0.f, 0.f));
  CK(h, ps::sara_analysis(h, h->S, h->tmp36, nullptr, ps::SARA_APPLY, 1.0f / 3.0f, 0.f, 0.f));
  CK(h, ps::weighted_l1(h, h->tmp36, h->T, dres + 4));
  CK(h, cudaMemcpyAsync(h->red_host, dres, 6 * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  CK(h, cudaStreamSynchronize(h->stream));
  out->violations = (int64_t)h->red_host[2];
  out->violations_raw = (int64_t)h->red_host[3];
  out->weighted_l1 = h->red_host[4];
  out->iterations = h->iterations;
  // Stopping rule of Section 5.5: every criterion that applies in the mode.
  int flags = 0;
  double rc = 0.0;
  for (int c = 0; c < h->cfg.stop_maps; ++c) rc = std::max(rc, out->rel_change[c]);
  if (rc <= h->cfg.rel_tol) flags |= PS_STOP_REL;
  bool fit = true;
  if (!ps::tv_mode(h->mode))
    for (int b = 0; b < h->nblocks; ++b) fit = fit && std::sqrt(bsum[b]) <= (1.0 + h->cfg.resid_tol) * h->eps_host[b];
  if (fit) flags |= PS_STOP_RESID;
  if (!ps::constrained_mode(h->mode) || 100.0 * (double)out->violations / (double)N <= h->cfg.np_tol)
    flags |= PS_STOP_NP;
  out->stop_flags = flags;
  out->converged = flags == (PS_STOP_REL | PS_STOP_RESID | PS_STOP_NP);
  return check_flags(h);
}

ps_status ps_apply_phi(ps_handle* h, const float* S, float* Y, int32_t device_ptrs) {
  if (!h || !S || !Y) return h ? fail(h, PS_EINVAL, "apply_phi: null pointer") : PS_EINVAL;
  CHECK_ALIGN(h, S, device_ptrs, "apply_phi");
  CHECK_ALIGN(h, Y, device_ptrs, "apply_phi");
  if (!h->have_meas) return fail(h, PS_ESTATE, "apply_phi: call ps_set_measurements first");
  if (h->M == 0) return PS_OK;
  const size_t N4 = 4 * (size_t)h->N, V = 4 * (size_t)h->M;
  const float* X = S;
  if (!device_ptrs) {
    CK(h, cudaMemcpyAsync(h->tmp4, S, N4 * sizeof(float), cudaMemcpyHostToDevice, h->stream));
    X = h->tmp4;
  }
  CK(h, ps::nufft_forward_grid(h, X));
  CK(h, ps::nufft_degrid(h, ps::DEG_APPLY, h->vtmp));
  if (device_ptrs) {
    CK(h, ps::scatter_vis(h, h->vtmp, (float2*)Y));
    return PS_OK;
  }
  float2* tmp = nullptr;
  CK(h, dalloc(h, &tmp, V));
  cudaError_t e = ps::scatter_vis(h, h->vtmp, tmp);
  if (e == cudaSuccess) e = cudaMemcpyAsync(Y, tmp, V * sizeof(float2), cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  dfree(h, tmp, V);
  CK(h, e);
  return PS_OK;
}

ps_status ps_apply_phi_adjoint(ps_handle* h, const float* Yin, float* S, int32_t device_ptrs) {
  if (!h || !Yin || !S) return h ? fail(h, PS_EINVAL, "apply_phi_adjoint: null pointer") : PS_EINVAL;
  CHECK_ALIGN(h, Yin, device_ptrs, "apply_phi_adjoint");
  CHECK_ALIGN(h, S, device_ptrs, "apply_phi_adjoint");
  if (!h->have_meas) return fail(h, PS_ESTATE, "apply_phi_adjoint: call ps_set_measurements first");
  const size_t N4 = 4 * (size_t)h->N, V = 4 * (size_t)h->M;
  float* out = device_ptrs ? S : h->tmp4;
  if (h->M == 0) {
    CK(h, cudaMemsetAsync(out, 0, N4 * sizeof(float), h->stream));
  } else if (device_ptrs) {
    CK(h, ps::gather_vis(h, (const float2*)Yin, h->vtmp));
  } else {
    float2* tmp = nullptr;
    CK(h, dalloc(h, &tmp, V));
    cudaError_t e = cudaMemcpyAsync(tmp, Yin, V * sizeof(float2), cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess) e = ps::gather_vis(h, tmp, h->vtmp);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    dfree(h, tmp, V);
    CK(h, e);
  }
  if (h->M > 0) {
    CK(h, ps::nufft_grid(h, h->vtmp, 0));
    CK(h, ps::nufft_adjoint_image(h, out));
  }
  if (!device_ptrs) return copy_out(h, h->tmp4, S, N4 * sizeof(float), 0);
  return PS_OK;
}

ps_status ps_apply_psi_adjoint(ps_handle* h, const float* S, float* A, int32_t device_ptrs) {
  if (!h || !S || !A) return h ? fail(h, PS_EINVAL, "apply_psi_adjoint: null pointer") : PS_EINVAL;
  CHECK_ALIGN(h, S, device_ptrs, "apply_psi_adjoint");
  CHECK_ALIGN(h, A, device_ptrs, "apply_psi_adjoint");
  const size_t N4 = 4 * (size_t)h->N;
  const float* X = S;
  float* coef = A;
  if (!device_ptrs) {
    ps_status st = ensure_tmp36(h);
    if (st != PS_OK) return st;
    CK(h, cudaMemcpyAsync(h->tmp4, S, N4 * sizeof(float), cudaMemcpyHostToDevice, h->stream));
    X = h->tmp4;
    coef = h->tmp36;
  }
  CK(h, ps::dirac_apply(h, X, coef, nullptr, ps::SARA_APPLY, 1.0f / 3.0f, 0.f, 0.f));
  CK(h, ps::sara_analysis(h, X, coef, nullptr, ps::SARA_APPLY, 1.0f / 3.0f, 0.f, 0.f));
  if (!device_ptrs) return copy_out(h, h->tmp36, A, 36 * (size_t)h->N * sizeof(float), 0);
  return PS_OK;
}

ps_status ps_apply_psi(ps_handle* h, const float* A, float* S, int32_t device_ptrs) {
  if (!h || !A || !S) return h ? fail(h, PS_EINVAL, "apply_psi: null pointer") : PS_EINVAL;
  CHECK_ALIGN(h, A, device_ptrs, "apply_psi");
  CHECK_ALIGN(h, S, device_ptrs, "apply_psi");
  const float* coef = A;
  float* out = S;
  if (!device_ptrs) {
    ps_status st = ensure_tmp36(h);
    if (st != PS_OK) return st;
    CK(h, cudaMemcpyAsync(h->tmp36, A, 36 * (size_t)h->N * sizeof(float), cudaMemcpyHostToDevice, h->stream));
    coef = h->tmp36;
    out = h->tmp4;
  }
  CK(h, ps::sara_synthesis(h, coef, out));
  if (!device_ptrs) return copy_out(h, h->tmp4, S, 4 * (size_t)h->N * sizeof(float), 0);
  return PS_OK;
}

ps_status ps_profile_stages(ps_handle* h, int32_t n_iter, double* stage_ms) {
  if (!h || !stage_ms || n_iter < 1) return h ? fail(h, PS_EINVAL, "profile_stages: bad arguments") : PS_EINVAL;
  if (!h->have_meas) return fail(h, PS_ESTATE, "profile_stages: call ps_set_measurements first");
  if (!h->derived_valid) {
    ps_status st = compute_derived(h);
    if (st != PS_OK) return st;
  }
  cudaEvent_t ev[PS_NSTAGES + 1];
  for (int i = 0; i <= PS_NSTAGES; ++i) CK(h, cudaEventCreate(&ev[i]));
  std::vector<double> acc(PS_NSTAGES, 0.0);
  cudaError_t e = cudaSuccess;
  for (int it = 0; it < n_iter && e == cudaSuccess; ++it) {
    e = one_iteration(h, ev);
    if (e == cudaSuccess) e = cudaEventSynchronize(ev[PS_NSTAGES]);
    for (int s = 0; s < PS_NSTAGES && e == cudaSuccess; ++s) {
      float ms = 0.f;
      e = cudaEventElapsedTime(&ms, ev[s], ev[s + 1]);
      acc[s] += ms;
    }
  }
  for (int i = 0; i <= PS_NSTAGES; ++i) cudaEventDestroy(ev[i]);
  CK(h, e);
  h->iterations += n_iter;
  for (int s = 0; s < PS_NSTAGES; ++s) stage_ms[s] = acc[s] / n_iter;
  return PS_OK;
}

// ---------------------------------------------------------------------------
// Autotuner: candidates per PS_TUNE_* slot, each timed on the handle's own data.
static const int kTuneCandidates[PS_TUNE_COUNT] = {3, 3, 5, 6};

// Mean milliseconds of `reps` launches of f after one untimed launch.
extern "C++" {
template <typename F>
ps_status tune_time(Handle* h, int reps, F f, double* ms) {
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  CK(h, cudaEventCreate(&e0));
  cudaError_t e = cudaEventCreate(&e1);
  if (e == cudaSuccess) e = f();
  if (e == cudaSuccess) e = cudaEventRecord(e0, h->stream);
  for (int r = 0; r < reps && e == cudaSuccess; ++r) e = f();
  if (e == cudaSuccess) e = cudaEventRecord(e1, h->stream);
  if (e == cudaSuccess) e = cudaEventSynchronize(e1);
  float t = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
  cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  CK(h, e);
  *ms = (double)t / reps;
  return PS_OK;
}
}  // extern "C++"

ps_status ps_autotune(ps_handle* h, int32_t reps, int32_t* choices, double* ms) {
  if (!h || reps < 1) return h ? fail(h, PS_EINVAL, "autotune: reps must be >= 1") : PS_EINVAL;
  if (!h->have_meas) return fail(h, PS_ESTATE, "autotune: call ps_set_measurements first");
  if (!h->derived_valid) {
    ps_status st = compute_derived(h);
    if (st != PS_OK) return st;
  }
  double best_ms[PS_TUNE_COUNT] = {0.0, 0.0, 0.0, 0.0};
  auto pick = [&](int slot, auto launch) -> ps_status {
    int best = 0;
    double best_t = 0.0;
    for (int v = 0; v < kTuneCandidates[slot]; ++v) {
      h->tune[slot] = v;
      double t = 0.0;
      ps_status st = tune_time(h, reps, launch, &t);
      if (st != PS_OK) return st;
      if (v == 0 || t < best_t) {
        best = v;
        best_t = t;
      }
    }
    h->tune[slot] = best;
    best_ms[slot] = best_t;
    return PS_OK;
  };
  // Analysis: the dual update of steps 5-6 as the iteration runs it (staged A and gamma W
  // reads), on scratch coefficients so the state's A is untouched.
  {
    ps_status st0 = ensure_tmp36(h);
    if (st0 != PS_OK) return st0;
    CK(h, cudaMemsetAsync(h->tmp36, 0, 36 * (size_t)h->N * sizeof(float), h->stream));
  }
  ps_status sta = pick(PS_TUNE_ANALYSIS, [&] {
    return ps::sara_analysis(h, h->S, h->tmp36, h->T, ps::SARA_DUAL, (float)(h->rho1 / 3.0), 0.f, 0.f);
  });
  if (sta != PS_OK) return sta;
  // Synthesis: Psi A of the current coefficients, written where it already is.
  ps_status st = pick(PS_TUNE_SYNTHESIS, [&] { return ps::sara_synthesis(h, h->A, h->PsiA); });
  if (st != PS_OK) return st;
  // Degridding as the iteration runs it (the dual update of steps 7-8 with its block sums),
  // from the spectrum of the current S, on a scratch copy of the dual: the candidates read and
  // write the visibility rows as in the iteration, and the state's dual is untouched.
  if (h->M > 0) {
    CK(h, ps::nufft_forward_grid(h, h->S));
    CK(h, cudaMemcpyAsync(h->vtmp, h->R, 4 * (size_t)h->M * sizeof(float2), cudaMemcpyDeviceToDevice, h->stream));
    float2* const R_state = h->R;
    h->R = h->vtmp;
    st = pick(PS_TUNE_DEGRID, [&] { return ps::nufft_degrid(h, ps::DEG_DUAL, nullptr); });
    h->R = R_state;
    if (st != PS_OK) return st;
    // Gridding: the current dual into the accumulator (an intermediate; phi^dagger B is kept).
    st = pick(PS_TUNE_GRID, [&] { return ps::nufft_grid(h, h->R, 1); });
    if (st != PS_OK) return st;
  }
  if (ps::tv_mode(h->mode)) h->derived_valid = false;   // the SARA synthesis timing wrote PsiA
  drop_graph(h);
  ++h->version;
  if (choices) std::memcpy(choices, h->tune, sizeof(h->tune));
  if (ms)
    for (int i = 0; i < PS_TUNE_COUNT; ++i) ms[i] = best_ms[i];
  return PS_OK;
}

ps_status ps_get_tuning(const ps_handle* h, int32_t* choices) {
  if (!h || !choices) return PS_EINVAL;
  std::memcpy(choices, h->tune, sizeof(h->tune));
  return PS_OK;
}

ps_status ps_set_tuning(ps_handle* h, const int32_t* choices) {
  if (!h || !choices) return h ? fail(h, PS_EINVAL, "set_tuning: null choices") : PS_EINVAL;
  for (int i = 0; i < PS_TUNE_COUNT; ++i)
    if (choices[i] < 0 || choices[i] >= kTuneCandidates[i])
      return fail(h, PS_EINVAL, "set_tuning: slot " + std::to_string(i) + " out of range");
  std::memcpy(h->tune, choices, sizeof(h->tune));
  drop_graph(h);
  ++h->version;
  return PS_OK;
}

int32_t ps_kernels_per_iteration(const ps_handle* h) {
  if (!h) return 0;
  int k = 1;                                   // k_primal
  if (ps::tv_mode(h->mode)) return k + 2 + (h->M > 0 ? 2 + 1 + 1 + 2 : 0);   // TV dual + adjoint, gradient chain
  if (h->mode != PS_NNLS) k += 2 * h->L;       // analysis + synthesis levels
  if (h->M > 0) k += 2 + 1 + 1 + 1 + 2;        // fwd rows/cols, degrid, block scale, grid, adj cols/rows
  return k;
}

ps_status ps_set_visibilities(ps_handle* h, const float* vis, int32_t device_ptrs) {
  if (!h || !vis) return h ? fail(h, PS_EINVAL, "set_visibilities: null pointer") : PS_EINVAL;
  if (!h->have_meas) return fail(h, PS_ESTATE, "set_visibilities: call ps_set_measurements first");
  CHECK_ALIGN(h, vis, device_ptrs, "set_visibilities");
  if (h->M == 0) return PS_OK;
  ps_status st = stage_in(h, vis, 4 * (size_t)h->M * sizeof(float2), device_ptrs, h->vtmp);
  if (st != PS_OK) return st;
  CK(h, ps::gather_vis(h, h->vtmp, h->Y));
  if (!device_ptrs) CK(h, cudaStreamSynchronize(h->stream));
  return PS_OK;
}

ps_status ps_get_rel_change(ps_handle* h, double* out4) {
  if (!h || !out4) return h ? fail(h, PS_EINVAL, "get_rel_change: null output") : PS_EINVAL;
  ps_status st = relc_enqueue(h);
  if (st != PS_OK) return st;
  CK(h, cudaStreamSynchronize(h->stream));
  return relc_finish(h, out4);
}

ps_status ps_rel_change_request(ps_handle* h) {
  if (!h) return PS_EINVAL;
  return relc_enqueue(h);
}

ps_status ps_rel_change_result(ps_handle* h, double* out4) {
  if (!h || !out4) return h ? fail(h, PS_EINVAL, "rel_change_result: null output") : PS_EINVAL;
  if (!h->relc_pending) return fail(h, PS_ESTATE, "rel_change_result: no ps_rel_change_request pending");
  CK(h, cudaEventSynchronize(h->relc_ev));
  return relc_finish(h, out4);
}

ps_status ps_max_abs_analysis(ps_handle* h, double* out) {
  if (!h || !out) return h ? fail(h, PS_EINVAL, "max_abs_analysis: null output") : PS_EINVAL;
  ps_status st = ensure_tmp36(h);
  if (st != PS_OK) return st;
  double* dres = h->red + (size_t)h->red_cap - 600;
  CK(h, ps::dirac_apply(h, h->S, h->tmp36, nullptr, ps::SARA_APPLY, 1.0f / 3.0f, 0.f, 0.f));
  CK(h, ps::sara_analysis(h, h->S, h->tmp36, nullptr, ps::SARA_APPLY, 1.0f / 3.0f, 0.f, 0.f));
  CK(h, ps::max_abs(h, h->tmp36, 36 * (size_t)h->N, dres + 8));
  CK(h, cudaMemcpyAsync(h->red_host, dres + 8, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  CK(h, cudaStreamSynchronize(h->stream));
  *out = h->red_host[0];
  return check_flags(h);
}

ps_status ps_debug_set_wait_polls(int32_t polls) {
  cudaError_t e = ps::set_wait_polls_sara(polls);
  if (e == cudaSuccess) e = ps::set_wait_polls_nufft(polls);
  // The copies run on the legacy stream, which non-blocking streams do not wait for.
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return fail(nullptr, PS_ECUDA, std::string("debug_set_wait_polls: ") + cudaGetErrorString(e));
  return PS_OK;
}

ps_status ps_wavelet_filters(double* out) {
  if (!out) return PS_EINVAL;
  double h[ps::kDb][ps::kMaxTaps];
  ps::daubechies_filters(h);
  std::memcpy(out, h, sizeof(h));
  return PS_OK;
}

}  // extern "C"
// Batches. Handles of one size class (same n and levels) keep their per-pixel state and SARA
// coefficients in class-wide slabs, problem after problem, so that the per-pixel sweep and
// the SARA transforms of the whole class run as single launches over 4 P maps (the kernels
// index maps across the consecutive problems); each problem's NUFFT chain stays on its own
// stream. The slabs are filled from the handles' own arrays when the batch is made and
// copied back when it is destroyed.
struct BatchClass {
  std::vector<Handle*> hs;
  size_t N = 0;
  int red_cap = 0;
  float *S = nullptr, *Z = nullptr, *C = nullptr, *D = nullptr, *Xb = nullptr, *PsiA = nullptr, *Adj = nullptr;
  float *A = nullptr, *T = nullptr, *ap0 = nullptr, *ap1 = nullptr;
  double* red = nullptr;
  cudaStream_t s_main = nullptr, s_sara = nullptr;
  cudaEvent_t ev_primal = nullptr, ev_sara = nullptr;
  bool fused = false;   // the last graph ran this class through the class-wide launches
};

struct ps_batch {
  std::vector<Handle*> hs;
  std::vector<uint64_t> versions;
  std::vector<cudaEvent_t> join;
  std::vector<cudaEvent_t> pre;    // each handle's own pending work, ordered before the batch's launches
  std::vector<BatchClass> classes;
  int64_t slab_bytes = 0;
  cudaEvent_t fork = nullptr;
  cudaEvent_t done = nullptr;      // the batch's launches, ordered before each handle's later work
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  cudaGraphExec_t graph = nullptr;
};

static ps_status batch_fail(cudaError_t e, const char* what) {
  ps::set_global_error(std::string(what) + ": " + cudaGetErrorString(e));
  return e == cudaErrorMemoryAllocation ? PS_ENOMEM : PS_ECUDA;
}

// The slab arrays of a class, in the order of the Handle fields they replace, with their
// per-problem sizes in floats (red: doubles).
struct SlabField {
  float* Handle::*hp;
  float* BatchClass::*cp;
  size_t per_N;   // floats per problem = per_N * N
};
static const SlabField kSlabFields[] = {
    {&Handle::S, &BatchClass::S, 4},    {&Handle::Z, &BatchClass::Z, 2},       {&Handle::C, &BatchClass::C, 4},
    {&Handle::D, &BatchClass::D, 2},    {&Handle::Xb, &BatchClass::Xb, 4},     {&Handle::PsiA, &BatchClass::PsiA, 4},
    {&Handle::Adj, &BatchClass::Adj, 4}, {&Handle::A, &BatchClass::A, 36},     {&Handle::T, &BatchClass::T, 36},
    {&Handle::approx, &BatchClass::ap0, 8}, {&Handle::approx2, &BatchClass::ap1, 8}};

static void free_class_slabs(BatchClass& c) {
  for (const SlabField& f : kSlabFields)
    if (c.*(f.cp)) {
      cudaFree(c.*(f.cp));
      c.*(f.cp) = nullptr;
    }
  if (c.red) cudaFree(c.red);
  c.red = nullptr;
  if (c.s_main) cudaStreamDestroy(c.s_main);
  if (c.s_sara) cudaStreamDestroy(c.s_sara);
  if (c.ev_primal) cudaEventDestroy(c.ev_primal);
  if (c.ev_sara) cudaEventDestroy(c.ev_sara);
  c.s_main = c.s_sara = nullptr;
  c.ev_primal = c.ev_sara = nullptr;
}

// Moves every handle of the class into freshly allocated slabs (device-to-device copies of its
// arrays, then its own arrays freed). On failure nothing has moved.
static cudaError_t move_class_into_slabs(BatchClass& c, int64_t* bytes) {
  const size_t P = c.hs.size(), N = c.N;
  cudaError_t e = cudaSuccess;
  for (const SlabField& f : kSlabFields)
    if (e == cudaSuccess) e = cudaMalloc((void**)&(c.*(f.cp)), P * f.per_N * N * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc((void**)&c.red, P * (size_t)c.red_cap * sizeof(double));
  int prio_lo = 0, prio_hi = 0;
  cudaDeviceGetStreamPriorityRange(&prio_lo, &prio_hi);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&c.s_main, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&c.s_sara, cudaStreamNonBlocking, prio_hi);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c.ev_primal, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c.ev_sara, cudaEventDisableTiming);
  for (size_t p = 0; p < P && e == cudaSuccess; ++p) {
    Handle* h = c.hs[p];
    for (const SlabField& f : kSlabFields)
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(c.*(f.cp) + p * f.per_N * N, h->*(f.hp), f.per_N * N * sizeof(float),
                            cudaMemcpyDeviceToDevice, h->stream);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(c.red + p * c.red_cap, h->red, (size_t)c.red_cap * sizeof(double), cudaMemcpyDeviceToDevice,
                          h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  }
  if (e != cudaSuccess) {
    cudaGetLastError();
    free_class_slabs(c);
    return e;
  }
  for (size_t p = 0; p < P; ++p) {
    Handle* h = c.hs[p];
    cudaFree(h->approx);   // approx2 lies in the same allocation
    h->approx2 = nullptr;
    for (const SlabField& f : kSlabFields) {
      if (f.hp != &Handle::approx && f.hp != &Handle::approx2) cudaFree(h->*(f.hp));
      h->*(f.hp) = c.*(f.cp) + p * f.per_N * N;
    }
    cudaFree(h->red);
    h->red = c.red + p * c.red_cap;
    const int64_t moved = (int64_t)(112 * N * sizeof(float) + (size_t)c.red_cap * sizeof(double));
    h->bytes -= moved;
    *bytes += moved;
    h->in_slab = true;
    drop_graph(h);   // the handle's own graphs hold the old addresses
    ++h->version;
  }
  return cudaSuccess;
}

// Copies every handle of the class back into arrays of its own and frees the slabs. A handle
// whose allocation fails stays in the slabs (which are then kept).
static void move_class_out_of_slabs(BatchClass& c, int64_t* bytes) {
  const size_t N = c.N;
  bool all_out = true;
  for (size_t p = 0; p < c.hs.size(); ++p) {
    Handle* h = c.hs[p];
    if (!h->in_slab) continue;
    cudaStreamSynchronize(h->stream);
    float* own[sizeof(kSlabFields) / sizeof(kSlabFields[0])] = {};
    double* red = nullptr;
    float* ap = nullptr;
    cudaError_t e = cudaMalloc((void**)&ap, 16 * N * sizeof(float));
    size_t k = 0;
    for (const SlabField& f : kSlabFields) {
      if (f.hp == &Handle::approx) own[k] = ap;
      else if (f.hp == &Handle::approx2) own[k] = ap ? ap + 8 * N : nullptr;
      else if (e == cudaSuccess) e = cudaMalloc((void**)&own[k], f.per_N * N * sizeof(float));
      ++k;
    }
    if (e == cudaSuccess) e = cudaMalloc((void**)&red, (size_t)c.red_cap * sizeof(double));
    k = 0;
    for (const SlabField& f : kSlabFields) {
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(own[k], h->*(f.hp), f.per_N * N * sizeof(float), cudaMemcpyDeviceToDevice, h->stream);
      ++k;
    }
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(red, h->red, (size_t)c.red_cap * sizeof(double), cudaMemcpyDeviceToDevice, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) {
      cudaGetLastError();
      k = 0;
      for (const SlabField& f : kSlabFields) {
        if (f.hp != &Handle::approx && f.hp != &Handle::approx2 && own[k]) cudaFree(own[k]);
        ++k;
      }
      if (ap) cudaFree(ap);
      if (red) cudaFree(red);
      all_out = false;
      continue;
    }
    k = 0;
    for (const SlabField& f : kSlabFields) h->*(f.hp) = own[k++];
    h->red = red;
    const int64_t moved = (int64_t)(112 * N * sizeof(float) + (size_t)c.red_cap * sizeof(double));
    h->bytes += moved;
    *bytes -= moved;
    h->in_slab = false;
    drop_graph(h);
    ++h->version;
  }
  if (all_out) free_class_slabs(c);
}

extern "C" void ps_batch_destroy(ps_batch* b) {
  if (!b) return;
  if (b->stream) cudaStreamSynchronize(b->stream);
  if (b->graph) cudaGraphExecDestroy(b->graph);
  for (BatchClass& c : b->classes)
    if (c.S) move_class_out_of_slabs(c, &b->slab_bytes);
  for (cudaEvent_t e : b->join) cudaEventDestroy(e);
  for (cudaEvent_t e : b->pre) cudaEventDestroy(e);
  if (b->fork) cudaEventDestroy(b->fork);
  if (b->done) cudaEventDestroy(b->done);
  if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
  delete b;
}

extern "C" ps_status ps_batch_create(ps_handle* const* handles, int32_t count, void* cuda_stream, ps_batch** out) {
  if (!handles || !out || count < 1) {
    ps::set_global_error("batch_create: need at least one handle and an output pointer");
    return PS_EINVAL;
  }
  *out = nullptr;
  ps_batch* b = new ps_batch();
  for (int i = 0; i < count; ++i) {
    Handle* h = handles[i];
    if (!h || !h->have_meas) {
      ps_batch_destroy(b);
      ps::set_global_error("batch_create: every handle needs ps_set_measurements first");
      return PS_ESTATE;
    }
    if (h->in_slab) {
      ps_batch_destroy(b);
      ps::set_global_error("batch_create: a handle belongs to another batch");
      return PS_EINVAL;
    }
    for (Handle* o : b->hs)
      if (o == h || o->stream == h->stream) {
        ps_batch_destroy(b);
        ps::set_global_error("batch_create: handles must be distinct and on distinct streams");
        return PS_EINVAL;
      }
    b->hs.push_back(h);
    b->versions.push_back(0);
  }
  cudaError_t e;
  if (cuda_stream) {
    b->stream = (cudaStream_t)cuda_stream;
  } else if ((e = cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking)) != cudaSuccess) {
    ps_batch_destroy(b);
    return batch_fail(e, "batch_create: stream");
  } else {
    b->own_stream = true;
  }
  if ((e = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming)) != cudaSuccess ||
      (e = cudaEventCreateWithFlags(&b->done, cudaEventDisableTiming)) != cudaSuccess) {
    ps_batch_destroy(b);
    return batch_fail(e, "batch_create: event");
  }
  b->join.resize(count, nullptr);
  b->pre.resize(count, nullptr);
  for (int i = 0; i < count; ++i)
    if ((e = cudaEventCreateWithFlags(&b->join[i], cudaEventDisableTiming)) != cudaSuccess ||
        (e = cudaEventCreateWithFlags(&b->pre[i], cudaEventDisableTiming)) != cudaSuccess) {
      ps_batch_destroy(b);
      return batch_fail(e, "batch_create: event");
    }
  // Size classes (n, levels) in order of first appearance; classes of two or more handles get slabs.
  for (Handle* h : b->hs) {
    BatchClass* c = nullptr;
    for (BatchClass& x : b->classes)
      if (x.hs[0]->n == h->n && x.hs[0]->L == h->L) c = &x;
    if (!c) {
      b->classes.emplace_back();
      c = &b->classes.back();
      c->N = h->N;
      c->red_cap = h->red_cap;
    }
    c->hs.push_back(h);
  }
  for (BatchClass& c : b->classes) {
    if (c.hs.size() < 2) continue;
    if ((e = move_class_into_slabs(c, &b->slab_bytes)) != cudaSuccess) {
      ps_batch_destroy(b);
      return batch_fail(e, "batch_create: class slabs");
    }
  }
  *out = b;
  return PS_OK;
}

// Whether a class can take the class-wide launches in this graph: two or more handles, all in
// the same SARA mode with the same step sizes, each with measurements. The class-wide SARA
// launches take the first handle's SARA launch choices (they depend on the image size only);
// each NUFFT chain keeps its handle's own.
static bool class_fusable(const BatchClass& c) {
  if (c.hs.size() < 2 || !c.S) return false;
  const Handle* a = c.hs[0];
  if (ps::tv_mode(a->mode)) return false;
  for (const Handle* h : c.hs)
    if (h->mode != a->mode || h->tau != a->tau || h->rho1 != a->rho1 || h->rho3 != a->rho3 || h->M == 0 || !h->aux)
      return false;
  return true;
}

// Capture one iteration of every handle: fork from the batch stream; per fusable class the
// class-wide per-pixel sweep, then its SARA chain beside the problems' NUFFT chains; every
// other handle's iteration on its own stream; join back.
static ps_status batch_build(ps_batch* b) {
  for (Handle* h : b->hs) {
    if (!h->derived_valid) {
      ps_status st = compute_derived(h);
      if (st != PS_OK) {
        ps::set_global_error("batch: " + h->err);
        return st;
      }
    }
    cudaError_t e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return batch_fail(e, "batch: handle stream");
  }
  if (b->graph) {
    cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
  }
  cudaGraph_t graph = nullptr;
  cudaError_t e = cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return batch_fail(e, "batch: begin capture");
  cudaError_t err = cudaEventRecord(b->fork, b->stream);
  auto index_of = [&](const Handle* h) {
    for (size_t i = 0; i < b->hs.size(); ++i)
      if (b->hs[i] == h) return i;
    return (size_t)0;
  };
  for (BatchClass& c : b->classes) {
    c.fused = class_fusable(c);
    if (!c.fused) {
      for (Handle* h : c.hs) {
        const size_t i = index_of(h);
        if (err == cudaSuccess) err = cudaStreamWaitEvent(h->stream, b->fork, 0);
        if (err == cudaSuccess) err = one_iteration(h);
        if (err == cudaSuccess) err = cudaEventRecord(b->join[i], h->stream);
        if (err == cudaSuccess) err = cudaStreamWaitEvent(b->stream, b->join[i], 0);
      }
      continue;
    }
    // A view of the class as one problem of 4 P maps over the slabs.
    Handle v = *c.hs[0];
    const int P = (int)c.hs.size();
    v.S = c.S, v.Z = c.Z, v.C = c.C, v.D = c.D, v.Xb = c.Xb, v.PsiA = c.PsiA, v.Adj = c.Adj;
    v.A = c.A, v.T = c.T, v.approx = c.ap0, v.approx2 = c.ap1, v.red = c.red;
    v.nmaps = 4 * P;
    v.problems = P;
    v.stream = c.s_main;
    if (err == cudaSuccess) err = cudaStreamWaitEvent(c.s_main, b->fork, 0);
    if (err == cudaSuccess) err = ps::primal_sweep(&v);
    if (err == cudaSuccess) err = cudaEventRecord(c.ev_primal, c.s_main);
    if (v.mode != PS_NNLS) {
      v.stream = c.s_sara;
      if (err == cudaSuccess) err = cudaStreamWaitEvent(c.s_sara, c.ev_primal, 0);
      if (err == cudaSuccess) err = sara_chain(&v);
      if (err == cudaSuccess) err = cudaEventRecord(c.ev_sara, c.s_sara);
      if (err == cudaSuccess) err = cudaStreamWaitEvent(b->stream, c.ev_sara, 0);
    } else if (err == cudaSuccess) {
      err = cudaStreamWaitEvent(b->stream, c.ev_primal, 0);
    }
    for (Handle* h : c.hs) {
      const size_t i = index_of(h);
      if (err == cudaSuccess) err = cudaStreamWaitEvent(h->stream, c.ev_primal, 0);
      if (err == cudaSuccess) err = nufft_chain(h, nullptr);
      if (err == cudaSuccess) err = cudaEventRecord(b->join[i], h->stream);
      if (err == cudaSuccess) err = cudaStreamWaitEvent(b->stream, b->join[i], 0);
    }
  }
  e = cudaStreamEndCapture(b->stream, &graph);
  if (err != cudaSuccess || e != cudaSuccess) {
    if (graph) cudaGraphDestroy(graph);
    return batch_fail(err != cudaSuccess ? err : e, "batch: capture");
  }
  e = cudaGraphInstantiate(&b->graph, graph, cudaGraphInstantiateFlagUseNodePriority);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) return batch_fail(e, "batch: instantiate");
  for (size_t i = 0; i < b->hs.size(); ++i) b->versions[i] = b->hs[i]->version;
  return PS_OK;
}

extern "C" ps_status ps_batch_iterate(ps_batch* b, int32_t n_iter) {
  if (!b || n_iter < 0) {
    ps::set_global_error("batch_iterate: bad arguments");
    return PS_EINVAL;
  }
  if (n_iter == 0) return PS_OK;
  bool stale = (b->graph == nullptr);
  for (size_t i = 0; i < b->hs.size(); ++i) stale = stale || (b->versions[i] != b->hs[i]->version);
  if (stale) {
    // The handles' streams may have pending work of their own: order it before the graph.
    for (Handle* h : b->hs) {
      cudaError_t e = cudaStreamSynchronize(h->stream);
      if (e != cudaSuccess) return batch_fail(e, "batch: handle stream");
    }
    ps_status st = batch_build(b);
    if (st != PS_OK) return st;
  }
  // Work already queued on a handle's own stream (a reweight, new thresholds, a state
  // upload) runs before the batch's iterations, and the handle's later work after them.
  for (size_t i = 0; i < b->hs.size(); ++i) {
    cudaError_t e = cudaEventRecord(b->pre[i], b->hs[i]->stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(b->stream, b->pre[i], 0);
    if (e != cudaSuccess) return batch_fail(e, "batch: ordering");
  }
  for (int i = 0; i < n_iter; ++i) {
    cudaError_t e = cudaGraphLaunch(b->graph, b->stream);
    if (e != cudaSuccess) return batch_fail(e, "batch: graph launch");
  }
  cudaError_t e = cudaEventRecord(b->done, b->stream);
  for (size_t i = 0; i < b->hs.size() && e == cudaSuccess; ++i) e = cudaStreamWaitEvent(b->hs[i]->stream, b->done, 0);
  if (e != cudaSuccess) return batch_fail(e, "batch: ordering");
  for (Handle* h : b->hs) h->iterations += n_iter;
  return PS_OK;
}

extern "C" ps_status ps_batch_synchronize(ps_batch* b) {
  if (!b) return PS_EINVAL;
  cudaError_t e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess) return batch_fail(e, "batch: synchronize");
  for (Handle* h : b->hs) {
    ps_status st = check_flags(h);
    if (st != PS_OK) {
      ps::set_global_error("batch: " + h->err);
      return st;
    }
  }
  return PS_OK;
}

#pragma GCC visibility pop

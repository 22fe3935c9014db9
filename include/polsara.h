/*
 * polsara.h - C ABI of the GB300 Polarized SARA primal-dual imager.
 *
 * Polarized SARA (Birdi, Repetti & Wiaux, arXiv:1801.02417) recovers the four
 * Stokes maps S = [I, Q, U, V] (N = n*n pixels each) from full-polarization
 * visibilities Y = phi(S) + E (Section 2.1, Eq. RIME_disc) by solving
 *   min_S,Z  f(phi(S)) + i_U(S) + gamma ||Psi^dagger S||_{W,1} + i_V(Z)
 *            + i_E1(S_:,1, Z_:,1) + i_E2(S_:,2:4, Z_:,2)          (Eq. min_gen2)
 * with the primal-dual iteration of Algorithm 1, reweighted by Algorithm 2.
 * Every step of the iteration runs in this library's CUDA kernels.
 *
 * Conventions shared by every call
 *   - Stokes maps: float32, 4 planes of n*n in the order I, Q, U, V; each plane is
 *     row-major, pixel (p, q) at centred coordinates x = q - n/2, y = p - n/2.
 *   - Visibilities: complex64 interleaved (re, im), M rows of 4 correlations in the
 *     paper's order RR, RL, LR, LL (Section 2.1: S^T L = [I+Q, U+iV, U-iV, I-Q]).
 *   - Frequencies: float64, M rows of (omega_u, omega_v) in radians per pixel
 *     (|omega| < pi); phi uses the phase exp(-i (omega_u x + omega_v y)) of Eq. RIME.
 *   - SARA coefficients: float32, 4 maps x 9 bases x n*n; basis 0 is Dirac, basis b
 *     (1..8) the periodic orthonormal Daubechies db_b Mallat transform with
 *     `levels` levels; the concatenation is scaled by 1/3 (tight frame).
 *     Mallat layout of one n*n basis array at level l (m = n >> (l-1), h = m/2):
 *     rows [0,h) cols [h,m) x-high/y-low, rows [h,m) cols [0,h) x-low/y-high,
 *     rows [h,m) cols [h,m) x-high/y-high; the coarsest approximation fills the
 *     top-left (n >> levels)^2 block.
 *   - `device_ptrs` = 1: pointers are CUDA device pointers read/written on the
 *     handle's stream, and must be 16-byte aligned (else PS_EINVAL); 0: host
 *     pointers (the call then synchronises the stream).
 *   - Ownership: inputs are copied; outputs go to caller-allocated buffers; the
 *     handle owns all its device state until ps_destroy.
 *   - Errors: every call returns a ps_status; ps_last_error() holds a message.
 *     No call aborts the process. A CUDA error leaves the handle unusable
 *     (PS_ECUDA); an invalid argument leaves it unchanged (PS_EINVAL).
 */
#ifndef POLSARA_H
#define POLSARA_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ps_handle ps_handle;

typedef enum {
  PS_OK = 0,
  PS_EINVAL = 1,      /* invalid argument (size, pointer, mode) */
  PS_ENOMEM = 2,      /* device allocation failed */
  PS_ECUDA = 3,       /* a CUDA runtime call or kernel failed */
  PS_ETIMEOUT = 4,    /* a bounded device wait gave up */
  PS_ENONFINITE = 5,  /* a NaN/Inf was detected in the state */
  PS_ESTATE = 6       /* call out of order (e.g. iterate before set_measurements) */
} ps_status;

/* Problem variants (Section 4.2, Section 4.3.4, Section 5.2). */
enum {
  PS_POLARIZED = 0,      /* Algorithm 1 in full: S, Z, A, B, C, D */
  PS_NO_CONSTRAINT = 1,  /* S, A, B only, with P_U' (Stokes I >= 0) */
  PS_NNLS = 2,           /* S, B only, with P_U' and g = 0: the initialisation of Alg. 2 */
  PS_SOC = 3,            /* not in the paper: the problem of PS_POLARIZED with the polarization
                            constraint (Eq. pol_const, a second-order cone per pixel) given one
                            dual C under the identity, C = C~ - rho3 P_P(C~/rho3) with the
                            closed-form cone projection, instead of the epigraph split of
                            Section 4.3.1: S, A, B, C only (no Z, D; 32 bytes/pixel less) */
  /* The TV problems of Section 4.4 (Algorithm 3, Eqs. Akiyama and Akiyama_2): data term
   * 1/2 ||Y L^-1 - phi(S) L^-1||^2 by its gradient 1/2 phi^dagger(phi(S) - Y) (no B, no l2
   * ball), sparsity prior sum_i mu_i ||grad S_i||_{2,1} (TV) or that plus sum_i nu_i
   * ||S_i||_1 (l1 + TV), grad = periodic forward differences; weights from
   * ps_set_tv_weights. The dual A of the prior lives in the SARA coefficient array:
   * A_tv of map c in its planes 0 (x) and 1 (y), A_l1 in plane 2 (ps_get/set_state). */
  PS_TV = 4,             /* TV with the polarization constraint: S, Z, A, C, D (steps 3-10) */
  PS_TV_NC = 5,          /* TV without it: S, A only, with P_U' (Stokes I >= 0) */
  PS_L1TV = 6,           /* l1 + TV with the constraint */
  PS_L1TV_NC = 7         /* l1 + TV without it */
};

typedef struct {
  int32_t n;             /* image side: power of two, 16 <= n <= 2048 */
  int32_t levels;        /* wavelet levels, 1 <= levels, n divisible by 2^levels */
  int32_t mode;          /* PS_POLARIZED | PS_NO_CONSTRAINT | PS_NNLS | PS_SOC | PS_TV .. PS_L1TV_NC */
  int32_t literal_ball;  /* 0: l2-ball radius eps (Moreau reading of Alg. 1 step 8);
                            1: the printed radius eps / rho2 */
  int32_t kernel_width;  /* NUFFT interpolation width W: 5, 7 or 9; 0 => 7 */
  int32_t stop_maps;     /* maps the relative-change rule of Eq. stop_crit takes: 3 = I, Q, U as printed
                            (the paper's V is zero), 4 or 0 = all four (V included; a map that stays
                            zero counts 0) */
  double tau, rho1, rho2, rho3;  /* step sizes; 0 => default of Section 4.3.3:
                                    rho1 = rho3 = 1, rho2 = 1/||phi||^2,
                                    tau = 0.99 / (sum of rho_i ||K_i||^2 in the mode) */
  double alpha;          /* NUFFT oversampling factor of the grid K = alpha n (Section 5.1 leaves it
                            open); 0 => 2, the only value accepted */
  double gamma;          /* gamma of Algorithm 1 step 6 (Section 4.2: it only affects the speed of
                            convergence); 0 => 1e-3 max|Psi^dagger phi^dagger Y| / ||phi||^2, computed by
                            ps_set_measurements (image units: phi^dagger phi peaks at ||phi||^2) */
  double noise_sigma;    /* sigma of the noise E (variance sigma^2 / 2 per real and imaginary part);
                            used only when ps_set_measurements receives eps = NULL, for the chi^2
                            bound of Section 5.1 */
  double rel_tol;        /* epsilon of Eq. stop_crit (relative change per map); 0 => 1e-5 */
  double resid_tol;      /* vartheta of Section 5.5: ||phi(S) - Y||_b <= (1 + vartheta) eps_b; 0 => 5e-3 */
  double np_tol;         /* varrho of Section 5.5: N_p <= varrho, in percent of the pixels; 0 => 0.5 */
  double zeta_sigma;     /* zeta = zeta_sigma x rms of the Stokes I residual image (Section 5.2); 0 => 3 */
} ps_config;

/* Criteria of the stopping rule of Section 5.5 (bits of ps_stats.stop_flags). */
enum {
  PS_STOP_REL = 1,     /* max_i ||S_i^(k+1) - S_i^(k)|| / ||S_i^(k)|| <= rel_tol over the first stop_maps
                          maps (Eq. stop_crit) */
  PS_STOP_RESID = 2,   /* ||phi(S) - Y||_b <= (1 + resid_tol) eps_b for every block */
  PS_STOP_NP = 4       /* N_p = 100 violations / N <= np_tol */
};

typedef struct {
  int32_t nblocks;          /* number of l2 blocks the next fields describe */
  int32_t stop_flags;       /* out: PS_STOP_* criteria met (criteria that do not apply in the mode count
                               as met: the residual rule in the TV modes, which have no l2 ball, and the
                               N_p rule in the modes without the polarization constraint) */
  double* block_residual;   /* out, nblocks entries (may be NULL): ||phi(S) - Y||_2 per block */
  double rel_change[4];     /* ||S_i^(k+1) - S_i^(k)|| / ||S_i^(k)|| of the last iteration (Eq. stop_crit),
                               0 for a map that stayed zero, +inf for a map that left zero */
  double zeta;              /* violation threshold used (Section 5.2) */
  int64_t violations;       /* pixels with -I + ||(Q,U,V)|| > zeta */
  int64_t violations_raw;   /* pixels with -I + ||(Q,U,V)|| > 0 */
  double weighted_l1;       /* sum |T .* Psi^dagger S| (gamma ||Psi^dagger S||_{W,1}) */
  int64_t iterations;       /* iterations run on this handle */
  int32_t converged;        /* out: 1 when every PS_STOP_* criterion holds (Section 5.5), else 0 */
  int32_t reserved;
} ps_stats;

/* Primal and dual state of Algorithm 1 (the warm start Algorithm 2 passes on).
 * Each pointer may be NULL to skip that array. Sizes: S, C: 4N floats; Z, D: 2N
 * floats; A: 36N floats; B: M x 4 complex64 (8M floats), rows in the caller's
 * visibility order. */
typedef struct {
  float* S; float* Z; float* A; float* B; float* C; float* D;
  int32_t device_ptrs;
  int32_t reserved;
} ps_state_view;

/* Create a handle for one imaging problem (Section 4). `cuda_stream` is a
 * cudaStream_t the handle launches on (NULL: the handle creates its own).
 * Validates cfg (n power of two, levels, mode). */
ps_status ps_create(const ps_config* cfg, void* cuda_stream, ps_handle** out);

/* Release every device buffer of the handle. NULL is accepted. */
void ps_destroy(ps_handle* h);

/* Message of the last failed call on `h` (or of the last failed ps_create when
 * h is NULL). Valid until the next call on the handle. */
const char* ps_last_error(const ps_handle* h);

/* Measurements of the data model Y = phi(S) + E (Section 2.1, Eq. RIME_disc) and
 * the l2 balls of the data-fidelity term (Eq. f_diff), one per block.
 *   M              rows (0 allowed: no data term)
 *   uv             M x 2 float64, radians per pixel, |omega| < pi
 *   vis            M x 4 complex64 (RR, RL, LR, LL)
 *   weights        M float32 per-row weights w_m >= 0 (phi = diag(w) F ...), NULL = 1
 *   nblocks        number of l2 blocks (>= 1 when M > 0)
 *   block_offsets  nblocks+1 int64, increasing, [0] = 0, [nblocks] = M
 *   eps            nblocks float64 radii eps_b > 0, or NULL: the chi^2 bound of Section 5.1 from
 *                  cfg.noise_sigma, eps_b^2 = (8 M_b + 2 sqrt(16 M_b)) sigma^2 / 2 (8 M_b real degrees
 *                  of freedom of variance sigma^2 / 2, two standard deviations above the mean;
 *                  PS_EINVAL if noise_sigma <= 0)
 *   device_ptrs    for uv, vis, weights (block_offsets and eps are host arrays)
 * Sorts the rows by interpolation tile, estimates ||phi||^2 by Lanczos iterations,
 * sets the default step sizes and (cfg.gamma = 0) the default gamma, fills the
 * thresholds with gamma W, W = 1, and resets the state to zero.
 * Precision: the Lanczos vectors and the operator products are FP32, the Lanczos
 * coefficients and their reductions FP64 (the estimate agrees with an FP64 Lanczos
 * within 1e-5 relative). The per-block l2 norms of step 8 and of the stopping rule
 * accumulate in FP64 across warps and CTAs; within one warp (at most 32 rows) the
 * partial sum is FP32. Both are departures from an all-FP64 reduction, bounded by
 * the per-operator tolerance. */
ps_status ps_set_measurements(ps_handle* h, int64_t M, const double* uv, const float* vis,
                              const float* weights, int32_t nblocks, const int64_t* block_offsets,
                              const double* eps, int32_t device_ptrs);

/* Soft-threshold sizes gamma W of Algorithm 1 step 6 (W >= 0: 4 x 9 x N floats in
 * the coefficient layout; NULL = all ones). gamma > 0, or 0 for the handle's gamma
 * (cfg.gamma, else the default computed by ps_set_measurements). */
ps_status ps_set_sara_weights(ps_handle* h, const float* W, double gamma, int32_t device_ptrs);

/* Current soft-threshold sizes gamma W (4 x 9 x N floats, coefficient layout). */
ps_status ps_get_sara_weights(ps_handle* h, float* out, int32_t device_ptrs);

/* Run n_iter iterations of Algorithm 1 (steps 3-12) in the handle's mode.
 * Asynchronous on the handle's stream (a CUDA graph of one iteration is replayed)
 * when `stats` is NULL. With `stats`, the call then computes the stopping-rule
 * statistics of the new state as ps_compute_stats does with the handle's zeta_sigma
 * (synchronises; PS_ENONFINITE if the state holds a NaN or infinity). */
ps_status ps_pd_iterate(ps_handle* h, int32_t n_iter, ps_stats* stats);

/* Reweighting of Algorithm 2 (Eq. weights): W = delta / (delta + |Psi^dagger S|),
 * thresholds gamma W with the gamma of the last ps_set_sara_weights. All primal and
 * dual state is kept (warm start). delta > 0. */
ps_status ps_reweight(ps_handle* h, double delta);

/* Switch the problem variant (PS_POLARIZED ... PS_L1TV_NC) keeping the state; step sizes
 * that were defaulted are recomputed for the new mode. Switching between the SARA modes
 * (0-3) and the TV modes (4-7) clears A (its layout differs). In the TV modes the data
 * gradient is Lipschitz with beta = ||phi||^2 / 2; the defaults are rho1 = beta / (2 ||Psi||^2),
 * rho3 = beta / 2 and tau = 0.99 / (beta / 2 + rho1 ||Psi||^2 [+ rho3 with the constraint]),
 * ||Psi||^2 = 8 (TV) or 9 (l1 + TV). */
ps_status ps_set_mode(ps_handle* h, int32_t mode);

/* Weights of the TV modes: tv[i] = mu_i > 0 of ||grad S_i||_{2,1}, l1[i] = nu_i >= 0 of
 * ||S_i||_1 (used by PS_L1TV and PS_L1TV_NC; may be null otherwise), i = I, Q, U, V
 * (Section 4.4, the thresholds Lambda of Algorithm 3 step 6). PS_EINVAL on negative or
 * non-finite values. */
ps_status ps_set_tv_weights(ps_handle* h, const double* tv, const double* l1);

/* Current Stokes maps S (4 x N floats). */
ps_status ps_get_stokes(ps_handle* h, float* out, int32_t device_ptrs);

/* Read or overwrite the primal/dual state (Algorithm 2 warm start). */
ps_status ps_get_state(ps_handle* h, const ps_state_view* view);
ps_status ps_set_state(ps_handle* h, const ps_state_view* view);

/* The handle's configuration with every default resolved: kernel_width, alpha and the
 * stopping tolerances as used, mode the current mode, and gamma the handle's gamma
 * (cfg.gamma, else the default that ps_set_measurements computed; 1 before it). */
ps_status ps_get_config(const ps_handle* h, ps_config* out);

/* Step sizes and the Lanczos estimate of ||phi||_sp^2 (Section 4.3.3). */
ps_status ps_get_params(ps_handle* h, double* tau, double* rho1, double* rho2, double* rho3,
                        double* opnorm_sq);

/* Stopping-rule statistics of Section 5.5 for the current S: per-block residual
 * norms, relative change of the last iteration, violation count N_p with
 * zeta = zeta_sigma * rms(Stokes I residual image) / PSF peak (Section 5.2; zeta_sigma
 * <= 0 takes the handle's), the weighted l1 objective, and which criteria of the
 * stopping rule hold with the handle's rel_tol, resid_tol and np_tol (stop_flags,
 * converged). The FP64 sums of the relative change also test the state: a NaN or an
 * infinity in S (which any non-finite dual reaches within one iteration) returns
 * PS_ENONFINITE. Synchronises the stream. */
ps_status ps_compute_stats(ps_handle* h, double zeta_sigma, ps_stats* out);

/* Operators of the method on caller data, using the handle's measurement set:
 *   ps_apply_phi          S (4 x N) -> Y = phi(S) (M x 4 complex64)    [Eq. meas_op]
 *   ps_apply_phi_adjoint  Y -> phi^dagger(Y) = Re(Phi^H Y L^H) (4 x N) [Alg. 1 step 3]
 *   ps_apply_psi_adjoint  S (4 x N) -> Psi^dagger S (4 x 9 x N)        [Section 4.1]
 *   ps_apply_psi          A (4 x 9 x N) -> Psi A (4 x N)               [Section 4.1]
 * Inputs and outputs may not alias. */
ps_status ps_apply_phi(ps_handle* h, const float* S, float* Y, int32_t device_ptrs);
ps_status ps_apply_phi_adjoint(ps_handle* h, const float* Y, float* S, int32_t device_ptrs);
ps_status ps_apply_psi_adjoint(ps_handle* h, const float* S, float* A, int32_t device_ptrs);
ps_status ps_apply_psi(ps_handle* h, const float* A, float* S, int32_t device_ptrs);

/* The Daubechies scaling filters db1..db8 the library uses (Section 4.1), built
 * on the host by spectral factorisation: out[8][16], row b-1 holds db_b's 2b taps
 * (zero padded). Needs no device. */
ps_status ps_wavelet_filters(double* out);

/* Stages of one iteration, in launch order (index into ps_profile_stages' output). */
enum {
  PS_STAGE_PRIMAL = 0,            /* k_primal: steps 3-4, 9-12, Dirac part of 5-6 */
  PS_STAGE_ANALYSIS = 1,          /* level-1 analysis (k_ana_l1): steps 5-6 on the finest details */
  PS_STAGE_ANALYSIS_COARSE = 2,   /* analysis levels 2..L: steps 5-6 on the coarser coefficients */
  PS_STAGE_SYNTHESIS_COARSE = 3,  /* synthesis levels L..2 (to the level-1 approximations) */
  PS_STAGE_SYNTHESIS = 4,         /* finest synthesis level (k_syn2_fine): Psi A for the next step 3 */
  PS_STAGE_FWD_FFT = 5,           /* k_fwd_rows + k_fwd_cols: F Z of step 7 */
  PS_STAGE_DEGRID = 6,            /* k_degrid: G, mixing, B~ and block-norm partials (step 7) */
  PS_STAGE_BALL = 7,              /* k_block_scale: step 8 */
  PS_STAGE_GRID = 8,              /* accumulator clear + k_grid: G^T of phi^dagger */
  PS_STAGE_ADJ_FFT = 9,           /* k_adj_cols + k_adj_rows: Z^T F^H of phi^dagger */
  PS_NSTAGES = 10
};

/* Run n_iter iterations launched one kernel at a time (no graph) with CUDA events
 * between the stages on the handle's stream, and write the mean milliseconds of
 * each stage to stage_ms[PS_NSTAGES]. The iterations advance the state like
 * ps_pd_iterate. Synchronises the stream. */
ps_status ps_profile_stages(ps_handle* h, int32_t n_iter, double* stage_ms);

/* Number of kernel launches in one iteration of the handle's current mode. */
int32_t ps_kernels_per_iteration(const ps_handle* h);

/* Allocation-free variant of ps_apply_psi: S = Psi A, the SARA synthesis, for
 * callers that cannot call cudaMalloc, such as code whose device memory is all
 * owned by another allocator (a framework's caching allocator or a fixed
 * pre-reserved pool) or that must not risk an allocation failing or stalling
 * mid-run. The paper has no counterpart of this entry point.
 *   A       device pointer, 4 x 9 x n*n floats in the coefficient layout
 *   S       device pointer, 4 x n*n floats (output)
 *   n       power of two, 16 <= n <= 256 (the limit of the static scratch)
 *   levels  n divisible by 2^levels
 *   cuda_stream  cudaStream_t to launch on (NULL: the legacy default stream)
 * Needs no handle and allocates nothing: the per-level scratch is a file-scope
 * device array of 2 x 32 x 128^2 floats (4 MiB) that every GPU loading the library
 * holds until process exit. The first call on a device (with that device current)
 * looks up the array's device address and uploads the filter taps; make that first
 * call before capturing a stream. All calls share the one array and leave their
 * intermediate values in it; it needs no clearing, but calls that overlap on the
 * GPU (different streams, or different host threads on the same device) race on it
 * and must be serialised by the caller. A and S must be 16-byte aligned pointers to
 * device (or managed) memory of the current device, else PS_EINVAL; sizes beyond the
 * limit return PS_EINVAL with a message in ps_last_error(NULL).
 * Asynchronous: the result is ready when the stream is synchronised. If a bounded
 * in-kernel wait for a bulk copy gives up, the tiles it served are left unwritten and
 * a device flag (cleared at the start of every call) is raised: ps_static_status
 * reports it. */
ps_status ps_apply_psi_static(const float* A, float* S, int32_t n, int32_t levels, void* cuda_stream);

/* Status of the last ps_apply_psi_static call on the current device: synchronises
 * `cuda_stream` (NULL: the legacy default stream), then returns PS_ETIMEOUT if one of
 * that call's bounded waits gave up (its S is then incomplete), else PS_OK. Allocates
 * nothing. Like ps_apply_psi_static, the paper has no counterpart of it. */
ps_status ps_static_status(void* cuda_stream);

/* Test hook of the failure path of the bounded in-kernel waits: the number of
 * polls a kernel makes on a bulk-copy barrier before it gives up, raises the error
 * flag that the next synchronising call reports as PS_ETIMEOUT, lets the copies in
 * flight land (a second wait with the full budget) and leaves its tile unwritten.
 * polls = 0 gives up at the first wait (deterministically); polls < 0 restores the
 * default (2^22). Applies to every handle and to ps_apply_psi_static on the current
 * device; call it with no kernel of this library in flight. No counterpart in the
 * paper. */
ps_status ps_debug_set_wait_polls(int32_t polls);

/* Replace the measurements Y of the current coverage (same rows, same caller
 * order, same blocks and radii) without re-sorting or re-estimating ||phi||: for a
 * new noise realisation or observation on the same uv tracks. The state is kept. */
ps_status ps_set_visibilities(ps_handle* h, const float* vis, int32_t device_ptrs);

/* Relative change ||S_i^(k+1) - S_i^(k)|| / ||S_i^(k)|| of the last iteration for the
 * four maps (Eq. stop_crit; 0 for a map that stayed zero, +inf for one that left zero),
 * from FP64 partials the iteration already wrote; cheaper than ps_compute_stats.
 * PS_ENONFINITE when those sums are not finite (a NaN or infinity in S).
 * Synchronises the handle's stream. */
ps_status ps_get_rel_change(ps_handle* h, double* out4);

/* The same relative change (Eq. stop_crit) without stalling the device, for solve loops that
 * test the stopping rule after every iteration: ps_rel_change_request enqueues on the handle's
 * stream the FP64 sums of the last iteration's partials and their copy (with the device error
 * flags) into host memory the library owns, and returns at once; ps_rel_change_result waits
 * for that copy only, not for work queued after it, and writes the four values as
 * ps_get_rel_change would have at the request (PS_ENONFINITE, PS_ETIMEOUT likewise). A loop
 * that requests after iteration k, launches iteration k + 1 and then reads the result keeps
 * the GPU busy while the host decides, and stops one iteration late. One request at a time:
 * a second request replaces the first, and a synchronous read (ps_get_rel_change,
 * ps_compute_stats, ps_pd_iterate with statistics) consumes it. ps_rel_change_result without a
 * pending request returns PS_ESTATE. */
ps_status ps_rel_change_request(ps_handle* h);
ps_status ps_rel_change_result(ps_handle* h, double* out4);

/* max_j |[Psi^dagger S]_j| over all four maps (FP32 values, exact maximum): the scale
 * from which reweighting schedules pick delta (Eq. weights). Synchronises. */
ps_status ps_max_abs_analysis(ps_handle* h, double* out);

/* Batches (many independent problems advanced together). One CUDA graph holds one
 * iteration of every handle of the batch, each on its own stream, forked from and
 * joined back to the batch stream, so one launch advances all problems and their
 * kernels overlap on the device. Handles keep their own state, mode and step sizes;
 * they must have distinct streams and measurements set. The graph is rebuilt when a
 * handle's mode or state changes. ps_batch_iterate orders the work already queued on
 * each handle's stream (a reweight, new thresholds) before its iterations, and each
 * handle's later calls after them. The batch does not own the handles. */
typedef struct ps_batch ps_batch;
ps_status ps_batch_create(ps_handle* const* handles, int32_t count, void* cuda_stream, ps_batch** out);
ps_status ps_batch_iterate(ps_batch* b, int32_t n_iter);   /* asynchronous on the batch stream */
ps_status ps_batch_synchronize(ps_batch* b);
void ps_batch_destroy(ps_batch* b);

/* Launch choices of the kernels (the paper runs the same operators in every
 * iteration of Algorithm 1 and prescribes no implementation; which launch shape is
 * fastest depends on the image size and on how the visibilities fill the uv plane,
 * so it is measured on the handle's own problem). Values index the candidates: */
enum {
  PS_TUNE_SYNTHESIS = 0,  /* finest synthesis level: 0 double-buffered subband staging (3 CTAs/SM),
                             1 single-buffered, refilled during the x-pass (4 CTAs/SM),
                             2 as 1 in persistent CTAs looping over (tile, map) units, the staging
                               running on from one unit into the next */
  PS_TUNE_DEGRID = 1,     /* 0 one row per thread over a work item,
                             1 one same-cell chunk per warp (broadcast stencil reads),
                             2 as 0 with registers capped for 6 CTAs per SM (W = 7; other widths
                               run 0) */
  PS_TUNE_GRID = 2,       /* 0 one warp per same-cell chunk (2 kernel cells per lane),
                             1 half-warps on alternate rows of a chunk (4 cells per lane),
                             2 lanes own (stencil row, channel pair) (W <= 8; W = 9 runs 0),
                             3 tensor cores: each chunk's block as a small matrix product
                               (TF32 hi/lo split, FP32 accumulation), kernel weights copied from a
                               per-row table made once per measurement set (W <= 8; W = 9 runs 0),
                             4 as 3 with the kernel weights evaluated in the kernel (no table
                               traffic) (W <= 8; W = 9 runs 0) */
  PS_TUNE_ANALYSIS = 3,   /* tiled analysis levels: 0 one (tile, basis, map) unit per CTA,
                             1 persistent (2 CTAs/SM looping over units, next unit's copies in flight),
                             2 level 1 with one CTA per (tile, map): the map's input tile copied once for
                               the 8 bases, each basis' staged A and gamma W in flight during the previous
                               basis (levels >= 2 as 0),
                             3 as 2 with one CTA per (tile, 4 bases, map),
                             4 as 3 with 512 threads per CTA (two columns per thread),
                             5 as 3 with one staging set, refilled for the next basis during its
                               row pass (3 CTAs/SM) */
  PS_TUNE_COUNT = 4
};

/* Autotuner: after ps_set_measurements, time every candidate of every PS_TUNE_*
 * slot on the handle's data (reps launches each, CUDA events on the handle's
 * stream, after one untimed launch) and keep the fastest. The state of the
 * iteration is unchanged (the timed launches run the analysis dual update on scratch
 * coefficients, recompute Psi A of the current A in place, run the degridding dual update
 * on a scratch copy of the data dual and grid the current dual into the gridding
 * accumulator, an intermediate; phi^dagger B is kept). Uses (and on first use allocates) the handle's
 * 36N operator scratch. choices (nullable) receives the
 * PS_TUNE_COUNT picks; ms (nullable) receives, per slot, the time of the pick in
 * milliseconds. Synchronises the stream. PS_ESTATE before measurements. */
ps_status ps_autotune(ps_handle* h, int32_t reps, int32_t* choices, double* ms);

/* Read / force the launch choices (PS_TUNE_COUNT int32; PS_EINVAL for a value
 * outside a slot's candidates). The defaults are 0. */
ps_status ps_get_tuning(const ps_handle* h, int32_t* choices);
ps_status ps_set_tuning(ps_handle* h, const int32_t* choices);

/* Measured FP32 throughput of the current device, the compute ceiling of the FP32
 * interpolation and wavelet kernels: independent FMA chains on every SM, packed FP32x2
 * (fma.rn.f32x2, packed = 1) or scalar (packed = 0); *flops_per_s counts 2 FLOPs per
 * FMA (a packed FMA is two). Allocates 4 bytes and a stream for the measurement,
 * synchronises. No counterpart in the paper. */
ps_status ps_fp32_peak(int32_t packed, double* flops_per_s);

/* Synchronise the handle's stream; reports a pending CUDA error. */
ps_status ps_synchronize(ps_handle* h);

/* Device bytes held by the handle (for admission control by memory footprint). */
int64_t ps_device_bytes(const ps_handle* h);

/* Estimate of the device bytes a handle would hold for (n, levels, M) before it is
 * created; 0 on invalid sizes. */
int64_t ps_estimate_bytes(int32_t n, int32_t levels, int64_t M);

#ifdef __cplusplus
}
#endif

#endif /* POLSARA_H */

/*
 * sr3d.h -- C ABI of the GB300 (sm_103a) library for the fast 3D single-image
 * super-resolution method of Tuador, Pham, Michetti, Basarab and Kouame,
 * "A Novel Fast 3D Single Image Super-Resolution Algorithm" (arXiv:2010.15491).
 *
 * Problem (Sec. II-A, eq. 1):  y = D H x + n.
 *   x   HR volume, sizes (m_h, n_h, s_h), stored C-order as x[s][n][m]
 *       (m fastest: the paper's lexicographic ordering).
 *   y   LR volume, sizes (m_h/dr, n_h/dc, s_h/ds), stored y[s][n][m].
 *   H   cyclic convolution with the PSF (eq. 2); the PSF centre tap, index
 *       floor(p/2) per axis, sits at the origin of the circulant.
 *   D   keeps sample 0 of every dr x dc x ds block (dr on m, dc on n, ds on s).
 *
 * Conventions shared by every entry point:
 *   - Real arrays hold the plan's element type: float for SR3D_F32 plans,
 *     double for SR3D_F64 plans.  Arguments named *_dev are device pointers
 *     owned by the caller, contiguous, 16-byte aligned; *_host are host
 *     pointers (pinned memory gives asynchronous copies).
 *   - The ADMM dual variable d holds 3*N_h elements, component-major:
 *     d[0..N_h) is the m-difference component, then n, then s
 *     (L = [D_m; D_n; D_s], periodic forward differences).
 *   - Every call is ordered on the plan's stream and returns after its result
 *     is complete.  A plan is not thread-safe; distinct plans are.
 *   - Return value: SR3D_OK (0) or a negative SR3D_ERR_* code; the message of
 *     the last failure on the calling thread is sr3d_last_error().  On error
 *     the outputs are unspecified; the plan stays usable unless the error is
 *     SR3D_ERR_CUDA.
 *
 * Supported sizes: every HR size is 2^a or 3*2^a, m_h a multiple of 32, n_h a
 * multiple of 8, 4 <= s_h, each HR size at most 2048; m_h/dr even;
 * d = dr*dc*ds at most 8.
 */
#ifndef SR3D_H
#define SR3D_H

#ifdef __cplusplus
extern "C" {
#endif

#define SR3D_OK                    0
#define SR3D_ERR_INVALID_ARG      -1  /* NULL pointer, non-positive size or weight */
#define SR3D_ERR_NOT_DIVISIBLE    -2  /* an HR size is not a multiple of its decimation factor */
#define SR3D_ERR_UNSUPPORTED_SIZE -3  /* a size outside the supported set above */
#define SR3D_ERR_SINGULAR         -4  /* sum of PSF taps is zero (ADMM DC class), or tau <= 0 */
#define SR3D_ERR_CUDA             -5  /* a CUDA runtime call failed */
#define SR3D_ERR_OOM              -6  /* device allocation failed */
#define SR3D_ERR_TIMEOUT          -7  /* a bounded device wait ran out */
#define SR3D_ERR_NUMERIC          -8  /* NaN or Inf in the objective / residual reductions */
#define SR3D_ERR_NOT_CONVERGED    -9  /* tol > 0 and max_iters reached; x and d are still written */

typedef struct sr3d_plan_s* sr3d_plan_t;

typedef enum { SR3D_F32 = 0, SR3D_F64 = 1 } sr3d_dtype;

/* Plan descriptor: the inputs of Algorithm 1 that do not change between
 * solves (y, H and the decimation; Sec. II-A and Algorithm 1 "Input"). */
typedef struct {
  int m_h, n_h, s_h;        /* HR sizes */
  int dr, dc, ds;           /* integer decimation factors, dividing m_h, n_h, s_h */
  const double* psf;        /* host PSF taps, psf[p_s][p_n][p_m]; copied at plan time */
  int p_m, p_n, p_s;        /* PSF sizes, 1 <= p_a <= HR size of axis a */
  int dtype;                /* sr3d_dtype: element type of every real array */
  void* stream;             /* cudaStream_t to run on; NULL = a stream the plan owns */
} sr3d_desc;

/* Statistics of sr3d_admm_tv.  Inputs: eval_every (evaluate the objective
 * and residuals every k-th iteration; 0 = only after the last one),
 * objective_hist (host array of hist_len doubles or NULL; entry i receives
 * the objective at the i-th evaluation).  Outputs: the rest, at the last
 * evaluation.  Residuals follow Boyd et al. (2011, Sec. 3.3) with A = L,
 * B = -I: primal ||Lx - u||, dual mu ||L^T (u - u_prev)||; the relative
 * values divide by max(||Lx||, ||u||) and mu ||L^T d||. */
typedef struct {
  int eval_every;
  double* objective_hist;
  int hist_len;
  int iters;                /* iterations run */
  int evals;                /* evaluations written */
  double objective;         /* 1/2 ||y - DHx||^2 + lambda sum_j ||(Lx)_j||_2 */
  double data_term;         /* 1/2 ||y - DHx||^2 */
  double tv_term;           /* sum_j ||(Lx)_j||_2 */
  double primal, dual;
  double primal_rel, dual_rel;
} sr3d_stats;

/* Plan: computes Lambda = DFT(PSF) (Algorithm 1 step 1, eq. 2), the Laplacian
 * symbol tables (steps 3-4) and FFT twiddles on the device, and allocates the
 * work buffers.  *out receives the plan.  Errors: INVALID_ARG, NOT_DIVISIBLE,
 * UNSUPPORTED_SIZE, OOM, CUDA. */
int sr3d_plan(sr3d_plan_t* out, const sr3d_desc* desc);

/* Frees the plan and everything it owns (safe with NULL). */
int sr3d_destroy(sr3d_plan_t plan);

/* Cap on the device memory any one plan may hold, process-wide (bytes <= 0:
 * no cap, the default).  A plan whose buffers would pass it fails as if
 * cudaMalloc had failed: sr3d_plan returns SR3D_ERR_OOM and frees everything
 * it had allocated; an entry point that allocates lazily (the ADMM dual and
 * residual buffers of the first sr3d_admm_tv, the CG vectors, the host-buffer
 * staging of sr3d_admm_tv_host) returns SR3D_ERR_OOM and the plan stays
 * usable.  For budgeting several plans on one device, and for testing the
 * out-of-memory path without exhausting the device.  Not in the paper.
 * Always returns SR3D_OK. */
int sr3d_set_plan_memory_limit(long long bytes);

/* Degradation operator of eq. (1) without noise: y_dev = D H x_dev
 * (HR x in, LR y out).  Used to synthesise observations.  Errors:
 * INVALID_ARG (NULL arrays), CUDA. */
int sr3d_forward(sr3d_plan_t plan, const void* x_dev, void* y_dev);

/* Sentinel for xbar_dev: the prior xbar is the nearest-neighbour replication
 * of y (each LR voxel copied to its dr x dc x ds block). */
#define SR3D_XBAR_NEAREST ((const void*)1)

/* 3D-FSR-l2-l2 (Sec. III-A, eq. 12): x_dev = argmin_x 1/2 ||y - DHx||^2
 * + tau/2 ||x - xbar||^2, tau = 2*lambda of eq. (5).  One batch of 3D FFT
 * passes, the per-aliasing-class solve of eq. (12), one inverse 3D FFT.
 * xbar_dev: NULL for xbar = 0, SR3D_XBAR_NEAREST, or a device HR array.
 * Errors: INVALID_ARG (tau <= 0 or NULL y/x), CUDA. */
int sr3d_tikhonov(sr3d_plan_t plan, const void* y_dev, const void* xbar_dev, double tau, void* x_dev);

/* 3D-FSR-l2-TV (Sec. III-B, Algorithm 1): ADMM for
 * min_x 1/2 ||y - DHx||^2 + lambda sum_j ||(Lx)_j||_2 with penalty rho (the
 * paper's mu).  Each iteration: x-update by eq. (12) with Gamma weights
 * (step 5a), isotropic soft threshold (5b), dual update (5c).
 *   x_dev   in: x0 when tau_init <= 0; out: x after the last iteration.
 *           With tau_init > 0, x0 = sr3d_tikhonov(y, SR3D_XBAR_NEAREST, tau_init).
 *   d_dev   NULL: d0 = 0 and the final d is discarded; else in: d0, out: d.
 *   u0 = L x0.  max_iters >= 0 iterations; tol > 0 stops early when both
 *   relative residuals fall below tol (tested every max(1, eval_every)
 *   iterations, on the device: the call waits once for the loop, not once
 *   per test; NOT_CONVERGED if max_iters is reached first); tol <= 0 runs
 *   exactly max_iters iterations.  stats may be NULL.
 * Errors: INVALID_ARG, SINGULAR (sum of PSF taps zero), NUMERIC, CUDA,
 * NOT_CONVERGED. */
int sr3d_admm_tv(sr3d_plan_t plan, const void* y_dev, void* x_dev, void* d_dev,
                 double lambda, double rho, int max_iters, double tol, double tau_init,
                 sr3d_stats* stats);

/* sr3d_admm_tv on host buffers: copies y_host (and x_host when
 * tau_init <= 0) to plan-owned device buffers, solves, copies x back to
 * x_host.  Same arguments and errors otherwise (d0 = 0, d discarded). */
int sr3d_admm_tv_host(sr3d_plan_t plan, const void* y_host, void* x_host,
                      double lambda, double rho, int max_iters, double tol, double tau_init,
                      sr3d_stats* stats);

/* Batched ADMM-TV over n volumes of uneven size and decimation (one plan
 * per volume; plans distinct and on non-default streams): for volume i,
 * sr3d_admm_tv(plans[i], y[i], x[i], NULL, lambda[i], rho[i], iters, 0,
 * tau_init[i], NULL).  The iterations of all volumes run as one CUDA graph
 * with one independent chain per volume, so small volumes execute
 * concurrently; the graph is cached and replayed while plans, buffers and
 * parameters repeat.  Serialised across host threads.  Not in the paper
 * (a throughput mode for many volumes).  Errors: INVALID_ARG, SINGULAR,
 * CUDA. */
int sr3d_admm_tv_batched(int n, sr3d_plan_t* plans, const void* const* y, void* const* x,
                         const double* lambda, const double* rho, const double* tau_init, int iters);

/* Message of the last failure on the calling thread ("" if none). */
const char* sr3d_last_error(void);

/* ---- Diagnostic entry points: one step of the hot path each, for parity
 * ---- tests against the oracle.  Same conventions as above. */

/* Lambda (eq. 2) in natural half-spectrum layout:
 * out_dev[k_s][k_n][k_m], k_m in [0, m_h/2], complex pairs (re, im) of the
 * plan's element type, unnormalised DFT. */
int sr3d_get_otf(sr3d_plan_t plan, void* out_dev);

/* Unnormalised forward 3D DFT of the real HR x_dev, same layout as
 * sr3d_get_otf. */
int sr3d_fft3(sr3d_plan_t plan, const void* x_dev, void* out_dev);

/* x-update of Algorithm 1 step 5a: x_dev = argmin 1/2||y - DHx||^2 +
 * rho/2 ||Lx - (u - d)||^2 given theta_dev = L^T (u - d) (HR real). */
int sr3d_xstep(sr3d_plan_t plan, const void* y_dev, const void* theta_dev, double rho, void* x_dev);

/* Steps 5b-5c of Algorithm 1 followed by the next step's Theta:
 * u = shrink(Lx + d_in, lambda/rho), d_out = d_in + Lx - u,
 * theta_out = L^T (u - d_out).  d_in and d_out must not overlap. */
int sr3d_tv_step(sr3d_plan_t plan, const void* x_dev, const void* d_in_dev, void* d_out_dev,
                 double lambda, double rho, void* theta_out_dev);

/* Autotuner (not in the paper): times candidate tile schedules (reps launches
 * each after one warm-up launch; reps < 1 takes 10) on the plan's own buffers -- the n pass's and the s pass's tile
 * widths (including widths that cover the m-slots with at most one step of
 * padding), the m passes' lines per CTA, and the TV kernel's planes per CTA
 * (including the counts whose grid fills whole waves of resident CTAs) --
 * keeps the fastest and caches the choice per geometry (sizes, decimation,
 * dtype) for the process; a later plan of the same geometry only applies the
 * cached choice.  Results are unchanged (the schedules only split the same
 * work differently); the work spectrum, Theta and dual buffers are
 * overwritten.  Errors: INVALID_ARG, CUDA, OOM. */
int sr3d_autotune(sr3d_plan_t plan, int reps);

/* The tile schedule the plan launches (the defaults, or the autotuner's
 * choice), and a way to set it.  Entries: [0] = m-slots per CTA of the n
 * pass, [1] = m-slots per CTA of the s pass (a multiple of d_r), [2] = s
 * planes each CTA of the TV kernel marches over (the last CTA along s takes
 * the remainder), [3] and [4] = lines per CTA of the forward and inverse m
 * passes (whole warps, at most the default of 256 threads).  set (may be
 * NULL) gives new values, entries <= 0 keeping the current one; results do
 * not depend on the schedule (it only splits the same work differently).
 * sched (may be NULL) receives the schedule in force.  Errors: INVALID_ARG
 * (a value the pass's kernel or the plan's solve-order buffers cannot take,
 * or fewer than 4 TV planes; nothing is changed), CUDA. */
int sr3d_schedule(sr3d_plan_t plan, const int set[5], int sched[5]);

/* Per-kernel accounting.  Kernel kinds: SR3D_K_TV (fused u/d/Theta step),
 * SR3D_K_RFFT_FWD / SR3D_K_RFFT_INV (real FFT along m), SR3D_K_FFTN_FWD /
 * SR3D_K_FFTN_INV (FFT along n), SR3D_K_FFTS (FFT along s, with the class
 * solve when solving), SR3D_K_OTHER (reductions, tables, copies),
 * SR3D_K_SETUP (every launch of sr3d_admm_tv before its first iteration:
 * LR spectrum, Tikhonov start, initial Theta).  Launches
 * are always counted.  With sr3d_profile(plan, 1) every launch made by an
 * entry point is also bracketed by CUDA events on the plan's stream and its
 * duration added to its kind (events add a few microseconds per launch).
 * sr3d_profile resets the totals; sr3d_profile_read copies them out
 * (ms[k] in milliseconds, launches[k]) for k < SR3D_NKINDS. */
#define SR3D_K_TV 0
#define SR3D_K_RFFT_FWD 1
#define SR3D_K_FFTN_FWD 2
#define SR3D_K_FFTS 3
#define SR3D_K_FFTN_INV 4
#define SR3D_K_RFFT_INV 5
#define SR3D_K_OTHER 6
#define SR3D_K_SETUP 7
#define SR3D_NKINDS 8
int sr3d_profile(sr3d_plan_t plan, int on);
int sr3d_profile_read(sr3d_plan_t plan, double ms[SR3D_NKINDS], long long launches[SR3D_NKINDS]);

/* Allocation-free Tikhonov solve (no counterpart in the paper: an
 * interface for callers that may not allocate device memory once running --
 * a reconstruction loop whose device-memory budget is fixed at start-up, or a
 * plug-in inside a host application that owns the device's memory pool --
 * where a cudaMalloc can fail, or stall the whole device while it
 * synchronises).  Same result as sr3d_plan + sr3d_tikhonov + sr3d_destroy for
 * the descriptor `desc` (desc->stream NULL = the legacy default stream), but
 * every piece of work memory is carved from one file-scope device array of
 * SR3D_NOALLOC_BYTES (8 MiB), held by every GPU that loads the library until
 * the process exits; the call makes no cudaMalloc/cudaFree and no allocating
 * library call.  The work memory is about 8 bytes per HR voxel in FP32 (16 in
 * FP64), so volumes up to about 2^19 HR voxels in FP32 (e.g. 128 x 64 x 64)
 * or 2^18 in FP64 fit; larger ones fail with SR3D_ERR_UNSUPPORTED_SIZE
 * before any work is queued.  The first call on a device looks up the
 * array's device address (once per device, with that device current); make
 * that first call before any stream capture.  The PSF is copied from host
 * memory on the stream and the call returns after the result is complete.
 * All calls share the array and every call overwrites it, so calls that
 * overlap on the GPU (other streams, other host threads) race; serialise
 * them.  Inputs and outputs are the caller's device arrays as in
 * sr3d_tikhonov. */
#define SR3D_NOALLOC_BYTES (8u << 20)
int sr3d_tikhonov_noalloc(const sr3d_desc* desc, const void* y_dev, const void* xbar_dev, double tau,
                          void* x_dev);

/* ---------------------------------------------------------------------------
 * Learned warm start (no counterpart in the paper, whose ADMM-TV of
 * Algorithm 1 starts from the Tikhonov solution of Eq. 12 and which argues
 * against learned super-resolution).  A 3D U-Net refines the Tikhonov
 * estimate into the ADMM starting point x0; sr3d_dual_init gives the dual
 * that is consistent with that x0.
 *
 * Network (channels C1 = 16, C2 = 32, C3 = 64; 3x3x3 convolutions with zero
 * padding and bias, each followed by ReLU; volumes [s][n][m]):
 *   e1 = conv(conv(x))               full size, C1
 *   e2 = conv(conv(maxpool(e1)))     half size, C2   (2x2x2 max pooling)
 *   e3 = conv(conv(maxpool(e2)))     quarter size, C3
 *   d2 = conv(conv([up(e3), e2]))    half size, C2   (nearest 2x upsampling,
 *   d1 = conv(conv([up(d2), e1]))    full size, C1    channel concatenation)
 *   out = sum_c w_h[c] d1[c] + b_h + x                (1x1x1 residual head)
 * Parameters are one flat FP32 vector of sr3d_unet_param_count() values: for
 * each of the ten 3x3x3 layers in the order above W[co][tap][ci] (tap =
 * (ks*3 + kn)*3 + km for the offset (ks-1, kn-1, km-1) in (s, n, m)) followed
 * by b[co]; then w_h[C1] and b_h.  Weights and activations are BF16 on the
 * tensor cores with FP32 accumulation; master weights and the Adam state are
 * FP32.  Sizes m, n, s must be positive multiples of 4.
 * ------------------------------------------------------------------------- */
typedef struct sr3d_unet_s* sr3d_unet_t;

/* number of FP32 parameters of the network above (353,281) */
long long sr3d_unet_param_count(void);

/* Creates a network with all parameters zero (the identity map: out = x) on
 * `stream` (NULL = legacy default stream).  Activation buffers are
 * allocated on first use of a size and kept until the size changes.  The
 * handle is freed by sr3d_unet_destroy (safe with NULL); a network is used by
 * one host thread at a time.  Errors of every sr3d_unet_* call: INVALID_ARG
 * (NULL arguments, a parameter or byte count that does not match, an unknown
 * path or activation index, sr3d_unet_read before any forward pass),
 * UNSUPPORTED_SIZE (m, n, s not positive multiples of 4), OOM, TIMEOUT (a
 * bounded tcgen05 wait ran out), CUDA. */
int sr3d_unet_create(sr3d_unet_t* out, void* stream);
int sr3d_unet_destroy(sr3d_unet_t net);

/* Copy the flat parameter vector from / to host memory (n must equal
 * sr3d_unet_param_count()); setting parameters also clears the Adam state. */
int sr3d_unet_set_params(sr3d_unet_t net, const float* params_host, long long n);
int sr3d_unet_get_params(sr3d_unet_t net, float* params_host, long long n);

/* out_dev = network(x_dev); both FP32 device arrays of m*n*s values in the
 * [s][n][m] layout (they may not alias).  Synchronises the stream. */
int sr3d_unet_forward(sr3d_unet_t net, int m, int n, int s, const float* x_dev, float* out_dev);

/* One training step on the pair (x_dev, target_dev) (FP32 device arrays as in
 * sr3d_unet_forward): loss = mean((network(x) - target)^2) is written to
 * *loss (if not NULL); the gradient of the loss with respect to the flat
 * parameters is copied to grad_host (if not NULL, FP32, param_count values);
 * with update != 0 the parameters then take one Adam step (beta1 0.9,
 * beta2 0.999, eps 1e-8, bias-corrected) of learning rate lr. */
int sr3d_unet_train_step(sr3d_unet_t net, int m, int n, int s, const float* x_dev, const float* target_dev,
                         double lr, double* loss, float* grad_host, int update);

/* Kernel path of the 3x3x3 convolutions.  The tcgen05 kernel (5th-generation
 * tensor cores: tcgen05.mma with TMEM accumulators, one thread issuing, a
 * persistent CTA per row marching over s) takes levels whose m extent is a
 * multiple of 128 with 16, 32 or 48 input and output channels; the mma.sync
 * kernel takes every shape.  SR3D_UNET_PATH_TCGEN05 (default): tcgen05 for
 * the shapes where it is the faster one (16 -> 16 and 16 -> 32 channels),
 * mma.sync for the rest; SR3D_UNET_PATH_MMA: mma.sync everywhere; SR3D_UNET_PATH_TCGEN05_ALL:
 * tcgen05 wherever it applies.  All compute the same convolution with FP32
 * accumulation (the order of the sums differs).  A tcgen05 wait that runs out
 * (about one second) makes the calling entry point return SR3D_ERR_TIMEOUT. */
#define SR3D_UNET_PATH_TCGEN05 0
#define SR3D_UNET_PATH_MMA 1
#define SR3D_UNET_PATH_TCGEN05_ALL 2
int sr3d_unet_set_path(sr3d_unet_t net, int path);

/* Test support for the bounded waits of the tcgen05 kernel: one CTA allocates
 * tensor memory as that kernel does, waits with the same bounded wait,
 * shortened to limit_cycles SM clock cycles (1 .. 2e9), on an mbarrier that
 * nothing arrives on (no MMA issued, none in flight), sets the network's
 * device error flag when the wait runs out, frees its tensor memory and
 * returns; the call then reports SR3D_ERR_TIMEOUT exactly as a forward or
 * training call would.  After a timeout of the real kernels the results of
 * that launch, and of any later launch on the stream, are to be discarded;
 * after this self-test the network stays usable.  Errors: INVALID_ARG,
 * TIMEOUT (the expected outcome), CUDA. */
int sr3d_unet_wait_selftest(sr3d_unet_t net, long long limit_cycles);

/* Copies an activation of the last forward pass (sr3d_unet_forward or
 * sr3d_unet_train_step) to host memory, for inspection and layer-by-layer
 * tests: which = 0 x, 1 e1a, 2 e1, 3 maxpool(e1), 4 e2a, 5 e2,
 * 6 maxpool(e2), 7 e3a, 8 e3, 9 d2a, 10 d2, 11 d1a, 12 d1 (BF16,
 * [voxel][channel] at the level's size, the first conv of each level named
 * with an "a"), 13 the output (FP32 [voxel]).  bytes must equal the
 * activation's size. */
int sr3d_unet_read(sr3d_unet_t net, int which, void* host, long long bytes);

/* KKT-consistent initial dual for sr3d_admm_tv started at x (no counterpart in
 * the paper, which starts from d = 0): with g = Lx (periodic forward
 * differences, Sec. III-B) and t = lambda / rho,
 *   d_j = t g_j / max(||g_j||, t)   (j = voxel, ||.|| over the 3 directions),
 * written as d_dev[3][V] in the plan's dtype; x_dev is an HR volume of the
 * plan.  Pass d_dev to sr3d_admm_tv together with x_dev as x0.  Errors:
 * INVALID_ARG (NULL arrays, lambda or rho not positive), CUDA. */
int sr3d_dual_init(sr3d_plan_t plan, const void* x_dev, double lambda, double rho, void* d_dev);

/* Replaces the plan's PSF (host taps psf[p_s][p_n][p_m], each size at most the
 * HR size of its axis): recomputes Lambda (Algorithm 1 step 1) and the
 * separable-PSF tables in the plan's buffers, without reallocating; later
 * calls use the new PSF.  Used to fit a PSF to data (many forward-model
 * evaluations with one plan).  Errors: INVALID_ARG, OOM, CUDA. */
int sr3d_set_psf(sr3d_plan_t plan, const double* psf, int p_m, int p_n, int p_s);

/* Other regularisers through the same Fourier-domain x-update (the
 * conclusion of the paper points to regularisation functions other than
 * Tikhonov and TV).
 *
 * sr3d_set_tv selects the TV of sr3d_admm_tv (and of the batched solve) on
 * this plan: SR3D_TV_ISOTROPIC (default, sum_j ||(Lx)_j||_2, Algorithm 1) or
 * SR3D_TV_ANISOTROPIC (sum_j sum_a |(D_a x)_j|): the u-step of step 5b then
 * shrinks each component separately, u_a = sign(nu_a) max(|nu_a| - lambda/rho,
 * 0); the x-update of step 5a and the dual step are unchanged; the statistics
 * report the matching TV term.  Errors: INVALID_ARG. */
#define SR3D_TV_ISOTROPIC 0
#define SR3D_TV_ANISOTROPIC 1
int sr3d_set_tv(sr3d_plan_t plan, int kind);

/* Tikhonov on the gradient: x_dev = argmin 1/2 ||y - DHx||^2 + tau/2 ||Lx||^2
 * (L the periodic forward differences of Sec. III-B).  Its normal equations
 * (H^T D^T D H + tau L^T L) x = H^T D^T y are those of the x-update of
 * Algorithm 1 step 5a with u - d = 0 and mu = tau, so it is one class solve of
 * eq. 12 with weights 1/(tau s_p) (the zero-frequency class solved exactly)
 * and one inverse 3D FFT.  Errors: INVALID_ARG (tau <= 0, NULL arrays),
 * SINGULAR (PSF taps sum to zero), CUDA. */
int sr3d_tikhonov_grad(sr3d_plan_t plan, const void* y_dev, double tau, void* x_dev);

/* The iterative comparator of Sec. IV: Table 1 solves eq. 5 both by the
 * closed form of eq. 12 and iteratively.  This entry solves the same problem
 * as sr3d_tikhonov (tau, xbar as there: NULL, SR3D_XBAR_NEAREST or a device
 * HR array not aliasing x) by conjugate gradients on the normal equations of
 * eq. 6, (H^T D^T D H + tau I) x = H^T D^T y + tau xbar, from x = 0: every
 * iteration applies H, the sampling mask D^T D and H^T through two 3D FFT
 * round trips of the library's FFT passes, with FP64 inner products.  Stops
 * after max_iters iterations or when ||r|| <= tol ||b|| (tol <= 0: exactly
 * max_iters).  *iters and *relres (if not NULL) receive the iterations run and
 * ||r|| / ||b||.  Errors: INVALID_ARG, NUMERIC, NOT_CONVERGED (tol > 0, x
 * still written), CUDA. */
int sr3d_tikhonov_cg(sr3d_plan_t plan, const void* y_dev, const void* xbar_dev, double tau, double tol,
                     int max_iters, void* x_dev, int* iters, double* relres);

/* The sums of the Gaussian PSF fit (Sec. IV estimates its PSF as a 3D
 * Gaussian against an HR reference): with yh = D H x_dev (the plan's PSF) and
 * y_dev an LR observation, moments[0..4] (host) receive, accumulated in FP64,
 * sum yh, sum yh^2, sum y, sum y^2 and sum yh*y -- everything the closed-form
 * gain a and offset b of min_{a,b} ||y - a yh - b||^2 and its residual need.
 * Errors: INVALID_ARG (NULL arguments), OOM, CUDA. */
int sr3d_psf_fit_moments(sr3d_plan_t plan, const void* x_dev, const void* y_dev, double moments[5]);

/* Separable-PSF fast path.  When the PSF is an outer product of three 1-D
 * factors (a Gaussian, for instance, as in the experiments of Sec. IV), the
 * eigenvalues of eq. 2 factor as Lambda(k_m, k_n, k_s) = L_m(k_m) L_n(k_n)
 * L_s(k_s), the 1-D DFTs of the wrapped factors.  sr3d_plan detects this (every
 * tap equal to the product of the PSF's marginal sums over the total squared,
 * to 1e-14 of the largest tap) and computes the three 1-D tables in FP64; the
 * class solve of eq. 12 then forms Lambda from them instead of reading the
 * stored 3-D Lambda (4 bytes less HBM traffic per voxel in FP32).  use = 1
 * enables the path (the default), 0 disables it, -1 only queries; *active (if
 * not NULL) receives 1 when the path is in use (enabled and the PSF
 * separable).  Results agree with the stored Lambda to rounding.  Errors:
 * INVALID_ARG (NULL plan), CUDA. */
int sr3d_separable(sr3d_plan_t plan, int use, int* active);

/* Plan facts for callers and tests: sizes[0..8] = m_h, n_h, s_h, m_l, n_l,
 * s_l, m-slots, m-pitch, dtype; bytes (if not NULL) = device memory the plan
 * holds.  Errors: INVALID_ARG (NULL plan or sizes). */
int sr3d_plan_info(sr3d_plan_t plan, int sizes[9], long long* bytes);

#ifdef __cplusplus
}
#endif
#endif /* SR3D_H */

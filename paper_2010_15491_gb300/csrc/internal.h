// Internal host-side interfaces of libsr3d: the plan object and the kernel
// launchers shared by the API translation unit and the kernel units.
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "common.cuh"

namespace sr3d {

// s-pass modes (kernel k_fft_s)
enum SMode {
  S_FWD = 0,       // forward transform along s
  S_INV = 1,       // inverse (unnormalised) transform along s
  S_TIK_GEN = 2,   // Tikhonov with zero / nearest-neighbour prior: build B, solve, inverse
  S_TIK_USER = 3,  // Tikhonov with a user prior: forward, B = conj(L) Y + tau Xbar, solve, inverse
  S_ADMM = 4,      // ADMM x-update: forward, B = conj(L) Y + mu Theta^, Gamma-weighted solve, inverse
  S_FOLD = 5,      // forward, then (1/d) sum_p L_p X_p per class into the LR spectrum
  S_MUL = 6,       // forward, X *= Lambda (natural layout or separable tables), inverse
  S_MULC = 7,      // forward, X *= conj(Lambda), inverse
};

// Arguments of the per-aliasing-class solve inside the s pass.
struct SolveArgs {
  const void* lam;     // Lambda in solve order (k_perm_lam)
  const void* yhat;    // LR spectrum in solve order (k_perm_yhat)
  void* lr_out;        // S_FOLD output, LR spectral layout
  const void* symM;    // 4 sin^2(pi k / M) tables (element type T)
  const void* symN;
  const void* symS;
  const void* twM;     // exp(-2 pi i q / M) tables (complex T)
  const void* twN;
  const void* twS;
  double alpha;        // tau (Tikhonov) or mu (ADMM)
  int nn_prior;        // S_TIK_GEN: 1 = nearest-neighbour prior, 0 = zero prior
  int M, N, S;
  int Ml, Nl, Sl;
  int dr, dc, ds;
  int Mlp;
  double* partial;     // per-CTA data-term partial sums (S_ADMM with statistics)
  // separable PSF: Lambda(km, kn, ks) = lamM[km] lamN[kn] lamS[ks] (complex T);
  // sep != 0 makes the class solve use these tables instead of `lam`
  const void* lamM;
  const void* lamN;
  const void* lamS;
  int sep;
  const void* lam_nat;  // Lambda in the natural spectral layout (S_MUL, S_MULC)
  // Batched ADMM s pass over `batch` volumes of one geometry stored one after
  // another (spectrum, solve-order LR spectrum, separable tables of M, N, S
  // entries each); batch <= 1: one volume.  batch_ny (tiles along n per
  // volume) is set by the launcher.
  int batch;
  int batch_ny;
};

struct Geometry {
  int M, N, S;        // sizes of the real volume
  int dr, dc, ds;     // aliasing groups (1,1,1 for LR transforms)
  int Ml, Nl, Sl;
  int Ms, Mp;         // m slots / pitch of the spectral layout
  FftAxis fm, fn, fs; // fm has length M/2
  int tw_s;           // s-pass tile width (multiple of dr)
  int g_s;            // s-pass tile height in n slots (multiple of dc)
  int tw_n;           // n-pass tile width
  int ts_tv;          // TV kernel: s planes per CTA (0 = default rule)
  int lm_f, lm_i;     // m passes (forward, inverse): lines per CTA (0 = default rule)
  long long V() const { return (long long)M * N * S; }
  long long spec_elems() const { return (long long)S * N * Mp; }
};

// Device state of the tolerance loop of sr3d_admm_tv (Algorithm 1, step 5).
struct TolCtl {
  int blocks;      // evaluation blocks the loop has run
  int max_blocks;  // blocks that fit in the iteration budget
  double tol;      // stop once primal_rel < tol and dual_rel < tol
};

struct Plan {
  int dtype;     // 0 float, 1 double
  size_t esz;    // element size
  Geometry hr, lr;
  double psf_sum;
  bool tv_aniso = false;   // u-step and TV term of the anisotropic TV (sr3d_set_tv)
  bool sep_avail = false;  // the PSF is an outer product of three 1-D factors
  bool sep_on = true;      // use the 1-D Lambda tables in the class solve when available
  void* lamM1 = nullptr; void* lamN1 = nullptr; void* lamS1 = nullptr;  // 1-D factor DFTs (complex)
  cudaStream_t stream;
  bool own_stream;
  // device buffers
  void* twM = nullptr; void* twN = nullptr; void* twS = nullptr;     // HR twiddles
  void* twMl = nullptr; void* twNl = nullptr; void* twSl = nullptr;  // LR twiddles
  void* symM = nullptr; void* symN = nullptr; void* symS = nullptr;
  void* lam = nullptr;    // HR spectral
  void* lam_solve = nullptr;   // Lambda in the solve order of the s pass
  void* yhat_solve = nullptr;  // LR spectrum in the same order
  long long lam_solve_cap = 0, yhat_solve_cap = 0;  // allocated elements
  int version = 0;             // bumped whenever the tile schedule changes
  void* yhat = nullptr;   // LR spectral
  void* spec = nullptr;   // HR spectral work
  void* theta = nullptr;  // HR real
  void* dbuf[2] = {nullptr, nullptr};  // ADMM dual, 3 V each
  void* psi = nullptr;                  // L^T u of the previous iteration
  void* xh = nullptr; void* yh = nullptr;  // staging for host-buffer calls
  void* fit_lr = nullptr;        // DHx of the PSF fit (LR real)
  double* fit_partial = nullptr; // its five FP64 sums: per-CTA partials, then the totals
  double* partial = nullptr;  // TV-kernel partial sums
  double* partial_s = nullptr;  // s-pass partial sums
  double* result = nullptr;   // finalize output (16 doubles)
  double* hist = nullptr;     // objective history (device)
  int hist_cap = 0;
  long long n_tv_blocks = 0, n_s_blocks = 0;
  long long bytes = 0;
  // per-kernel accounting (sr3d_profile)
  bool prof_on = false;
  int kind_override = -1;  // >= 0: account every launch to this kind
  int prof_cap = 0, prof_n = 0;
  cudaEvent_t* prof_ev = nullptr;  // 2 * prof_cap events
  int* prof_kind = nullptr;
  double prof_ms[8] = {0};
  long long launches[8] = {0};
  // CUDA graph of two ADMM iterations (x-step + TV step twice, dual buffers
  // swapped), replayed by sr3d_admm_tv for iterations without statistics
  cudaGraphExec_t iter_graph = nullptr;
  const void* ig_x = nullptr;
  const void* ig_d0 = nullptr;
  const void* ig_d1 = nullptr;
  double ig_thr = 0, ig_rho = 0;
  long long ig_launches[8] = {0};
  // CUDA graphs of one evaluation block of sr3d_admm_tv with statistics:
  // every-1 iterations, the iteration that evaluates (statistics kernels in
  // the last two), the finalize and the copy of its results to pinned host
  // memory.  One graph per dual-buffer parity at the start of the block.
  cudaGraphExec_t eval_graph[2] = {nullptr, nullptr};
  const void* eg_x = nullptr;
  const void* eg_d[2] = {nullptr, nullptr};
  const void* eg_hist = nullptr;
  const void* eg_partial = nullptr;
  double eg_thr = 0, eg_rho = 0, eg_lam = 0;
  int eg_every = 0;
  long long eg_launches[2][8] = {};
  int* hcount = nullptr;       // device: objective-history entries written by graph replays
  // graphs of the device-side tolerance loop (a WHILE node over evaluation
  // blocks), one per dual-buffer parity, keyed like eval_graph; the launches
  // of the gate ahead of the loop and of one block (its gate included)
  cudaGraphExec_t tol_graph[2] = {nullptr, nullptr};
  long long tg_first[2][8] = {};
  long long tg_block[2][8] = {};
  struct TolCtl* tolctl = nullptr;  // device state of that loop
  // conjugate-gradient comparator (sr3d_tikhonov_cg): r, p, Ap, a temporary,
  // per-CTA FP64 partial sums and the scalars rr, pAp, rr_new
  void* cg_buf[4] = {nullptr, nullptr, nullptr, nullptr};
  double* cg_partial = nullptr;
  double* cg_scal = nullptr;
  double* res_host = nullptr;  // pinned host copy of the finalize results
};

// ---- launchers (kernels_fft.cu) ----
cudaError_t launch_rfft_m_fwd(const Plan& p, const Geometry& g, const void* in, void* out, const void* tw);
cudaError_t launch_rfft_m_inv(const Plan& p, const Geometry& g, const void* in, void* out, const void* tw,
                              double scale);
cudaError_t launch_fft_n(const Plan& p, const Geometry& g, void* spec, const void* tw, bool inverse);
cudaError_t launch_fft_s(const Plan& p, const Geometry& g, void* spec, const void* tw, int mode, bool stats,
                         const SolveArgs* sv);
long long s_pass_blocks(const Geometry& g);
long long solve_lam_elems(const Geometry& g);
long long solve_yhat_elems(const Geometry& g);
cudaError_t launch_perm_lam(const Plan& p, const void* lam, void* out);
cudaError_t launch_perm_yhat(const Plan& p, const void* yh, void* out);

// ---- launchers (kernels_tv.cu) ----
// mode 0: ADMM step (shrink + dual update); mode 1: initial Theta = L^T (L x - d)
// ADMM TV step (isotropic or anisotropic as the plan, no statistics) over
// `batch` volumes of the plan's geometry stored one after another (x, theta:
// V each; din, dout: 3V each); the vectorised kernel only (tv_batchable).
cudaError_t launch_tv_batched(const Plan& p, int batch, const void* x, const void* din, void* dout, void* theta,
                              double thr);
bool tv_batchable(const Plan& p);
cudaError_t launch_tv(const Plan& p, const void* x, const void* din, void* dout, void* theta, void* psi,
                      double thr, int mode, bool stats);
long long tv_blocks(const Geometry& g);
int tv_default_ts(const Geometry& g);
// planes-per-CTA values for the autotuner to time (at most cap, into out)
int tv_ts_candidates(const Plan& p, int* out, int cap);
cudaError_t launch_finalize(const Plan& p, int hist_index, double lam_tv, double mu, double inv_nl,
                            bool with_data);
// The stopping test of Algorithm 1 (step 5) made on the device for the
// graph loop of sr3d_admm_tv; see k_tol_gate.
cudaError_t launch_tol_gate(const Plan& p, int count, cudaGraphConditionalHandle loop,
                            cudaGraphConditionalHandle next, bool has_next);
cudaError_t launch_twiddle(const Plan& p, void* tw, int n);
cudaError_t launch_symbol(const Plan& p, void* sym, int n);
cudaError_t launch_wrap_psf(const Plan& p, void* out, const double* psf_dev, int pm, int pn, int ps);
cudaError_t launch_export_half(const Plan& p, const void* spec, void* out);

cudaError_t launch_dft_factor(const Plan& p, void* out, const double* f_dev, int pf, int n);
// conjugate-gradient comparator (kernels_cg.cu)
constexpr int CG_BLOCKS = 1024;
cudaError_t launch_zero_fill(const Plan& p, const void* y, void* z);
cudaError_t launch_nn_replicate(const Plan& p, const void* y, void* xb);
cudaError_t launch_mask_lattice(const Plan& p, void* v);
cudaError_t launch_cg_init(const Plan& p, const void* hty, const void* xbar, double tau, void* x, void* r, void* pv);
cudaError_t launch_cg_ap(const Plan& p, void* w_ap, const void* pv, double tau);
cudaError_t launch_cg_update(const Plan& p, void* x, void* r, const void* pv, const void* ap);
cudaError_t launch_cg_dir(const Plan& p, const void* r, void* pv);
cudaError_t launch_cg_reduce(const Plan& p, int slot, int copy_from, int copy_to);
// partial: 5 * CG_BLOCKS doubles; out: 5 doubles (device)
cudaError_t launch_fit_moments(const Plan& p, const void* yh, const void* y, double* partial, double* out);
// KKT-consistent initial dual from x (unet.cu)
cudaError_t launch_dual_init(const Plan& p, const void* x, double thr, void* d);
// sets the calling thread's last-error text (api.cu) and returns code
int record_error(int code, const char* msg);

}  // namespace sr3d

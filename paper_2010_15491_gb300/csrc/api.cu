// C ABI of libsr3d (declared in include/sr3d.h): plan construction and the
// solver entry points.  Every numerical step runs in the kernels of
// kernels_fft.cu and kernels_tv.cu; this file validates arguments, owns
// device memory and sequences launches on the plan's stream.
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <cmath>
#include <functional>
#include <map>
#include <mutex>
#include <tuple>
#include <string>
#include <algorithm>
#include <atomic>
#include <initializer_list>
#include <vector>

#include "fft_host.cuh"
#include "internal.h"
#include "sr3d.h"

using namespace sr3d;

struct sr3d_plan_s {
  Plan p;
};

static thread_local std::string g_err;

static int fail(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_err = buf;
  return code;
}

int sr3d::record_error(int code, const char* msg) { return fail(code, "%s", msg); }

#define CK(call)                                                                                  \
  do {                                                                                            \
    cudaError_t e_ = (call);                                                                      \
    if (e_ != cudaSuccess)                                                                        \
      return fail(e_ == cudaErrorMemoryAllocation ? SR3D_ERR_OOM : SR3D_ERR_CUDA, "%s: %s", #call, \
                  cudaGetErrorString(e_));                                                        \
  } while (0)

// Launch accounting: counts every launch by kind and, when profiling is on,
// brackets it with events on the plan's stream (resolved at sync_plan).
static cudaError_t prof_begin(Plan& p, int kind) {
  if (p.kind_override >= 0) kind = p.kind_override;
  p.launches[kind]++;
  if (!p.prof_on || p.prof_n >= p.prof_cap) return cudaSuccess;
  p.prof_kind[p.prof_n] = kind;
  return cudaEventRecord(p.prof_ev[2 * p.prof_n], p.stream);
}
static cudaError_t prof_end(Plan& p) {
  if (!p.prof_on || p.prof_n >= p.prof_cap) return cudaSuccess;
  cudaError_t e = cudaEventRecord(p.prof_ev[2 * p.prof_n + 1], p.stream);
  p.prof_n++;
  return e;
}
#define LAUNCH(kind, call)                                   \
  do {                                                       \
    CK(prof_begin(p, kind));                                 \
    CK(call);                                                \
    CK(prof_end(p));                                         \
  } while (0)

#define TRY(call)              \
  do {                         \
    int r_ = (call);           \
    if (r_ != SR3D_OK) return r_; \
  } while (0)

// ---------------------------------------------------------------------------
// geometry
// ---------------------------------------------------------------------------
static bool is_pow2(int n) { return n > 0 && (n & (n - 1)) == 0; }
static bool supported_len(int n) { return is_pow2(n) || (n % 3 == 0 && is_pow2(n / 3)); }

// Elements per thread e (largest allowed that divides n) and Stockham radices
// (each dividing e).  Powers of two: e <= 16 (float) or 8 (double); 3 * 2^a:
// e <= 12.  Must agree with Emax<T> in common.cuh.
static FftAxis make_axis(int n, size_t esz) {
  FftAxis f;
  memset(&f, 0, sizeof(f));
  f.n = n;
  if (n % 3 == 0) {
    const int cand[3] = {12, 6, 3};
    for (int c : cand)
      if (c <= n && n % c == 0) { f.e = c; break; }
  } else {
    const int p2 = esz == 4 ? 16 : 8;
    const int cand[5] = {16, 8, 4, 2, 1};
    for (int c : cand)
      if (c <= p2 && c <= n && n % c == 0) { f.e = c; break; }
  }
  int rest = n;
  if (rest % 3 == 0) {
    f.radix[f.nst++] = 3;
    rest /= 3;
    const int rads[3] = {4, 2, 1};
    for (int r : rads)
      while (r > 1 && rest % r == 0 && f.e % r == 0) { f.radix[f.nst++] = r; rest /= r; }
    return f;
  }
  // powers of two: [remainder, P, P, ...] with P = e when e is the full
  // 16 (float) or 8 (double): later stages then use one radix only
  int big = 0, pw = f.e;
  while (rest % pw == 0 && pw > 1) { rest /= pw; ++big; }
  if (rest > 1) f.radix[f.nst++] = rest;  // 2, 4 or 8 (< pw, divides e)
  for (int i = 0; i < big; ++i) f.radix[f.nst++] = pw;
  return f;
}

static Geometry make_geom(int M, int N, int S, int dr, int dc, int ds, size_t csz) {
  Geometry g;
  memset(&g, 0, sizeof(g));
  g.M = M; g.N = N; g.S = S;
  g.dr = dr; g.dc = dc; g.ds = ds;
  g.Ml = M / dr; g.Nl = N / dc; g.Sl = S / ds;
  g.Ms = (g.Ml / 2 + 1) * dr;
  g.Mp = (g.Ms + 1) & ~1;
  g.fm = make_axis(M / 2, csz / 2);
  g.fn = make_axis(N, csz / 2);
  g.fs = make_axis(S, csz / 2);
  // n pass: TW slots x N rows, TW * N / e threads
  {
    const int tpl = N / g.fn.e;
    int tw = 256 / tpl;
    tw = tw < 1 ? 1 : (tw > 64 ? 64 : tw);
    if (tw > 1) tw &= ~1;
    while (tw > 1 && (size_t)tw * N * csz > 96 * 1024) tw /= 2;
    const int cap = (g.Ms + 1) & ~1;
    if (tw > cap) tw = cap;
    g.tw_n = tw;
  }
  // s pass: TW (multiple of dr) slots x G = dc n-slots x S planes
  {
    const int tpl = S / g.fs.e;
    g.g_s = dc;
    int target = 256 / (dc * tpl);
    if (target < 1) target = 1;
    int tw = ((target + dr - 1) / dr) * dr;
    if (tw % 2) tw += dr;  // even when possible: keeps rows 16-byte aligned
    const int cap = ((g.Ms + 2 * dr - 1) / (2 * dr)) * (2 * dr);
    if (tw > cap) tw = cap;
    while (tw > dr && ((long long)tw * dc * tpl > 512 || (size_t)tw * dc * S * csz > 160 * 1024)) tw -= dr;
    g.tw_s = tw;
  }
  return g;
}

static int validate_lengths(const Geometry& g, size_t csz) {
  const int lens[3] = {g.M / 2, g.N, g.S};
  for (int n : lens)
    if (n >= 1 && !supported_len(n)) return fail(SR3D_ERR_UNSUPPORTED_SIZE, "FFT length %d is not 2^a or 3*2^a", n);
  if ((long long)g.tw_s * g.g_s * (g.S / g.fs.e) > 512 || (size_t)g.tw_s * g.g_s * g.S * csz > 200 * 1024 ||
      (long long)g.tw_n * (g.N / g.fn.e) > 256 || (g.M / 2) / g.fm.e > 256)
    return fail(SR3D_ERR_UNSUPPORTED_SIZE, "s-pass tile does not fit (S=%d, dc=%d)", g.S, g.dc);
  return SR3D_OK;
}

// Cap on the device bytes one plan may hold (0 = none); see
// sr3d_set_plan_memory_limit.  A plan that would pass it fails with
// SR3D_ERR_OOM exactly as if cudaMalloc had failed.
static std::atomic<long long> g_plan_mem_limit{0};

static int dmalloc(Plan& p, void** ptr, size_t bytes) {
  const long long cap = g_plan_mem_limit.load();
  if (cap > 0 && p.bytes + (long long)bytes > cap) {
    *ptr = nullptr;
    return fail(SR3D_ERR_OOM, "plan memory limit: %lld bytes held + %zu requested > %lld", p.bytes, bytes, cap);
  }
  cudaError_t e = cudaMalloc(ptr, bytes);
  if (e != cudaSuccess) {
    *ptr = nullptr;
    cudaGetLastError();
    return fail(e == cudaErrorMemoryAllocation ? SR3D_ERR_OOM : SR3D_ERR_CUDA, "cudaMalloc(%zu): %s", bytes,
                cudaGetErrorString(e));
  }
  p.bytes += (long long)bytes;
  return SR3D_OK;
}

static void free_plan(Plan& p) {
  void* bufs[] = {p.twM, p.twN, p.twS, p.twMl, p.twNl, p.twSl, p.symM, p.symN, p.symS, p.lam, p.lam_solve,
                  p.yhat_solve, p.yhat, p.spec,
                  p.theta, p.dbuf[0], p.dbuf[1], p.psi, p.xh, p.yh, p.partial, p.partial_s, p.result, p.hist,
                  p.lamM1, p.lamN1, p.lamS1, p.cg_buf[0], p.cg_buf[1], p.cg_buf[2], p.cg_buf[3],
                  p.cg_partial, p.cg_scal, p.fit_lr, p.fit_partial};
  for (void* b : bufs)
    if (b) cudaFree(b);
  if (p.iter_graph) cudaGraphExecDestroy(p.iter_graph);
  for (auto& g : p.eval_graph)
    if (g) cudaGraphExecDestroy(g);
  for (auto& g : p.tol_graph)
    if (g) cudaGraphExecDestroy(g);
  if (p.hcount) cudaFree(p.hcount);
  if (p.tolctl) cudaFree(p.tolctl);
  if (p.res_host) cudaFreeHost(p.res_host);
  if (p.own_stream && p.stream) cudaStreamDestroy(p.stream);
  for (int i = 0; i < 2 * p.prof_cap; ++i) cudaEventDestroy(p.prof_ev[i]);
  delete[] p.prof_ev;
  delete[] p.prof_kind;
}

// Is the PSF an outer product f_s x f_n x f_m?  With T the sum of its taps,
// the factors are its marginal sums and psf = f_s f_n f_m / T^2 exactly when
// it is separable; accepted if every tap agrees to rounding (1e-14 of the
// largest).  fm absorbs the 1 / T^2.
static bool separable_factors(const double* psf, int pm, int pn, int ps, std::vector<double>& fm,
                              std::vector<double>& fn, std::vector<double>& fs) {
  fm.assign(pm, 0.0);
  fn.assign(pn, 0.0);
  fs.assign(ps, 0.0);
  double tot = 0.0, big = 0.0;
  for (int a = 0; a < ps; ++a)
    for (int b = 0; b < pn; ++b)
      for (int c = 0; c < pm; ++c) {
        const double v = psf[((long long)a * pn + b) * pm + c];
        fs[a] += v;
        fn[b] += v;
        fm[c] += v;
        tot += v;
        big = std::max(big, std::fabs(v));
      }
  if (tot == 0.0 || big == 0.0) return false;
  const double it2 = 1.0 / (tot * tot);
  for (int a = 0; a < ps; ++a)
    for (int b = 0; b < pn; ++b)
      for (int c = 0; c < pm; ++c) {
        const double v = psf[((long long)a * pn + b) * pm + c];
        if (std::fabs(v - fs[a] * fn[b] * fm[c] * it2) > 1e-14 * big) return false;
      }
  for (double& v : fm) v *= it2;
  return true;
}

// Lambda = DFT of the origin-wrapped PSF (Algorithm 1 step 1) into p.lam and
// its solve-order copy; for a separable PSF also the three 1-D factor DFTs.
// Uses p.theta as scratch; synchronises the stream.
static int compute_lambda(Plan& p, const double* psf, int pm, int pn, int ps) {
  const Geometry& g = p.hr;
  const size_t csz = 2 * p.esz;
  const long long np = (long long)pm * pn * ps;
  double psum = 0;
  for (long long i = 0; i < np; ++i) psum += psf[i];
  p.psf_sum = psum;
  void* psf_dev = nullptr;
  cudaError_t e = cudaMalloc(&psf_dev, (size_t)np * sizeof(double));
  if (e != cudaSuccess) return fail(SR3D_ERR_OOM, "PSF upload: %s", cudaGetErrorString(e));
  e = cudaMemcpyAsync(psf_dev, psf, (size_t)np * sizeof(double), cudaMemcpyHostToDevice, p.stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(p.theta, 0, (size_t)g.V() * p.esz, p.stream);
  if (e == cudaSuccess) e = launch_wrap_psf(p, p.theta, (const double*)psf_dev, pm, pn, ps);
  if (e == cudaSuccess) e = launch_rfft_m_fwd(p, g, p.theta, p.lam, p.twM);
  if (e == cudaSuccess) e = launch_fft_n(p, g, p.lam, p.twN, false);
  if (e == cudaSuccess) e = launch_fft_s(p, g, p.lam, p.twS, S_FWD, false, nullptr);
  if (e == cudaSuccess) e = launch_perm_lam(p, p.lam, p.lam_solve);
  if (e == cudaSuccess) e = cudaStreamSynchronize(p.stream);
  cudaFree(psf_dev);
  if (e != cudaSuccess) return fail(SR3D_ERR_CUDA, "Lambda: %s", cudaGetErrorString(e));
  // separable PSF: the 1-D factor DFTs, whose products the class solve uses
  std::vector<double> fm, fn, fs;
  p.sep_avail = false;
  if (separable_factors(psf, pm, pn, ps, fm, fn, fs)) {
    if (!p.lamM1) TRY(dmalloc(p, &p.lamM1, (size_t)g.M * csz));
    if (!p.lamN1) TRY(dmalloc(p, &p.lamN1, (size_t)g.N * csz));
    if (!p.lamS1) TRY(dmalloc(p, &p.lamS1, (size_t)g.S * csz));
    double* fdev = nullptr;
    const size_t nf = fm.size() + fn.size() + fs.size();
    CK(cudaMalloc(&fdev, nf * sizeof(double)));
    std::vector<double> all(fm);
    all.insert(all.end(), fn.begin(), fn.end());
    all.insert(all.end(), fs.begin(), fs.end());
    e = cudaMemcpyAsync(fdev, all.data(), nf * sizeof(double), cudaMemcpyHostToDevice, p.stream);
    if (e == cudaSuccess) e = launch_dft_factor(p, p.lamM1, fdev, pm, g.M);
    if (e == cudaSuccess) e = launch_dft_factor(p, p.lamN1, fdev + fm.size(), pn, g.N);
    if (e == cudaSuccess) e = launch_dft_factor(p, p.lamS1, fdev + fm.size() + fn.size(), ps, g.S);
    if (e == cudaSuccess) e = cudaStreamSynchronize(p.stream);
    cudaFree(fdev);
    if (e != cudaSuccess) return fail(SR3D_ERR_CUDA, "Lambda (separable PSF): %s", cudaGetErrorString(e));
    p.sep_avail = true;
  }
  return SR3D_OK;
}

static SolveArgs solve_args(const Plan& p, int mode_alpha_nn, double alpha) {
  SolveArgs sv;
  memset(&sv, 0, sizeof(sv));
  const Geometry& g = p.hr;
  sv.lam = p.lam_solve;
  sv.yhat = p.yhat_solve;
  sv.lr_out = p.yhat;
  sv.symM = p.symM; sv.symN = p.symN; sv.symS = p.symS;
  sv.twM = p.twM; sv.twN = p.twN; sv.twS = p.twS;
  sv.alpha = alpha;
  sv.nn_prior = mode_alpha_nn;
  sv.M = g.M; sv.N = g.N; sv.S = g.S;
  sv.Ml = g.Ml; sv.Nl = g.Nl; sv.Sl = g.Sl;
  sv.dr = g.dr; sv.dc = g.dc; sv.ds = g.ds;
  sv.Mlp = p.lr.Mp;
  sv.partial = p.partial_s;
  sv.lamM = p.lamM1; sv.lamN = p.lamN1; sv.lamS = p.lamS1;
  sv.sep = (p.sep_avail && p.sep_on) ? 1 : 0;
  sv.lam_nat = p.lam;
  return sv;
}

// ---------------------------------------------------------------------------
// pipelines
// ---------------------------------------------------------------------------
static int lr_spectrum(Plan& p, const void* y) {
  LAUNCH(SR3D_K_RFFT_FWD, launch_rfft_m_fwd(p, p.lr, y, p.yhat, p.twMl));
  LAUNCH(SR3D_K_FFTN_FWD, launch_fft_n(p, p.lr, p.yhat, p.twNl, false));
  LAUNCH(SR3D_K_FFTS, launch_fft_s(p, p.lr, p.yhat, p.twSl, S_FWD, false, nullptr));
  LAUNCH(SR3D_K_OTHER, launch_perm_yhat(p, p.yhat, p.yhat_solve));
  return SR3D_OK;
}

static int hr_forward_partial(Plan& p, const void* x) {
  LAUNCH(SR3D_K_RFFT_FWD, launch_rfft_m_fwd(p, p.hr, x, p.spec, p.twM));
  LAUNCH(SR3D_K_FFTN_FWD, launch_fft_n(p, p.hr, p.spec, p.twN, false));
  return SR3D_OK;
}

static int hr_inverse_partial(Plan& p, void* x) {
  LAUNCH(SR3D_K_FFTN_INV, launch_fft_n(p, p.hr, p.spec, p.twN, true));
  LAUNCH(SR3D_K_RFFT_INV, launch_rfft_m_inv(p, p.hr, p.spec, x, p.twM, 1.0 / (double)p.hr.V()));
  return SR3D_OK;
}

static int tikhonov_core(Plan& p, const void* xbar, double tau, void* x) {
  if (xbar && xbar != SR3D_XBAR_NEAREST) {
    TRY(hr_forward_partial(p, xbar));
    SolveArgs sv = solve_args(p, 0, tau);
    LAUNCH(SR3D_K_FFTS, launch_fft_s(p, p.hr, p.spec, p.twS, S_TIK_USER, false, &sv));
  } else {
    SolveArgs sv = solve_args(p, xbar == SR3D_XBAR_NEAREST ? 1 : 0, tau);
    LAUNCH(SR3D_K_FFTS, launch_fft_s(p, p.hr, p.spec, p.twS, S_TIK_GEN, false, &sv));
  }
  return hr_inverse_partial(p, x);
}

static int xstep_core(Plan& p, const void* theta, double mu, void* x, bool stats) {
  TRY(hr_forward_partial(p, theta));
  SolveArgs sv = solve_args(p, 0, mu);
  LAUNCH(SR3D_K_FFTS, launch_fft_s(p, p.hr, p.spec, p.twS, S_ADMM, stats, &sv));
  return hr_inverse_partial(p, x);
}

static int sync_plan(Plan& p);

// One ADMM iteration without statistics: x-step from Theta, then the TV step
// (u, d_in -> d_out, next Theta).
static int admm_iteration(Plan& p, void* x, const void* din, void* dout, double thr, double rho);

// Runs n >= 2 iterations (n even) through the cached two-iteration graph,
// capturing it first when the buffers or parameters changed.
static int admm_iterations_graph(Plan& p, void* x, void* d0, void* d1, double thr, double rho, int n) {
  if (!p.iter_graph || p.ig_x != x || p.ig_d0 != d0 || p.ig_d1 != d1 || p.ig_thr != thr || p.ig_rho != rho) {
    if (p.iter_graph) {
      cudaGraphExecDestroy(p.iter_graph);
      p.iter_graph = nullptr;
    }
    long long before[8];
    for (int k = 0; k < 8; ++k) before[k] = p.launches[k];
    cudaGraph_t graph = nullptr;
    CK(cudaStreamBeginCapture(p.stream, cudaStreamCaptureModeThreadLocal));
    int rc = admm_iteration(p, x, d0, d1, thr, rho);
    if (rc == SR3D_OK) rc = admm_iteration(p, x, d1, d0, thr, rho);
    cudaError_t ec = cudaStreamEndCapture(p.stream, &graph);
    if (rc != SR3D_OK) {
      if (graph) cudaGraphDestroy(graph);
      return rc;
    }
    if (ec != cudaSuccess) return fail(SR3D_ERR_CUDA, "graph capture: %s", cudaGetErrorString(ec));
    ec = cudaGraphInstantiate(&p.iter_graph, graph, 0);
    cudaGraphDestroy(graph);
    if (ec != cudaSuccess) {
      p.iter_graph = nullptr;
      return fail(SR3D_ERR_CUDA, "graph instantiate: %s", cudaGetErrorString(ec));
    }
    for (int k = 0; k < 8; ++k) {
      p.ig_launches[k] = p.launches[k] - before[k];
      p.launches[k] = before[k];
    }
    p.ig_x = x; p.ig_d0 = d0; p.ig_d1 = d1; p.ig_thr = thr; p.ig_rho = rho;
  }
  for (int i = 0; i + 2 <= n; i += 2) {
    CK(cudaGraphLaunch(p.iter_graph, p.stream));
    for (int k = 0; k < 8; ++k) p.launches[k] += p.ig_launches[k];
  }
  return SR3D_OK;
}

static int admm_iteration(Plan& p, void* x, const void* din, void* dout, double thr, double rho) {
  TRY(xstep_core(p, p.theta, rho, x, false));
  LAUNCH(SR3D_K_TV, launch_tv(p, x, din, dout, p.theta, p.psi, thr, 0, false));
  return SR3D_OK;
}

static void drop_eval_graphs(Plan& p) {
  for (cudaGraphExec_t* gs : {p.eval_graph, p.tol_graph})
    for (int i = 0; i < 2; ++i)
      if (gs[i]) {
        cudaGraphExecDestroy(gs[i]);
        gs[i] = nullptr;
      }
}

// One evaluation block: iterations 1..every, statistics kernels in the last
// two (the dual residual needs L^T u of the iteration before), the finalize
// (objective history indexed on the device) and, when to_host, the copy of
// its results to pinned host memory.  d0 -> d1 -> d0 ... through the block.
static int admm_eval_block(Plan& p, void* x, void* d0, void* d1, double thr, double rho, double lambda,
                           int every, bool to_host = true) {
  void* a = d0;
  void* b = d1;
  for (int j = 1; j <= every; ++j) {
    const bool eval_now = j == every;
    const bool stats_now = eval_now || j + 1 == every;
    TRY(xstep_core(p, p.theta, rho, x, eval_now));
    LAUNCH(SR3D_K_TV, launch_tv(p, x, a, b, p.theta, p.psi, thr, 0, stats_now));
    void* t = a;
    a = b;
    b = t;
  }
  LAUNCH(SR3D_K_OTHER, launch_finalize(p, -2, lambda, rho, 1.0 / (double)p.lr.V(), true));
  if (to_host) CK(cudaMemcpyAsync(p.res_host, p.result, 11 * sizeof(double), cudaMemcpyDeviceToHost, p.stream));
  return SR3D_OK;
}

// Keys the cached evaluation-block and tolerance-loop graphs: drops them
// when the buffers or parameters they were captured with changed.
static void key_eval_graphs(Plan& p, void* x, void* d0, void* d1, double thr, double rho, double lambda, int every,
                            int par) {
  if (p.eg_x != x || p.eg_thr != thr || p.eg_rho != rho || p.eg_lam != lambda || p.eg_every != every ||
      p.eg_hist != p.hist || p.eg_partial != p.partial || p.eg_d[par] != d0 || p.eg_d[1 - par] != d1) {
    drop_eval_graphs(p);
    p.eg_x = x; p.eg_thr = thr; p.eg_rho = rho; p.eg_lam = lambda; p.eg_every = every;
    p.eg_hist = p.hist; p.eg_partial = p.partial;
    p.eg_d[par] = d0; p.eg_d[1 - par] = d1;
  }
}

// Replays the evaluation block whose dual buffers start as (d0, d1),
// capturing it first when buffers or parameters changed.  par selects the
// cached graph (0: first buffer order seen, 1: the swapped order).
static int admm_eval_block_graph(Plan& p, void* x, void* d0, void* d1, double thr, double rho, double lambda,
                                 int every, int par) {
  key_eval_graphs(p, x, d0, d1, thr, rho, lambda, every, par);
  cudaGraphExec_t& ge = p.eval_graph[par];
  if (!ge) {
    long long before[8];
    for (int k = 0; k < 8; ++k) before[k] = p.launches[k];
    cudaGraph_t graph = nullptr;
    CK(cudaStreamBeginCapture(p.stream, cudaStreamCaptureModeThreadLocal));
    const int rc = admm_eval_block(p, x, d0, d1, thr, rho, lambda, every);
    cudaError_t ec = cudaStreamEndCapture(p.stream, &graph);
    if (rc != SR3D_OK) {
      if (graph) cudaGraphDestroy(graph);
      return rc;
    }
    if (ec != cudaSuccess) return fail(SR3D_ERR_CUDA, "graph capture: %s", cudaGetErrorString(ec));
    ec = cudaGraphInstantiate(&ge, graph, 0);
    cudaGraphDestroy(graph);
    if (ec != cudaSuccess) {
      ge = nullptr;
      return fail(SR3D_ERR_CUDA, "graph instantiate: %s", cudaGetErrorString(ec));
    }
    for (int k = 0; k < 8; ++k) {
      p.eg_launches[par][k] = p.launches[k] - before[k];
      p.launches[k] = before[k];
    }
  }
  CK(cudaGraphLaunch(ge, p.stream));
  for (int k = 0; k < 8; ++k) p.launches[k] += p.eg_launches[par][k];
  return SR3D_OK;
}

// Captures work() on the plan's stream into g, an existing graph (a
// conditional node's body or the loop graph itself); *last, when given,
// receives the one node the captured work ends on.
template <class F>
static int capture_to(Plan& p, cudaGraph_t g, F&& work, cudaGraphNode_t* last) {
  CK(cudaStreamBeginCaptureToGraph(p.stream, g, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
  int rc = work();
  if (rc == SR3D_OK && last) {
    cudaStreamCaptureStatus st;
    const cudaGraphNode_t* deps = nullptr;
    size_t nd = 0;
    const cudaError_t e = cudaStreamGetCaptureInfo(p.stream, &st, nullptr, nullptr, &deps, nullptr, &nd);
    if (e != cudaSuccess || nd != 1 || !deps)
      rc = fail(SR3D_ERR_CUDA, "graph capture: the captured work does not end on one node");
    else
      *last = deps[0];
  }
  cudaGraph_t out = nullptr;
  const cudaError_t ec = cudaStreamEndCapture(p.stream, &out);
  if (rc != SR3D_OK) return rc;
  if (ec != cudaSuccess) return fail(SR3D_ERR_CUDA, "graph capture: %s", cudaGetErrorString(ec));
  return SR3D_OK;
}

// Adds a conditional node of the given type after dep; *body receives the
// graph it runs (owned by the node).
static int add_conditional(cudaGraph_t g, cudaGraphNode_t dep, cudaGraphConditionalHandle h,
                           cudaGraphConditionalNodeType type, cudaGraph_t* body) {
  cudaGraphNodeParams cp = {};
  cp.type = cudaGraphNodeTypeConditional;
  cp.conditional.handle = h;
  cp.conditional.type = type;
  cp.conditional.size = 1;
  cudaGraphNode_t node;
  CK(cudaGraphAddNode(&node, g, &dep, nullptr, 1, &cp));
  *body = cp.conditional.phGraph_out[0];
  return SR3D_OK;
}

// The tolerance loop of Algorithm 1 as one graph, replayed without the host
// between blocks: a gate (k_tol_gate) on the evaluation made before it, then
// a WHILE node whose body runs one evaluation block and the gate again.
// For odd `every` a block swaps the dual buffers, so the body holds two
// blocks, the second under an IF node set by the first block's gate, and
// leaves the buffers in the order it found them.  The caller has written
// p.tolctl (blocks = 0, the block budget, tol) and p.hcount.
static int admm_tol_graph(Plan& p, void* x, void* d0, void* d1, double thr, double rho, double lambda, int every,
                          int par) {
  key_eval_graphs(p, x, d0, d1, thr, rho, lambda, every, par);
  cudaGraphExec_t& ge = p.tol_graph[par];
  if (!ge) {
    long long base[8], mark[8];
    for (int k = 0; k < 8; ++k) base[k] = mark[k] = p.launches[k];
    auto counted = [&](long long* out) {
      for (int k = 0; k < 8; ++k) {
        out[k] = p.launches[k] - mark[k];
        mark[k] = p.launches[k];
      }
    };
    cudaGraph_t g = nullptr;
    CK(cudaGraphCreate(&g, 0));
    struct Owner {
      cudaGraph_t g;
      ~Owner() { cudaGraphDestroy(g); }
    } owner{g};
    cudaGraphConditionalHandle loop;
    CK(cudaGraphConditionalHandleCreate(&loop, g, 0, 0));
    cudaGraphNode_t gate = nullptr;
    TRY(capture_to(p, g, [&]() -> int {
      LAUNCH(SR3D_K_OTHER, launch_tol_gate(p, 0, loop, loop, false));
      return SR3D_OK;
    }, &gate));
    counted(p.tg_first[par]);
    cudaGraph_t body = nullptr;
    TRY(add_conditional(g, gate, loop, cudaGraphCondTypeWhile, &body));
    const bool two = (every & 1) != 0;
    cudaGraphConditionalHandle next = 0;
    if (two) CK(cudaGraphConditionalHandleCreate(&next, body, 0, 0));
    cudaGraphNode_t end_a = nullptr;
    TRY(capture_to(p, body, [&]() -> int {
      TRY(admm_eval_block(p, x, d0, d1, thr, rho, lambda, every, false));
      LAUNCH(SR3D_K_OTHER, launch_tol_gate(p, 1, loop, next, two));
      return SR3D_OK;
    }, two ? &end_a : nullptr));
    counted(p.tg_block[par]);
    if (two) {
      cudaGraph_t second = nullptr;
      TRY(add_conditional(body, end_a, next, cudaGraphCondTypeIf, &second));
      TRY(capture_to(p, second, [&]() -> int {
        TRY(admm_eval_block(p, x, d1, d0, thr, rho, lambda, every, false));
        LAUNCH(SR3D_K_OTHER, launch_tol_gate(p, 1, loop, loop, false));
        return SR3D_OK;
      }, nullptr));
    }
    for (int k = 0; k < 8; ++k) p.launches[k] = base[k];
    const cudaError_t ec = cudaGraphInstantiate(&ge, g, 0);
    if (ec != cudaSuccess) {
      ge = nullptr;
      return fail(SR3D_ERR_CUDA, "graph instantiate: %s", cudaGetErrorString(ec));
    }
  }
  CK(cudaGraphLaunch(ge, p.stream));
  return SR3D_OK;
}

static int sync_plan(Plan& p) {
  CK(cudaStreamSynchronize(p.stream));
  for (int i = 0; i < p.prof_n; ++i) {
    float ms = 0;
    CK(cudaEventElapsedTime(&ms, p.prof_ev[2 * i], p.prof_ev[2 * i + 1]));
    p.prof_ms[p.prof_kind[i]] += ms;
  }
  p.prof_n = 0;
  return SR3D_OK;
}

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
extern "C" {

const char* sr3d_last_error(void) { return g_err.c_str(); }

int sr3d_plan(sr3d_plan_t* out, const sr3d_desc* d) {
  if (!out || !d) return fail(SR3D_ERR_INVALID_ARG, "NULL argument");
  *out = nullptr;
  if (d->m_h <= 0 || d->n_h <= 0 || d->s_h <= 0 || d->dr <= 0 || d->dc <= 0 || d->ds <= 0)
    return fail(SR3D_ERR_INVALID_ARG, "sizes and decimation factors must be positive");
  if (!d->psf || d->p_m <= 0 || d->p_n <= 0 || d->p_s <= 0) return fail(SR3D_ERR_INVALID_ARG, "missing PSF");
  if (d->dtype != SR3D_F32 && d->dtype != SR3D_F64) return fail(SR3D_ERR_INVALID_ARG, "dtype must be F32 or F64");
  if (d->m_h % d->dr || d->n_h % d->dc || d->s_h % d->ds)
    return fail(SR3D_ERR_NOT_DIVISIBLE, "HR sizes (%d,%d,%d) not divisible by (%d,%d,%d)", d->m_h, d->n_h, d->s_h,
                d->dr, d->dc, d->ds);
  if (d->p_m > d->m_h || d->p_n > d->n_h || d->p_s > d->s_h)
    return fail(SR3D_ERR_INVALID_ARG, "PSF larger than the volume");
  if (d->m_h % 32 || d->n_h % 8 || d->s_h < 4 || d->m_h > 2048 || d->n_h > 2048 || d->s_h > 2048 ||
      !supported_len(d->m_h) || !supported_len(d->n_h) || !supported_len(d->s_h))
    return fail(SR3D_ERR_UNSUPPORTED_SIZE,
                "HR sizes must be 2^a or 3*2^a, m_h %% 32 == 0, n_h %% 8 == 0, 4 <= s_h, all <= 2048");
  if ((d->m_h / d->dr) % 2) return fail(SR3D_ERR_UNSUPPORTED_SIZE, "m_h / dr must be even");
  if (d->dr * d->dc * d->ds > 8) return fail(SR3D_ERR_UNSUPPORTED_SIZE, "dr*dc*ds must be at most 8");

  sr3d_plan_s* h = new sr3d_plan_s();
  Plan& p = h->p;
  p.dtype = d->dtype;
  p.esz = p.dtype ? 8 : 4;
  const size_t csz = 2 * p.esz;
  p.hr = make_geom(d->m_h, d->n_h, d->s_h, d->dr, d->dc, d->ds, csz);
  p.lr = make_geom(p.hr.Ml, p.hr.Nl, p.hr.Sl, 1, 1, 1, csz);
  int rc = validate_lengths(p.hr, csz);
  if (rc == SR3D_OK) rc = validate_lengths(p.lr, csz);
  if (rc != SR3D_OK) {
    delete h;
    return rc;
  }
  double psum = 0;
  const long long np = (long long)d->p_m * d->p_n * d->p_s;
  for (long long i = 0; i < np; ++i) psum += d->psf[i];
  p.psf_sum = psum;

  if (d->stream) {
    p.stream = (cudaStream_t)d->stream;
    p.own_stream = false;
  } else {
    cudaError_t e = cudaStreamCreateWithFlags(&p.stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
      delete h;
      return fail(SR3D_ERR_CUDA, "cudaStreamCreate: %s", cudaGetErrorString(e));
    }
    p.own_stream = true;
  }

  auto body = [&]() -> int {
    const Geometry& g = p.hr;
    const Geometry& l = p.lr;
    TRY(dmalloc(p, &p.twM, (size_t)g.M * csz));
    TRY(dmalloc(p, &p.twN, (size_t)g.N * csz));
    TRY(dmalloc(p, &p.twS, (size_t)g.S * csz));
    TRY(dmalloc(p, &p.twMl, (size_t)l.M * csz));
    TRY(dmalloc(p, &p.twNl, (size_t)l.N * csz));
    TRY(dmalloc(p, &p.twSl, (size_t)l.S * csz));
    TRY(dmalloc(p, &p.symM, (size_t)g.M * p.esz));
    TRY(dmalloc(p, &p.symN, (size_t)g.N * p.esz));
    TRY(dmalloc(p, &p.symS, (size_t)g.S * p.esz));
    TRY(dmalloc(p, &p.lam, (size_t)g.spec_elems() * csz));
    TRY(dmalloc(p, &p.spec, (size_t)g.spec_elems() * csz));
    TRY(dmalloc(p, &p.yhat, (size_t)l.spec_elems() * csz));
    p.lam_solve_cap = solve_lam_elems(g);
    p.yhat_solve_cap = solve_yhat_elems(g);
    TRY(dmalloc(p, &p.lam_solve, (size_t)p.lam_solve_cap * csz));
    TRY(dmalloc(p, &p.yhat_solve, (size_t)p.yhat_solve_cap * csz));
    TRY(dmalloc(p, &p.theta, (size_t)g.V() * p.esz));
    p.n_tv_blocks = tv_blocks(g);
    p.n_s_blocks = s_pass_blocks(g);
    TRY(dmalloc(p, (void**)&p.partial, (size_t)p.n_tv_blocks * 6 * sizeof(double)));
    TRY(dmalloc(p, (void**)&p.partial_s, (size_t)p.n_s_blocks * sizeof(double)));
    TRY(dmalloc(p, (void**)&p.result, 16 * sizeof(double)));
    CK(launch_twiddle(p, p.twM, g.M));
    CK(launch_twiddle(p, p.twN, g.N));
    CK(launch_twiddle(p, p.twS, g.S));
    CK(launch_twiddle(p, p.twMl, l.M));
    CK(launch_twiddle(p, p.twNl, l.N));
    CK(launch_twiddle(p, p.twSl, l.S));
    CK(launch_symbol(p, p.symM, g.M));
    CK(launch_symbol(p, p.symN, g.N));
    CK(launch_symbol(p, p.symS, g.S));
    TRY(compute_lambda(p, d->psf, d->p_m, d->p_n, d->p_s));
    return SR3D_OK;
  };
  rc = body();
  if (rc != SR3D_OK) {
    free_plan(p);
    delete h;
    return rc;
  }
  *out = h;
  return SR3D_OK;
}

int sr3d_set_plan_memory_limit(long long bytes) {
  g_plan_mem_limit.store(bytes > 0 ? bytes : 0);
  return SR3D_OK;
}

int sr3d_destroy(sr3d_plan_t plan) {
  if (!plan) return SR3D_OK;
  cudaStreamSynchronize(plan->p.stream);
  free_plan(plan->p);
  delete plan;
  return SR3D_OK;
}

int sr3d_profile(sr3d_plan_t plan, int on) {
  if (!plan) return fail(SR3D_ERR_INVALID_ARG, "NULL argument");
  Plan& p = plan->p;
  TRY(sync_plan(p));
  if (on && !p.prof_ev) {
    const int cap = 4096;
    p.prof_ev = new cudaEvent_t[2 * cap];
    p.prof_kind = new int[cap];
    for (int i = 0; i < 2 * cap; ++i) {
      cudaError_t e = cudaEventCreate(&p.prof_ev[i]);
      if (e != cudaSuccess) {
        p.prof_cap = i / 2;
        return fail(SR3D_ERR_CUDA, "cudaEventCreate: %s", cudaGetErrorString(e));
      }
      p.prof_cap = (i + 1) / 2;
    }
  }
  p.prof_on = on != 0;
  p.prof_n = 0;
  for (int k = 0; k < 8; ++k) {
    p.prof_ms[k] = 0;
    p.launches[k] = 0;
  }
  return SR3D_OK;
}

int sr3d_profile_read(sr3d_plan_t plan, double ms[SR3D_NKINDS], long long launches[SR3D_NKINDS]) {
  if (!plan || !ms || !launches) return fail(SR3D_ERR_INVALID_ARG, "NULL argument");
  Plan& p = plan->p;
  TRY(sync_plan(p));
  for (int k = 0; k < SR3D_NKINDS; ++k) {
    ms[k] = p.prof_ms[k];
    launches[k] = p.launches[k];
  }
  return SR3D_OK;
}

int sr3d_plan_info(sr3d_plan_t plan, int sizes[9], long long* bytes) {
  if (!plan || !sizes) return fail(SR3D_ERR_INVALID_ARG, "NULL argument");
  const Plan& p = plan->p;
  const int v[9] = {p.hr.M, p.hr.N, p.hr.S, p.hr.Ml, p.hr.Nl, p.hr.Sl, p.hr.Ms, p.hr.Mp, p.dtype};
  for (int i = 0; i < 9; ++i) sizes[i] = v[i];
  if (bytes) *bytes = p.bytes;
  return SR3D_OK;
}

static int realloc_partials(Plan& p);

// Tile widths the n pass and the s pass (with its class solve) accept for
// this volume: the launch limits of their kernels and, for the s pass, the
// solve-order buffers allocated with the plan.
static bool tw_n_valid(const Geometry& g, size_t csz, int tw) {
  const int tpl = g.N / g.fn.e;
  const int cap = (g.Ms + 1) & ~1;
  return tw >= 1 && tw <= 64 && tw <= cap && tw * tpl <= 256 && (size_t)tw * g.N * csz <= 96 * 1024 &&
         (tw == 1 || tw % 2 == 0);
}

static bool tw_s_valid(const Plan& p, const Geometry& g, size_t csz, int tw) {
  const int tpl = g.S / g.fs.e;
  const int cap = ((g.Ms + 2 * g.dr - 1) / (2 * g.dr)) * (2 * g.dr);
  if (tw < g.dr || tw % g.dr || tw > cap || (long long)tw * g.g_s * tpl > 512 ||
      (size_t)tw * g.g_s * g.S * csz > 160 * 1024)
    return false;
  Geometry gc = g;
  gc.tw_s = tw;
  return solve_lam_elems(gc) <= p.lam_solve_cap && solve_yhat_elems(gc) <= p.yhat_solve_cap;
}

int sr3d_schedule(sr3d_plan_t plan, const int set[5], int sched[5]) {
  if (!plan) return fail(SR3D_ERR_INVALID_ARG, "NULL plan");
  Plan& p = plan->p;
  Geometry& g = p.hr;
  const size_t csz = 2 * p.esz;
  if (set) {
    if (set[0] > 0 && !tw_n_valid(g, csz, set[0]))
      return fail(SR3D_ERR_INVALID_ARG, "n-pass tile width %d does not fit this volume", set[0]);
    if (set[1] > 0 && !tw_s_valid(p, g, csz, set[1]))
      return fail(SR3D_ERR_INVALID_ARG, "s-pass tile width %d does not fit this volume", set[1]);
    // at least 4 planes per CTA: the per-CTA partial sums are sized for that
    if (set[2] > 0 && set[2] < 4) return fail(SR3D_ERR_INVALID_ARG, "TV planes per CTA must be >= 4");
    for (int k = 3; k < 5; ++k)
      if (set[k] > 0 && !m_lines_valid(g, set[k]))
        return fail(SR3D_ERR_INVALID_ARG, "m-pass lines per CTA %d: need whole warps within 256 threads", set[k]);
    const int v[5] = {g.tw_n, g.tw_s, g.ts_tv, g.lm_f, g.lm_i};
    int w[5];
    bool change = false;
    for (int k = 0; k < 5; ++k) {
      w[k] = set[k] > 0 ? set[k] : v[k];
      change |= w[k] != v[k];
    }
    if (change) {
      TRY(sync_plan(p));
      g.tw_n = w[0];
      g.tw_s = w[1];
      g.ts_tv = w[2];
      g.lm_f = w[3];
      g.lm_i = w[4];
      TRY(realloc_partials(p));
      CK(launch_perm_lam(p, p.lam, p.lam_solve));  // Lambda in the new solve order
      if (p.iter_graph) {  // captured launches hold the old grids
        cudaGraphExecDestroy(p.iter_graph);
        p.iter_graph = nullptr;
      }
      drop_eval_graphs(p);
      ++p.version;
      TRY(sync_plan(p));
    }
  }
  if (sched) {
    int L, Hp, threads;
    size_t smem;
    sched[0] = g.tw_n;
    sched[1] = g.tw_s;
    sched[2] = g.ts_tv > 0 ? g.ts_tv : tv_default_ts(g);
    m_launch_shape(g, csz, g.lm_f, L, Hp, threads, smem);
    sched[3] = L;
    m_launch_shape(g, csz, g.lm_i, L, Hp, threads, smem);
    sched[4] = L;
  }
  return SR3D_OK;
}

int sr3d_dual_init(sr3d_plan_t plan, const void* x, double lambda, double rho, void* d) {
  if (!plan || !x || !d) return fail(SR3D_ERR_INVALID_ARG, "NULL argument");
  if (!(rho > 0) || !(lambda > 0)) return fail(SR3D_ERR_INVALID_ARG, "need rho > 0 and lambda > 0");
  Plan& p = plan->p;
  LAUNCH(SR3D_K_OTHER, launch_dual_init(p, x, lambda / rho, d));
  return sync_plan(p);
}

int sr3d_set_psf(sr3d_plan_t plan, const double* psf, int p_m, int p_n, int p_s) {
  if (!plan || !psf || p_m <= 0 || p_n <= 0 || p_s <= 0) return fail(SR3D_ERR_INVALID_ARG, "missing PSF");
  Plan& p = plan->p;
  if (p_m > p.hr.M || p_n > p.hr.N || p_s > p.hr.S) return fail(SR3D_ERR_INVALID_ARG, "PSF larger than the volume");
  TRY(sync_plan(p));
  const bool sep_before = p.sep_avail;
  TRY(compute_lambda(p, psf, p_m, p_n, p_s));
  if (p.sep_avail != sep_before) {  // captured solve arguments change with the separable path
    if (p.iter_graph) {
      cudaGraphExecDestroy(p.iter_graph);
      p.iter_graph = nullptr;
    }
    drop_eval_graphs(p);
    ++p.version;
  }
  return SR3D_OK;
}

int sr3d_set_tv(sr3d_plan_t plan, int kind) {
  if (!plan) return fail(SR3D_ERR_INVALID_ARG, "NULL argument");
  if (kind != SR3D_TV_ISOTROPIC && kind != SR3D_TV_ANISOTROPIC)
    return fail(SR3D_ERR_INVALID_ARG, "kind must be SR3D_TV_ISOTROPIC or SR3D_TV_ANISOTROPIC");
  Plan& p = plan->p;
  const bool aniso = kind == SR3D_TV_ANISOTROPIC;
  if (aniso != p.tv_aniso) {
    TRY(sync_plan(p));
    p.tv_aniso = aniso;
    if (p.iter_graph) {  // captured launches hold the other TV kernel
      cudaGraphExecDestroy(p.iter_graph);
      p.iter_graph = nullptr;
    }
    drop_eval_graphs(p);
    ++p.version;
  }
  return SR3D_OK;
}

int sr3d_tikhonov_grad(sr3d_plan_t plan, const void* y, double tau, void* x) {
  if (!plan || !y || !x) return fail(SR3D_ERR_INVALID_ARG, "NULL argument");
  if (!(tau > 0) || !std::isfinite(tau)) return fail(SR3D_ERR_INVALID_ARG, "tau must be positive");
  Plan& p = plan->p;
  if (p.psf_sum == 0.0) return fail(SR3D_ERR_SINGULAR, "PSF taps sum to zero: the zero-frequency class is singular");
  TRY(lr_spectrum(p, y));
  // the ADMM x-step with Theta = 0 and mu = tau: a zero spectrum for F Theta
  CK(cudaMemsetAsync(p.spec, 0, (size_t)p.hr.spec_elems() * 2 * p.esz, p.stream));
  SolveArgs sv = solve_args(p, 0, tau);
  LAUNCH(SR3D_K_FFTS, launch_fft_s(p, p.hr, p.spec, p.twS, S_ADMM, false, &sv));
  TRY(hr_inverse_partial(p, x));
  return sync_plan(p);
}

// w = H^T D^T D H v through two FFT round trips (Lambda, then conj(Lambda))
static int apply_normal(Plan& p, const void* v, void* w, void* tmp) {
  SolveArgs sv = solve_args(p, 0, 1.0);
  TRY(hr_forward_partial(p, v));
  LAUNCH(SR3D_K_FFTS, launch_fft_s(p, p.hr, p.spec, p.twS, S_MUL, false, &sv));
  TRY(hr_inverse_partial(p, tmp));
  LAUNCH(SR3D_K_OTHER, launch_mask_lattice(p, tmp));
  TRY(hr_forward_partial(p, tmp));
  LAUNCH(SR3D_K_FFTS, launch_fft_s(p, p.hr, p.spec, p.twS, S_MULC, false, &sv));
  return hr_inverse_partial(p, w);
}

static int read_scalar(Plan& p, int slot, double* out) {
  CK(cudaMemcpyAsync(out, p.cg_scal + slot, sizeof(double), cudaMemcpyDeviceToHost, p.stream));
  return sync_plan(p);
}

int sr3d_tikhonov_cg(sr3d_plan_t plan, const void* y, const void* xbar, double tau, double tol, int max_iters,
                     void* x, int* iters, double* relres) {
  if (!plan || !y || !x) return fail(SR3D_ERR_INVALID_ARG, "NULL argument");
  if (!(tau > 0) || !std::isfinite(tau) || max_iters < 0)
    return fail(SR3D_ERR_INVALID_ARG, "need tau > 0 and max_iters >= 0");
  if (xbar == x) return fail(SR3D_ERR_INVALID_ARG, "x and xbar must differ");
  Plan& p = plan->p;
  const size_t vb = (size_t)p.hr.V() * p.esz;
  for (auto& b : p.cg_buf)
    if (!b) TRY(dmalloc(p, &b, vb));
  if (!p.cg_partial) TRY(dmalloc(p, (void**)&p.cg_partial, CG_BLOCKS * sizeof(double)));
  if (!p.cg_scal) TRY(dmalloc(p, (void**)&p.cg_scal, 8 * sizeof(double)));
  void* r = p.cg_buf[0];
  void* pv = p.cg_buf[1];
  void* w = p.cg_buf[2];
  void* tmp = p.cg_buf[3];
  // b = H^T D^T y + tau xbar
  SolveArgs sv = solve_args(p, 0, 1.0);
  LAUNCH(SR3D_K_OTHER, launch_zero_fill(p, y, tmp));
  TRY(hr_forward_partial(p, tmp));
  LAUNCH(SR3D_K_FFTS, launch_fft_s(p, p.hr, p.spec, p.twS, S_MULC, false, &sv));
  TRY(hr_inverse_partial(p, w));
  const void* xb = nullptr;
  if (xbar == SR3D_XBAR_NEAREST) {
    LAUNCH(SR3D_K_OTHER, launch_nn_replicate(p, y, tmp));
    xb = tmp;
  } else if (xbar) {
    xb = xbar;
  }
  LAUNCH(SR3D_K_OTHER, launch_cg_init(p, w, xb, tau, x, r, pv));
  LAUNCH(SR3D_K_OTHER, launch_cg_reduce(p, 2, -1, 0));  // r.r
  double rr = 0;
  TRY(read_scalar(p, 2, &rr));
  const double bb = rr;
  int k = 0;
  while (k < max_iters && !(tol > 0 && rr <= tol * tol * bb)) {
    TRY(apply_normal(p, pv, w, tmp));
    LAUNCH(SR3D_K_OTHER, launch_cg_ap(p, w, pv, tau));         // w = A p; p.Ap
    LAUNCH(SR3D_K_OTHER, launch_cg_reduce(p, 1, 2, 0));        // rr <- rr_new, pAp
    LAUNCH(SR3D_K_OTHER, launch_cg_update(p, x, r, pv, w));    // x, r; r.r
    LAUNCH(SR3D_K_OTHER, launch_cg_reduce(p, 2, -1, 0));       // rr_new
    LAUNCH(SR3D_K_OTHER, launch_cg_dir(p, r, pv));             // p
    ++k;
    if (tol > 0) TRY(read_scalar(p, 2, &rr));
  }
  TRY(read_scalar(p, 2, &rr));
  if (!std::isfinite(rr)) return fail(SR3D_ERR_NUMERIC, "NaN/Inf in the CG residual");
  if (iters) *iters = k;
  if (relres) *relres = bb > 0 ? std::sqrt(rr / bb) : 0.0;
  if (tol > 0 && rr > tol * tol * bb) return fail(SR3D_ERR_NOT_CONVERGED, "max_iters=%d reached before tol=%g", max_iters, tol);
  return SR3D_OK;
}

int sr3d_separable(sr3d_plan_t plan, int use, int* active) {
  if (!plan) return fail(SR3D_ERR_INVALID_ARG, "NULL argument");
  Plan& p = plan->p;
  if (use >= 0 && (use != 0) != p.sep_on) {
    TRY(sync_plan(p));
    p.sep_on = use != 0;
    if (p.iter_graph) {  // captured launches carry the old solve arguments
      cudaGraphExecDestroy(p.iter_graph);
      p.iter_graph = nullptr;
    }
    drop_eval_graphs(p);
    ++p.version;
  }
  if (active) *active = (p.sep_avail && p.sep_on) ? 1 : 0;
  return SR3D_OK;
}

int sr3d_forward(sr3d_plan_t plan, const void* x, void* y) {
  if (!plan || !x || !y) return fail(SR3D_ERR_INVALID_ARG, "NULL argument");
  Plan& p = plan->p;
  TRY(hr_forward_partial(p, x));
  SolveArgs sv = solve_args(p, 0, 1.0);
  LAUNCH(SR3D_K_FFTS, launch_fft_s(p, p.hr, p.spec, p.twS, S_FOLD, false, &sv));
  LAUNCH(SR3D_K_FFTS, launch_fft_s(p, p.lr, p.yhat, p.twSl, S_INV, false, nullptr));
  LAUNCH(SR3D_K_FFTN_INV, launch_fft_n(p, p.lr, p.yhat, p.twNl, true));
  LAUNCH(SR3D_K_RFFT_INV, launch_rfft_m_inv(p, p.lr, p.yhat, y, p.twMl, 1.0 / (double)p.lr.V()));
  return sync_plan(p);
}

int sr3d_psf_fit_moments(sr3d_plan_t plan, const void* x, const void* y, double moments[5]) {
  if (!plan || !x || !y || !moments) return fail(SR3D_ERR_INVALID_ARG, "NULL argument");
  Plan& p = plan->p;
  if (!p.fit_lr) TRY(dmalloc(p, &p.fit_lr, (size_t)p.lr.V() * p.esz));
  if (!p.fit_partial) TRY(dmalloc(p, (void**)&p.fit_partial, (size_t)(5 * CG_BLOCKS + 5) * sizeof(double)));
  TRY(hr_forward_partial(p, x));
  SolveArgs sv = solve_args(p, 0, 1.0);
  LAUNCH(SR3D_K_FFTS, launch_fft_s(p, p.hr, p.spec, p.twS, S_FOLD, false, &sv));
  LAUNCH(SR3D_K_FFTS, launch_fft_s(p, p.lr, p.yhat, p.twSl, S_INV, false, nullptr));
  LAUNCH(SR3D_K_FFTN_INV, launch_fft_n(p, p.lr, p.yhat, p.twNl, true));
  LAUNCH(SR3D_K_RFFT_INV, launch_rfft_m_inv(p, p.lr, p.yhat, p.fit_lr, p.twMl, 1.0 / (double)p.lr.V()));
  LAUNCH(SR3D_K_OTHER, launch_fit_moments(p, p.fit_lr, y, p.fit_partial, p.fit_partial + 5 * CG_BLOCKS));
  CK(cudaMemcpyAsync(moments, p.fit_partial + 5 * CG_BLOCKS, 5 * sizeof(double), cudaMemcpyDeviceToHost, p.stream));
  return sync_plan(p);
}

int sr3d_tikhonov(sr3d_plan_t plan, const void* y, const void* xbar, double tau, void* x) {
  if (!plan || !y || !x) return fail(SR3D_ERR_INVALID_ARG, "NULL argument");
  if (!(tau > 0) || !std::isfinite(tau)) return fail(SR3D_ERR_INVALID_ARG, "tau must be positive and finite");
  Plan& p = plan->p;
  TRY(lr_spectrum(p, y));
  TRY(tikhonov_core(p, xbar, tau, x));
  return sync_plan(p);
}

int sr3d_get_otf(sr3d_plan_t plan, void* out) {
  if (!plan || !out) return fail(SR3D_ERR_INVALID_ARG, "NULL argument");
  Plan& p = plan->p;
  LAUNCH(SR3D_K_OTHER, launch_export_half(p, p.lam, out));
  return sync_plan(p);
}

int sr3d_fft3(sr3d_plan_t plan, const void* x, void* out) {
  if (!plan || !x || !out) return fail(SR3D_ERR_INVALID_ARG, "NULL argument");
  Plan& p = plan->p;
  TRY(hr_forward_partial(p, x));
  LAUNCH(SR3D_K_FFTS, launch_fft_s(p, p.hr, p.spec, p.twS, S_FWD, false, nullptr));
  LAUNCH(SR3D_K_OTHER, launch_export_half(p, p.spec, out));
  return sync_plan(p);
}

int sr3d_xstep(sr3d_plan_t plan, const void* y, const void* theta, double rho, void* x) {
  if (!plan || !y || !theta || !x) return fail(SR3D_ERR_INVALID_ARG, "NULL argument");
  if (!(rho > 0)) return fail(SR3D_ERR_INVALID_ARG, "rho must be positive");
  Plan& p = plan->p;
  if (p.psf_sum == 0.0) return fail(SR3D_ERR_SINGULAR, "PSF taps sum to zero");
  TRY(lr_spectrum(p, y));
  TRY(xstep_core(p, theta, rho, x, false));
  return sync_plan(p);
}

int sr3d_tv_step(sr3d_plan_t plan, const void* x, const void* din, void* dout, double lambda, double rho,
                 void* theta) {
  if (!plan || !x || !din || !dout || !theta) return fail(SR3D_ERR_INVALID_ARG, "NULL argument");
  if (!(rho > 0) || lambda < 0) return fail(SR3D_ERR_INVALID_ARG, "need rho > 0 and lambda >= 0");
  if (din == dout) return fail(SR3D_ERR_INVALID_ARG, "d_in and d_out must differ");
  Plan& p = plan->p;
  LAUNCH(SR3D_K_TV, launch_tv(p, x, din, dout, theta, nullptr, lambda / rho, 0, false));
  return sync_plan(p);
}

static int ensure_admm_buffers(Plan& p, bool need_psi) {
  const size_t dbytes = (size_t)3 * p.hr.V() * p.esz;
  if (!p.dbuf[0]) TRY(dmalloc(p, &p.dbuf[0], dbytes));
  if (!p.dbuf[1]) TRY(dmalloc(p, &p.dbuf[1], dbytes));
  if (need_psi && !p.psi) TRY(dmalloc(p, &p.psi, (size_t)p.hr.V() * p.esz));
  return SR3D_OK;
}

static int ensure_hist(Plan& p, int n) {
  if (n <= p.hist_cap) return SR3D_OK;
  if (p.hist) {
    cudaFree(p.hist);
    p.bytes -= (long long)p.hist_cap * sizeof(double);
    p.hist = nullptr;
    p.hist_cap = 0;  // stays 0 if the allocation below fails
  }
  TRY(dmalloc(p, (void**)&p.hist, (size_t)n * sizeof(double)));
  p.hist_cap = n;
  return SR3D_OK;
}

int sr3d_admm_tv(sr3d_plan_t plan, const void* y, void* x, void* d_dev, double lambda, double rho, int max_iters,
                 double tol, double tau_init, sr3d_stats* stats) {
  if (!plan || !y || !x) return fail(SR3D_ERR_INVALID_ARG, "NULL argument");
  if (!(rho > 0) || !(lambda >= 0) || max_iters < 0 || !std::isfinite(rho) || !std::isfinite(lambda))
    return fail(SR3D_ERR_INVALID_ARG, "need rho > 0, lambda >= 0, max_iters >= 0");
  Plan& p = plan->p;
  if (p.psf_sum == 0.0) return fail(SR3D_ERR_SINGULAR, "PSF taps sum to zero: the zero-frequency class is singular");
  const bool want_stats = stats != nullptr || tol > 0;
  int every = stats ? stats->eval_every : 0;
  if (tol > 0 && every <= 0) every = 1;
  TRY(ensure_admm_buffers(p, want_stats));
  const int max_evals = want_stats ? (every > 0 ? max_iters / every + 1 : 1) : 0;
  if (want_stats) TRY(ensure_hist(p, max_evals > 0 ? max_evals : 1));

  void* dcur = d_dev ? d_dev : p.dbuf[0];
  void* dnext = d_dev ? p.dbuf[0] : p.dbuf[1];
  const double thr = lambda / rho;
  {
    p.kind_override = SR3D_K_SETUP;
    struct Reset { Plan& p; ~Reset() { p.kind_override = -1; } } reset{p};
    TRY(lr_spectrum(p, y));
    if (tau_init > 0) TRY(tikhonov_core(p, SR3D_XBAR_NEAREST, tau_init, x));
    if (!d_dev) CK(cudaMemsetAsync(dcur, 0, (size_t)3 * p.hr.V() * p.esz, p.stream));
    // Theta^0 = L^T (u0 - d0) with u0 = L x0
    LAUNCH(SR3D_K_TV, launch_tv(p, x, dcur, nullptr, p.theta, p.psi, thr, 1, want_stats));
  }
  int evals = 0, it = 0;
  bool converged = false;
  double res[16] = {0};
  if (!want_stats && !p.prof_on && p.stream != nullptr && max_iters >= 3) {
    // fixed iterations: the first runs eagerly (every kernel is loaded and
    // configured before any capture), then the two-iteration graph is
    // replayed; an odd last iteration runs eagerly
    auto eager = [&]() -> int {
      TRY(admm_iteration(p, x, dcur, dnext, thr, rho));
      void* t = dcur;
      dcur = dnext;
      dnext = t;
      ++it;
      return SR3D_OK;
    };
    TRY(eager());
    const int pairs = (max_iters - it) / 2;
    TRY(admm_iterations_graph(p, x, dcur, dnext, thr, rho, 2 * pairs));
    it += 2 * pairs;
    if (it < max_iters) TRY(eager());
  }
  // with statistics: after the first evaluation (all kernels loaded), whole
  // evaluation blocks run as replayed graphs.  With tol > 0 one graph loops
  // over the blocks and makes the stopping test on the device (the host waits
  // once, after it); without, the blocks are queued back to back.
  const bool block_graphs = want_stats && every >= 1 && !p.prof_on && p.stream != nullptr;
  const bool dev_loop = block_graphs && tol > 0;
  if (block_graphs) {
    if (!p.hcount) TRY(dmalloc(p, (void**)&p.hcount, sizeof(int)));
    if (!p.res_host) CK(cudaHostAlloc((void**)&p.res_host, 16 * sizeof(double), cudaHostAllocDefault));
  }
  if (dev_loop && !p.tolctl) TRY(dmalloc(p, (void**)&p.tolctl, sizeof(TolCtl)));
  void* const d_first = dcur;
  for (int k = it + 1; k <= max_iters; ++k) {
    if (dev_loop && evals > 0 && (k - 1) % every == 0 && k - 1 + every <= max_iters) {
      const TolCtl c = {0, (max_iters - (k - 1)) / every, tol};
      CK(cudaMemcpyAsync(p.tolctl, &c, sizeof c, cudaMemcpyHostToDevice, p.stream));
      CK(cudaMemcpyAsync(p.hcount, &evals, sizeof(int), cudaMemcpyHostToDevice, p.stream));
      const int par = dcur == d_first ? 0 : 1;
      TRY(admm_tol_graph(p, x, dcur, dnext, thr, rho, lambda, every, par));
      int* const blocks_host = reinterpret_cast<int*>(p.res_host + 12);
      CK(cudaMemcpyAsync(p.res_host, p.result, 11 * sizeof(double), cudaMemcpyDeviceToHost, p.stream));
      CK(cudaMemcpyAsync(blocks_host, &p.tolctl->blocks, sizeof(int), cudaMemcpyDeviceToHost, p.stream));
      TRY(sync_plan(p));
      const int b = *blocks_host;
      for (int j = 0; j < 8; ++j) p.launches[j] += p.tg_first[par][j] + b * p.tg_block[par][j];
      evals += b;
      it = k - 1 + b * every;
      k = it;
      if ((every & 1) && (b & 1)) {
        void* t = dcur;
        dcur = dnext;
        dnext = t;
      }
      memcpy(res, p.res_host, 11 * sizeof(double));
      if (res[10] != 0.0) return fail(SR3D_ERR_NUMERIC, "NaN/Inf in the objective or residuals at iteration %d", it);
      if (res[8] < tol && res[9] < tol) {
        converged = true;
        break;
      }
      continue;  // the block budget is spent: the iterations left run below
    }
    if (block_graphs && !dev_loop && evals > 0 && (k - 1) % every == 0 && k - 1 + every <= max_iters) {
      CK(cudaMemcpyAsync(p.hcount, &evals, sizeof(int), cudaMemcpyHostToDevice, p.stream));
      const int par = dcur == d_first ? 0 : 1;
      TRY(admm_eval_block_graph(p, x, dcur, dnext, thr, rho, lambda, every, par));
      if (every & 1) {
        void* t = dcur;
        dcur = dnext;
        dnext = t;
      }
      ++evals;
      it = k - 1 + every;
      k = it;
      if (tol > 0) {
        TRY(sync_plan(p));
        memcpy(res, p.res_host, 11 * sizeof(double));
        if (res[10] != 0.0) return fail(SR3D_ERR_NUMERIC, "NaN/Inf in the objective or residuals at iteration %d", it);
        if (res[8] < tol && res[9] < tol) {
          converged = true;
          break;
        }
      }
      continue;
    }
    const bool eval_now = want_stats && ((every > 0 && k % every == 0) || k == max_iters);
    const bool stats_now = want_stats && (eval_now || (every > 0 && (k + 1) % every == 0) || k + 1 == max_iters);
    TRY(xstep_core(p, p.theta, rho, x, eval_now));
    LAUNCH(SR3D_K_TV, launch_tv(p, x, dcur, dnext, p.theta, p.psi, thr, 0, stats_now));
    void* t = dcur;
    dcur = dnext;
    dnext = t;
    it = k;
    if (eval_now) {
      LAUNCH(SR3D_K_OTHER, launch_finalize(p, evals < p.hist_cap ? evals : -1, lambda, rho, 1.0 / (double)p.lr.V(), true));
      ++evals;
      // ahead of the device loop its first gate makes this evaluation's test
      if (tol > 0 && !(dev_loop && k % every == 0 && k + every <= max_iters)) {
        CK(cudaMemcpyAsync(res, p.result, 11 * sizeof(double), cudaMemcpyDeviceToHost, p.stream));
        TRY(sync_plan(p));
        if (res[10] != 0.0) return fail(SR3D_ERR_NUMERIC, "NaN/Inf in the objective or residuals at iteration %d", k);
        if (res[8] < tol && res[9] < tol) {
          converged = true;
          break;
        }
      }
    }
  }
  if (d_dev && dcur != d_dev)
    CK(cudaMemcpyAsync(d_dev, dcur, (size_t)3 * p.hr.V() * p.esz, cudaMemcpyDeviceToDevice, p.stream));
  if (want_stats && evals > 0) {
    CK(cudaMemcpyAsync(res, p.result, 11 * sizeof(double), cudaMemcpyDeviceToHost, p.stream));
    if (stats && stats->objective_hist && stats->hist_len > 0) {
      const int n = evals < stats->hist_len ? evals : stats->hist_len;
      CK(cudaMemcpyAsync(stats->objective_hist, p.hist, (size_t)n * sizeof(double), cudaMemcpyDeviceToHost,
                         p.stream));
    }
  }
  TRY(sync_plan(p));
  if (stats) {
    stats->iters = it;
    stats->evals = evals;
    stats->objective = res[0];
    stats->data_term = res[1];
    stats->tv_term = res[2];
    stats->primal = res[3];
    stats->dual = res[4];
    stats->primal_rel = res[8];
    stats->dual_rel = res[9];
  }
  if (want_stats && evals > 0 && res[10] != 0.0) return fail(SR3D_ERR_NUMERIC, "NaN/Inf in the objective or residuals");
  if (tol > 0 && !converged) return fail(SR3D_ERR_NOT_CONVERGED, "max_iters=%d reached before tol=%g", max_iters, tol);
  return SR3D_OK;
}

int sr3d_admm_tv_host(sr3d_plan_t plan, const void* y_host, void* x_host, double lambda, double rho, int max_iters,
                      double tol, double tau_init, sr3d_stats* stats) {
  if (!plan || !y_host || !x_host) return fail(SR3D_ERR_INVALID_ARG, "NULL argument");
  Plan& p = plan->p;
  const size_t xb = (size_t)p.hr.V() * p.esz, yb = (size_t)p.lr.V() * p.esz;
  if (!p.xh) TRY(dmalloc(p, &p.xh, xb));
  if (!p.yh) TRY(dmalloc(p, &p.yh, yb));
  CK(cudaMemcpyAsync(p.yh, y_host, yb, cudaMemcpyHostToDevice, p.stream));
  if (!(tau_init > 0)) CK(cudaMemcpyAsync(p.xh, x_host, xb, cudaMemcpyHostToDevice, p.stream));
  const int rc = sr3d_admm_tv(plan, p.yh, p.xh, nullptr, lambda, rho, max_iters, tol, tau_init, stats);
  if (rc != SR3D_OK && rc != SR3D_ERR_NOT_CONVERGED) return rc;
  CK(cudaMemcpyAsync(x_host, p.xh, xb, cudaMemcpyDeviceToHost, p.stream));
  TRY(sync_plan(p));
  return rc;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Autotuner: times candidate tile schedules of the n pass, the s pass (with
// its class solve) and the TV kernel on the plan's own buffers, keeps the
// fastest and caches the choice per geometry for the process.
// ---------------------------------------------------------------------------
using TuneKey = std::tuple<int, int, int, int, int, int, int>;
struct TuneVal { int tw_n, tw_s, ts_tv, lm_f, lm_i; };
static std::mutex g_tune_mu;
static std::map<TuneKey, TuneVal> g_tune;

static int time_ms(Plan& p, int reps, float* ms, const std::function<int()>& f) {
  cudaEvent_t a, b;
  CK(cudaEventCreate(&a));
  CK(cudaEventCreate(&b));
  int rc = f();  // warm-up (also loads the kernel)
  if (rc == SR3D_OK && cudaEventRecord(a, p.stream) == cudaSuccess) {
    for (int i = 0; i < reps && rc == SR3D_OK; ++i) rc = f();
    cudaEventRecord(b, p.stream);
    cudaEventSynchronize(b);
    cudaEventElapsedTime(ms, a, b);
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  return rc;
}

// Tile widths to time: the given ones, plus every multiple of step up to hi
// whose tiles cover the ms m-slots with at most one step of padding (the
// m-slot count of a half spectrum, (m_l / 2 + 1) d_r, is rarely a power of
// two, and a nearly empty last tile costs a whole CTA lifetime per row).
static std::vector<int> pad_candidates(std::initializer_list<int> base, int ms, int step, int hi) {
  std::vector<int> out(base);
  for (int tw = step; tw <= hi; tw += step) {
    const int pad = (ms + tw - 1) / tw * tw - ms;
    if (pad <= step && std::find(out.begin(), out.end(), tw) == out.end()) out.push_back(tw);
  }
  return out;
}

static int realloc_partials(Plan& p) {
  const long long ns = s_pass_blocks(p.hr);
  if (ns > p.n_s_blocks || !p.partial_s) {
    if (p.partial_s) {
      cudaFree(p.partial_s);
      p.bytes -= (long long)p.n_s_blocks * sizeof(double);
      p.partial_s = nullptr;
    }
    const long long n = ns > p.n_s_blocks ? ns : p.n_s_blocks;
    TRY(dmalloc(p, (void**)&p.partial_s, (size_t)n * sizeof(double)));
    p.n_s_blocks = n;
  }
  return SR3D_OK;
}

extern "C" int sr3d_autotune(sr3d_plan_t plan, int reps) {
  if (!plan) return fail(SR3D_ERR_INVALID_ARG, "NULL argument");
  Plan& p = plan->p;
  Geometry& g = p.hr;
  const size_t csz = 2 * p.esz;
  const TuneKey key{g.M, g.N, g.S, g.dr, g.dc, g.ds, p.dtype};
  TuneVal best{g.tw_n, g.tw_s, g.ts_tv, g.lm_f, g.lm_i};
  bool cached = false;
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune.find(key);
    if (it != g_tune.end()) {
      best = it->second;
      cached = true;
    }
  }
  if (reps < 1) reps = 10;  // a window of a few hundred microseconds per candidate
  const bool prof = p.prof_on;
  p.prof_on = false;
  struct Restore { Plan& p; bool on; ~Restore() { p.prof_on = on; } } restore{p, prof};
  if (!cached) {
    TRY(ensure_admm_buffers(p, false));
    CK(cudaMemsetAsync(p.spec, 0, (size_t)g.spec_elems() * csz, p.stream));
    CK(cudaMemsetAsync(p.yhat_solve, 0, (size_t)solve_yhat_elems(g) * csz, p.stream));
    CK(cudaMemsetAsync(p.dbuf[0], 0, (size_t)3 * g.V() * p.esz, p.stream));
    CK(cudaMemsetAsync(p.theta, 0, (size_t)g.V() * p.esz, p.stream));
    // n pass tile width
    {
      float bt = 1e30f;
      for (int tw : pad_candidates({g.tw_n / 2, g.tw_n, g.tw_n * 2, g.tw_n * 4}, g.Ms, 2, 64)) {
        if (!tw_n_valid(g, csz, tw)) continue;
        g.tw_n = tw;
        float ms = 0;
        TRY(time_ms(p, reps, &ms, [&]() -> int {
          CK(launch_fft_n(p, g, p.spec, p.twN, false));
          CK(launch_fft_n(p, g, p.spec, p.twN, true));
          return SR3D_OK;
        }));
        if (ms < bt) { bt = ms; best.tw_n = tw; }
      }
      g.tw_n = best.tw_n;
    }
    // m passes: lines per CTA (whole warps), forward and inverse apart; at
    // most eight values spread down from the default
    {
      std::vector<int> cand;
      for (int L = 256; L >= 1; --L)
        if (m_lines_valid(g, L)) cand.push_back(L);
      const size_t stride = (cand.size() + 7) / 8;
      float bf = 1e30f, bi = 1e30f;
      for (size_t ci = 0; ci < cand.size(); ci += stride) {
        const int L = cand[ci];
        g.lm_f = g.lm_i = L;
        float ms = 0;
        TRY(time_ms(p, reps, &ms, [&]() -> int {
          CK(launch_rfft_m_fwd(p, g, p.theta, p.spec, p.twM));
          return SR3D_OK;
        }));
        if (ms < bf) { bf = ms; best.lm_f = L; }
        TRY(time_ms(p, reps, &ms, [&]() -> int {
          CK(launch_rfft_m_inv(p, g, p.spec, p.theta, p.twM, 1.0));
          return SR3D_OK;
        }));
        if (ms < bi) { bi = ms; best.lm_i = L; }
      }
      g.lm_f = best.lm_f;
      g.lm_i = best.lm_i;
    }
    // s pass (ADMM class solve) tile width; Lambda is re-permuted per candidate
    {
      const int cap = ((g.Ms + 2 * g.dr - 1) / (2 * g.dr)) * (2 * g.dr);
      float bt = 1e30f;
      const int tw0 = g.tw_s;
      for (int tw : pad_candidates({tw0 / 2, tw0, tw0 * 2}, g.Ms, g.dr, cap)) {
        tw = (tw / g.dr) * g.dr;
        if (!tw_s_valid(p, g, csz, tw)) continue;
        g.tw_s = tw;
        TRY(realloc_partials(p));
        CK(launch_perm_lam(p, p.lam, p.lam_solve));
        SolveArgs sv = solve_args(p, 0, 1e-2);
        float ms = 0;
        TRY(time_ms(p, reps, &ms, [&]() -> int {
          CK(launch_fft_s(p, g, p.spec, p.twS, S_ADMM, false, &sv));
          return SR3D_OK;
        }));
        if (ms < bt) { bt = ms; best.tw_s = tw; }
      }
      g.tw_s = best.tw_s;
    }
    // TV planes per CTA
    {
      float bt = 1e30f;
      int cand[8];
      const int nc = tv_ts_candidates(p, cand, 8);
      for (int ci = 0; ci < nc; ++ci) {
        const int ts = cand[ci];
        g.ts_tv = ts;
        float ms = 0;
        TRY(time_ms(p, reps, &ms, [&]() -> int {
          CK(launch_tv(p, p.theta, p.dbuf[0], p.dbuf[1], p.spec, nullptr, 1.0, 0, false));
          return SR3D_OK;
        }));
        if (ms < bt) { bt = ms; best.ts_tv = ts; }
      }
    }
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune[key] = best;
  }
  g.tw_n = best.tw_n;
  g.tw_s = best.tw_s;
  g.ts_tv = best.ts_tv;
  g.lm_f = best.lm_f;
  g.lm_i = best.lm_i;
  {
    Geometry gc = g;
    if (solve_lam_elems(gc) > p.lam_solve_cap || solve_yhat_elems(gc) > p.yhat_solve_cap)
      g.tw_s = make_geom(g.M, g.N, g.S, g.dr, g.dc, g.ds, csz).tw_s;  // cached choice does not fit: default
  }
  ++p.version;
  TRY(realloc_partials(p));
  CK(launch_perm_lam(p, p.lam, p.lam_solve));
  if (p.iter_graph) {
    cudaGraphExecDestroy(p.iter_graph);
    p.iter_graph = nullptr;
  }
  drop_eval_graphs(p);
  TRY(sync_plan(p));
  return SR3D_OK;
}

// ---------------------------------------------------------------------------
// Batched solve of many volumes of uneven size and decimation.
//
// Every volume keeps its own plan and stream, and the per-volume set-up (LR
// spectrum, Tikhonov start, initial Theta) is launched on the plans' streams.
// Volumes that share a geometry, a tile schedule, lambda, rho, the TV kind and
// a separable PSF (FP32) form a group: their iterates, duals, Theta, spectra,
// solve-order LR spectra and separable Lambda tables are copied into buffers
// that hold the group's volumes one after another, and each ADMM iteration of
// the group is six launches (m, n, s passes with the class solve, n, m, TV)
// over all of them; the m and n passes treat the volumes' planes as more
// planes, the s pass and the TV kernel take the volume from their grid.  Other
// volumes run their own six launches.  The iterations run as one CUDA graph
// that forks from a capture stream into one chain per group or single volume
// (two ADMM iterations each) and joins back, replayed iters/2 times, so the
// chains run concurrently; the graph and the group buffers are cached for
// repeated calls with the same plans, buffers and parameters.
// ---------------------------------------------------------------------------
struct BatchGroup {
  std::vector<int> vols;         // volume indices of the call, in order
  const sr3d_plan_s* lead = nullptr;
  void* x = nullptr;             // B V reals
  void* d[2] = {nullptr, nullptr};  // B 3V reals each
  void* theta = nullptr;         // B V reals
  void* spec = nullptr;          // B spectra
  void* yhat = nullptr;          // B solve-order LR spectra
  void* lam[3] = {nullptr, nullptr, nullptr};  // B M, B N, B S separable factors
  int cur = 0;                   // which of d[] holds the current dual
};

struct BatchGraph {
  cudaGraphExec_t exec = nullptr;
  std::vector<const void*> key_ptr;
  std::vector<double> key_val;
  std::vector<cudaEvent_t> ev;  // fork/join events
  cudaStream_t main = nullptr;
  long long launches[8] = {0};
  // grouping of the last call and its buffers
  std::vector<BatchGroup> groups;
  std::vector<const void*> gkey_ptr;
  std::vector<double> gkey_val;
  // the set-up graph (per-volume set-up, the copies into the group buffers
  // and, for an odd iteration count, the first iteration), its key, launch
  // counts, and whether the grouping has run its set-up eagerly once
  cudaGraphExec_t setup_exec = nullptr;
  std::vector<const void*> skey_ptr;
  std::vector<double> skey_val;
  long long setup_launches[8] = {0};
  bool setup_warm = false;
};
static std::mutex g_batch_mu;
static BatchGraph g_batch;

static void free_groups() {
  for (BatchGroup& G : g_batch.groups) {
    void* bufs[] = {G.x, G.d[0], G.d[1], G.theta, G.spec, G.yhat, G.lam[0], G.lam[1], G.lam[2]};
    for (void* q : bufs)
      if (q) cudaFree(q);
  }
  g_batch.groups.clear();
}

// a volume that can join a group: FP32, separable PSF in use, vectorised TV
static bool groupable(const Plan& p) { return p.dtype == SR3D_F32 && p.sep_avail && p.sep_on && tv_batchable(p); }

// Groups of two or more volumes (see above); singletons are not listed.
static int build_groups(int n, sr3d_plan_t* plans, const double* lambda, const double* rho) {
  std::vector<bool> used(n, false);
  std::vector<BatchGroup> out;
  for (int i = 0; i < n; ++i) {
    if (used[i] || !groupable(plans[i]->p)) continue;
    const Plan& a = plans[i]->p;
    BatchGroup G;
    G.vols.push_back(i);
    for (int j = i + 1; j < n; ++j) {
      if (used[j] || !groupable(plans[j]->p)) continue;
      const Plan& b = plans[j]->p;
      const Geometry &ga = a.hr, &gb = b.hr;
      if (ga.M == gb.M && ga.N == gb.N && ga.S == gb.S && ga.dr == gb.dr && ga.dc == gb.dc && ga.ds == gb.ds &&
          ga.tw_n == gb.tw_n && ga.tw_s == gb.tw_s && ga.ts_tv == gb.ts_tv && ga.lm_f == gb.lm_f &&
          ga.lm_i == gb.lm_i && a.tv_aniso == b.tv_aniso && lambda[i] == lambda[j] && rho[i] == rho[j])
        G.vols.push_back(j);
    }
    if (G.vols.size() < 2) continue;
    for (int v : G.vols) used[v] = true;
    G.lead = plans[i];
    out.push_back(G);
  }
  free_groups();
  g_batch.groups = out;
  for (BatchGroup& G : g_batch.groups) {
    const Plan& p = G.lead->p;
    const Geometry& g = p.hr;
    const size_t B = G.vols.size(), csz = 2 * p.esz;
    const size_t sizes[9] = {B * g.V() * p.esz, 3 * B * g.V() * p.esz, 3 * B * g.V() * p.esz, B * g.V() * p.esz,
                             B * g.spec_elems() * csz, B * solve_yhat_elems(g) * csz, B * g.M * csz, B * g.N * csz,
                             B * g.S * csz};
    void** dst[9] = {&G.x, &G.d[0], &G.d[1], &G.theta, &G.spec, &G.yhat, &G.lam[0], &G.lam[1], &G.lam[2]};
    for (int k = 0; k < 9; ++k) {
      cudaError_t e = cudaMalloc(dst[k], sizes[k]);
      if (e != cudaSuccess) {
        *dst[k] = nullptr;
        cudaGetLastError();
        free_groups();
        return fail(e == cudaErrorMemoryAllocation ? SR3D_ERR_OOM : SR3D_ERR_CUDA, "batched group buffers: %s",
                    cudaGetErrorString(e));
      }
    }
  }
  return SR3D_OK;
}

// One ADMM iteration of a group (the six passes over all of its volumes) on
// the lead plan's stream: dual d[cur] in, d[1 - cur] out.
static int group_iteration(BatchGroup& G, double thr, double rho) {
  Plan& p = const_cast<Plan&>(G.lead->p);
  const int B = (int)G.vols.size();
  Geometry gB = p.hr;  // the m and n passes see the volumes' planes as more planes
  gB.S *= B;
  SolveArgs sv = solve_args(p, 0, rho);
  sv.yhat = G.yhat;
  sv.lamM = G.lam[0];
  sv.lamN = G.lam[1];
  sv.lamS = G.lam[2];
  sv.sep = 1;
  sv.batch = B;
  LAUNCH(SR3D_K_RFFT_FWD, launch_rfft_m_fwd(p, gB, G.theta, G.spec, p.twM));
  LAUNCH(SR3D_K_FFTN_FWD, launch_fft_n(p, gB, G.spec, p.twN, false));
  LAUNCH(SR3D_K_FFTS, launch_fft_s(p, p.hr, G.spec, p.twS, S_ADMM, false, &sv));
  LAUNCH(SR3D_K_FFTN_INV, launch_fft_n(p, gB, G.spec, p.twN, true));
  LAUNCH(SR3D_K_RFFT_INV, launch_rfft_m_inv(p, gB, G.spec, G.x, p.twM, 1.0 / (double)p.hr.V()));
  LAUNCH(SR3D_K_TV, launch_tv_batched(p, B, G.x, G.d[G.cur], G.d[1 - G.cur], G.theta, thr));
  G.cur = 1 - G.cur;
  return SR3D_OK;
}

static int batch_events(size_t n) {
  while (g_batch.ev.size() < n + 1) {
    cudaEvent_t e;
    CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    g_batch.ev.push_back(e);
  }
  if (!g_batch.main) CK(cudaStreamCreateWithFlags(&g_batch.main, cudaStreamNonBlocking));
  return SR3D_OK;
}

extern "C" int sr3d_admm_tv_batched(int n, sr3d_plan_t* plans, const void* const* y, void* const* x,
                                    const double* lambda, const double* rho, const double* tau_init, int iters) {
  if (n <= 0 || !plans || !y || !x || !lambda || !rho || !tau_init || iters < 0)
    return fail(SR3D_ERR_INVALID_ARG, "NULL argument or non-positive count");
  for (int i = 0; i < n; ++i) {
    if (!plans[i] || !y[i] || !x[i]) return fail(SR3D_ERR_INVALID_ARG, "NULL plan or buffer %d", i);
    if (!(rho[i] > 0) || !(lambda[i] >= 0)) return fail(SR3D_ERR_INVALID_ARG, "volume %d: need rho > 0, lambda >= 0", i);
    if (plans[i]->p.psf_sum == 0.0) return fail(SR3D_ERR_SINGULAR, "volume %d: PSF taps sum to zero", i);
    if (plans[i]->p.stream == nullptr) return fail(SR3D_ERR_INVALID_ARG, "volume %d: plan on the legacy stream", i);
    for (int j = 0; j < i; ++j)
      if (plans[j] == plans[i]) return fail(SR3D_ERR_INVALID_ARG, "plan %d repeated", i);
  }
  std::lock_guard<std::mutex> lk(g_batch_mu);
  TRY(batch_events((size_t)n));
  // grouping (cached while the plans, their versions and parameters repeat)
  {
    std::vector<const void*> gp;
    std::vector<double> gv;
    for (int i = 0; i < n; ++i) {
      gp.push_back(plans[i]);
      gv.push_back((double)plans[i]->p.version);
      gv.push_back(lambda[i]);
      gv.push_back(rho[i]);
    }
    if (gp != g_batch.gkey_ptr || gv != g_batch.gkey_val) {
      for (cudaGraphExec_t* ge : {&g_batch.exec, &g_batch.setup_exec})
        if (*ge) {
          cudaGraphExecDestroy(*ge);
          *ge = nullptr;
        }
      g_batch.setup_warm = false;
      g_batch.gkey_ptr.clear();
      TRY(build_groups(n, plans, lambda, rho));
      g_batch.gkey_ptr = gp;
      g_batch.gkey_val = gv;
    }
  }
  std::vector<int> group_of(n, -1);
  for (int k = 0; k < (int)g_batch.groups.size(); ++k)
    for (int v : g_batch.groups[k].vols) group_of[v] = k;
  std::vector<void*> dcur(n), dnext(n);
  // set-up on every plan's stream, then the group members' state into the
  // group buffers on the lead's stream after each member's set-up
  auto setup_all = [&]() -> int {
    for (int i = 0; i < n; ++i) {
      Plan& p = plans[i]->p;
      p.kind_override = SR3D_K_SETUP;
      struct Reset { Plan& p; ~Reset() { p.kind_override = -1; } } reset{p};
      TRY(lr_spectrum(p, y[i]));
      if (tau_init[i] > 0) TRY(tikhonov_core(p, SR3D_XBAR_NEAREST, tau_init[i], x[i]));
      CK(cudaMemsetAsync(dcur[i], 0, (size_t)3 * p.hr.V() * p.esz, p.stream));
      LAUNCH(SR3D_K_TV, launch_tv(p, x[i], dcur[i], nullptr, p.theta, p.psi, lambda[i] / rho[i], 1, false));
    }
    for (BatchGroup& G : g_batch.groups) {
      Plan& L = const_cast<Plan&>(G.lead->p);
      const Geometry& g = L.hr;
      const size_t csz = 2 * L.esz, vb = (size_t)g.V() * L.esz;
      for (size_t j = 0; j < G.vols.size(); ++j) {
        Plan& p = plans[G.vols[j]]->p;
        if (&p != &L) {
          CK(cudaEventRecord(g_batch.ev[G.vols[j]], p.stream));
          CK(cudaStreamWaitEvent(L.stream, g_batch.ev[G.vols[j]], 0));
        }
        unsigned char* xb = (unsigned char*)G.x + j * vb;
        unsigned char* tb = (unsigned char*)G.theta + j * vb;
        unsigned char* yb = (unsigned char*)G.yhat + j * (size_t)solve_yhat_elems(g) * csz;
        CK(cudaMemcpyAsync(xb, x[G.vols[j]], vb, cudaMemcpyDeviceToDevice, L.stream));
        CK(cudaMemcpyAsync(tb, p.theta, vb, cudaMemcpyDeviceToDevice, L.stream));
        CK(cudaMemcpyAsync(yb, p.yhat_solve, (size_t)solve_yhat_elems(g) * csz, cudaMemcpyDeviceToDevice, L.stream));
        CK(cudaMemcpyAsync((unsigned char*)G.lam[0] + j * g.M * csz, p.lamM1, g.M * csz, cudaMemcpyDeviceToDevice, L.stream));
        CK(cudaMemcpyAsync((unsigned char*)G.lam[1] + j * g.N * csz, p.lamN1, g.N * csz, cudaMemcpyDeviceToDevice, L.stream));
        CK(cudaMemcpyAsync((unsigned char*)G.lam[2] + j * g.S * csz, p.lamS1, g.S * csz, cudaMemcpyDeviceToDevice, L.stream));
      }
      CK(cudaMemsetAsync(G.d[0], 0, 3 * G.vols.size() * vb, L.stream));
    }
    return SR3D_OK;
  };
  for (int i = 0; i < n; ++i) {
    TRY(ensure_admm_buffers(plans[i]->p, false));
    dcur[i] = plans[i]->p.dbuf[0];
    dnext[i] = plans[i]->p.dbuf[1];
  }
  for (BatchGroup& G : g_batch.groups) G.cur = 0;
  // the chains: a group (its lead's index) or a single volume
  std::vector<int> chain;
  for (int i = 0; i < n; ++i)
    if (group_of[i] < 0) chain.push_back(i);
  for (const BatchGroup& G : g_batch.groups) chain.push_back(G.vols[0]);
  auto chain_iteration = [&](int i) -> int {
    if (group_of[i] >= 0) {
      BatchGroup& G = g_batch.groups[group_of[i]];
      return group_iteration(G, lambda[i] / rho[i], rho[i]);
    }
    Plan& p = plans[i]->p;
    TRY(admm_iteration(p, x[i], dcur[i], dnext[i], lambda[i] / rho[i], rho[i]));
    std::swap(dcur[i], dnext[i]);
    return SR3D_OK;
  };
  auto eager_iteration = [&]() -> int {
    for (int i : chain) TRY(chain_iteration(i));
    return SR3D_OK;
  };
  bool profiling = false;
  for (int i = 0; i < n; ++i) profiling |= plans[i]->p.prof_on;
  // main waits for every plan's queued work / every plan's stream waits for main
  auto join_to_main = [&]() -> int {
    for (int i = 0; i < n; ++i) {
      CK(cudaEventRecord(g_batch.ev[i], plans[i]->p.stream));
      CK(cudaStreamWaitEvent(g_batch.main, g_batch.ev[i], 0));
    }
    return SR3D_OK;
  };
  auto fork_from_main = [&]() -> int {
    CK(cudaEventRecord(g_batch.ev[n], g_batch.main));
    for (int i = 0; i < n; ++i) CK(cudaStreamWaitEvent(plans[i]->p.stream, g_batch.ev[n], 0));
    return SR3D_OK;
  };
  int it = 0;
  if (profiling || !g_batch.setup_warm) {
    // eager: the first call of a grouping loads and configures every kernel
    // before any capture; the first iteration runs eagerly too
    TRY(setup_all());
    if (iters > 0) {
      TRY(eager_iteration());
      it = 1;
    }
    if (!profiling) g_batch.setup_warm = true;
  } else {
    // the set-up as one graph from the main stream, with the first iteration
    // when the count is odd (the pairs then cover the rest)
    const int first = iters & 1;
    std::vector<const void*> kp;
    std::vector<double> kv;
    for (int i = 0; i < n; ++i) {
      kp.push_back(y[i]);
      kp.push_back(x[i]);
      kp.push_back(dcur[i]);
      kv.push_back(tau_init[i]);
    }
    for (const BatchGroup& G : g_batch.groups) kp.push_back(G.x);
    kv.push_back((double)first);
    if (!g_batch.setup_exec || kp != g_batch.skey_ptr || kv != g_batch.skey_val) {
      if (g_batch.setup_exec) {
        cudaGraphExecDestroy(g_batch.setup_exec);
        g_batch.setup_exec = nullptr;
      }
      std::vector<long long> before(8 * (size_t)n);
      for (int i = 0; i < n; ++i)
        for (int k = 0; k < 8; ++k) before[8 * i + k] = plans[i]->p.launches[k];
      cudaGraph_t graph = nullptr;
      CK(cudaStreamBeginCapture(g_batch.main, cudaStreamCaptureModeThreadLocal));
      int rc = fork_from_main();
      if (rc == SR3D_OK) rc = setup_all();
      if (rc == SR3D_OK && first) rc = eager_iteration();
      if (rc == SR3D_OK) rc = join_to_main();
      const cudaError_t ee = cudaStreamEndCapture(g_batch.main, &graph);
      if (rc != SR3D_OK || ee != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        if (rc != SR3D_OK) return rc;
        return fail(SR3D_ERR_CUDA, "batched set-up graph capture: %s", cudaGetErrorString(ee));
      }
      const cudaError_t ei = cudaGraphInstantiate(&g_batch.setup_exec, graph, 0);
      cudaGraphDestroy(graph);
      if (ei != cudaSuccess) {
        g_batch.setup_exec = nullptr;
        return fail(SR3D_ERR_CUDA, "batched set-up graph instantiate: %s", cudaGetErrorString(ei));
      }
      for (int k = 0; k < 8; ++k) g_batch.setup_launches[k] = 0;
      for (int i = 0; i < n; ++i)
        for (int k = 0; k < 8; ++k) {
          g_batch.setup_launches[k] += plans[i]->p.launches[k] - before[8 * i + k];
          plans[i]->p.launches[k] = before[8 * i + k];
        }
      g_batch.skey_ptr = kp;
      g_batch.skey_val = kv;
    } else if (first) {
      // the captured iteration advanced the dual buffers of every chain
      for (int i : chain) {
        if (group_of[i] >= 0) {
          BatchGroup& G = g_batch.groups[group_of[i]];
          G.cur = 1 - G.cur;
        } else {
          std::swap(dcur[i], dnext[i]);
        }
      }
    }
    TRY(join_to_main());
    CK(cudaGraphLaunch(g_batch.setup_exec, g_batch.main));
    for (int k = 0; k < 8; ++k) plans[0]->p.launches[k] += g_batch.setup_launches[k];
    TRY(fork_from_main());
    it = first;
  }
  const int pairs = profiling ? 0 : (iters - it) / 2;  // per-launch events are not captured
  if (pairs > 0) {
    std::vector<const void*> kp;
    std::vector<double> kv;
    for (int i = 0; i < n; ++i) {
      kp.push_back(plans[i]);
      kp.push_back(x[i]);
      kp.push_back(dcur[i]);
      kv.push_back(lambda[i]);
      kv.push_back(rho[i]);
      kv.push_back((double)plans[i]->p.version);
    }
    for (const BatchGroup& G : g_batch.groups) {
      kp.push_back(G.x);
      kv.push_back((double)G.cur);
    }
    if (!g_batch.exec || kp != g_batch.key_ptr || kv != g_batch.key_val) {
      if (g_batch.exec) {
        cudaGraphExecDestroy(g_batch.exec);
        g_batch.exec = nullptr;
      }
      std::vector<long long> before(8 * (size_t)n);
      for (int i = 0; i < n; ++i)
        for (int k = 0; k < 8; ++k) before[8 * i + k] = plans[i]->p.launches[k];
      // each chain's two iterations captured into one graph after a common
      // root; a chain's kernels get a priority that rises as its work falls,
      // so the CTAs of the short, latency-bound chains are dispatched ahead of
      // the queued CTAs of the long ones instead of in their tails
      cudaGraph_t graph = nullptr;
      CK(cudaGraphCreate(&graph, 0));
      struct Owner {
        cudaGraph_t g;
        ~Owner() { cudaGraphDestroy(g); }
      } owner{graph};
      cudaGraphNode_t root;
      CK(cudaGraphAddEmptyNode(&root, graph, nullptr, 0));
      int prio_least = 0, prio_greatest = 0;
      CK(cudaDeviceGetStreamPriorityRange(&prio_least, &prio_greatest));
      std::vector<double> work(chain.size());
      for (size_t c = 0; c < chain.size(); ++c) {
        const int i = chain[c];
        if (group_of[i] >= 0)
          work[c] = (double)g_batch.groups[group_of[i]].vols.size() * (double)plans[i]->p.hr.V();
        else
          work[c] = (double)plans[i]->p.hr.V();
      }
      std::vector<int> rank(chain.size());  // 0 = least work
      for (size_t c = 0; c < chain.size(); ++c) {
        int r = 0;
        for (size_t o = 0; o < chain.size(); ++o) r += (work[o] < work[c] || (work[o] == work[c] && o < c)) ? 1 : 0;
        rank[c] = r;
      }
      std::vector<cudaGraphNode_t> seen{root};
      for (size_t c = 0; c < chain.size(); ++c) {
        const int i = chain[c];
        Plan& p = plans[i]->p;
        CK(cudaStreamBeginCaptureToGraph(p.stream, graph, &root, nullptr, 1, cudaStreamCaptureModeThreadLocal));
        int rc = chain_iteration(i);
        if (rc == SR3D_OK) rc = chain_iteration(i);
        cudaGraph_t out = nullptr;
        const cudaError_t ee = cudaStreamEndCapture(p.stream, &out);
        if (rc != SR3D_OK) return rc;
        if (ee != cudaSuccess) return fail(SR3D_ERR_CUDA, "batched graph capture: %s", cudaGetErrorString(ee));
        const int prio = chain.size() > 1
                             ? prio_greatest + (int)((long long)(prio_least - prio_greatest) * rank[c] /
                                                     (long long)(chain.size() - 1))
                             : prio_least;
        size_t nn = 0;
        CK(cudaGraphGetNodes(graph, nullptr, &nn));
        std::vector<cudaGraphNode_t> nodes(nn);
        CK(cudaGraphGetNodes(graph, nodes.data(), &nn));
        for (cudaGraphNode_t nd : nodes) {
          if (std::find(seen.begin(), seen.end(), nd) != seen.end()) continue;
          seen.push_back(nd);
          cudaGraphNodeType t;
          CK(cudaGraphNodeGetType(nd, &t));
          if (t != cudaGraphNodeTypeKernel) continue;
          cudaLaunchAttributeValue v;
          memset(&v, 0, sizeof(v));
          v.priority = prio;
          CK(cudaGraphKernelNodeSetAttribute(nd, cudaLaunchAttributePriority, &v));
        }
      }
      cudaError_t ee = cudaGraphInstantiate(&g_batch.exec, graph, cudaGraphInstantiateFlagUseNodePriority);
      if (ee != cudaSuccess) {
        g_batch.exec = nullptr;
        return fail(SR3D_ERR_CUDA, "batched graph instantiate: %s", cudaGetErrorString(ee));
      }
      for (int k = 0; k < 8; ++k) g_batch.launches[k] = 0;
      for (int i = 0; i < n; ++i)
        for (int k = 0; k < 8; ++k) {
          g_batch.launches[k] += plans[i]->p.launches[k] - before[8 * i + k];
          plans[i]->p.launches[k] = before[8 * i + k];
        }
      g_batch.key_ptr = kp;
      g_batch.key_val = kv;
    }
    // the graph starts after every plan's queued work; later work on the
    // plans' streams starts after it
    TRY(join_to_main());
    for (int r = 0; r < pairs; ++r) {
      CK(cudaGraphLaunch(g_batch.exec, g_batch.main));
      for (int k = 0; k < 8; ++k) plans[0]->p.launches[k] += g_batch.launches[k];
    }
    TRY(fork_from_main());
    it += 2 * pairs;
  }
  while (it < iters) {
    TRY(eager_iteration());
    ++it;
  }
  // the groups' iterates back to the callers' buffers
  for (BatchGroup& G : g_batch.groups) {
    Plan& L = const_cast<Plan&>(G.lead->p);
    const size_t vb = (size_t)L.hr.V() * L.esz;
    for (size_t j = 0; j < G.vols.size(); ++j)
      CK(cudaMemcpyAsync(x[G.vols[j]], (unsigned char*)G.x + j * vb, vb, cudaMemcpyDeviceToDevice, L.stream));
    CK(cudaEventRecord(g_batch.ev[G.vols[0]], L.stream));
    for (size_t j = 1; j < G.vols.size(); ++j)
      CK(cudaStreamWaitEvent(plans[G.vols[j]]->p.stream, g_batch.ev[G.vols[0]], 0));
  }
  for (int i = 0; i < n; ++i) TRY(sync_plan(plans[i]->p));
  return SR3D_OK;
}

// ---------------------------------------------------------------------------
// Allocation-free Tikhonov solve.
//
// For callers that may not allocate device memory once they are running: a
// reconstruction loop whose device-memory budget is fixed at start-up, or a
// plug-in inside a host application that owns the device's memory pool.  All
// the work memory (twiddle and symbol tables, Lambda, the LR spectrum, the HR
// spectrum) lives in one file-scope device array of SR3D_NOALLOC_BYTES, so
// every GPU that loads this library holds it until the process exits.  The
// first call on a device looks up the array's device address; it should come
// before any stream capture.  Calls share the array: calls that overlap on the
// GPU race.
// ---------------------------------------------------------------------------
static __device__ __align__(256) unsigned char g_noalloc_scratch[SR3D_NOALLOC_BYTES];

static std::mutex g_noalloc_mu;
static void* g_noalloc_dev_ptr[256];  // device address of g_noalloc_scratch, per device

// Set-up, once per device, with that device current: the host-side name of a
// __device__ array is only a stand-in, so the kernels get its device address.
static int noalloc_scratch(void** out) {
  int dev = 0;
  CK(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 256) return fail(SR3D_ERR_INVALID_ARG, "device ordinal %d out of range", dev);
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (!g_noalloc_dev_ptr[dev]) {
    void* ptr = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
    if (e != cudaSuccess || !ptr)
      return fail(SR3D_ERR_CUDA, "cudaGetSymbolAddress(scratch): %s", cudaGetErrorString(e));
    g_noalloc_dev_ptr[dev] = ptr;
  }
  *out = g_noalloc_dev_ptr[dev];
  return SR3D_OK;
}

extern "C" int sr3d_tikhonov_noalloc(const sr3d_desc* d, const void* y, const void* xbar, double tau, void* x) {
  if (!d || !y || !x || !d->psf) return fail(SR3D_ERR_INVALID_ARG, "NULL argument");
  if (!(tau > 0) || !std::isfinite(tau)) return fail(SR3D_ERR_INVALID_ARG, "tau must be positive and finite");
  if (d->m_h <= 0 || d->n_h <= 0 || d->s_h <= 0 || d->dr <= 0 || d->dc <= 0 || d->ds <= 0 || d->p_m <= 0 ||
      d->p_n <= 0 || d->p_s <= 0)
    return fail(SR3D_ERR_INVALID_ARG, "sizes and decimation factors must be positive");
  if (d->dtype != SR3D_F32 && d->dtype != SR3D_F64) return fail(SR3D_ERR_INVALID_ARG, "dtype must be F32 or F64");
  if (d->m_h % d->dr || d->n_h % d->dc || d->s_h % d->ds)
    return fail(SR3D_ERR_NOT_DIVISIBLE, "HR sizes not divisible by the decimation factors");
  if (d->p_m > d->m_h || d->p_n > d->n_h || d->p_s > d->s_h)
    return fail(SR3D_ERR_INVALID_ARG, "PSF larger than the volume");
  if (d->m_h % 32 || d->n_h % 8 || d->s_h < 4 || d->m_h > 2048 || d->n_h > 2048 || d->s_h > 2048 ||
      !supported_len(d->m_h) || !supported_len(d->n_h) || !supported_len(d->s_h) || (d->m_h / d->dr) % 2 ||
      d->dr * d->dc * d->ds > 8)
    return fail(SR3D_ERR_UNSUPPORTED_SIZE, "sizes outside the supported set of sr3d_plan");

  Plan p;
  p.dtype = d->dtype;
  p.esz = p.dtype ? 8 : 4;
  const size_t csz = 2 * p.esz;
  p.hr = make_geom(d->m_h, d->n_h, d->s_h, d->dr, d->dc, d->ds, csz);
  p.lr = make_geom(p.hr.Ml, p.hr.Nl, p.hr.Sl, 1, 1, 1, csz);
  TRY(validate_lengths(p.hr, csz));
  TRY(validate_lengths(p.lr, csz));
  p.stream = (cudaStream_t)d->stream;
  p.own_stream = false;

  // carve the scratch array: 256-byte aligned pieces
  const long long np = (long long)d->p_m * d->p_n * d->p_s;
  const Geometry& g = p.hr;
  const Geometry& l = p.lr;
  const size_t sizes[13] = {(size_t)g.M * csz, (size_t)g.N * csz, (size_t)g.S * csz, (size_t)l.M * csz,
                            (size_t)l.N * csz, (size_t)l.S * csz, (size_t)g.M * p.esz, (size_t)g.N * p.esz,
                            (size_t)g.S * p.esz, (size_t)solve_lam_elems(g) * csz, (size_t)g.spec_elems() * csz,
                            (size_t)l.spec_elems() * csz, (size_t)solve_yhat_elems(g) * csz};
  size_t need = 0, off[14];
  for (int i = 0; i < 13; ++i) {
    off[i] = need;
    need += (sizes[i] + 255) & ~(size_t)255;
  }
  off[13] = need;
  need += ((size_t)np * sizeof(double) + 255) & ~(size_t)255;
  if (need > (size_t)SR3D_NOALLOC_BYTES)
    return fail(SR3D_ERR_UNSUPPORTED_SIZE,
                "volume needs %zu bytes of work memory; the allocation-free path holds %u (use sr3d_plan)", need,
                (unsigned)SR3D_NOALLOC_BYTES);
  void* base = nullptr;
  TRY(noalloc_scratch(&base));
  unsigned char* b = (unsigned char*)base;
  p.twM = b + off[0]; p.twN = b + off[1]; p.twS = b + off[2];
  p.twMl = b + off[3]; p.twNl = b + off[4]; p.twSl = b + off[5];
  p.symM = b + off[6]; p.symN = b + off[7]; p.symS = b + off[8];
  p.lam_solve = b + off[9];
  p.lam_solve_cap = solve_lam_elems(g);
  p.yhat_solve_cap = solve_yhat_elems(g);
  p.spec = b + off[10];
  p.yhat = b + off[11];
  p.yhat_solve = b + off[12];
  // scratch reuse without aliasing inside any kernel: the wrapped PSF (a real
  // HR volume) sits in the solve-order region until Lambda is formed in the
  // spec region; the permutation then overwrites the solve-order region
  p.theta = p.lam_solve;
  p.lam = p.spec;
  double* psf_dev = (double*)(b + off[13]);

  CK(launch_twiddle(p, p.twM, g.M));
  CK(launch_twiddle(p, p.twN, g.N));
  CK(launch_twiddle(p, p.twS, g.S));
  CK(launch_twiddle(p, p.twMl, l.M));
  CK(launch_twiddle(p, p.twNl, l.N));
  CK(launch_twiddle(p, p.twSl, l.S));
  CK(launch_symbol(p, p.symM, g.M));
  CK(launch_symbol(p, p.symN, g.N));
  CK(launch_symbol(p, p.symS, g.S));
  CK(cudaMemcpyAsync(psf_dev, d->psf, (size_t)np * sizeof(double), cudaMemcpyHostToDevice, p.stream));
  CK(cudaMemsetAsync(p.theta, 0, (size_t)g.V() * p.esz, p.stream));  // the wrap fills only the PSF taps
  CK(launch_wrap_psf(p, p.theta, psf_dev, d->p_m, d->p_n, d->p_s));
  // Lambda: wrapped PSF -> spectrum (spec region) -> solve order
  CK(launch_rfft_m_fwd(p, g, p.theta, p.lam, p.twM));
  CK(launch_fft_n(p, g, p.lam, p.twN, false));
  CK(launch_fft_s(p, g, p.lam, p.twS, S_FWD, false, nullptr));
  CK(launch_perm_lam(p, p.lam, p.lam_solve));
  TRY(lr_spectrum(p, y));
  TRY(tikhonov_core(p, xbar, tau, x));
  CK(cudaStreamSynchronize(p.stream));
  return SR3D_OK;
}

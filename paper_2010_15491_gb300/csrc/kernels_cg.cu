// Vector kernels of the conjugate-gradient comparator: conjugate gradients on
// the normal equations of eq. 6, (H^T D^T D H + tau I) x = H^T D^T y + tau xbar,
// the iterative way of solving eq. 5 that Table 1 compares with the closed
// form of eq. 12.  The operator applications run through the FFT passes
// (s-pass modes S_MUL / S_MULC); these kernels do the sampling mask, the
// vector updates and the FP64 inner products.  alpha and beta are formed on
// the device from the reduced scalars, so an iteration never waits for the
// host:
//   scal[0] = r.r (current), scal[1] = p.Ap, scal[2] = r.r (new).
#include "internal.h"

namespace sr3d {

namespace {

constexpr int CG_THREADS = 256;

__device__ __forceinline__ double cg_warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// block sum of v into partial[blockIdx.x]
__device__ __forceinline__ void cg_block_sum(double v, double* __restrict__ partial) {
  __shared__ double red[CG_THREADS / 32];
  v = cg_warp_sum(v);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x < 32) {
    double t = threadIdx.x < CG_THREADS / 32 ? red[threadIdx.x] : 0.0;
    t = cg_warp_sum(t);
    if (threadIdx.x == 0) partial[blockIdx.x] = t;
  }
}

// z = D^T y: y's LR samples on the lattice (sample 0 of each block), 0 elsewhere
template <typename T>
__global__ void k_zero_fill(const T* __restrict__ y, T* __restrict__ z, int M, int N, int S, int dr, int dc, int ds) {
  const long long V = (long long)M * N * S;
  const int Ml = M / dr, Nl = N / dc;
  for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < V; v += (long long)gridDim.x * blockDim.x) {
    const int m = (int)(v % M), n = (int)((v / M) % N), s = (int)(v / ((long long)M * N));
    T val = 0;
    if (m % dr == 0 && n % dc == 0 && s % ds == 0)
      val = y[((long long)(s / ds) * Nl + n / dc) * Ml + m / dr];
    z[v] = val;
  }
}

// xbar = nearest-neighbour replication of y over each dr x dc x ds block
template <typename T>
__global__ void k_nn_replicate(const T* __restrict__ y, T* __restrict__ xb, int M, int N, int S, int dr, int dc,
                               int ds) {
  const long long V = (long long)M * N * S;
  const int Ml = M / dr, Nl = N / dc;
  for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < V; v += (long long)gridDim.x * blockDim.x) {
    const int m = (int)(v % M), n = (int)((v / M) % N), s = (int)(v / ((long long)M * N));
    xb[v] = y[((long long)(s / ds) * Nl + n / dc) * Ml + m / dr];
  }
}

// v = D^T D v: keep the lattice samples
template <typename T>
__global__ void k_mask_lattice(T* __restrict__ v, int M, int N, int S, int dr, int dc, int ds) {
  const long long V = (long long)M * N * S;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < V; i += (long long)gridDim.x * blockDim.x) {
    const int m = (int)(i % M), n = (int)((i / M) % N), s = (int)(i / ((long long)M * N));
    if (m % dr || n % dc || s % ds) v[i] = 0;
  }
}

// x = 0, r = p = b = hty + tau xbar (xbar may be NULL); partial: r.r
template <typename T>
__global__ void k_cg_init(const T* __restrict__ hty, const T* __restrict__ xbar, T tau, T* __restrict__ x,
                          T* __restrict__ r, T* __restrict__ p, long long V, double* __restrict__ partial) {
  double acc = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < V; i += (long long)gridDim.x * blockDim.x) {
    T b = hty[i];
    if (xbar) b += tau * xbar[i];
    x[i] = 0;
    r[i] = b;
    p[i] = b;
    acc += (double)b * b;
  }
  cg_block_sum(acc, partial);
}

// Ap = w + tau p (in place over w); partial: p.Ap
template <typename T>
__global__ void k_cg_ap(T* __restrict__ w, const T* __restrict__ p, T tau, long long V, double* __restrict__ partial) {
  double acc = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < V; i += (long long)gridDim.x * blockDim.x) {
    const T pi = p[i];
    const T a = w[i] + tau * pi;
    w[i] = a;
    acc += (double)pi * a;
  }
  cg_block_sum(acc, partial);
}

// alpha = rr / pAp; x += alpha p; r -= alpha Ap; partial: r.r
template <typename T>
__global__ void k_cg_update(T* __restrict__ x, T* __restrict__ r, const T* __restrict__ p, const T* __restrict__ ap,
                            const double* __restrict__ scal, long long V, double* __restrict__ partial) {
  const T alpha = (T)(scal[0] / scal[1]);
  double acc = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < V; i += (long long)gridDim.x * blockDim.x) {
    x[i] += alpha * p[i];
    const T ri = r[i] - alpha * ap[i];
    r[i] = ri;
    acc += (double)ri * ri;
  }
  cg_block_sum(acc, partial);
}

// beta = rr_new / rr; p = r + beta p
template <typename T>
__global__ void k_cg_dir(const T* __restrict__ r, T* __restrict__ p, const double* __restrict__ scal, long long V) {
  const T beta = (T)(scal[2] / scal[0]);
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < V; i += (long long)gridDim.x * blockDim.x)
    p[i] = r[i] + beta * p[i];
}

// scal[slot] = sum of the CG_BLOCKS partials (fixed order); then, if
// copy_from >= 0, scal[copy_to] = scal[copy_from] (read before any write)
__global__ void k_cg_reduce(const double* __restrict__ partial, double* __restrict__ scal, int slot, int copy_from,
                            int copy_to) {
  __shared__ double red[CG_THREADS];
  double acc = 0.0;
  for (int i = threadIdx.x; i < CG_BLOCKS; i += CG_THREADS) acc += partial[i];
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int st = CG_THREADS / 2; st > 0; st >>= 1) {
    if (threadIdx.x < st) red[threadIdx.x] += red[threadIdx.x + st];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    if (copy_from >= 0) scal[copy_to] = scal[copy_from];
    scal[slot] = red[0];
  }
}

// The five sums of the Gaussian PSF fit's gain/offset least squares:
// partial[k * gridDim.x + block] for k = 0..4 of sum yh, sum yh^2, sum y,
// sum y^2, sum yh y (FP64 accumulation).
template <typename T>
__global__ void k_fit_moments(const T* __restrict__ yh, const T* __restrict__ y, long long n,
                              double* __restrict__ partial) {
  double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0, a4 = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const double h = (double)yh[i], v = (double)y[i];
    a0 += h;
    a1 += h * h;
    a2 += v;
    a3 += v * v;
    a4 += h * v;
  }
  cg_block_sum(a0, partial);
  __syncthreads();
  cg_block_sum(a1, partial + gridDim.x);
  __syncthreads();
  cg_block_sum(a2, partial + 2 * gridDim.x);
  __syncthreads();
  cg_block_sum(a3, partial + 3 * gridDim.x);
  __syncthreads();
  cg_block_sum(a4, partial + 4 * gridDim.x);
}

// out[k] = sum of row k of partial (nb entries each, fixed order), k < 5
__global__ void k_fit_moments_final(const double* __restrict__ partial, int nb, double* __restrict__ out) {
  __shared__ double red[CG_THREADS];
  for (int k = 0; k < 5; ++k) {
    double acc = 0.0;
    for (int i = threadIdx.x; i < nb; i += CG_THREADS) acc += partial[k * nb + i];
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int st = CG_THREADS / 2; st > 0; st >>= 1) {
      if (threadIdx.x < st) red[threadIdx.x] += red[threadIdx.x + st];
      __syncthreads();
    }
    if (threadIdx.x == 0) out[k] = red[0];
    __syncthreads();
  }
}

}  // namespace

cudaError_t launch_fit_moments(const Plan& p, const void* yh, const void* y, double* partial, double* out) {
  const long long n = p.lr.V();
  if (p.dtype)
    k_fit_moments<double><<<CG_BLOCKS, CG_THREADS, 0, p.stream>>>((const double*)yh, (const double*)y, n, partial);
  else
    k_fit_moments<float><<<CG_BLOCKS, CG_THREADS, 0, p.stream>>>((const float*)yh, (const float*)y, n, partial);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_fit_moments_final<<<1, CG_THREADS, 0, p.stream>>>(partial, CG_BLOCKS, out);
  return cudaGetLastError();
}

cudaError_t launch_zero_fill(const Plan& p, const void* y, void* z) {
  const Geometry& g = p.hr;
  if (p.dtype)
    k_zero_fill<double><<<CG_BLOCKS, CG_THREADS, 0, p.stream>>>((const double*)y, (double*)z, g.M, g.N, g.S, g.dr,
                                                               g.dc, g.ds);
  else
    k_zero_fill<float><<<CG_BLOCKS, CG_THREADS, 0, p.stream>>>((const float*)y, (float*)z, g.M, g.N, g.S, g.dr, g.dc,
                                                              g.ds);
  return cudaGetLastError();
}

cudaError_t launch_nn_replicate(const Plan& p, const void* y, void* xb) {
  const Geometry& g = p.hr;
  if (p.dtype)
    k_nn_replicate<double><<<CG_BLOCKS, CG_THREADS, 0, p.stream>>>((const double*)y, (double*)xb, g.M, g.N, g.S, g.dr,
                                                                  g.dc, g.ds);
  else
    k_nn_replicate<float><<<CG_BLOCKS, CG_THREADS, 0, p.stream>>>((const float*)y, (float*)xb, g.M, g.N, g.S, g.dr,
                                                                 g.dc, g.ds);
  return cudaGetLastError();
}

cudaError_t launch_mask_lattice(const Plan& p, void* v) {
  const Geometry& g = p.hr;
  if (p.dtype)
    k_mask_lattice<double><<<CG_BLOCKS, CG_THREADS, 0, p.stream>>>((double*)v, g.M, g.N, g.S, g.dr, g.dc, g.ds);
  else
    k_mask_lattice<float><<<CG_BLOCKS, CG_THREADS, 0, p.stream>>>((float*)v, g.M, g.N, g.S, g.dr, g.dc, g.ds);
  return cudaGetLastError();
}

cudaError_t launch_cg_init(const Plan& p, const void* hty, const void* xbar, double tau, void* x, void* r, void* pv) {
  const long long V = p.hr.V();
  if (p.dtype)
    k_cg_init<double><<<CG_BLOCKS, CG_THREADS, 0, p.stream>>>((const double*)hty, (const double*)xbar, tau,
                                                             (double*)x, (double*)r, (double*)pv, V, p.cg_partial);
  else
    k_cg_init<float><<<CG_BLOCKS, CG_THREADS, 0, p.stream>>>((const float*)hty, (const float*)xbar, (float)tau,
                                                            (float*)x, (float*)r, (float*)pv, V, p.cg_partial);
  return cudaGetLastError();
}

cudaError_t launch_cg_ap(const Plan& p, void* w_ap, const void* pv, double tau) {
  const long long V = p.hr.V();
  if (p.dtype)
    k_cg_ap<double><<<CG_BLOCKS, CG_THREADS, 0, p.stream>>>((double*)w_ap, (const double*)pv, tau, V, p.cg_partial);
  else
    k_cg_ap<float><<<CG_BLOCKS, CG_THREADS, 0, p.stream>>>((float*)w_ap, (const float*)pv, (float)tau, V,
                                                          p.cg_partial);
  return cudaGetLastError();
}

cudaError_t launch_cg_update(const Plan& p, void* x, void* r, const void* pv, const void* ap) {
  const long long V = p.hr.V();
  if (p.dtype)
    k_cg_update<double><<<CG_BLOCKS, CG_THREADS, 0, p.stream>>>((double*)x, (double*)r, (const double*)pv,
                                                               (const double*)ap, p.cg_scal, V, p.cg_partial);
  else
    k_cg_update<float><<<CG_BLOCKS, CG_THREADS, 0, p.stream>>>((float*)x, (float*)r, (const float*)pv,
                                                              (const float*)ap, p.cg_scal, V, p.cg_partial);
  return cudaGetLastError();
}

cudaError_t launch_cg_dir(const Plan& p, const void* r, void* pv) {
  const long long V = p.hr.V();
  if (p.dtype)
    k_cg_dir<double><<<CG_BLOCKS, CG_THREADS, 0, p.stream>>>((const double*)r, (double*)pv, p.cg_scal, V);
  else
    k_cg_dir<float><<<CG_BLOCKS, CG_THREADS, 0, p.stream>>>((const float*)r, (float*)pv, p.cg_scal, V);
  return cudaGetLastError();
}

cudaError_t launch_cg_reduce(const Plan& p, int slot, int copy_from, int copy_to) {
  k_cg_reduce<<<1, CG_THREADS, 0, p.stream>>>(p.cg_partial, p.cg_scal, slot, copy_from, copy_to);
  return cudaGetLastError();
}

}  // namespace sr3d

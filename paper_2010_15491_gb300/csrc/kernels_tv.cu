// ADMM-TV voxel kernels (Algorithm 1 steps 5b, 5c and the Theta of step 5a),
// FP64 reductions for the objective and residuals, and plan-time helpers.
#include <math.h>

#include "internal.h"

namespace sr3d {

constexpr int TM = 32;  // tile along m (one warp)
constexpr int TN = 8;   // tile along n
constexpr int NQ = 6;   // reduced quantities of the TV kernel

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// One CTA covers m in [m0, m0+32) x n in [n0, n0+8) and marches over the s
// planes [s0, s0+TS).  For each plane it evaluates, on the tile plus a
// one-voxel halo at -m and -n, g = Lx (periodic forward differences),
// nu = g + d, u = shrink(nu, thr), d' = nu - u and rho = u - d'; then
// Theta = L^T rho on the tile, using rho of the previous plane (kept in a
// register) for the s component.
// MODE 0: ADMM step.  MODE 1: initial Theta with u = Lx and d unchanged.
// STATS: per-CTA FP64 sums of ||g||, ||d'-d||^2, ||g||^2, ||u||^2,
// (L^T u - psi)^2, (L^T d')^2; psi (= L^T u of the previous iteration) is
// read and overwritten in place.
//
// Thread (lm, ln) owns tile voxel (m0+lm, n0+ln): its loads are aligned,
// coalesced rows.  The 41 halo voxels of the rho region and the 84 of the x
// region are second positions of the first threads.  x of plane s+2 and d of
// plane s+1 are loaded into registers while plane s is computed; x planes
// rotate through three shared buffers.
template <typename T, int MODE, bool STATS>
__global__ void __launch_bounds__(TM* TN) k_tv(const T* __restrict__ x, const T* __restrict__ din,
                                               T* __restrict__ dout, T* __restrict__ theta, T* __restrict__ psi,
                                               int M, int N, int S, int TS, T thr, double* __restrict__ partial) {
  constexpr int XW = TM + 2, XH = TN + 2;  // x plane with halo -1..+1
  constexpr int RW = TM + 1, RH = TN + 1;  // rho plane with halo -1
  constexpr int NC = STATS ? 6 : 3;
  constexpr int NXH = 2 * XW + 2 * TN;      // x halo positions (84)
  constexpr int NRH = RW + TN;              // rho halo positions (41)
  __shared__ T xs[3][XH * XW];
  __shared__ T rs[NC][RH * RW];
  const int lm = threadIdx.x, ln = threadIdx.y, tid = ln * TM + lm;
  const int m0 = blockIdx.x * TM, n0 = blockIdx.y * TN, s0 = blockIdx.z * TS;
  const long long V = (long long)M * N * S;
  const long long P = (long long)M * N;
  const int s_end = min(S, s0 + TS);

  // x positions: interior (ln+1, lm+1) and, for tid < NXH, one halo cell
  const bool has_xh = tid < NXH;
  int xh_r = 0, xh_c = 0;
  if (has_xh) {
    if (tid < XW) { xh_r = 0; xh_c = tid; }
    else if (tid < 2 * XW) { xh_r = XH - 1; xh_c = tid - XW; }
    else if (tid < 2 * XW + TN) { xh_r = 1 + tid - 2 * XW; xh_c = 0; }
    else { xh_r = 1 + tid - 2 * XW - TN; xh_c = XW - 1; }
  }
  const long long xo_in = (long long)((n0 + ln) % N) * M + (m0 + lm) % M;
  const long long xo_h = (long long)((n0 - 1 + xh_r + N) % N) * M + (m0 - 1 + xh_c + M) % M;
  // rho positions: interior (ln+1, lm+1) and, for tid < NRH, one halo cell
  const bool has_rh = tid < NRH;
  int rh_r = 0, rh_c = 0;
  if (has_rh) {
    if (tid < RW) { rh_r = 0; rh_c = tid; }
    else { rh_r = 1 + tid - RW; rh_c = 0; }
  }
  const long long ro_h = (long long)((n0 - 1 + rh_r + N) % N) * M + (m0 - 1 + rh_c + M) % M;
  const int own = (ln + 1) * RW + (lm + 1);
  const int hpos = rh_r * RW + rh_c;

  auto plane_of = [&](int s) -> long long { return (long long)((s + S) % S) * P; };
  T xin_n = 0, xh_n = 0;  // prefetched x (plane s+2)
  T di_n[3] = {0, 0, 0}, dh_n[3] = {0, 0, 0};  // prefetched d (plane s+1)
  T di[3], dh[3];
  auto load_x = [&](int s, T& a, T& b) {
    const long long pl = plane_of(s);
    a = __ldg(&x[pl + xo_in]);
    if (has_xh) b = __ldg(&x[pl + xo_h]);
  };
  auto store_x = [&](T* buf, T a, T b) {
    buf[(ln + 1) * XW + lm + 1] = a;
    if (has_xh) buf[xh_r * XW + xh_c] = b;
  };
  auto load_d = [&](int s, T* a, T* b) {
    const long long pl = plane_of(s);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      a[c] = __ldg(&din[c * V + pl + xo_in]);
      if (has_rh) b[c] = __ldg(&din[c * V + pl + ro_h]);
    }
  };

  double q[NQ] = {0, 0, 0, 0, 0, 0};
  T r2prev = 0, u2prev = 0, d2prev = 0;
  {
    T a, b = 0;
    load_x(s0 - 1, a, b);
    store_x(xs[0], a, b);
    load_x(s0, a, b);
    store_x(xs[1], a, b);
    load_d(s0 - 1, di, dh);
  }
  __syncthreads();
  int cur = 0;  // buffer of plane s; s+1 in (cur+1)%3, s+2 goes to (cur+2)%3
  for (int s = s0 - 1; s < s_end; ++s) {
    const bool more_x = s + 2 <= s_end;
    const bool more_d = s + 1 < s_end;
    if (more_x) load_x(s + 2, xin_n, xh_n);
    if (more_d) load_d(s + 1, di_n, dh_n);
    const T* xc = xs[cur];
    const T* xn = xs[(cur + 1) % 3];
    const long long pl = plane_of(s);
    const bool own_plane = s >= s0;
    // phase 1: u, d', rho at a position of the rho region
    auto point = [&](int rr, int cc, const T* dv, long long gi, bool interior) {
      const int i = rr * RW + cc;
      const T xv = xc[rr * XW + cc];
      const T g0 = xc[rr * XW + cc + 1] - xv;
      const T g1 = xc[(rr + 1) * XW + cc] - xv;
      const T g2 = xn[rr * XW + cc] - xv;
      T u0, u1, u2, e0, e1, e2;
      if (MODE == 1) {
        u0 = g0; u1 = g1; u2 = g2;
        e0 = dv[0]; e1 = dv[1]; e2 = dv[2];
      } else {
        const T v0 = g0 + dv[0], v1 = g1 + dv[1], v2 = g2 + dv[2];
        const T nrm = sqrt(v0 * v0 + v1 * v1 + v2 * v2);
        const T sc = nrm > thr ? (nrm - thr) / nrm : (T)0;
        u0 = v0 * sc; u1 = v1 * sc; u2 = v2 * sc;
        e0 = v0 - u0; e1 = v1 - u1; e2 = v2 - u2;
      }
      if (STATS) {
        rs[0][i] = u0; rs[1][i] = u1; rs[2][i] = u2;
        rs[3][i] = e0; rs[4][i] = e1; rs[5][i] = e2;
      } else {
        rs[0][i] = u0 - e0; rs[1][i] = u1 - e1; rs[2][i] = u2 - e2;
      }
      if (interior && own_plane) {
        if (MODE == 0) {
          dout[gi] = e0; dout[V + gi] = e1; dout[2 * V + gi] = e2;
        }
        if (STATS) {
          const double gg = (double)g0 * g0 + (double)g1 * g1 + (double)g2 * g2;
          q[0] += sqrt(gg);
          const double p0 = (double)e0 - dv[0], p1 = (double)e1 - dv[1], p2 = (double)e2 - dv[2];
          q[1] += p0 * p0 + p1 * p1 + p2 * p2;
          q[2] += gg;
          q[3] += (double)u0 * u0 + (double)u1 * u1 + (double)u2 * u2;
        }
      }
    };
    point(ln + 1, lm + 1, di, pl + xo_in, true);
    if (has_rh) point(rh_r, rh_c, dh, pl + ro_h, false);
    if (more_x) store_x(xs[(cur + 2) % 3], xin_n, xh_n);
    __syncthreads();
    // phase 2: Theta = L^T rho on the tile
    {
      const int left = own - 1, down = own - RW;
      T r2, u2c = 0, d2c = 0;
      if (STATS) {
        u2c = rs[2][own];
        d2c = rs[5][own];
        r2 = u2c - d2c;
      } else {
        r2 = rs[2][own];
      }
      if (own_plane) {
        const long long gi = pl + xo_in;
        T th;
        if (STATS) {
          const T psi_v = (rs[0][left] - rs[0][own]) + (rs[1][down] - rs[1][own]) + (u2prev - u2c);
          const T ltd = (rs[3][left] - rs[3][own]) + (rs[4][down] - rs[4][own]) + (d2prev - d2c);
          th = psi_v - ltd;
          if (MODE == 0) {
            const double dl = (double)psi_v - (double)psi[gi];
            q[4] += dl * dl;
          }
          psi[gi] = psi_v;
          q[5] += (double)ltd * ltd;
        } else {
          th = (rs[0][left] - rs[0][own]) + (rs[1][down] - rs[1][own]) + (r2prev - r2);
        }
        theta[gi] = th;
      }
      r2prev = r2;
      u2prev = u2c;
      d2prev = d2c;
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      di[c] = di_n[c];
      dh[c] = dh_n[c];
    }
    (void)hpos;
    __syncthreads();
    cur = (cur + 1) % 3;
  }
  if (STATS) {
    __shared__ double red[NQ][TM * TN / 32];
    const int lane = tid & 31, warp = tid >> 5;
#pragma unroll
    for (int k = 0; k < NQ; ++k) {
      const double v = warp_sum_d(q[k]);
      if (lane == 0) red[k][warp] = v;
    }
    __syncthreads();
    if (tid < NQ) {
      double v = 0;
      for (int w = 0; w < TM * TN / 32; ++w) v += red[tid][w];
      const long long b = ((long long)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
      partial[b * NQ + tid] = v;
    }
  }
}

static int tv_ts(const Geometry& g) {
  // planes per CTA: aim for a few CTAs per SM-slot while keeping the
  // one-plane priming overhead small
  if (g.S >= 256) return 16;
  if (g.S >= 64) return 8;
  return 4;
}

long long tv_blocks(const Geometry& g) {
  const int ts = tv_ts(g);
  return (long long)((g.M + TM - 1) / TM) * ((g.N + TN - 1) / TN) * ((g.S + ts - 1) / ts);
}

template <typename T, int MODE, bool STATS>
static cudaError_t tv_k(const Plan& p, const void* x, const void* din, void* dout, void* theta, void* psi,
                        double thr) {
  const Geometry& g = p.hr;
  const int ts = tv_ts(g);
  dim3 grid((g.M + TM - 1) / TM, (g.N + TN - 1) / TN, (g.S + ts - 1) / ts);
  dim3 block(TM, TN);
  k_tv<T, MODE, STATS><<<grid, block, 0, p.stream>>>((const T*)x, (const T*)din, (T*)dout, (T*)theta, (T*)psi,
                                                     g.M, g.N, g.S, ts, (T)thr, p.partial);
  return cudaGetLastError();
}

template <typename T>
static cudaError_t tv_t(const Plan& p, const void* x, const void* din, void* dout, void* theta, void* psi,
                        double thr, int mode, bool stats) {
  if (mode == 0)
    return stats ? tv_k<T, 0, true>(p, x, din, dout, theta, psi, thr)
                 : tv_k<T, 0, false>(p, x, din, dout, theta, psi, thr);
  return stats ? tv_k<T, 1, true>(p, x, din, dout, theta, psi, thr)
               : tv_k<T, 1, false>(p, x, din, dout, theta, psi, thr);
}

cudaError_t launch_tv(const Plan& p, const void* x, const void* din, void* dout, void* theta, void* psi,
                      double thr, int mode, bool stats) {
  return p.dtype ? tv_t<double>(p, x, din, dout, theta, psi, thr, mode, stats)
                 : tv_t<float>(p, x, din, dout, theta, psi, thr, mode, stats);
}

// ---------------------------------------------------------------------------
// finalize: deterministic sum of the per-CTA partials (fixed order), then
// objective and residuals.  out[0..9] = objective, data term, TV term,
// primal, dual, ||Lx||, ||u||, mu ||L^T d||, primal_rel, dual_rel; out[10] =
// 1 if any of them is NaN/Inf.  hist[idx] = objective when idx >= 0.
// ---------------------------------------------------------------------------
__global__ void k_finalize(const double* __restrict__ ptv, long long ntv, const double* __restrict__ ps,
                           long long ns, double lam_tv, double mu, double inv_nl, int with_data,
                           double* __restrict__ out, double* __restrict__ hist, int hidx) {
  __shared__ double red[NQ + 1][256];
  const int tid = threadIdx.x;
  double acc[NQ + 1] = {0, 0, 0, 0, 0, 0, 0};
  for (long long b = tid; b < ntv; b += blockDim.x)
    for (int k = 0; k < NQ; ++k) acc[k] += ptv[b * NQ + k];
  if (with_data)
    for (long long b = tid; b < ns; b += blockDim.x) acc[NQ] += ps[b];
  for (int k = 0; k <= NQ; ++k) red[k][tid] = acc[k];
  __syncthreads();
  for (int st = blockDim.x / 2; st > 0; st >>= 1) {
    if (tid < st)
      for (int k = 0; k <= NQ; ++k) red[k][tid] += red[k][tid + st];
    __syncthreads();
  }
  if (tid == 0) {
    const double tv = red[0][0];
    const double data = with_data ? 0.5 * red[NQ][0] * inv_nl : 0.0;
    const double primal = sqrt(red[1][0]);
    const double nlx = sqrt(red[2][0]);
    const double nu = sqrt(red[3][0]);
    const double dual = mu * sqrt(red[4][0]);
    const double nltd = mu * sqrt(red[5][0]);
    const double obj = data + lam_tv * tv;
    const double den_p = fmax(nlx, nu);
    out[0] = obj;
    out[1] = data;
    out[2] = tv;
    out[3] = primal;
    out[4] = dual;
    out[5] = nlx;
    out[6] = nu;
    out[7] = nltd;
    out[8] = den_p > 0 ? primal / den_p : 0.0;
    out[9] = nltd > 0 ? dual / nltd : 0.0;
    bool bad = false;
    for (int k = 0; k < 10; ++k) bad |= !isfinite(out[k]);
    out[10] = bad ? 1.0 : 0.0;
    if (hidx >= 0 && hist) hist[hidx] = obj;
  }
}

cudaError_t launch_finalize(const Plan& p, int hist_index, double lam_tv, double mu, double inv_nl,
                            bool with_data) {
  k_finalize<<<1, 256, 0, p.stream>>>(p.partial, p.n_tv_blocks, p.partial_s, p.n_s_blocks, lam_tv, mu, inv_nl,
                                      with_data ? 1 : 0, p.result, p.hist, hist_index);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// plan-time tables and helpers
// ---------------------------------------------------------------------------
template <typename T>
__global__ void k_twiddle(cplx<T>* tw, int n) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= n) return;
  double sn, cs;
  sincospi(-2.0 * (double)q / (double)n, &sn, &cs);  // exp(-2 pi i q / n)
  tw[q] = mkc((T)cs, (T)sn);
}

template <typename T>
__global__ void k_symbol(T* sym, int n) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const double s = sinpi((double)k / (double)n);
  sym[k] = (T)(4.0 * s * s);  // |exp(2 pi i k / n) - 1|^2
}

template <typename T>
__global__ void k_wrap_psf(T* out, const double* __restrict__ psf, int pm, int pn, int ps, int M, int N, int S) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= pm * pn * ps) return;
  const int a = i / (pn * pm), b = (i / pm) % pn, c = i % pm;
  const int s = ((a - ps / 2) % S + S) % S;
  const int n = ((b - pn / 2) % N + N) % N;
  const int m = ((c - pm / 2) % M + M) % M;
  out[((long long)s * N + n) * M + m] = (T)psf[i];
}

template <typename T>
__global__ void k_export_half(const cplx<T>* __restrict__ spec, cplx<T>* __restrict__ out, int M, int N, int S,
                              int Ml, int Nl, int dr, int dc, int Mp) {
  const int Hc = M / 2 + 1;
  const long long total = (long long)S * N * Hc;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const int km = (int)(i % Hc);
    const int kn = (int)((i / Hc) % N);
    const int ks = (int)(i / ((long long)Hc * N));
    bool cj;
    const int slot = mslot_of(km, M, Ml, dr, cj);
    const int kn2 = cj ? (N - kn) % N : kn;
    const int ks2 = cj ? (S - ks) % S : ks;
    const cplx<T> v = spec[((long long)ks2 * N + nslot(kn2, Nl, dc)) * Mp + slot];
    out[i] = cj ? conjc(v) : v;
  }
}

cudaError_t launch_twiddle(const Plan& p, void* tw, int n) {
  const int b = (n + 255) / 256;
  if (p.dtype) k_twiddle<double><<<b, 256, 0, p.stream>>>((double2*)tw, n);
  else k_twiddle<float><<<b, 256, 0, p.stream>>>((float2*)tw, n);
  return cudaGetLastError();
}

cudaError_t launch_symbol(const Plan& p, void* sym, int n) {
  const int b = (n + 255) / 256;
  if (p.dtype) k_symbol<double><<<b, 256, 0, p.stream>>>((double*)sym, n);
  else k_symbol<float><<<b, 256, 0, p.stream>>>((float*)sym, n);
  return cudaGetLastError();
}

cudaError_t launch_wrap_psf(const Plan& p, void* out, const double* psf_dev, int pm, int pn, int ps) {
  const int n = pm * pn * ps;
  const int b = (n + 255) / 256;
  const Geometry& g = p.hr;
  if (p.dtype) k_wrap_psf<double><<<b, 256, 0, p.stream>>>((double*)out, psf_dev, pm, pn, ps, g.M, g.N, g.S);
  else k_wrap_psf<float><<<b, 256, 0, p.stream>>>((float*)out, psf_dev, pm, pn, ps, g.M, g.N, g.S);
  return cudaGetLastError();
}

cudaError_t launch_export_half(const Plan& p, const void* spec, void* out) {
  const Geometry& g = p.hr;
  const int blocks = 1024;
  if (p.dtype)
    k_export_half<double><<<blocks, 256, 0, p.stream>>>((const double2*)spec, (double2*)out, g.M, g.N, g.S, g.Ml,
                                                        g.Nl, g.dr, g.dc, g.Mp);
  else
    k_export_half<float><<<blocks, 256, 0, p.stream>>>((const float2*)spec, (float2*)out, g.M, g.N, g.S, g.Ml,
                                                       g.Nl, g.dr, g.dc, g.Mp);
  return cudaGetLastError();
}

}  // namespace sr3d

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
// MODE 0: ADMM step (isotropic shrink).  MODE 1: initial Theta with u = Lx
// and d unchanged.  MODE 2: ADMM step of the anisotropic TV (componentwise
// shrink: d' = clamp(nu, -thr, thr), u = nu - d'; TV term sum_a |g_a|).
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
      } else if (MODE == 2) {  // anisotropic: d' = clamp(nu, -thr, thr), u = nu - d'
        const T v0 = g0 + dv[0], v1 = g1 + dv[1], v2 = g2 + dv[2];
        e0 = fmin(fmax(v0, -thr), thr); e1 = fmin(fmax(v1, -thr), thr); e2 = fmin(fmax(v2, -thr), thr);
        u0 = v0 - e0; u1 = v1 - e1; u2 = v2 - e2;
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
        if (MODE != 1) {
          dout[gi] = e0; dout[V + gi] = e1; dout[2 * V + gi] = e2;
        }
        if (STATS) {
          const double gg = (double)g0 * g0 + (double)g1 * g1 + (double)g2 * g2;
          q[0] += MODE == 2 ? fabs((double)g0) + fabs((double)g1) + fabs((double)g2) : sqrt(gg);
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
          if (MODE != 1) {
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

// ---------------------------------------------------------------------------
// Vectorised variant for FP32 volumes whose m_h is a multiple of the tile
// width W (128, else 96, else 64): a CTA of 32 x 9 threads covers m in
// [m0, m0+W) x n in [n0, n0+8); warps 0-7 own the tile rows, lanes below W/4
// four consecutive m voxels each (float4 loads and stores).  Warp 8, the halo warp, copies the x and d halo rows and columns
// and evaluates the -n halo row and the -m halo column of the rho region, so
// that every warp evaluates about one row per plane (a tile warp that also
// took the halo row held the others at the plane's barrier).  Same algebra, modes
// and statistics as k_tv; the statistics of a thread's four voxels are summed
// in FP32 (sqrtf for ||g||) and accumulated over its planes in compensated
// FP32 (Kahan), then reduced across the CTA in FP64 (FP64 arithmetic is slow
// on this GPU).  Shared rows are padded so that m0 sits at column 4 (16-byte
// aligned); column 3 is m0-1 and column 4+W is m0+W.
// ---------------------------------------------------------------------------
constexpr int V4W = 136;  // padded row length (floats), for every tile width W <= 128

__device__ __forceinline__ float4 ld4(const float* p) { return __ldg(reinterpret_cast<const float4*>(p)); }
__device__ __forceinline__ void st4(float* p, float4 v) { *reinterpret_cast<float4*>(p) = v; }
__device__ __forceinline__ float4 lds4(const float* p) { return *reinterpret_cast<const float4*>(p); }
__device__ __forceinline__ float f4(const float4& v, int i) { return i == 0 ? v.x : i == 1 ? v.y : i == 2 ? v.z : v.w; }

// asynchronous global -> shared copies (cp.async, completion by wait_group)
__device__ __forceinline__ void cp16(float* dst, const float* src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp4(float* dst, const float* src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

template <int W, int MODE, bool STATS>
__global__ void __launch_bounds__(32 * (TN + 1), 3) k_tv4(const float* __restrict__ x, const float* __restrict__ din,
                                             float* __restrict__ dout, float* __restrict__ theta,
                                             float* __restrict__ psi, int M, int N, int S, int TS, float thr,
                                             double* __restrict__ partial, int zper) {
  constexpr int XR = TN + 2;  // x rows n0-1 .. n0+8
  constexpr int RR = TN + 1;  // rho / d rows n0-1 .. n0+7
  extern __shared__ __align__(16) float sm4[];
  float* xs = sm4;                       // [3][XR][V4W]: x planes s, s+1, s+2
  float* ds = xs + 3 * XR * V4W;         // [2][3][RR][V4W]: d planes s, s+1
  float* rs = ds + 2 * 3 * RR * V4W;     // [NC][RR][V4W]
  constexpr int XP = XR * V4W, DP = 3 * RR * V4W, RP = RR * V4W;
  const int lm = threadIdx.x, ln = threadIdx.y, tid = ln * 32 + lm;
  const bool halo_warp = ln == TN;
  static_assert(W == 64 || W == 96 || W == 128, "tile width");
  const bool act = W == 128 || lm < W / 4;  // lanes that own four voxels of a tile row (all at W = 128)
  const long long V = (long long)M * N * S;
  // volume of a batch (z blocks zper per volume, volumes one after another;
  // the statistics variants are never batched)
  const int vb = STATS ? 0 : (int)(blockIdx.z / zper);
  x += vb * V;
  din += 3 * vb * V;
  dout += 3 * vb * V;
  theta += vb * V;
  psi += vb * V;
  const int m0 = blockIdx.x * W, n0 = blockIdx.y * TN, s0 = (blockIdx.z - vb * zper) * TS;
  const long long P = (long long)M * N;
  const int s_end = min(S, s0 + TS);
  const int mc = 4 + 4 * lm;  // shared column of the thread's first voxel
  const long long o_in = (long long)(n0 + ln) * M + m0 + 4 * lm;            // interior (warps 0-7)
  const long long o_hr = (long long)((n0 - 1 + N) % N) * M + m0 + 4 * lm;  // row n0-1 (halo warp)
  const long long o_xr = (long long)((n0 + TN) % N) * M + m0 + 4 * lm;     // row n0+8 (halo warp, x only)
  // halo warp: lane < 10 -> x column m0-1 of row n0-1+lane; 10 <= lane < 20 -> column m0+128
  const bool xcol = halo_warp && lm < 20;
  const int xc_row = lm < 10 ? lm : lm - 10;
  const int xc_col = lm < 10 ? 3 : 4 + W;
  const long long o_xc = (long long)((n0 - 1 + xc_row + N) % N) * M + (lm < 10 ? (m0 - 1 + M) % M : (m0 + W) % M);
  // halo warp: lane < RR -> d (and rho) column m0-1 of row n0-1+lane
  const bool rcol = halo_warp && lm < RR;
  const long long o_rc = (long long)((n0 - 1 + lm + N) % N) * M + (m0 - 1 + M) % M;
  auto plane_of = [&](int s) -> long long { return (long long)((s + S) % S) * P; };

  auto fetch_x = [&](int s, float* buf) {
    const long long pl = plane_of(s);
    if (!halo_warp) {
      if (act) cp16(buf + (ln + 1) * V4W + mc, x + pl + o_in);
    } else {
      if (act) {
        cp16(buf + mc, x + pl + o_hr);
        cp16(buf + (XR - 1) * V4W + mc, x + pl + o_xr);
      }
      if (xcol) cp4(buf + xc_row * V4W + xc_col, x + pl + o_xc);
    }
  };
  auto fetch_d = [&](int s, float* buf) {
    const long long pl = plane_of(s);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      if (!halo_warp) {
        if (act) cp16(buf + k * RP + (ln + 1) * V4W + mc, din + k * V + pl + o_in);
      } else {
        if (act) cp16(buf + k * RP + mc, din + k * V + pl + o_hr);
        if (rcol) cp4(buf + k * RP + lm * V4W + 3, din + k * V + pl + o_rc);
      }
    }
  };

  // per-thread statistics: compensated (Kahan) FP32 sums over the thread's
  // planes, converted to FP64 once for the CTA reduction (FP64 arithmetic is
  // slow on this GPU)
  float qs[NQ] = {0, 0, 0, 0, 0, 0}, qc[NQ] = {0, 0, 0, 0, 0, 0};
  auto kadd = [&](int k, float v) {
    const float y = v - qc[k];
    const float t = qs[k] + y;
    qc[k] = (t - qs[k]) - y;
    qs[k] = t;
  };
  float4 r2prev = make_float4(0, 0, 0, 0), u2prev = r2prev, e2prev = r2prev;
  fetch_x(s0 - 1, xs);
  fetch_x(s0, xs + XP);
  fetch_d(s0 - 1, ds);
  cp_commit();
  cp_wait_all();
  __syncthreads();
  int cur = 0;
  for (int s = s0 - 1; s < s_end; ++s) {
    const int it = s - (s0 - 1);
    if (s + 2 <= s_end) fetch_x(s + 2, xs + ((cur + 2) % 3) * XP);
    if (s + 1 < s_end) fetch_d(s + 1, ds + ((it + 1) & 1) * DP);
    cp_commit();
    const float* xc = xs + cur * XP;
    const float* xn = xs + ((cur + 1) % 3) * XP;
    const float* dd = ds + (it & 1) * DP;
    const long long pl = plane_of(s);
    const bool own_plane = s >= s0;

    // one voxel of the rho region: shrink, dual, rho into shared row rr, column cc
    auto voxel = [&](int rr, int cc, float g0, float g1, float g2, float d0, float d1, float d2, float& u0,
                     float& u1, float& u2, float& e0, float& e1, float& e2, bool store) {
      if (MODE == 1) {
        u0 = g0; u1 = g1; u2 = g2;
        e0 = d0; e1 = d1; e2 = d2;
      } else if (MODE == 2) {  // anisotropic: d' = clamp(nu, -thr, thr), u = nu - d'
        const float v0 = g0 + d0, v1 = g1 + d1, v2 = g2 + d2;
        e0 = fminf(fmaxf(v0, -thr), thr); e1 = fminf(fmaxf(v1, -thr), thr); e2 = fminf(fmaxf(v2, -thr), thr);
        u0 = v0 - e0; u1 = v1 - e1; u2 = v2 - e2;
      } else {
        const float v0 = g0 + d0, v1 = g1 + d1, v2 = g2 + d2;
        const float nrm = sqrtf(v0 * v0 + v1 * v1 + v2 * v2);
        const float sc = nrm > thr ? (nrm - thr) / nrm : 0.f;
        u0 = v0 * sc; u1 = v1 * sc; u2 = v2 * sc;
        e0 = v0 - u0; e1 = v1 - u1; e2 = v2 - u2;
      }
      if (!store) return;
      const int i = rr * V4W + cc;
      if (STATS) {
        rs[0 * RP + i] = u0; rs[1 * RP + i] = u1; rs[2 * RP + i] = u2;
        rs[3 * RP + i] = e0; rs[4 * RP + i] = e1; rs[5 * RP + i] = e2;
      } else {
        rs[0 * RP + i] = u0 - e0; rs[1 * RP + i] = u1 - e1; rs[2 * RP + i] = u2 - e2;
      }
    };
    // lanes of a tile row (all 32 at W = 128); the right x neighbour of a
    // thread's last voxel and the left rho neighbour of its first are the
    // next / previous lane's (shuffles instead of strided shared loads)
    const unsigned amask = W == 128 ? 0xffffffffu : ((1u << (W / 4)) - 1u);
    // four voxels of shared row xr (x rows xr, xr+1; rho / d row xr), columns mc..mc+3
    auto quad = [&](int xr, bool interior) {
      const float4 a = lds4(xc + xr * V4W + mc);
      float a4;
      if (STATS) {
        a4 = xc[xr * V4W + mc + 4];  // (registers of the statistics variants at their limit)
      } else {
        a4 = __shfl_down_sync(amask, a.x, 1);
        if (lm == W / 4 - 1) a4 = xc[xr * V4W + mc + 4];  // halo column m0 + W
      }
      const float4 b = lds4(xc + (xr + 1) * V4W + mc);
      const float4 c = lds4(xn + xr * V4W + mc);
      const float4 dv0 = lds4(dd + 0 * RP + xr * V4W + mc);
      const float4 dv1 = lds4(dd + 1 * RP + xr * V4W + mc);
      const float4 dv2 = lds4(dd + 2 * RP + xr * V4W + mc);
      float e0v[4], e1v[4], e2v[4], u0v[4], u1v[4], u2v[4];
      float f0 = 0.f, f1 = 0.f, f2 = 0.f, f3 = 0.f;  // the quad's partial sums (FP32, 4 terms)
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const float xv = f4(a, i);
        const float g0 = (i < 3 ? f4(a, i + 1) : a4) - xv;
        const float g1 = f4(b, i) - xv;
        const float g2 = f4(c, i) - xv;
        float u0, u1, u2;
        // the statistics variants (six values per voxel, registers at their
        // limit) store each voxel as it is formed; the step variants store
        // the quad below
        voxel(xr, mc + i, g0, g1, g2, f4(dv0, i), f4(dv1, i), f4(dv2, i), u0, u1, u2, e0v[i], e1v[i], e2v[i], STATS);
        u0v[i] = u0;
        u1v[i] = u1;
        u2v[i] = u2;
        if (STATS && interior && own_plane) {
          const float gg = g0 * g0 + g1 * g1 + g2 * g2;
          f0 += MODE == 2 ? fabsf(g0) + fabsf(g1) + fabsf(g2) : sqrtf(gg);
          const float p0 = e0v[i] - f4(dv0, i), p1 = e1v[i] - f4(dv1, i), p2 = e2v[i] - f4(dv2, i);
          f1 += p0 * p0 + p1 * p1 + p2 * p2;
          f2 += gg;
          f3 += u0 * u0 + u1 * u1 + u2 * u2;
        }
      }
      // the quad's rho as one 16-byte store per component (conflict-free,
      // where four scalar stores per component at a four-float lane stride
      // were four-way bank conflicts)
      if (!STATS) {
        float* r = rs + xr * V4W + mc;
        st4(r + 0 * RP, make_float4(u0v[0] - e0v[0], u0v[1] - e0v[1], u0v[2] - e0v[2], u0v[3] - e0v[3]));
        st4(r + 1 * RP, make_float4(u1v[0] - e1v[0], u1v[1] - e1v[1], u1v[2] - e1v[2], u1v[3] - e1v[3]));
        st4(r + 2 * RP, make_float4(u2v[0] - e2v[0], u2v[1] - e2v[1], u2v[2] - e2v[2], u2v[3] - e2v[3]));
      }
      if (STATS && interior && own_plane) {
        kadd(0, f0);
        kadd(1, f1);
        kadd(2, f2);
        kadd(3, f3);
      }
      if (MODE != 1 && interior && own_plane) {
        const long long gi = pl + o_in;
        st4(dout + gi, make_float4(e0v[0], e0v[1], e0v[2], e0v[3]));
        st4(dout + V + gi, make_float4(e1v[0], e1v[1], e1v[2], e1v[3]));
        st4(dout + 2 * V + gi, make_float4(e2v[0], e2v[1], e2v[2], e2v[3]));
      }
    };
    if (act) {
      if (!halo_warp) quad(ln + 1, true);
      else quad(0, false);
    }
    if (rcol) {
      // halo column m0-1 (shared column 3), row lm
      const int xr = lm;
      const float xv = xc[xr * V4W + 3];
      float u0, u1, u2, e0, e1, e2;
      voxel(xr, 3, xc[xr * V4W + 4] - xv, xc[(xr + 1) * V4W + 3] - xv, xn[xr * V4W + 3] - xv,
            dd[0 * RP + xr * V4W + 3], dd[1 * RP + xr * V4W + 3], dd[2 * RP + xr * V4W + 3], u0, u1, u2, e0, e1,
            e2, true);
    }
    __syncthreads();
    // phase 2: Theta = L^T rho for the four interior voxels (tile warps)
    if (!halo_warp && act) {
      const int row = (ln + 1) * V4W + mc;
      const int up = ln * V4W + mc;
      float4 own0, own1, own2, up1;
      float4 u_0, u_1, u_2, e_0, e_1, e_2, uup1, eup1;
      float left0, ul = 0.f, el = 0.f;
      if (STATS) {
        u_0 = lds4(rs + 0 * RP + row); u_1 = lds4(rs + 1 * RP + row); u_2 = lds4(rs + 2 * RP + row);
        e_0 = lds4(rs + 3 * RP + row); e_1 = lds4(rs + 4 * RP + row); e_2 = lds4(rs + 5 * RP + row);
        uup1 = lds4(rs + 1 * RP + up); eup1 = lds4(rs + 4 * RP + up);
        own0 = make_float4(u_0.x - e_0.x, u_0.y - e_0.y, u_0.z - e_0.z, u_0.w - e_0.w);
        own1 = make_float4(u_1.x - e_1.x, u_1.y - e_1.y, u_1.z - e_1.z, u_1.w - e_1.w);
        own2 = make_float4(u_2.x - e_2.x, u_2.y - e_2.y, u_2.z - e_2.z, u_2.w - e_2.w);
        up1 = make_float4(uup1.x - eup1.x, uup1.y - eup1.y, uup1.z - eup1.z, uup1.w - eup1.w);
        ul = rs[0 * RP + row - 1];
        el = rs[3 * RP + row - 1];
        left0 = ul - el;
      } else {
        own0 = lds4(rs + 0 * RP + row); own1 = lds4(rs + 1 * RP + row); own2 = lds4(rs + 2 * RP + row);
        up1 = lds4(rs + 1 * RP + up);
        left0 = __shfl_up_sync(amask, own0.w, 1);
        if (lm == 0) left0 = rs[0 * RP + row - 1];  // halo column m0 - 1
      }
      if (own_plane) {
        float th[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const float lft = i == 0 ? left0 : f4(own0, i - 1);
          th[i] = (lft - f4(own0, i)) + (f4(up1, i) - f4(own1, i)) + (f4(r2prev, i) - f4(own2, i));
        }
        const long long gi = pl + o_in;
        st4(theta + gi, make_float4(th[0], th[1], th[2], th[3]));
        if (STATS) {
          float pv[4];
          float f5 = 0.f;
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            const float lu = i == 0 ? ul : f4(u_0, i - 1);
            const float le = i == 0 ? el : f4(e_0, i - 1);
            const float psi_v = (lu - f4(u_0, i)) + (f4(uup1, i) - f4(u_1, i)) + (f4(u2prev, i) - f4(u_2, i));
            const float ltd = (le - f4(e_0, i)) + (f4(eup1, i) - f4(e_1, i)) + (f4(e2prev, i) - f4(e_2, i));
            pv[i] = psi_v;
            f5 += ltd * ltd;
          }
          kadd(5, f5);
          if (MODE != 1) {
            const float4 old = ld4(psi + gi);
            float f4s = 0.f;
#pragma unroll
            for (int i = 0; i < 4; ++i) {
              const float dl = pv[i] - f4(old, i);
              f4s += dl * dl;
            }
            kadd(4, f4s);
          }
          st4(psi + gi, make_float4(pv[0], pv[1], pv[2], pv[3]));
        }
      }
      r2prev = own2;
      if (STATS) {
        u2prev = u_2;
        e2prev = e_2;
      }
    }
    cp_wait_all();
    __syncthreads();
    cur = (cur + 1) % 3;
  }
  if (STATS) {
    __shared__ double red[NQ][TN];  // the tile warps' sums (the halo warp adds none)
    const int lane = tid & 31, warp = tid >> 5;
#pragma unroll
    for (int k = 0; k < NQ; ++k) {
      const double v = warp_sum_d((double)qs[k] - (double)qc[k]);
      if (lane == 0 && warp < TN) red[k][warp] = v;
    }
    __syncthreads();
    if (tid < NQ) {
      double v = 0;
      for (int w = 0; w < TN; ++w) v += red[tid][w];
      const long long b = ((long long)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
      partial[b * NQ + tid] = v;
    }
  }
}

static size_t tv4_smem(bool stats) {
  return sizeof(float) * ((size_t)3 * (TN + 2) * V4W + (size_t)2 * 3 * (TN + 1) * V4W +
                          (size_t)(stats ? 6 : 3) * (TN + 1) * V4W);
}

// tile width of the vectorised kernel for this plan (0: the general kernel)
static int tv4_width(const Plan& p) {
  if (p.dtype != 0 || p.hr.N % TN != 0) return 0;
  const int M = p.hr.M;
  return M % 128 == 0 ? 128 : M % 96 == 0 ? 96 : M % 64 == 0 ? 64 : 0;
}
static bool tv_vec4(const Plan& p) { return tv4_width(p) > 0; }

int tv_default_ts(const Geometry& g) {
  // planes per CTA: a few CTAs per SM while keeping the one-plane priming
  // overhead small
  if (g.S >= 256) return 16;
  if (g.S >= 64) return 8;
  return 4;
}

static int tv_ts(const Geometry& g) { return g.ts_tv > 0 ? g.ts_tv : tv_default_ts(g); }

// resident CTAs per SM of the plain ADMM-step TV kernel the plan launches
template <typename T>
static cudaError_t tv_per_sm(const Plan& p, int* per_sm) {
  if (tv_vec4(p)) {
    // the three widths share the launch bounds and the shared-memory size
    const size_t smem = tv4_smem(false);
    cudaError_t e = cudaFuncSetAttribute(k_tv4<128, 0, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, k_tv4<128, 0, false>, 32 * (TN + 1), smem);
  }
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, k_tv<T, 0, false>, TM * TN, 0);
}

int tv_ts_candidates(const Plan& p, int* out, int cap) {
  const Geometry& g = p.hr;
  int n = 0;
  auto add = [&](int ts) {
    if (ts < 4 || ts > g.S || n >= cap) return;
    for (int i = 0; i < n; ++i)
      if (out[i] == ts) return;
    out[n++] = ts;
  };
  for (int ts : {4, 8, 16, 32}) add(ts);
  // Every CTA marches over the same number of planes, so a partly filled last
  // wave of CTAs holds the bandwidth of a few SMs for a whole CTA lifetime:
  // add the plane counts whose grid fills 1..4 waves of resident CTAs.
  int dev = 0, sms = 0, per_sm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess) e = p.dtype ? tv_per_sm<double>(p, &per_sm) : tv_per_sm<float>(p, &per_sm);
  if (e != cudaSuccess || per_sm <= 0) {
    cudaGetLastError();
    return n;
  }
  const long long tiles = tv_vec4(p) ? (long long)(g.M / tv4_width(p)) * (g.N / TN)
                                     : (long long)((g.M + TM - 1) / TM) * ((g.N + TN - 1) / TN);
  const long long slots = (long long)sms * per_sm;
  for (int w = 1; w <= 4; ++w) {
    const long long zmax = w * slots / tiles;  // CTAs along s that fit in w waves
    if (zmax >= 1) add((int)((g.S + zmax - 1) / zmax));
  }
  return n;
}

long long tv_blocks(const Geometry& g) {
  // an upper bound covering both variants (the vectorised one has 4x fewer m
  // tiles) and every planes-per-CTA choice of at least 4
  const int ts = 4;
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

template <int W, int MODE, bool STATS>
static cudaError_t tv4_k(const Plan& p, const void* x, const void* din, void* dout, void* theta, void* psi,
                         double thr) {
  const Geometry& g = p.hr;
  const int ts = tv_ts(g);
  dim3 grid(g.M / W, g.N / TN, (g.S + ts - 1) / ts);
  dim3 block(32, TN + 1);  // eight tile warps and the halo warp
  const size_t smem = tv4_smem(STATS);
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k_tv4<W, MODE, STATS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  k_tv4<W, MODE, STATS><<<grid, block, smem, p.stream>>>((const float*)x, (const float*)din, (float*)dout,
                                                   (float*)theta, (float*)psi, g.M, g.N, g.S, ts, (float)thr,
                                                   p.partial, (int)grid.z);
  return cudaGetLastError();
}

template <int W, int MODE>
static cudaError_t tv4_batch_k(const Plan& p, int batch, const void* x, const void* din, void* dout, void* theta,
                               double thr) {
  const Geometry& g = p.hr;
  const int ts = tv_ts(g);
  const int zper = (g.S + ts - 1) / ts;
  dim3 grid(g.M / W, g.N / TN, zper * batch);
  dim3 block(32, TN + 1);
  const size_t smem = tv4_smem(false);
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k_tv4<W, MODE, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  // theta doubles as the (unused) psi argument
  k_tv4<W, MODE, false><<<grid, block, smem, p.stream>>>((const float*)x, (const float*)din, (float*)dout,
                                                        (float*)theta, (float*)theta, g.M, g.N, g.S, ts, (float)thr,
                                                        nullptr, zper);
  return cudaGetLastError();
}

bool tv_batchable(const Plan& p) { return tv_vec4(p); }

cudaError_t launch_tv_batched(const Plan& p, int batch, const void* x, const void* din, void* dout, void* theta,
                              double thr) {
  const int w = tv4_width(p);
  const bool an = p.tv_aniso;
  if (w == 128) return an ? tv4_batch_k<128, 2>(p, batch, x, din, dout, theta, thr) : tv4_batch_k<128, 0>(p, batch, x, din, dout, theta, thr);
  if (w == 96) return an ? tv4_batch_k<96, 2>(p, batch, x, din, dout, theta, thr) : tv4_batch_k<96, 0>(p, batch, x, din, dout, theta, thr);
  if (w == 64) return an ? tv4_batch_k<64, 2>(p, batch, x, din, dout, theta, thr) : tv4_batch_k<64, 0>(p, batch, x, din, dout, theta, thr);
  return cudaErrorNotSupported;
}

template <int W>
static cudaError_t tv4_w(const Plan& p, const void* x, const void* din, void* dout, void* theta, void* psi, double thr,
                         int mode, bool stats) {
  if (mode == 0)
    return stats ? tv4_k<W, 0, true>(p, x, din, dout, theta, psi, thr) : tv4_k<W, 0, false>(p, x, din, dout, theta, psi, thr);
  if (mode == 2)
    return stats ? tv4_k<W, 2, true>(p, x, din, dout, theta, psi, thr) : tv4_k<W, 2, false>(p, x, din, dout, theta, psi, thr);
  return stats ? tv4_k<W, 1, true>(p, x, din, dout, theta, psi, thr) : tv4_k<W, 1, false>(p, x, din, dout, theta, psi, thr);
}

template <typename T>
static cudaError_t tv_t(const Plan& p, const void* x, const void* din, void* dout, void* theta, void* psi,
                        double thr, int mode, bool stats) {
  if (mode == 0 && p.tv_aniso) mode = 2;  // the plan's TV is anisotropic
  const int w = tv4_width(p);
  if (w == 128) return tv4_w<128>(p, x, din, dout, theta, psi, thr, mode, stats);
  if (w == 96) return tv4_w<96>(p, x, din, dout, theta, psi, thr, mode, stats);
  if (w == 64) return tv4_w<64>(p, x, din, dout, theta, psi, thr, mode, stats);
  if (mode == 0)
    return stats ? tv_k<T, 0, true>(p, x, din, dout, theta, psi, thr)
                 : tv_k<T, 0, false>(p, x, din, dout, theta, psi, thr);
  if (mode == 2)
    return stats ? tv_k<T, 2, true>(p, x, din, dout, theta, psi, thr)
                 : tv_k<T, 2, false>(p, x, din, dout, theta, psi, thr);
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
                           double* __restrict__ out, double* __restrict__ hist, int hidx, int* __restrict__ hcount,
                           int hcap) {
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
    if (hidx == -2 && hcount) {  // index kept on the device (graph replays)
      const int i = *hcount;
      if (i < hcap && hist) hist[i] = obj;
      *hcount = i + 1;
    } else if (hidx >= 0 && hist) {
      hist[hidx] = obj;
    }
  }
}

// The stopping test of Algorithm 1 (step 5), made on the device so that a
// graph can loop over evaluation blocks without the host: after the
// evaluation in res (k_finalize's output) the loop goes on while a relative
// residual is at or above tol, nothing is NaN/Inf and blocks are left.
// count = 0 for the gate ahead of the loop, 1 after a block.  When has_next,
// the condition of the second block of a two-block body gets the same value.
__global__ void k_tol_gate(const double* __restrict__ res, TolCtl* __restrict__ c, int count,
                           cudaGraphConditionalHandle loop, cudaGraphConditionalHandle next, int has_next) {
  const int b = c->blocks + count;
  c->blocks = b;
  const bool converged = res[8] < c->tol && res[9] < c->tol;
  const unsigned go = (res[10] == 0.0 && !converged && b < c->max_blocks) ? 1u : 0u;
  cudaGraphSetConditional(loop, go);
  if (has_next) cudaGraphSetConditional(next, go);
}

cudaError_t launch_tol_gate(const Plan& p, int count, cudaGraphConditionalHandle loop,
                            cudaGraphConditionalHandle next, bool has_next) {
  k_tol_gate<<<1, 1, 0, p.stream>>>(p.result, p.tolctl, count, loop, next, has_next ? 1 : 0);
  return cudaGetLastError();
}

// number of CTAs (and partial-sum rows) of the TV variant the plan launches
static long long tv_launch_blocks(const Plan& p) {
  const Geometry& g = p.hr;
  const int ts = tv_ts(g);
  const long long mt = tv_vec4(p) ? g.M / tv4_width(p) : (g.M + TM - 1) / TM;
  return mt * ((g.N + TN - 1) / TN) * ((g.S + ts - 1) / ts);
}

cudaError_t launch_finalize(const Plan& p, int hist_index, double lam_tv, double mu, double inv_nl,
                            bool with_data) {
  // the partials of the CTAs the current schedules launch (the buffers hold
  // the largest grid any schedule has used)
  k_finalize<<<1, 256, 0, p.stream>>>(p.partial, tv_launch_blocks(p), p.partial_s, s_pass_blocks(p.hr), lam_tv, mu,
                                      inv_nl, with_data ? 1 : 0, p.result, p.hist, hist_index, p.hcount, p.hist_cap);
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

// 1-D DFT of one factor f (length pf, centre tap pf/2 wrapped to the origin)
// of a separable PSF: out[k] = sum_j f[j] exp(-2 pi i k ((j - pf/2) mod n) / n),
// in FP64 with the exact integer phase (k * j') mod n
template <typename T>
__global__ void k_dft_factor(cplx<T>* __restrict__ out, const double* __restrict__ f, int pf, int n) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  double re = 0.0, im = 0.0;
  for (int j = 0; j < pf; ++j) {
    const long long jw = ((j - pf / 2) % n + n) % n;
    const long long w = (jw * k) % n;
    double sn, cs;
    sincospi(-2.0 * (double)w / (double)n, &sn, &cs);
    re += f[j] * cs;
    im += f[j] * sn;
  }
  out[k] = mkc((T)re, (T)im);
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
    const cplx<T> v = spec[((long long)ks2 * N + kn2) * Mp + slot];
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

cudaError_t launch_dft_factor(const Plan& p, void* out, const double* f_dev, int pf, int n) {
  const int b = (n + 255) / 256;
  if (p.dtype) k_dft_factor<double><<<b, 256, 0, p.stream>>>((cplx<double>*)out, f_dev, pf, n);
  else k_dft_factor<float><<<b, 256, 0, p.stream>>>((cplx<float>*)out, f_dev, pf, n);
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

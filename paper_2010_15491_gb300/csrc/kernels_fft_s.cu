// s pass of the 3D transforms fused with the per-aliasing-class solve of
// eq. (12) (Tikhonov) and of the x-update of Algorithm 1 step 5a (ADMM), the
// spectral multiplies of the CG comparator, and the solve-order permutations
// of Lambda and of the LR spectrum.  Spectral layout: see kernels_fft.cu.
#include "fft.cuh"
#include "fft_ct.cuh"
#include "fft_host.cuh"
#include "internal.h"

namespace sr3d {

template <typename T> struct Lim;
template <> struct Lim<float> { static constexpr float big = 3.0e38f; };
template <> struct Lim<double> { static constexpr double big = 1.0e300; };

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
// ---------------------------------------------------------------------------
// s pass with the class solve.  Tile: m-slots [a0, a0+TW) x n-slots
// [b0, b0+G) x all S planes; TW is a multiple of dr and G of dc, so the tile
// holds whole aliasing classes.
// ---------------------------------------------------------------------------
template <typename C, typename T>
__device__ __forceinline__ C box_factor(const C* __restrict__ tw, int n, int da, int k) {
  // sum_{q < da} exp(-2 pi i k q / n): DFT of the nearest-neighbour block along one axis
  C r = czero<C>();
  for (int q = 0; q < da; ++q) r = r + __ldg(&tw[(int)(((long long)k * q) % n)]);
  return r;
}

constexpr int DMAX = 8;  // largest supported d = dr*dc*ds

// Solve order of the per-class constants: for the s-pass CTA bc = (by, bx),
// class c of the tile (c = gm + GMc * (gn + GNc * is)) and member q
// (q = pm + dr * (pn + dc * ps)), Lambda sits at (bc * d + q) * ncls + c and
// the LR spectrum at bc * ncls + c, so the solve's loads are contiguous
// across a warp.  solve_layout gives the tile sizes shared by the kernels
// and the permutations.
struct SolveTile {
  int GMc, GNc, ncls, Gm, gx;
};
__host__ __device__ __forceinline__ SolveTile solve_layout(int Ms, int TW, int G, int dr, int dc, int Sl) {
  SolveTile t;
  t.GMc = TW / dr;
  t.GNc = G / dc;
  t.ncls = t.GMc * t.GNc * Sl;
  t.Gm = Ms / dr;
  t.gx = (Ms + TW - 1) / TW;
  return t;
}

// Per-aliasing-class solve of eq. (12) (Tikhonov, w = 1/tau) or of the
// Gamma-weighted x-update of Algorithm 1 step 5a (ADMM, w_p = 1/(mu s_p)) on
// a tile held in shared memory, and the fold of S_FOLD.  DR_/DC_/DS_ > 0 fix
// the class shape at compile time; 0 takes it from sv.  Returns this
// thread's share of sum_i |Y_i - (1/d) sum_p Lambda_p X_p|^2 (STATS).
template <typename T, int MODE, bool STATS, int DR_, int DC_, int DS_>
__device__ __forceinline__ double solve_tile(cplx<T>* sm, int TW, int G, int a0, int b0, int Ms, const SolveArgs& sv,
                                             int tid, int nthr, int vb) {
  using C = cplx<T>;
  const int dr = DR_ > 0 ? DR_ : sv.dr, dc = DR_ > 0 ? DC_ : sv.dc, ds = DR_ > 0 ? DS_ : sv.ds;
  const int d = dr * dc * ds;
  const T dd = (T)d;
  const SolveTile tl = solve_layout(Ms, TW, G, dr, dc, sv.Sl);
  const int ncls = tl.ncls;
  const long long bc = (long long)blockIdx.y * gridDim.x + blockIdx.x;
  const C* __restrict__ lamc = reinterpret_cast<const C*>(sv.lam) + bc * d * ncls;
  const C* __restrict__ yhc = reinterpret_cast<const C*>(sv.yhat) + bc * ncls;
  const T* __restrict__ symM = reinterpret_cast<const T*>(sv.symM);
  const T* __restrict__ symN = reinterpret_cast<const T*>(sv.symN);
  const T* __restrict__ symS = reinterpret_cast<const T*>(sv.symS);
  // separable PSF: Lambda of a member is the product of three 1-D factor DFTs
  // the volume's separable tables (vb > 0 only in a batched ADMM s pass)
  const C* __restrict__ lamM = reinterpret_cast<const C*>(sv.lamM) + (long long)vb * sv.M;
  const C* __restrict__ lamN = reinterpret_cast<const C*>(sv.lamN) + (long long)vb * sv.N;
  const C* __restrict__ lamS = reinterpret_cast<const C*>(sv.lamS) + (long long)vb * sv.S;
  const T alpha = (T)sv.alpha;
  const T ialpha = (T)(1.0 / sv.alpha);
  double acc = 0.0;
#pragma unroll 1
  for (int c = tid; c < ncls; c += nthr) {
    const int gm = c % tl.GMc;
    const int rest = c / tl.GMc;
    const int gn = rest % tl.GNc;
    const int is = rest / tl.GNc;
    const int g = a0 / dr + gm;
    if (g >= tl.Gm) continue;
    const int jl = b0 / dc + gn;
    if (MODE == S_FOLD) {
      C tsum = czero<C>();
      for (int q = 0; q < d; ++q) {
        const int pm = q % dr, pn = (q / dr) % dc, ps = q / (dr * dc);
        const int si = ((is + ps * sv.Sl) * G + gn * dc + pn) * TW + gm * dr + pm;
        const C a_ = sv.sep ? cmul(cmul(__ldg(&lamM[g + pm * sv.Ml]), __ldg(&lamN[jl + pn * sv.Nl])),
                                   __ldg(&lamS[is + ps * sv.Sl]))
                            : __ldg(&lamc[(long long)q * ncls + c]);
        tsum = tsum + cmul(a_, sm[si]);
      }
      reinterpret_cast<C*>(sv.lr_out)[((long long)is * sv.Nl + jl) * sv.Mlp + g] = tsum * (T)(1.0 / d);
      continue;
    }
    const C Yc = __ldg(&yhc[c]);
    const bool dc_cls = (MODE == S_ADMM) && g == 0 && jl == 0 && is == 0;
    if constexpr (DR_ > 0 && MODE == S_ADMM) {
      // compile-time class shape: Lambda in registers, B parked in the tile,
      // the dr + dc + ds symbol values instead of d weights
      constexpr int D = DR_ * DC_ * DS_;
      T sMv[DR_], sNv[DC_], sSv[DS_];
#pragma unroll
      for (int i = 0; i < DR_; ++i) sMv[i] = __ldg(&symM[g + i * sv.Ml]);
#pragma unroll
      for (int i = 0; i < DC_; ++i) sNv[i] = __ldg(&symN[jl + i * sv.Nl]);
#pragma unroll
      for (int i = 0; i < DS_; ++i) sSv[i] = __ldg(&symS[is + i * sv.Sl]);
      const int sbase = (is * G + gn * DC_) * TW + gm * DR_;
      const int splane = sv.Sl * G * TW;
      auto sidx = [&](int q) { return sbase + (q / (DR_ * DC_)) * splane + ((q / DR_) % DC_) * TW + q % DR_; };
      auto wgt = [&](int q) -> T {
        if (dc_cls && q == 0) return (T)0;
        return (T)1 / (alpha * (sMv[q % DR_] + sNv[(q / DR_) % DC_] + sSv[q / (DR_ * DC_)]));
      };
      C lmn[DR_ * DC_], lsv[DS_];
      if (sv.sep) {
#pragma unroll
        for (int i = 0; i < DS_; ++i) lsv[i] = __ldg(&lamS[is + i * sv.Sl]);
#pragma unroll
        for (int j = 0; j < DC_; ++j) {
          const C ln = __ldg(&lamN[jl + j * sv.Nl]);
#pragma unroll
          for (int i = 0; i < DR_; ++i) lmn[i + DR_ * j] = cmul(__ldg(&lamM[g + i * sv.Ml]), ln);
        }
      }
      C av[D];
      int qs = 0;
      T best = (T)-1;
#pragma unroll
      for (int q = 0; q < D; ++q) {
        const C a_ = sv.sep ? cmul(lmn[q % (DR_ * DC_)], lsv[q / (DR_ * DC_)]) : __ldg(&lamc[(long long)q * ncls + c]);
        av[q] = a_;
        const int si = sidx(q);
        sm[si] = cmulc(a_, Yc) + sm[si] * alpha;  // B = conj(Lambda) Y + mu F Theta
        const T key = (dc_cls && q == 0) ? Lim<T>::big : norm2(a_) * wgt(q);
        if (key > best) { best = key; qs = q; }
      }
      T Sp = 0, ws = 0;
      C Tp = czero<C>(), as = czero<C>(), bs = czero<C>();
#pragma unroll
      for (int q = 0; q < D; ++q) {
        const C B = sm[sidx(q)];
        const T w = wgt(q);
        if (q == qs) {
          as = av[q]; bs = B; ws = w;
        } else {
          Sp += norm2(av[q]) * w;
          Tp = Tp + cmul(av[q], B) * w;
        }
      }
      C Xs, ratio;
      if (dc_cls) {
        const T inv = (T)1 / norm2(as);
        Xs = (bs * (dd + Sp) - cmulc(as, Tp)) * inv;
        ratio = cmul(bs, as) * inv;
      } else {
        const T iD = (T)1 / (dd + Sp + norm2(as) * ws);
        Xs = (bs * (dd + Sp) - cmulc(as, Tp)) * (ws * iD);
        ratio = (Tp + cmul(as, bs) * ws) * iD;
      }
      C tsum = czero<C>();
#pragma unroll
      for (int q = 0; q < D; ++q) {
        const int si = sidx(q);
        const C X = (q == qs) ? Xs : (sm[si] - cmulc(av[q], ratio)) * wgt(q);
        sm[si] = conjc(X);
        if (STATS) tsum = tsum + cmul(av[q], X);
      }
      if (STATS) {
        const C R = Yc - tsum * (T)(1.0 / D);
        const double wg = (g == 0 || 2 * g == sv.Ml) ? 1.0 : 2.0;
        acc += wg * (double)norm2(R);
      }
      continue;
    }
    C av[DMAX], bv[DMAX];
    T wv[DMAX];
    int si[DMAX];
    int qs = 0;
    T best = (T)-1;
#pragma unroll
    for (int q = 0; q < DMAX; ++q) {
      if (q < d) {
        const int pm = q % dr, pn = (q / dr) % dc, ps = q / (dr * dc);
        const int ks = is + ps * sv.Sl, kn = jl + pn * sv.Nl, km = g + pm * sv.Ml;
        si[q] = (ks * G + gn * dc + pn) * TW + gm * dr + pm;
        const C a_ = sv.sep ? cmul(cmul(__ldg(&lamM[km]), __ldg(&lamN[kn])), __ldg(&lamS[ks]))
                            : __ldg(&lamc[(long long)q * ncls + c]);
        C B = cmulc(a_, Yc);  // conj(Lambda_p) Y: F H^H D^H y at this frequency
        T w;
        if (MODE == S_ADMM) {
          B = B + sm[si[q]] * alpha;  // + mu F Theta
          const T sy = __ldg(&symM[km]) + __ldg(&symN[kn]) + __ldg(&symS[ks]);
          w = (dc_cls && q == 0) ? (T)0 : (T)1 / (alpha * sy);  // Gamma / mu
        } else {
          if (MODE == S_TIK_USER) B = B + sm[si[q]] * alpha;  // + tau F xbar
          if (MODE == S_TIK_GEN && sv.nn_prior) {
            const C bx = cmul(cmul(box_factor<C, T>(reinterpret_cast<const C*>(sv.twM), sv.M, dr, km),
                                   box_factor<C, T>(reinterpret_cast<const C*>(sv.twN), sv.N, dc, kn)),
                              box_factor<C, T>(reinterpret_cast<const C*>(sv.twS), sv.S, ds, ks));
            B = B + cmul(Yc, bx) * alpha;  // + tau F xbar, xbar = nearest-neighbour y
          }
          w = ialpha;
        }
        const T key = (dc_cls && q == 0) ? Lim<T>::big : norm2(a_) * w;
        if (key > best) { best = key; qs = q; }
        av[q] = a_;
        bv[q] = B;
        wv[q] = w;
      }
    }
    // Sherman-Morrison on the class block diag(1/w) + (1/d) conj(a) a^T with
    // the dominant member p* = qs kept out of the sums (no cancellation).
    T Sp = 0;
    C Tp = czero<C>(), as = czero<C>(), bs = czero<C>();
    T ws = 0;
#pragma unroll
    for (int q = 0; q < DMAX; ++q) {
      if (q < d) {
        if (q == qs) {
          as = av[q]; bs = bv[q]; ws = wv[q];
        } else {
          Sp += norm2(av[q]) * wv[q];
          Tp = Tp + cmul(av[q], bv[q]) * wv[q];
        }
      }
    }
    C Xs, ratio;
    if (dc_cls) {
      // zero frequency: Gamma singular, the class is solved exactly
      const T inv = (T)1 / norm2(as);
      Xs = (bs * (dd + Sp) - cmulc(as, Tp)) * inv;
      ratio = cmul(bs, as) * inv;  // B_* / conj(Lambda_*)
    } else {
      const T iD = (T)1 / (dd + Sp + norm2(as) * ws);
      Xs = (bs * (dd + Sp) - cmulc(as, Tp)) * (ws * iD);
      ratio = (Tp + cmul(as, bs) * ws) * iD;
    }
    C tsum = czero<C>();
#pragma unroll
    for (int q = 0; q < DMAX; ++q) {
      if (q < d) {
        const C X = (q == qs) ? Xs : (bv[q] - cmulc(av[q], ratio)) * wv[q];
        sm[si[q]] = conjc(X);  // conjugated: the inverse runs through the forward engine
        if (STATS) tsum = tsum + cmul(av[q], X);
      }
    }
    if (STATS) {
      const C R = Yc - tsum * (T)(1.0 / d);
      const double wgt = (g == 0 || 2 * g == sv.Ml) ? 1.0 : 2.0;
      acc += wgt * (double)norm2(R);
    }
  }
  return acc;
}

template <typename T, int EMAX, int MODE, bool STATS, int NC, int DR_, int DC_, int DS_>
__global__ void __launch_bounds__(NC > 0 ? 256 : 512, NC > 0 ? 3 : 1) k_fft_s(cplx<T>* __restrict__ spec, LAxis a, int Ms, int Mp, int Nn, int TW, int G, SolveArgs sv,
                        const cplx<T>* __restrict__ twS, int ndc, int nNl) {
  using C = cplx<T>;
  extern __shared__ __align__(16) unsigned char smraw[];
  C* sm = reinterpret_cast<C*>(smraw);
  const int S = NC > 0 ? NC : a.N;
  // volume of a batch (batched S_ADMM only; see SolveArgs::batch)
  const int ny = sv.batch_ny > 0 ? sv.batch_ny : (int)gridDim.y;
  const int vb = blockIdx.y / ny;
  const int a0 = blockIdx.x * TW, b0 = (blockIdx.y - vb * ny) * G;
  spec += (long long)vb * S * Nn * Mp;
  const int tv = min(TW, Ms - a0);
  const int nthr = blockDim.x, tid = threadIdx.x;
  const int rowlen = G * TW;
  const long long plane = (long long)Nn * Mp;
  const int t = tid % TW, gi = (tid / TW) % G, tl = tid / (TW * G), tpl = NC > 0 ? NC / ct_e(NC) : S / a.f.e;
  (void)tpl;
  const bool ok = t < tv;
  // tile row gi = gn * dc + pn holds n = b0 / dc + gn + pn * Nl (dc, Nl of the n axis)
  const int nrow = b0 / ndc + gi / ndc + (gi % ndc) * nNl;
  C* col = spec + (long long)nrow * Mp + a0 + t;
  C* line = sm + gi * TW + t;
  C* tws = sm + S * rowlen;
  if constexpr (NC > 0) ct_load_twiddles(tws, twS, NC);
  auto ld = [&](int s) -> C {
    if (!ok) return czero<C>();
    const C v = col[s * plane];
    return MODE == S_INV ? conjc(v) : v;
  };
  auto st = [&](int s, C v) {
    if (ok) col[s * plane] = MODE == S_FWD ? v : conjc(v);
  };
  if (MODE == S_FWD || MODE == S_INV) {
    if constexpr (NC > 0) ct_line_gg<NC>(ld, st, line, rowlen, tl, tws, 1);
    else fft_line_gg<T, EMAX>(ld, st, line, rowlen, a.f, tl, tpl, twS, 1);
    return;
  }
  if (MODE != S_TIK_GEN) {
    if constexpr (NC > 0) ct_line_gs<NC>(ld, line, rowlen, tl, tws, 1);
    else fft_line_gs<T, EMAX>(ld, line, rowlen, a.f, tl, tpl, twS, 1);
  }

  if (MODE == S_MUL || MODE == S_MULC) {
    // multiply every frequency of the tile by Lambda (or its conjugate)
    __syncthreads();
    const C* __restrict__ lamn = reinterpret_cast<const C*>(sv.lam_nat);
    const C* __restrict__ lamM = reinterpret_cast<const C*>(sv.lamM);
    const C* __restrict__ lamN = reinterpret_cast<const C*>(sv.lamN);
    const C* __restrict__ lamS = reinterpret_cast<const C*>(sv.lamS);
    for (int i = tid; i < S * rowlen; i += nthr) {
      const int ks = i / rowlen, rem = i - ks * rowlen, r = rem / TW, c = rem - r * TW;
      if (c >= tv) continue;
      const int n = b0 / ndc + r / ndc + (r % ndc) * nNl;
      const int slot = a0 + c;
      C lv;
      if (sv.sep) {
        const int km = (slot / sv.dr) + (slot % sv.dr) * sv.Ml;  // slot g*dr + p holds frequency g + p*Ml
        lv = cmul(cmul(__ldg(&lamM[km]), __ldg(&lamN[n])), __ldg(&lamS[ks]));
      } else {
        lv = __ldg(&lamn[((long long)ks * Nn + n) * Mp + slot]);
      }
      const C X = MODE == S_MUL ? cmul(sm[i], lv) : cmulc(lv, sm[i]);
      sm[i] = conjc(X);  // conjugated: the inverse runs through the forward engine
    }
    __syncthreads();
  }
  if (MODE >= S_TIK_GEN && MODE <= S_FOLD) {
    double acc = solve_tile<T, MODE, STATS, DR_, DC_, DS_>(sm, TW, G, a0, b0, Ms, sv, tid, nthr, vb);
    if (STATS) {
      double* red = reinterpret_cast<double*>(tws + (NC > 0 ? NC : 0));  // 32 slots after the tile (and twiddles)
      acc = warp_sum(acc);
      const int lane = tid & 31, warp = tid >> 5;
      if (lane == 0) red[warp] = acc;
      __syncthreads();
      if (warp == 0) {
        double v = (lane < (nthr + 31) / 32) ? red[lane] : 0.0;
        v = warp_sum(v);
        if (lane == 0) sv.partial[(long long)blockIdx.y * gridDim.x + blockIdx.x] = v;
      }
    }
    __syncthreads();
  }
  if (MODE == S_FOLD) return;
  if constexpr (NC > 0) ct_line_sg<NC>(line, st, rowlen, tl, tws, 1);
  else fft_line_sg<T, EMAX>(line, st, rowlen, a.f, tl, tpl, twS, 1);
}

// ---------------------------------------------------------------------------
// Register-resident s pass of the ADMM x-update (Algorithm 1 step 5a) for the
// compile-time s lengths in FP32 with the class shape DR x DC x DS fixed at
// compile time.  After the forward transform's last stage, thread tl of a
// line holds the frequencies k = tl + TPL r (r < E; E = 16 elements and
// TPL = S/16 threads per line for S = 2^a, E = 12 for S = 3 * 2^a) in
// registers, so the DS members k, k + S/DS, ... of an aliasing class along s
// are in the same thread (S/DS = TPL E/DS), and those frequencies are exactly
// the inputs of the inverse transform's first stage.  The class's DR x DC members in the (m, n) plane sit in QN = DR * DC
// adjacent lanes of one warp (lane layout q + QN * (gm + GMc * tl), q = pm +
// DR * pn), and the solve exchanges only per-class scalars by warp shuffles
// (the Sherman-Morrison sums of the other lanes' members, as the butterfly
// delivers them).  Each element crosses shared memory four times (one round
// trip per transform) instead of going through a shared tile for the solve.
// Same system as solve_tile (B = conj(Lambda) Y + mu F Theta, the
// zero-frequency class solved exactly), but every member is formed with its
// own term kept out of the sums, so no member needs a dominant-member search.
// ---------------------------------------------------------------------------
// 1/x: the hardware approximation refined by one Newton-Raphson step
// r <- r (2 - x r) (a few units in the last place; x normal and positive here)
__device__ __forceinline__ float rcp_nr(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r * fmaf(-x, r, 2.0f);
}

template <int S, bool STATS, int DR, int DC, int DS>
__global__ void __launch_bounds__(256, 3) k_fft_s_admm_reg(float2* __restrict__ spec, int Ms, int Mp, int Nn, int TW,
                                                         SolveArgs sv, const float2* __restrict__ twS, int nNl) {
  constexpr int E = ct_e(S), TPL = S / E, NST = ct_nst(S);
  constexpr int QN = DR * DC, D = DR * DC * DS, RS = E / DS, SL = S / DS;
  static_assert(QN == 1 || QN == 2 || QN == 4, "class members in the (m, n) plane: 1, 2 or 4 lanes");
  static_assert(E % DS == 0, "the s members of a class must share a thread");
  extern __shared__ __align__(16) unsigned char smraw[];
  float2* sm = reinterpret_cast<float2*>(smraw);
  const int GMc = TW / DR;
  const int rowlen = DC * TW;
  const int tid = threadIdx.x;
  const int q = tid % QN, rest = tid / QN;
  const int gm = rest % GMc, tl = rest / GMc;
  const int pm = q % DR, pn = q / DR;
  const int t = gm * DR + pm;  // m-slot of the tile
  const int a0 = blockIdx.x * TW;
  // volume of a batch (sv.batch_ny tiles along n per volume, volumes one after
  // another); the solve-order LR spectrum follows from the block index alone
  const int ny = sv.batch_ny > 0 ? sv.batch_ny : (int)gridDim.y;
  const int vb = blockIdx.y / ny;
  const int jl = blockIdx.y - vb * ny;  // LR n frequency of the tile's class row (G = DC rows)
  const bool cls_ok = a0 + gm * DR < Ms;  // whole classes: Ms and TW are multiples of DR
  const long long plane = (long long)Nn * Mp;
  spec += (long long)vb * S * plane;
  float2* col = spec + (long long)(jl + pn * nNl) * Mp + a0 + t;
  float2* line = sm + pn * TW + t;
  float2* tws = sm + S * rowlen;
  ct_load_twiddles(tws, twS, S);

  float2 v[E];
  // forward transform: every stage but the last through shared memory (the
  // first one loads straight from global memory, E loads in flight), the last
  // into registers: v[r] = frequency tl + TPL r
  auto ld = [&](int j) -> float2 { return cls_ok ? col[(long long)j * plane] : make_float2(0.f, 0.f); };
  ct_run_to<S, 0, NST - 1, false>(ld, line, rowlen, tl, tws, 1);
  ct_last_to_regs<S, false>(line, rowlen, tl, tws, 1, v);

  // per-class solve
  const int g = cls_ok ? a0 / DR + gm : 0;
  const int km = g + pm * sv.Ml, kn = jl + pn * sv.Nl;
  const float* __restrict__ symS = reinterpret_cast<const float*>(sv.symS);
  const float2* __restrict__ lamS = reinterpret_cast<const float2*>(sv.lamS) + (long long)vb * S;
  const float sMN = __ldg(&reinterpret_cast<const float*>(sv.symM)[km]) +
                    __ldg(&reinterpret_cast<const float*>(sv.symN)[kn]);
  float2 lmn = make_float2(0.f, 0.f);
  if (sv.sep)
    lmn = cmul(__ldg(&reinterpret_cast<const float2*>(sv.lamM)[(long long)vb * sv.M + km]),
               __ldg(&reinterpret_cast<const float2*>(sv.lamN)[(long long)vb * sv.N + kn]));
  const long long bc = (long long)blockIdx.y * gridDim.x + blockIdx.x;
  const int ncls = GMc * sv.Sl;
  const float2* __restrict__ lamc = reinterpret_cast<const float2*>(sv.lam) + bc * D * ncls;
  const float2* __restrict__ yhc = reinterpret_cast<const float2*>(sv.yhat) + bc * ncls;
  const float alpha = (float)sv.alpha;
  const float dd = (float)D;
  const int lane = tid & 31;
  const int gbase = lane - q;  // first lane of this class's group
  double acc = 0.0;
#pragma unroll
  for (int cr = 0; cr < RS; ++cr) {
    const int is = tl + TPL * cr;  // LR s frequency of the class
    const int c = gm + GMc * is;
    const float2 Yc = cls_ok ? __ldg(&yhc[c]) : make_float2(0.f, 0.f);
    const bool dc_cls = cls_ok && g == 0 && jl == 0 && is == 0;
    // members: Lambda a, mu s (den0), w = 1 / (mu s), B, key |a|^2 w, a B w
    float2 av[DS], bv[DS], tv[DS];
    float sv_[DS], wv[DS], kv[DS];
    float Sown = 0.f;
    float2 Town = make_float2(0.f, 0.f);
#pragma unroll
    for (int ps = 0; ps < DS; ++ps) {
      const int qq = q + QN * ps;
      const int ks = is + ps * SL;
      float2 a_ = make_float2(0.f, 0.f);
      float mus = 1.f, w = 0.f;
      if (cls_ok) {
        a_ = sv.sep ? cmul(lmn, __ldg(&lamS[ks])) : __ldg(&lamc[(long long)qq * ncls + c]);
        mus = alpha * (sMN + __ldg(&symS[ks]));
        w = (dc_cls && qq == 0) ? 0.f : rcp_nr(mus);  // Gamma / mu; singular at the zero frequency
      }
      av[ps] = a_;
      sv_[ps] = mus;
      wv[ps] = w;
      bv[ps] = cmulc(a_, Yc) + v[cr + ps * RS] * alpha;  // B = conj(Lambda) Y + mu F Theta
      kv[ps] = norm2(a_) * w;
      tv[ps] = cmul(a_, bv[ps]) * w;
      Sown += kv[ps];
      Town = Town + tv[ps];
    }
    // sums over the members held by the other lanes of the class, without
    // subtraction: the butterfly's received values are exactly those sums
    float So = 0.f;
    float2 To = make_float2(0.f, 0.f);
    if (QN > 1) {
      So = __shfl_xor_sync(0xffffffffu, Sown, 1);
      To.x = __shfl_xor_sync(0xffffffffu, Town.x, 1);
      To.y = __shfl_xor_sync(0xffffffffu, Town.y, 1);
      if (QN > 2) {
        const float s2 = __shfl_xor_sync(0xffffffffu, Sown + So, 2);
        const float t2x = __shfl_xor_sync(0xffffffffu, Town.x + To.x, 2);
        const float t2y = __shfl_xor_sync(0xffffffffu, Town.y + To.y, 2);
        So += s2;
        To.x += t2x;
        To.y += t2y;
      }
    }
    // Each member by Sherman-Morrison with itself kept out of the sums (no
    // cancellation for any member):
    //   X_p = (B_p (d + S_-p) - conj(Lambda_p) T_-p) / (mu s_p (d + S_-p) + |Lambda_p|^2).
    // The zero-frequency class (Gamma singular at its member 0; one class in
    // the volume) is solved exactly from member 0; its warp takes that branch.
    float2 ratio0 = make_float2(0.f, 0.f);
    const bool dc_warp = __any_sync(0xffffffffu, dc_cls);
    if (dc_warp) {
      float2 r = make_float2(0.f, 0.f);
      if (dc_cls && q == 0) r = cmul(bv[0], av[0]) * (1.f / norm2(av[0]));  // B_0 / conj(Lambda_0)
      if (QN > 1) {
        r.x = __shfl_sync(0xffffffffu, r.x, gbase);
        r.y = __shfl_sync(0xffffffffu, r.y, gbase);
      }
      ratio0 = r;
    }
    float2 tsum = make_float2(0.f, 0.f);
#pragma unroll
    for (int ps = 0; ps < DS; ++ps) {
      float Sm = So;
      float2 Tm = To;
#pragma unroll
      for (int o = 0; o < DS; ++o)
        if (o != ps) {
          Sm += kv[o];
          Tm = Tm + tv[o];
        }
      float2 X = (bv[ps] * (dd + Sm) - cmulc(av[ps], Tm)) * rcp_nr(sv_[ps] * (dd + Sm) + norm2(av[ps]));
      if (dc_warp && dc_cls) {
        X = (q == 0 && ps == 0) ? (bv[0] * (dd + Sm) - cmulc(av[0], Tm)) * (1.f / norm2(av[0]))
                                : (bv[ps] - cmulc(av[ps], ratio0)) * wv[ps];
      }
      v[cr + ps * RS] = conjc(X);  // conjugated: the inverse runs through the forward engine
      if (STATS) tsum = tsum + cmul(av[ps], X);
    }
    if (STATS) {
#pragma unroll
      for (int o = 1; o < QN; o <<= 1) {
        tsum.x += __shfl_xor_sync(0xffffffffu, tsum.x, o);
        tsum.y += __shfl_xor_sync(0xffffffffu, tsum.y, o);
      }
      if (cls_ok && q == 0) {
        const float2 R = Yc - tsum * (1.f / (float)D);
        const double wg = (g == 0 || 2 * g == sv.Ml) ? 1.0 : 2.0;
        acc += wg * (double)norm2(R);
      }
    }
  }
  if (STATS) {
    double* red = reinterpret_cast<double*>(tws + S);
    acc = warp_sum(acc);
    const int warp = tid >> 5;
    if (lane == 0) red[warp] = acc;
    __syncthreads();
    if (warp == 0) {
      double s_ = (lane < (int)((blockDim.x + 31) / 32)) ? red[lane] : 0.0;
      s_ = warp_sum(s_);
      if (lane == 0) sv.partial[bc] = s_;
    }
  }
  // inverse transform, stage 0 from the registers
  __syncthreads();  // every thread has read its forward last-stage inputs
  ct_first_from_regs<S, false>(v, line, rowlen, tl);
  __syncthreads();
  // the store addresses are formed again here rather than kept live (in
  // registers) from the loads through the whole solve
  asm volatile("" : "+l"(col));
  auto st = [&](int j, float2 x) {
    if (cls_ok) col[(long long)j * plane] = conjc(x);
  };
  ct_run<S, 1, false, true, false>(CtNone{}, st, line, rowlen, tl, tws, 1);
}

template <int S, bool STATS, int DR, int DC, int DS>
static cudaError_t fft_s_admm_reg(const Plan& p, const Geometry& g, void* spec, const void* tw, const SolveArgs& sv) {
  const int TW = g.tw_s;
  size_t smem = (size_t)(S * TW * DC + S) * sizeof(float2);
  if (STATS) smem += 32 * sizeof(double);
  const int nb = sv.batch > 1 ? sv.batch : 1;
  SolveArgs svb = sv;
  svb.batch_ny = g.N / DC;
  dim3 grid((g.Ms + TW - 1) / TW, (g.N / DC) * nb);
  cudaError_t e;
  if ((e = allow_smem(k_fft_s_admm_reg<S, STATS, DR, DC, DS>, smem)) != cudaSuccess) return e;
  k_fft_s_admm_reg<S, STATS, DR, DC, DS><<<grid, TW * DC * (S / ct_e(S)), smem, p.stream>>>(
      (float2*)spec, g.Ms, g.Mp, g.N, TW, svb, (const float2*)tw, g.Nl);
  return cudaGetLastError();
}

// the register-resident ADMM s pass for the compile-time lengths and the class
// shapes of the benchmark set (2x2x2, 2x2x1, 1x1x4); cudaErrorNotSupported otherwise
template <int S>
static cudaError_t fft_s_admm_reg_shape(const Plan& p, const Geometry& g, void* spec, const void* tw, bool stats,
                                        const SolveArgs& sv) {
  if (g.dr == 2 && g.dc == 2 && g.ds == 2)
    return stats ? fft_s_admm_reg<S, true, 2, 2, 2>(p, g, spec, tw, sv) : fft_s_admm_reg<S, false, 2, 2, 2>(p, g, spec, tw, sv);
  if (g.dr == 1 && g.dc == 1 && g.ds == 4)
    return stats ? fft_s_admm_reg<S, true, 1, 1, 4>(p, g, spec, tw, sv) : fft_s_admm_reg<S, false, 1, 1, 4>(p, g, spec, tw, sv);
  if (g.dr == 2 && g.dc == 2 && g.ds == 1)
    return stats ? fft_s_admm_reg<S, true, 2, 2, 1>(p, g, spec, tw, sv) : fft_s_admm_reg<S, false, 2, 2, 1>(p, g, spec, tw, sv);
  return cudaErrorNotSupported;
}

template <typename T, int EMAX, int MODE, bool STATS, int NC, int DR_ = 0, int DC_ = 0, int DS_ = 0>
static cudaError_t fft_s_k(const Plan& p, const Geometry& g, void* spec, const void* tw, const SolveArgs& sv) {
  const int tpl = g.S / g.fs.e;
  const int TW = g.tw_s, G = g.g_s;
  size_t smem = (size_t)g.S * TW * G * sizeof(cplx<T>);
  if (NC > 0) smem += (size_t)NC * sizeof(cplx<T>);
  if (STATS) smem += 32 * sizeof(double);  // the CTA's reduction slots
  const int nb = (MODE == S_ADMM && sv.batch > 1) ? sv.batch : 1;
  SolveArgs svb = sv;
  svb.batch_ny = g.N / G;
  dim3 grid((g.Ms + TW - 1) / TW, (g.N / G) * nb);
  LAxis a = laxis(g.S, g.Sl, g.ds, g.fs);
  cudaError_t e;
  if ((e = allow_smem(k_fft_s<T, EMAX, MODE, STATS, NC, DR_, DC_, DS_>, smem)) != cudaSuccess) return e;
  k_fft_s<T, EMAX, MODE, STATS, NC, DR_, DC_, DS_><<<grid, TW * G * tpl, smem, p.stream>>>((cplx<T>*)spec, a, g.Ms, g.Mp, g.N, TW,
                                                                          G, svb, (const cplx<T>*)tw, g.dc, g.Nl);
  return cudaGetLastError();
}

template <typename T, int EMAX>
static cudaError_t fft_s_e(const Plan& p, const Geometry& g, void* spec, const void* tw, int mode, bool stats,
                           const SolveArgs& sv) {
  switch (mode) {
    case S_FWD: return fft_s_k<T, EMAX, S_FWD, false, 0>(p, g, spec, tw, sv);
    case S_INV: return fft_s_k<T, EMAX, S_INV, false, 0>(p, g, spec, tw, sv);
    case S_TIK_GEN: return fft_s_k<T, EMAX, S_TIK_GEN, false, 0>(p, g, spec, tw, sv);
    case S_TIK_USER: return fft_s_k<T, EMAX, S_TIK_USER, false, 0>(p, g, spec, tw, sv);
    case S_ADMM:
      if constexpr (sizeof(T) == 4 && EMAX == 12) {
        const int sl = ct_len<T>(g.S, g.fs);
        if ((sl == 96 || sl == 192) && g.tw_s * g.g_s * (sl / 12) <= 256) {
          const cudaError_t r = sl == 192 ? fft_s_admm_reg_shape<192>(p, g, spec, tw, stats, sv)
                                          : fft_s_admm_reg_shape<96>(p, g, spec, tw, stats, sv);
          if (r != cudaErrorNotSupported) return r;
        }
      }
      if constexpr (sizeof(T) == 4 && EMAX == 16) {
        const int sl = ct_len<T>(g.S, g.fs);
        if ((sl == 64 || sl == 128 || sl == 256) && g.tw_s * g.g_s * (sl / 16) <= 256) {
          const cudaError_t r = sl == 256   ? fft_s_admm_reg_shape<256>(p, g, spec, tw, stats, sv)
                                : sl == 128 ? fft_s_admm_reg_shape<128>(p, g, spec, tw, stats, sv)
                                            : fft_s_admm_reg_shape<64>(p, g, spec, tw, stats, sv);
          if (r != cudaErrorNotSupported) return r;
          if (sl == 256)
            return stats ? fft_s_k<T, EMAX, S_ADMM, true, 256>(p, g, spec, tw, sv)
                         : fft_s_k<T, EMAX, S_ADMM, false, 256>(p, g, spec, tw, sv);
        }
        if (g.dr == 2 && g.dc == 2 && g.ds == 1)
          return stats ? fft_s_k<T, EMAX, S_ADMM, true, 0, 2, 2, 1>(p, g, spec, tw, sv)
                       : fft_s_k<T, EMAX, S_ADMM, false, 0, 2, 2, 1>(p, g, spec, tw, sv);
      }
      return stats ? fft_s_k<T, EMAX, S_ADMM, true, 0>(p, g, spec, tw, sv)
                   : fft_s_k<T, EMAX, S_ADMM, false, 0>(p, g, spec, tw, sv);
    case S_FOLD: return fft_s_k<T, EMAX, S_FOLD, false, 0>(p, g, spec, tw, sv);
    case S_MUL:
    case S_MULC:
      if constexpr (sizeof(T) == 4 && EMAX == 16) {
        if (ct_len<T>(g.S, g.fs) == 256 && g.tw_s * g.g_s * (256 / 16) <= 256)
          return mode == S_MUL ? fft_s_k<T, EMAX, S_MUL, false, 256>(p, g, spec, tw, sv)
                               : fft_s_k<T, EMAX, S_MULC, false, 256>(p, g, spec, tw, sv);
      }
      return mode == S_MUL ? fft_s_k<T, EMAX, S_MUL, false, 0>(p, g, spec, tw, sv)
                           : fft_s_k<T, EMAX, S_MULC, false, 0>(p, g, spec, tw, sv);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_fft_s(const Plan& p, const Geometry& g, void* spec, const void* tw, int mode, bool stats,
                         const SolveArgs* sv) {
  SolveArgs z;
  if (!sv) {
    memset(&z, 0, sizeof(z));
    sv = &z;
  }
  const bool f3 = fam3(g.fs);
  if (p.dtype)
    return f3 ? fft_s_e<double, Emax<double>::p3>(p, g, spec, tw, mode, stats, *sv)
              : fft_s_e<double, Emax<double>::p2>(p, g, spec, tw, mode, stats, *sv);
  return f3 ? fft_s_e<float, Emax<float>::p3>(p, g, spec, tw, mode, stats, *sv)
            : fft_s_e<float, Emax<float>::p2>(p, g, spec, tw, mode, stats, *sv);
}


// ---------------------------------------------------------------------------
// solve-order permutations of Lambda (plan time) and of the LR spectrum
// (once per solve); see solve_layout.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void k_perm_lam(const cplx<T>* __restrict__ lam, cplx<T>* __restrict__ out, int Ms, int Mp, int N,
                           int TW, int G, int dr, int dc, int ds, int Sl, long long total) {
  const SolveTile tl = solve_layout(Ms, TW, G, dr, dc, Sl);
  const int d = dr * dc * ds;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    const int c = (int)(idx % tl.ncls);
    const long long rest = idx / tl.ncls;
    const int q = (int)(rest % d);
    const long long bc = rest / d;
    const int a0 = (int)(bc % tl.gx) * TW, b0 = (int)(bc / tl.gx) * G;
    const int gm = c % tl.GMc, gn = (c / tl.GMc) % tl.GNc, is = c / (tl.GMc * tl.GNc);
    const int pm = q % dr, pn = (q / dr) % dc, ps = q / (dr * dc);
    cplx<T> v = czero<cplx<T>>();
    if (a0 / dr + gm < tl.Gm)
      v = lam[((long long)(is + ps * Sl) * N + b0 / dc + gn + pn * (N / dc)) * Mp + a0 + gm * dr + pm];
    out[idx] = v;
  }
}

template <typename T>
__global__ void k_perm_yhat(const cplx<T>* __restrict__ yh, cplx<T>* __restrict__ out, int Ms, int TW, int G,
                            int dr, int dc, int Sl, int Nl, int Mlp, long long total) {
  const SolveTile tl = solve_layout(Ms, TW, G, dr, dc, Sl);
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    const int c = (int)(idx % tl.ncls);
    const long long bc = idx / tl.ncls;
    const int a0 = (int)(bc % tl.gx) * TW, b0 = (int)(bc / tl.gx) * G;
    const int gm = c % tl.GMc, gn = (c / tl.GMc) % tl.GNc, is = c / (tl.GMc * tl.GNc);
    const int g = a0 / dr + gm, jl = b0 / dc + gn;
    out[idx] = g < tl.Gm ? yh[((long long)is * Nl + jl) * Mlp + g] : czero<cplx<T>>();
  }
}

long long solve_lam_elems(const Geometry& g) {
  const SolveTile tl = solve_layout(g.Ms, g.tw_s, g.g_s, g.dr, g.dc, g.Sl);
  return (long long)tl.gx * (g.N / g.g_s) * (g.dr * g.dc * g.ds) * tl.ncls;
}

long long solve_yhat_elems(const Geometry& g) {
  const SolveTile tl = solve_layout(g.Ms, g.tw_s, g.g_s, g.dr, g.dc, g.Sl);
  return (long long)tl.gx * (g.N / g.g_s) * tl.ncls;
}

cudaError_t launch_perm_lam(const Plan& p, const void* lam, void* out) {
  const Geometry& g = p.hr;
  const long long total = solve_lam_elems(g);
  const int blocks = (int)((total + 255) / 256 < 4096 ? (total + 255) / 256 : 4096);
  if (p.dtype)
    k_perm_lam<double><<<blocks, 256, 0, p.stream>>>((const double2*)lam, (double2*)out, g.Ms, g.Mp, g.N, g.tw_s,
                                                     g.g_s, g.dr, g.dc, g.ds, g.Sl, total);
  else
    k_perm_lam<float><<<blocks, 256, 0, p.stream>>>((const float2*)lam, (float2*)out, g.Ms, g.Mp, g.N, g.tw_s,
                                                    g.g_s, g.dr, g.dc, g.ds, g.Sl, total);
  return cudaGetLastError();
}

cudaError_t launch_perm_yhat(const Plan& p, const void* yh, void* out) {
  const Geometry& g = p.hr;
  const long long total = solve_yhat_elems(g);
  const int blocks = (int)((total + 255) / 256 < 4096 ? (total + 255) / 256 : 4096);
  if (p.dtype)
    k_perm_yhat<double><<<blocks, 256, 0, p.stream>>>((const double2*)yh, (double2*)out, g.Ms, g.tw_s, g.g_s, g.dr,
                                                      g.dc, g.Sl, g.Nl, p.lr.Mp, total);
  else
    k_perm_yhat<float><<<blocks, 256, 0, p.stream>>>((const float2*)yh, (float2*)out, g.Ms, g.tw_s, g.g_s, g.dr,
                                                     g.dc, g.Sl, g.Nl, p.lr.Mp, total);
  return cudaGetLastError();
}

long long s_pass_blocks(const Geometry& g) {
  return (long long)((g.Ms + g.tw_s - 1) / g.tw_s) * (g.N / g.g_s);
}

}  // namespace sr3d

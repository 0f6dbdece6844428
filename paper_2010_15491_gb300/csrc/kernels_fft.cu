// FFT passes of the 3D transforms along m and n (the s pass with the
// per-aliasing-class solve is in kernels_fft_s.cu).
//
// Spectral layout of a real volume x[s][n][m] (sizes M, N, S): complex
// spec[k_s][n-slot][m-slot] with
//   m-slot g*dr + p  <->  m-frequency g + p*Ml, g in [0, Ml/2]   (Ml = M/dr)
//   n and s natural.
// Every frequency either is stored or has its conjugate stored (the m axis
// is real), and the d = dr*dc*ds members of each aliasing class of eq. (8)
// sit in dr adjacent m-slots of the dc rows j, j+Nl, ... on ds planes, so the
// s pass can solve a class from one shared-memory tile.
//
// Per solve the passes are: real FFT along m (packed half-length complex
// transform), strided FFT along n, FFT along s fused with the class solve
// and the inverse s FFT, inverse n FFT, inverse real FFT along m.
#include "fft.cuh"
#include "fft_ct.cuh"
#include "fft_host.cuh"
#include "internal.h"

namespace sr3d {


// ---------------------------------------------------------------------------
// m pass, forward: L real lines of length M -> Ms slots each.
// ---------------------------------------------------------------------------
template <typename T, int EMAX, int NC>
__global__ void __launch_bounds__(256, 2) k_rfft_m_fwd(const T* __restrict__ in, long long nlines, cplx<T>* __restrict__ out, MAxis a,
                             int L, int Hp, const cplx<T>* __restrict__ twM) {
  using C = cplx<T>;
  extern __shared__ __align__(16) unsigned char smraw[];
  C* sm = reinterpret_cast<C*>(smraw);
  const int H = NC > 0 ? NC : a.H;
  const int tpl = NC > 0 ? NC / ct_e(NC) : H / a.f.e;
  const long long line0 = (long long)blockIdx.x * L;
  const C* inc = reinterpret_cast<const C*>(in);  // (x[2j], x[2j+1]) as one complex
  const C* tw = twM;
  {
    const int l = threadIdx.x / tpl, tl = threadIdx.x - l * tpl;
    const long long gl = line0 + l;
    const bool ok = gl < nlines;
    const C* src = inc + gl * H;
    auto ld = [&](int j) -> C { return ok ? __ldg(&src[j]) : czero<C>(); };
    if constexpr (NC > 0) {
      C* tws = sm + L * Hp;  // table of the M = 2H roots
      ct_load_twiddles(tws, twM, 2 * NC);
      tw = tws;
      ct_line_gs<NC, true>(ld, sm + l * Hp, 1, tl, tws, 2);
    } else {
      fft_line_gs<T, EMAX>(ld, sm + l * Hp, 1, a.f, tl, tpl, twM, 2);
    }
  }
  auto pos = [](int i) { return NC > 0 ? ct_pos<true>(i) : i; };
  // split the packed transform: X[k] = E[k] + W^k O[k], E/O from Z[k], conj(Z[H-k])
  auto emit = [&](int l, int slot, int k, bool cj) {
    const long long gl = line0 + l;
    const C zk = sm[l * Hp + pos(k == H ? 0 : k)];
    const C zc = conjc(sm[l * Hp + pos(k == 0 ? 0 : H - k)]);
    const C e = (zk + zc) * (T)0.5;
    const C o = mul_mi(zk - zc) * (T)0.5;
    const C X = e + cmul(NC > 0 ? tw[k] : __ldg(&twM[k]), o);
    out[gl * a.Mp + slot] = cj ? conjc(X) : X;
  };
  if constexpr (NC > 0) {
    // slot -> (frequency, conjugate) once per CTA; a warp writes 32 slots of a line
    short2* tab = reinterpret_cast<short2*>(sm + L * Hp + 2 * NC);
    for (int i = threadIdx.x; i < a.Ms; i += blockDim.x) {
      const int grp = i / a.dr, p = i - grp * a.dr;
      int k = grp + p * a.Ml;
      const bool cj = k > H;
      if (cj) k = a.M - k;
      tab[i] = make_short2((short)k, (short)cj);
    }
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int l = warp; l < L; l += nw) {
      if (line0 + l >= nlines) break;
      for (int slot = lane; slot < a.Ms; slot += 32) {
        const short2 t = tab[slot];
        emit(l, slot, t.x, t.y != 0);
      }
    }
  } else {
    for (int i = threadIdx.x; i < L * a.Ms; i += blockDim.x) {
      const int l = i / a.Ms, slot = i - l * a.Ms;
      if (line0 + l >= nlines) continue;
      const int grp = slot / a.dr, p = slot - grp * a.dr;
      int k = grp + p * a.Ml;
      const bool cj = k > H;
      if (cj) k = a.M - k;
      emit(l, slot, k, cj);
    }
  }
}

// ---------------------------------------------------------------------------
// m pass, inverse: Ms slots -> M reals per line, times `scale`.
// ---------------------------------------------------------------------------
template <typename T, int EMAX, int NC>
__global__ void __launch_bounds__(256, 2) k_rfft_m_inv(const cplx<T>* __restrict__ in, long long nlines, T* __restrict__ out, MAxis a,
                             int L, int Hp, const cplx<T>* __restrict__ twM, T scale) {
  using C = cplx<T>;
  extern __shared__ __align__(16) unsigned char smraw[];
  C* sm = reinterpret_cast<C*>(smraw);
  const int H = NC > 0 ? NC : a.H;
  const int tpl = NC > 0 ? NC / ct_e(NC) : H / a.f.e;
  const C* tw = twM;
  C* slots = sm + L * Hp + (NC > 0 ? 2 * NC : 0);  // NC > 0: the CTA's L slot rows, staged
  short2* stab = reinterpret_cast<short2*>(slots + (NC > 0 ? L * a.Mp : 0));  // NC > 0: k -> (slot, conj)
  if constexpr (NC > 0) {
    for (int k = threadIdx.x; k <= H; k += blockDim.x) {
      bool c;
      const int sl = mslot_of(k, a.M, a.Ml, a.dr, c);
      stab[k] = make_short2((short)sl, (short)c);
    }
    C* tws = sm + L * Hp;
    // the L rows of Mp complex are contiguous in global memory: 16-byte async copies
    const long long line0s = (long long)blockIdx.x * L;
    const long long nrows = (nlines - line0s) < L ? (nlines - line0s) : L;
    const float* src = reinterpret_cast<const float*>(in + line0s * a.Mp);
    float* dst = reinterpret_cast<float*>(slots);
    const int n16 = (int)(nrows * a.Mp / 2);  // Mp even: whole 16-byte chunks
    for (int i = threadIdx.x; i < n16; i += blockDim.x) {
      const unsigned dsh = (unsigned)__cvta_generic_to_shared(dst + 4 * i);
      asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(dsh), "l"(src + 4 * i) : "memory");
    }
    asm volatile("cp.async.commit_group;\n" ::: "memory");
    for (int i = threadIdx.x; i < 2 * NC; i += blockDim.x) tws[i] = __ldg(&twM[i]);
    asm volatile("cp.async.wait_group 0;\n" ::: "memory");
    __syncthreads();
    tw = tws;
  }
  const long long line0 = (long long)blockIdx.x * L;
  const int l = threadIdx.x / tpl, tl = threadIdx.x - l * tpl;
  const long long gl = line0 + l;
  const bool ok = gl < nlines;
  const C* row = NC > 0 ? slots + (long long)l * a.Mp : in + gl * a.Mp;
  // Z[k] = E'[k] + i O'[k] from X[k] and conj(X[H-k]); the inverse runs
  // through the forward engine on conj(Z)
  auto ld = [&](int k) -> C {
    if (!ok) return czero<C>();
    bool c1, c2;
    int s1, s2;
    if constexpr (NC > 0) {
      const short2 t1 = stab[k], t2 = stab[H - k];
      s1 = t1.x; c1 = t1.y != 0;
      s2 = t2.x; c2 = t2.y != 0;
    } else {
      s1 = mslot_of(k, a.M, a.Ml, a.dr, c1);
      s2 = mslot_of(H - k, a.M, a.Ml, a.dr, c2);
    }
    C xk = NC > 0 ? row[s1] : __ldg(&row[s1]);
    if (c1) xk = conjc(xk);
    C xh = NC > 0 ? row[s2] : __ldg(&row[s2]);
    if (!c2) xh = conjc(xh);  // conj(X[H-k])
    const C e = xk + xh;
    const C o = cmulc(NC > 0 ? tw[k] : __ldg(&twM[k]), xk - xh);  // W^-k (X[k] - conj(X[H-k]))
    return conjc(e + mul_i(o));
  };
  C* outc = reinterpret_cast<C*>(out) + gl * H;
  auto st = [&](int j, C r) {
    if (ok) outc[j] = mkc(r.x * scale, -r.y * scale);
  };
  if constexpr (NC > 0) ct_line_gg<NC, true>(ld, st, sm + l * Hp, 1, tl, tw, 2);
  else fft_line_gg<T, EMAX>(ld, st, sm + l * Hp, 1, a.f, tl, tpl, twM, 2);
}

// ---------------------------------------------------------------------------
// m passes with the real-FFT split in registers (FP32, compile-time lengths,
// d_r = 1 or 2).  After the last stage of the half-length transform (length
// NC = M/2, E elements and TPL = NC/E threads per line), thread tl holds Z[k]
// for k = tl + TPL r, r < E.  The split of the real transform pairs Z[g] with
// Z[NC - g], which sits in lane (TPL - tl) mod TPL at r' = E - 1 - r (lane 0:
// itself, r' = E - r), so one warp shuffle per pair replaces the shared-
// memory round trip of the split:
//   E = (Z[g] + conj Z[NC-g]) / 2,  O = -i (Z[g] - conj Z[NC-g]) / 2,
//   X[g] = E + W^g O,  X[NC-g] = conj(E - W^g O)   (W = exp(-2 pi i / M)).
// With d_r = 2 the slots 2g and 2g+1 hold X[g] and conj(X[NC-g]) (frequency
// g + NC, conjugated), i.e. E + W^g O and E - W^g O: one 16-byte store per g,
// and the inverse pass reads the same 16 bytes to form its inputs for g and
// NC - g.  The inverse input set of thread tl (k = tl + TPL m) is the same
// index set, so the first inverse stage runs from registers.
// ---------------------------------------------------------------------------
template <int NC, int DR>
__global__ void __launch_bounds__(256, 2) k_rfft_m_fwd2(const float* __restrict__ in, long long nlines,
                                                      float2* __restrict__ out, int Mp, int L, int Hp,
                                                      const float2* __restrict__ twM) {
  constexpr int E = ct_e(NC), TPL = NC / E, HE = E / 2;
  constexpr int NST = ct_nst(NC);
  extern __shared__ __align__(16) unsigned char smraw[];
  float2* sm = reinterpret_cast<float2*>(smraw);
  float2* tws = sm + L * Hp;  // the M = 2 NC roots
  ct_load_twiddles(tws, twM, 2 * NC);
  const int l = threadIdx.x / TPL, tl = threadIdx.x % TPL;
  const long long gl = (long long)blockIdx.x * L + l;
  const bool ok = gl < nlines;
  const float2* src = reinterpret_cast<const float2*>(in) + gl * NC;  // (x[2j], x[2j+1]) as one complex
  float2* line = sm + l * Hp;
  auto ld = [&](int j) -> float2 { return ok ? __ldg(&src[j]) : make_float2(0.f, 0.f); };
  ct_run_to<NC, 0, NST - 1, true>(ld, line, 1, tl, tws, 2);
  float2 v[E];  // v[r] = Z[tl + TPL r]
  ct_last_to_regs<NC, true>(line, 1, tl, tws, 2, v);
  const int lane = threadIdx.x & 31;
  const int partner = lane - tl + ((TPL - tl) & (TPL - 1));
  float2* orow = out + gl * Mp;
#pragma unroll
  for (int r = 0; r <= HE; ++r) {
    float2 zh;
    if (r < HE) {
      float2 recv;
      recv.x = __shfl_sync(0xffffffffu, v[E - 1 - r].x, partner);
      recv.y = __shfl_sync(0xffffffffu, v[E - 1 - r].y, partner);
      zh = tl == 0 ? v[(E - r) % E] : recv;
    } else {
      zh = v[HE];  // g = NC/2 (lane 0 only)
    }
    const int g = tl + TPL * r;
    const float2 zc = conjc(zh);
    const float2 e = (v[r] + zc) * 0.5f;
    const float2 o = mul_mi(v[r] - zc) * 0.5f;
    const float2 t = cmul(tws[r < HE ? g : NC / 2], o);
    if (ok && (r < HE || tl == 0)) {
      const float2 xp = e + t, xm = e - t;
      if constexpr (DR == 2) {
        reinterpret_cast<float4*>(orow)[g] = make_float4(xp.x, xp.y, xm.x, xm.y);
      } else {
        orow[g] = xp;
        if (r < HE || tl != 0) orow[NC - g] = conjc(xm);  // g = NC/2: the same slot
      }
    }
  }
}

template <int NC, int DR>
__global__ void __launch_bounds__(256, 2) k_rfft_m_inv2(const float2* __restrict__ in, long long nlines,
                                                      float* __restrict__ out, int Mp, int L, int Hp,
                                                      const float2* __restrict__ twM, float scale) {
  constexpr int E = ct_e(NC), TPL = NC / E, HE = E / 2;
  extern __shared__ __align__(16) unsigned char smraw[];
  float2* sm = reinterpret_cast<float2*>(smraw);
  float2* tws = sm + L * Hp;
  ct_load_twiddles(tws, twM, 2 * NC);
  const int l = threadIdx.x / TPL, tl = threadIdx.x % TPL;
  const long long gl = (long long)blockIdx.x * L + l;
  const bool ok = gl < nlines;
  const float2* row = in + gl * Mp;
  // pairs g = tl + TPL m: X[g] and conj(X[NC - g])
  float2 xk[HE + 1], xh[HE + 1];
#pragma unroll
  for (int m = 0; m <= HE; ++m) {
    const int g = tl + TPL * m;
    const bool act = ok && (m < HE || tl == 0);
    xk[m] = make_float2(0.f, 0.f);
    xh[m] = make_float2(0.f, 0.f);
    if (act) {
      if constexpr (DR == 2) {
        const float4 q4 = __ldg(reinterpret_cast<const float4*>(row) + g);
        xk[m] = make_float2(q4.x, q4.y);
        xh[m] = make_float2(q4.z, q4.w);
      } else {
        xk[m] = __ldg(&row[g]);
        xh[m] = conjc(__ldg(&row[NC - g]));
      }
    }
  }
  // inverse inputs (the forward engine on conjugated data): z[m] = Zi[tl + TPL m]
  float2 z[E];
  const int lane = threadIdx.x & 31;
  const int partner = lane - tl + ((TPL - tl) & (TPL - 1));
#pragma unroll
  for (int m = 0; m <= HE; ++m) {
    const int g = tl + TPL * m;
    const float2 e = xk[m] + xh[m];
    const float2 o = cmulc(tws[m < HE ? g : NC / 2], xk[m] - xh[m]);  // W^-g (X[g] - conj X[NC-g])
    const float2 zg = conjc(e + mul_i(o));                            // input g
    const float2 zp = e - mul_i(o);                                   // input NC - g
    if (m < HE) {
      z[m] = zg;
      float2 recv;
      recv.x = __shfl_sync(0xffffffffu, zp.x, partner);
      recv.y = __shfl_sync(0xffffffffu, zp.y, partner);
      if (tl != 0) z[E - 1 - m] = recv;
      else if (m >= 1) z[E - m] = zp;
    } else if (tl == 0) {
      z[HE] = zg;
    }
  }
  // stage 0 from the registers
  float2* line = sm + l * Hp;
  ct_first_from_regs<NC, true>(z, line, 1, tl);
  __syncthreads();
  float2* outc = reinterpret_cast<float2*>(out) + gl * NC;
  auto st = [&](int j, float2 r) {
    if (ok) outc[j] = make_float2(r.x * scale, -r.y * scale);
  };
  ct_run<NC, 1, false, true, true>(CtNone{}, st, line, 1, tl, tws, 2);
}

// ---------------------------------------------------------------------------
// n pass: tile of TW m-slots x all N rows of one s plane.
// ---------------------------------------------------------------------------
template <typename T, int EMAX, bool INV, int NC>
__global__ void __launch_bounds__(256, 2) k_fft_n(cplx<T>* __restrict__ spec, LAxis a, int Ms, int Mp, int TW,
                        const cplx<T>* __restrict__ twN) {
  using C = cplx<T>;
  extern __shared__ __align__(16) unsigned char smraw[];
  C* sm = reinterpret_cast<C*>(smraw);
  const int N = NC > 0 ? NC : a.N;
  const int a0 = blockIdx.x * TW;
  const int tv = min(TW, Ms - a0);
  C* base = spec + (long long)blockIdx.y * N * Mp + a0;
  const int t = threadIdx.x % TW, tl = threadIdx.x / TW, tpl = NC > 0 ? NC / ct_e(NC) : N / a.f.e;
  const bool ok = t < tv;
  C* col = base + t;
  auto ld = [&](int k) -> C {
    if (!ok) return czero<C>();
    const C v = col[(long long)k * Mp];
    return INV ? conjc(v) : v;
  };
  auto st = [&](int k, C v) {
    if (ok) col[(long long)k * Mp] = INV ? conjc(v) : v;
  };
  if constexpr (NC > 0) {
    C* tws = sm + N * TW;
    ct_load_twiddles(tws, twN, NC);
    ct_line_gg<NC>(ld, st, sm + t, TW, tl, tws, 1);
  } else {
    fft_line_gg<T, EMAX>(ld, st, sm + t, TW, a.f, tl, tpl, twN, 1);
  }
}

template <typename T, int EMAX, int NC>
static cudaError_t rfft_fwd_k(const Plan& p, const Geometry& g, const void* in, void* out, const void* tw) {
  int L, Hp, threads;
  size_t smem;
  m_launch_shape(g, sizeof(cplx<T>), g.lm_f, L, Hp, threads, smem);
  if (NC > 0) {
    Hp = ct_line_pitch<true>(NC);
    smem = (size_t)(L * Hp + 2 * NC) * sizeof(cplx<T>) + (size_t)g.Ms * sizeof(short2);  // + slot table
  }
  const long long nlines = (long long)g.S * g.N;
  const unsigned blocks = (unsigned)((nlines + L - 1) / L);
  MAxis a = maxis(g);
  cudaError_t e;
  if ((e = allow_smem(k_rfft_m_fwd<T, EMAX, NC>, smem)) != cudaSuccess) return e;
  k_rfft_m_fwd<T, EMAX, NC><<<blocks, threads, smem, p.stream>>>((const T*)in, nlines, (cplx<T>*)out, a, L, Hp,
                                                                (const cplx<T>*)tw);
  return cudaGetLastError();
}

template <typename T, int EMAX, int NC>
static cudaError_t rfft_inv_k(const Plan& p, const Geometry& g, const void* in, void* out, const void* tw,
                              double scale) {
  int L, Hp, threads;
  size_t smem;
  m_launch_shape(g, sizeof(cplx<T>), g.lm_i, L, Hp, threads, smem);
  if (NC > 0) {
    Hp = ct_line_pitch<true>(NC);
    smem = (size_t)(L * Hp + 2 * NC + L * g.Mp) * sizeof(cplx<T>) + (size_t)(NC + 1) * sizeof(short2);
  }
  const long long nlines = (long long)g.S * g.N;
  const unsigned blocks = (unsigned)((nlines + L - 1) / L);
  MAxis a = maxis(g);
  cudaError_t e;
  if ((e = allow_smem(k_rfft_m_inv<T, EMAX, NC>, smem)) != cudaSuccess) return e;
  k_rfft_m_inv<T, EMAX, NC><<<blocks, threads, smem, p.stream>>>((const cplx<T>*)in, nlines, (T*)out, a, L, Hp,
                                                                (const cplx<T>*)tw, (T)scale);
  return cudaGetLastError();
}

template <int NC, int DR>
static cudaError_t rfft_fwd2_k(const Plan& p, const Geometry& g, const void* in, void* out, const void* tw) {
  int L, Hp, threads;
  size_t smem;
  m_launch_shape(g, sizeof(float2), g.lm_f, L, Hp, threads, smem);
  Hp = ct_line_pitch<true>(NC);
  smem = (size_t)(L * Hp + 2 * NC) * sizeof(float2);
  const long long nlines = (long long)g.S * g.N;
  const unsigned blocks = (unsigned)((nlines + L - 1) / L);
  cudaError_t e;
  if ((e = allow_smem(k_rfft_m_fwd2<NC, DR>, smem)) != cudaSuccess) return e;
  k_rfft_m_fwd2<NC, DR><<<blocks, threads, smem, p.stream>>>((const float*)in, nlines, (float2*)out, g.Mp, L, Hp,
                                                           (const float2*)tw);
  return cudaGetLastError();
}

template <int NC, int DR>
static cudaError_t rfft_inv2_k(const Plan& p, const Geometry& g, const void* in, void* out, const void* tw,
                               double scale) {
  int L, Hp, threads;
  size_t smem;
  m_launch_shape(g, sizeof(float2), g.lm_i, L, Hp, threads, smem);
  Hp = ct_line_pitch<true>(NC);
  smem = (size_t)(L * Hp + 2 * NC) * sizeof(float2);
  const long long nlines = (long long)g.S * g.N;
  const unsigned blocks = (unsigned)((nlines + L - 1) / L);
  cudaError_t e;
  if ((e = allow_smem(k_rfft_m_inv2<NC, DR>, smem)) != cudaSuccess) return e;
  k_rfft_m_inv2<NC, DR><<<blocks, threads, smem, p.stream>>>((const float2*)in, nlines, (float*)out, g.Mp, L, Hp,
                                                           (const float2*)tw, (float)scale);
  return cudaGetLastError();
}

// the register-split m passes: FP32, compile-time half length, d_r 1 or 2
template <int DR>
static cudaError_t rfft2_fwd_len(const Plan& p, const Geometry& g, const void* in, void* out, const void* tw) {
  switch (ct_len<float>(g.M / 2, g.fm)) {
    case 32: return rfft_fwd2_k<32, DR>(p, g, in, out, tw);
    case 64: return rfft_fwd2_k<64, DR>(p, g, in, out, tw);
    case 128: return rfft_fwd2_k<128, DR>(p, g, in, out, tw);
    case 256: return rfft_fwd2_k<256, DR>(p, g, in, out, tw);
    case 512: return rfft_fwd2_k<512, DR>(p, g, in, out, tw);
    case 48: return rfft_fwd2_k<48, DR>(p, g, in, out, tw);
    case 96: return rfft_fwd2_k<96, DR>(p, g, in, out, tw);
    case 192: return rfft_fwd2_k<192, DR>(p, g, in, out, tw);
  }
  return cudaErrorNotSupported;
}
template <int DR>
static cudaError_t rfft2_inv_len(const Plan& p, const Geometry& g, const void* in, void* out, const void* tw,
                                 double scale) {
  switch (ct_len<float>(g.M / 2, g.fm)) {
    case 32: return rfft_inv2_k<32, DR>(p, g, in, out, tw, scale);
    case 64: return rfft_inv2_k<64, DR>(p, g, in, out, tw, scale);
    case 128: return rfft_inv2_k<128, DR>(p, g, in, out, tw, scale);
    case 256: return rfft_inv2_k<256, DR>(p, g, in, out, tw, scale);
    case 512: return rfft_inv2_k<512, DR>(p, g, in, out, tw, scale);
    case 48: return rfft_inv2_k<48, DR>(p, g, in, out, tw, scale);
    case 96: return rfft_inv2_k<96, DR>(p, g, in, out, tw, scale);
    case 192: return rfft_inv2_k<192, DR>(p, g, in, out, tw, scale);
  }
  return cudaErrorNotSupported;
}

template <typename T>
static cudaError_t rfft_fwd_t(const Plan& p, const Geometry& g, const void* in, void* out, const void* tw) {
  if constexpr (sizeof(T) == 4) {
    if (ct_len<T>(g.M / 2, g.fm) > 0 && (g.dr == 1 || g.dr == 2))
      return g.dr == 2 ? rfft2_fwd_len<2>(p, g, in, out, tw) : rfft2_fwd_len<1>(p, g, in, out, tw);
    switch (ct_len<T>(g.M / 2, g.fm)) {
      case 32: return rfft_fwd_k<T, 16, 32>(p, g, in, out, tw);
      case 64: return rfft_fwd_k<T, 16, 64>(p, g, in, out, tw);
      case 128: return rfft_fwd_k<T, 16, 128>(p, g, in, out, tw);
      case 256: return rfft_fwd_k<T, 16, 256>(p, g, in, out, tw);
      case 512: return rfft_fwd_k<T, 16, 512>(p, g, in, out, tw);
      case 48: return rfft_fwd_k<T, 12, 48>(p, g, in, out, tw);
      case 96: return rfft_fwd_k<T, 12, 96>(p, g, in, out, tw);
      case 192: return rfft_fwd_k<T, 12, 192>(p, g, in, out, tw);
    }
  }
  if (fam3(g.fm)) return rfft_fwd_k<T, Emax<T>::p3, 0>(p, g, in, out, tw);
  return rfft_fwd_k<T, Emax<T>::p2, 0>(p, g, in, out, tw);
}

template <typename T>
static cudaError_t rfft_inv_t(const Plan& p, const Geometry& g, const void* in, void* out, const void* tw,
                              double scale) {
  if constexpr (sizeof(T) == 4) {
    if (ct_len<T>(g.M / 2, g.fm) > 0 && (g.dr == 1 || g.dr == 2))
      return g.dr == 2 ? rfft2_inv_len<2>(p, g, in, out, tw, scale) : rfft2_inv_len<1>(p, g, in, out, tw, scale);
    switch (ct_len<T>(g.M / 2, g.fm)) {
      case 32: return rfft_inv_k<T, 16, 32>(p, g, in, out, tw, scale);
      case 64: return rfft_inv_k<T, 16, 64>(p, g, in, out, tw, scale);
      case 128: return rfft_inv_k<T, 16, 128>(p, g, in, out, tw, scale);
      case 256: return rfft_inv_k<T, 16, 256>(p, g, in, out, tw, scale);
      case 512: return rfft_inv_k<T, 16, 512>(p, g, in, out, tw, scale);
      case 48: return rfft_inv_k<T, 12, 48>(p, g, in, out, tw, scale);
      case 96: return rfft_inv_k<T, 12, 96>(p, g, in, out, tw, scale);
      case 192: return rfft_inv_k<T, 12, 192>(p, g, in, out, tw, scale);
    }
  }
  if (fam3(g.fm)) return rfft_inv_k<T, Emax<T>::p3, 0>(p, g, in, out, tw, scale);
  return rfft_inv_k<T, Emax<T>::p2, 0>(p, g, in, out, tw, scale);
}

template <typename T, int EMAX, int NC>
static cudaError_t fft_n_e(const Plan& p, const Geometry& g, void* spec, const void* tw, bool inverse) {
  const int tpl = g.N / g.fn.e;
  const int TW = g.tw_n;
  size_t smem = (size_t)g.N * TW * sizeof(cplx<T>);
  if (NC > 0) smem += (size_t)NC * sizeof(cplx<T>);
  dim3 grid((g.Ms + TW - 1) / TW, g.S);
  LAxis a = laxis(g.N, g.Nl, g.dc, g.fn);
  cudaError_t e;
  if (inverse) {
    if ((e = allow_smem(k_fft_n<T, EMAX, true, NC>, smem)) != cudaSuccess) return e;
    k_fft_n<T, EMAX, true, NC><<<grid, TW * tpl, smem, p.stream>>>((cplx<T>*)spec, a, g.Ms, g.Mp, TW,
                                                                  (const cplx<T>*)tw);
  } else {
    if ((e = allow_smem(k_fft_n<T, EMAX, false, NC>, smem)) != cudaSuccess) return e;
    k_fft_n<T, EMAX, false, NC><<<grid, TW * tpl, smem, p.stream>>>((cplx<T>*)spec, a, g.Ms, g.Mp, TW,
                                                                   (const cplx<T>*)tw);
  }
  return cudaGetLastError();
}

cudaError_t launch_rfft_m_fwd(const Plan& p, const Geometry& g, const void* in, void* out, const void* tw) {
  return p.dtype ? rfft_fwd_t<double>(p, g, in, out, tw) : rfft_fwd_t<float>(p, g, in, out, tw);
}

cudaError_t launch_rfft_m_inv(const Plan& p, const Geometry& g, const void* in, void* out, const void* tw,
                              double scale) {
  return p.dtype ? rfft_inv_t<double>(p, g, in, out, tw, scale) : rfft_inv_t<float>(p, g, in, out, tw, scale);
}

cudaError_t launch_fft_n(const Plan& p, const Geometry& g, void* spec, const void* tw, bool inverse) {
  const bool f3 = fam3(g.fn);
  if (p.dtype)
    return f3 ? fft_n_e<double, Emax<double>::p3, 0>(p, g, spec, tw, inverse)
              : fft_n_e<double, Emax<double>::p2, 0>(p, g, spec, tw, inverse);
  switch (ct_len<float>(g.N, g.fn)) {
    case 64: return fft_n_e<float, 16, 64>(p, g, spec, tw, inverse);
    case 128: return fft_n_e<float, 16, 128>(p, g, spec, tw, inverse);
    case 256: return fft_n_e<float, 16, 256>(p, g, spec, tw, inverse);
    case 512: return fft_n_e<float, 16, 512>(p, g, spec, tw, inverse);
    case 48: return fft_n_e<float, 12, 48>(p, g, spec, tw, inverse);
    case 96: return fft_n_e<float, 12, 96>(p, g, spec, tw, inverse);
    case 192: return fft_n_e<float, 12, 192>(p, g, spec, tw, inverse);
  }
  if (f3) return fft_n_e<float, Emax<float>::p3, 0>(p, g, spec, tw, inverse);
  return fft_n_e<float, Emax<float>::p2, 0>(p, g, spec, tw, inverse);
}

}  // namespace sr3d

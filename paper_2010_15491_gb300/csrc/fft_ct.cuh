// Compile-time-planned FFT lines for the hot lengths (FP32).
//
// Same Stockham formulation as fft.cuh, but the length N, the radices, the
// threads per line and every index are compile-time constants, so there are
// no runtime divisions or predicated stage loops, and twiddles come from a
// shared-memory table.  A thread owns E elements per stage: E = 16 for
// N = 2^a (radices [N / 16^b, 16, ..., 16]) and E = 12 for N = 3 * 2^a
// (radices [3 or 6, 4, ..., 4]); N / E threads per line.  The first stage
// loads straight from global memory and the last stage stores straight to
// global memory.
#pragma once
#include "fft.cuh"

namespace sr3d {

constexpr int ct_e(int n) { return n % 3 == 0 ? 12 : 16; }
constexpr int ct_rem(int n, int p) { return n % p == 0 ? ct_rem(n / p, p) : n; }
constexpr int ct_big(int n, int p) { return n % p == 0 ? 1 + ct_big(n / p, p) : 0; }
constexpr int ct_nst(int n) {
  return ct_e(n) == 16 ? ct_big(n, 16) + (ct_rem(n, 16) > 1 ? 1 : 0) : ct_big(n, 4) + 1;
}
// radix of stage i
constexpr int ct_radix(int n, int i) {
  return ct_e(n) == 16 ? ((ct_rem(n, 16) > 1 && i == 0) ? ct_rem(n, 16) : 16) : (i == 0 ? ct_rem(n, 4) : 4);
}
// product of the radices before stage i
constexpr int ct_ns(int n, int i) { return i == 0 ? 1 : ct_ns(n, i - 1) * ct_radix(n, i - 1); }

template <int N> __host__ __device__ constexpr bool ct_supported() {
  return N == 32 || N == 64 || N == 128 || N == 256 || N == 512 || N == 48 || N == 96 || N == 192;
}

// Shared-memory position of line element i: with PAD one spare slot follows
// every 16 elements, which spreads the first stage's stride-R stores over
// the banks (used by the contiguous-line m pass).
template <bool PAD> __device__ __forceinline__ int ct_pos(int i) { return PAD ? i + (i >> 4) : i; }
template <bool PAD> __host__ __device__ constexpr int ct_line_pitch(int n) {
  // padded length rounded to 4 (mod 16) complex, so that consecutive lines
  // start 8 banks apart
  return PAD ? ((n + n / 16 + 1 + 15) / 16) * 16 + 4 : n;
}

// Stage I of the length-N transform on one line.  FIRST: inputs from ld;
// LAST: outputs to st; otherwise shared memory in place (barrier between
// the loads and the stores, and after the stores).
template <int N, int I, bool FIRST, bool LAST, bool PAD, class Ld, class St>
__device__ __forceinline__ void ct_stage(const Ld& ld, const St& st, float2* line, int es, int tl,
                                         const float2* __restrict__ tws, int twstep) {
  constexpr int E = ct_e(N);
  constexpr int R = ct_radix(N, I);
  constexpr int NS = ct_ns(N, I);
  constexpr int TPL = N / E;
  constexpr int NB = E / R;
  constexpr int NR = N / R;
  constexpr int STEP = N / (NS * R);
  float2 v[E];
#pragma unroll
  for (int u = 0; u < NB; ++u) {
    const int j = tl + u * TPL;
    const int jm = j % NS;
#pragma unroll
    for (int r = 0; r < R; ++r) {
      float2 a;
      if constexpr (FIRST) a = ld(j + r * NR);
      else a = line[ct_pos<PAD>(j + r * NR) * es];
      if constexpr (NS > 1)
        if (r > 0) a = cmul(a, tws[jm * r * STEP * twstep]);
      v[u * R + r] = a;
    }
  }
  if constexpr (!FIRST && !LAST) __syncthreads();
  if constexpr (FIRST && LAST) __syncthreads();  // single stage: every load before any store
#pragma unroll
  for (int u = 0; u < NB; ++u) {
    Dft<R, float2, float>::run(&v[u * R]);
    const int j = tl + u * TPL;
    const int jm = j % NS;
    const int base = (j - jm) * R + jm;
#pragma unroll
    for (int r = 0; r < R; ++r) {
      if constexpr (LAST) st(base + r * NS, v[u * R + r]);
      else line[ct_pos<PAD>(base + r * NS) * es] = v[u * R + r];
    }
  }
  if constexpr (!LAST) __syncthreads();
}

struct CtNone {
  __device__ float2 operator()(int) const { return make_float2(0.f, 0.f); }
  __device__ void operator()(int, float2) const {}
};

// Stages I.. of the length-N transform.  G_IN: stage 0 reads through ld
// (global); G_OUT: the last stage writes through st (global); otherwise the
// line lives in shared memory.
template <int N, int I, bool G_IN, bool G_OUT, bool PAD, class Ld, class St>
__device__ __forceinline__ void ct_run(const Ld& ld, const St& st, float2* line, int es, int tl,
                                       const float2* __restrict__ tws, int twstep) {
  constexpr int NST = ct_nst(N);
  if constexpr (I < NST) {
    ct_stage<N, I, G_IN && I == 0, G_OUT && I == NST - 1, PAD>(ld, st, line, es, tl, tws, twstep);
    ct_run<N, I + 1, G_IN, G_OUT, PAD>(ld, st, line, es, tl, tws, twstep);
  }
}

// Stages I .. END-1 (END < number of stages): stage 0 reads through ld, every
// stage writes the line in shared memory (barrier after each).
template <int N, int I, int END, bool PAD, class Ld>
__device__ __forceinline__ void ct_run_to(const Ld& ld, float2* line, int es, int tl, const float2* __restrict__ tws,
                                          int twstep) {
  if constexpr (I < END) {
    ct_stage<N, I, I == 0, false, PAD>(ld, CtNone{}, line, es, tl, tws, twstep);
    ct_run_to<N, I + 1, END, PAD>(ld, line, es, tl, tws, twstep);
  }
}

// The last stage from the line in shared memory (complete, after a barrier)
// into registers: v[q] = X[tl + TPL q], q < E.  Its butterfly j = tl + u TPL
// (u < E / R) reads j + r NS (NS = N / R) and yields output j + r NS =
// tl + TPL (u + (E / R) r).
template <int N, bool PAD>
__device__ __forceinline__ void ct_last_to_regs(const float2* line, int es, int tl, const float2* __restrict__ tws,
                                                int twstep, float2* v) {
  constexpr int I = ct_nst(N) - 1;
  constexpr int E = ct_e(N), R = ct_radix(N, I), NS = ct_ns(N, I), TPL = N / E, NB = E / R;
  static_assert(NS * R == N, "the last stage spans the line");
#pragma unroll
  for (int u = 0; u < NB; ++u) {
    const int j = tl + u * TPL;
    float2 w[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
      float2 a = line[ct_pos<PAD>(j + r * NS) * es];
      if (r > 0) a = cmul(a, tws[j * r * twstep]);
      w[r] = a;
    }
    Dft<R, float2, float>::run(w);
#pragma unroll
    for (int r = 0; r < R; ++r) v[u + NB * r] = w[r];
  }
}

// The first stage (no twiddles) from registers z[q] = x[tl + TPL q], q < E,
// into the line in shared memory; no barrier.  Butterfly j = tl + u TPL takes
// inputs j + r N / R0 = tl + TPL (u + (E / R0) r) and writes j R0 + r.
template <int N, bool PAD>
__device__ __forceinline__ void ct_first_from_regs(const float2* z, float2* line, int es, int tl) {
  constexpr int E = ct_e(N), R0 = ct_radix(N, 0), TPL = N / E, NB = E / R0;
#pragma unroll
  for (int u = 0; u < NB; ++u) {
    float2 w[R0];
#pragma unroll
    for (int r = 0; r < R0; ++r) w[r] = z[u + r * NB];
    Dft<R0, float2, float>::run(w);
    const int j = tl + u * TPL;
#pragma unroll
    for (int r = 0; r < R0; ++r) line[ct_pos<PAD>(j * R0 + r) * es] = w[r];
  }
}

// global -> global.  Every load precedes the first barrier and every store
// follows it, so ld and st may alias.
template <int N, bool PAD = false, class Ld, class St>
__device__ __forceinline__ void ct_line_gg(const Ld& ld, const St& st, float2* line, int es, int tl,
                                           const float2* __restrict__ tws, int twstep) {
  ct_run<N, 0, true, true, PAD>(ld, st, line, es, tl, tws, twstep);
}

// global -> shared (natural order, after a barrier)
template <int N, bool PAD = false, class Ld>
__device__ __forceinline__ void ct_line_gs(const Ld& ld, float2* line, int es, int tl,
                                           const float2* __restrict__ tws, int twstep) {
  ct_run<N, 0, true, false, PAD>(ld, CtNone{}, line, es, tl, tws, twstep);
}

// shared (complete, after a barrier) -> global
template <int N, bool PAD = false, class St>
__device__ __forceinline__ void ct_line_sg(float2* line, const St& st, int es, int tl,
                                           const float2* __restrict__ tws, int twstep) {
  ct_run<N, 0, false, true, PAD>(CtNone{}, st, line, es, tl, tws, twstep);
}

// Copies the n-entry twiddle table to shared memory (all threads; barrier).
__device__ __forceinline__ void ct_load_twiddles(float2* dst, const float2* __restrict__ src, int n) {
  for (int i = threadIdx.x; i < n; i += blockDim.x) dst[i] = __ldg(&src[i]);
  __syncthreads();
}

}  // namespace sr3d

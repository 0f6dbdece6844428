// Compile-time-planned FFT lines for the hot power-of-two lengths (FP32).
//
// Same Stockham formulation as fft.cuh, but the length N, the radices
// ([N / 16^a, 16, ..., 16]), the threads per line (N / 16) and every index
// are compile-time constants, so there are no runtime divisions or
// predicated stage loops, and twiddles come from a shared-memory table.
// A thread owns 16 elements per stage; the first stage loads them straight
// from global memory and the last stage stores straight to global memory.
#pragma once
#include "fft.cuh"

namespace sr3d {

constexpr int ct_rem(int n) { return n % 16 == 0 ? ct_rem(n / 16) : n; }
constexpr int ct_big(int n) { return n % 16 == 0 ? 1 + ct_big(n / 16) : 0; }
constexpr int ct_nst(int n) { return ct_big(n) + (ct_rem(n) > 1 ? 1 : 0); }
// radix of stage i
constexpr int ct_radix(int n, int i) { return (ct_rem(n) > 1 && i == 0) ? ct_rem(n) : 16; }
// product of the radices before stage i
constexpr int ct_ns(int n, int i) { return i == 0 ? 1 : ct_ns(n, i - 1) * ct_radix(n, i - 1); }

template <int N> __host__ __device__ constexpr bool ct_supported() {
  return N == 32 || N == 64 || N == 128 || N == 256 || N == 512;
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
  constexpr int R = ct_radix(N, I);
  constexpr int NS = ct_ns(N, I);
  constexpr int TPL = N / 16;
  constexpr int NB = 16 / R;
  constexpr int NR = N / R;
  constexpr int STEP = N / (NS * R);
  float2 v[16];
#pragma unroll
  for (int u = 0; u < NB; ++u) {
    const int j = tl + u * TPL;
    const int jm = j & (NS - 1);
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
    const int jm = j & (NS - 1);
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

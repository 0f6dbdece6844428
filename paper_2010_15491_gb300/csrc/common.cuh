// Shared device helpers: complex arithmetic on float2 / double2 and the
// small descriptors that every pass kernel takes by value.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace sr3d {

template <typename T> struct CplxOf;
template <> struct CplxOf<float> { using type = float2; };
template <> struct CplxOf<double> { using type = double2; };
template <typename T> using cplx = typename CplxOf<T>::type;

__host__ __device__ __forceinline__ float2 mkc(float a, float b) { return make_float2(a, b); }
__host__ __device__ __forceinline__ double2 mkc(double a, double b) { return make_double2(a, b); }

#define SR3D_COPS(C, R)                                                                                  \
  __device__ __forceinline__ C operator+(C a, C b) { return mkc(a.x + b.x, a.y + b.y); }                 \
  __device__ __forceinline__ C operator-(C a, C b) { return mkc(a.x - b.x, a.y - b.y); }                 \
  __device__ __forceinline__ C operator*(C a, R s) { return mkc(a.x * s, a.y * s); }                     \
  __device__ __forceinline__ C cmul(C a, C b) { return mkc(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); } \
  /* conj(a) * b */                                                                                      \
  __device__ __forceinline__ C cmulc(C a, C b) { return mkc(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x); } \
  __device__ __forceinline__ C conjc(C a) { return mkc(a.x, -a.y); }                                     \
  __device__ __forceinline__ C mul_i(C a) { return mkc(-a.y, a.x); }                                     \
  __device__ __forceinline__ C mul_mi(C a) { return mkc(a.y, -a.x); }                                    \
  __device__ __forceinline__ R norm2(C a) { return a.x * a.x + a.y * a.y; }

SR3D_COPS(float2, float)
SR3D_COPS(double2, double)
#undef SR3D_COPS

template <typename C> __device__ __forceinline__ C czero() { C c; c.x = 0; c.y = 0; return c; }

// Largest elements-per-thread of the FFT engine (register budget): powers of
// two use up to 16 (float) / 8 (double) per thread, the 3 * 2^a family 12.
template <typename T> struct Emax {
  static constexpr int p2 = sizeof(T) == 4 ? 16 : 8;
  static constexpr int p3 = 12;
};

// One FFT axis: line length n, elements per thread e (n / e threads per
// line), and the radix of each Stockham stage (product = n).
struct FftAxis {
  int n;
  int e;
  int nst;
  int radix[8];
};

// m axis of a spectral array: real length M, packed half length H = M/2,
// aliasing group size dr, LR length Ml = M/dr, slots Ms, pitch Mp (complex).
// Slot (g, p) = g*dr + p holds HR frequency g + p*Ml, g in [0, Ml/2].
struct MAxis {
  int M, H, Ml, dr, Ms, Mp;
  FftAxis f;  // transform of length H
};

// n (or s) axis: length N, aliasing group size dc, LR length Nl.
struct LAxis {
  int N, Nl, dc;
  FftAxis f;
};

// Location of m-frequency k (0 <= k < M) in the slot layout: the slot and
// whether the stored value must be conjugated (the value at M - k).  Along a
// line of spatial (n, s) that is the whole story; in the 3D spectrum the
// conjugate partner also has negated n and s frequencies.
__device__ __forceinline__ int mslot_of(int k, int M, int Ml, int dr, bool& cj) {
  int r = k % Ml, p = k / Ml;
  if (2 * r <= Ml) { cj = false; return r * dr + p; }
  int k2 = M - k;
  cj = true;
  return (Ml - r) * dr + k2 / Ml;
}

}  // namespace sr3d

// Batched 1D FFT engine in shared memory.
//
// A CTA transforms several lines at once.  Each line of length n is owned by
// tpl = n / e threads; every Stockham stage (self-sorting, decimation in
// time) loads e elements per thread into registers, applies the twiddles,
// barriers, runs e / R radix-R butterflies and stores back in place, so the
// shared footprint is one tile.  The first stage reads its inputs straight
// from global memory (all e loads of a thread in flight at once) and the last
// stage writes straight to global memory, so a two-stage length such as
// 256 = 16 x 16 crosses shared memory once.  Radices 2, 3, 4, 8 and 16 cover
// every length 2^a and 3 * 2^a (radix 6 serves the compile-time plans of
// fft_ct.cuh).  The transform is the unnormalised forward DFT
// X[k] = sum_j x[j] exp(-2 pi i j k / n); inverses conjugate on the way in
// and out.  Butterfly constants are the exact values cos(2 pi j / 16),
// sin(2 pi j / 16) and sqrt(3)/2 written as decimal literals.
#pragma once
#include <type_traits>

#include "common.cuh"

namespace sr3d {

template <int R, typename C, typename T> struct Dft;

template <typename C, typename T> struct Dft<2, C, T> {
  __device__ __forceinline__ static void run(C* v) {
    C a = v[0];
    v[0] = a + v[1];
    v[1] = a - v[1];
  }
};

template <typename C, typename T> struct Dft<3, C, T> {
  __device__ __forceinline__ static void run(C* v) {
    const T k = (T)0.86602540378443864676;  // sqrt(3)/2
    C s = v[1] + v[2];
    C t = v[0] - s * (T)0.5;
    C u = mul_mi(v[1] - v[2]) * k;
    v[0] = v[0] + s;
    v[1] = t + u;
    v[2] = t - u;
  }
};

template <typename C, typename T> struct Dft<4, C, T> {
  __device__ __forceinline__ static void run(C* v) {
    C a0 = v[0] + v[2], a1 = v[0] - v[2];
    C a2 = v[1] + v[3], a3 = mul_mi(v[1] - v[3]);
    v[0] = a0 + a2;
    v[2] = a0 - a2;
    v[1] = a1 + a3;
    v[3] = a1 - a3;
  }
};

// 6 = 2 x 3: length-3 transforms of the even and odd inputs, the odd ones
// turned by exp(-2 pi i k / 6), then X[k] = A[k] + B[k], X[k + 3] = A[k] - B[k].
template <typename C, typename T> struct Dft<6, C, T> {
  __device__ __forceinline__ static void run(C* v) {
    const T k = (T)0.86602540378443864676;  // sqrt(3)/2
    C a[3] = {v[0], v[2], v[4]};
    C b[3] = {v[1], v[3], v[5]};
    Dft<3, C, T>::run(a);
    Dft<3, C, T>::run(b);
    const C b1 = mkc((T)0.5 * b[1].x + k * b[1].y, (T)0.5 * b[1].y - k * b[1].x);    // * exp(-i pi/3)
    const C b2 = mkc((T)-0.5 * b[2].x + k * b[2].y, (T)-0.5 * b[2].y - k * b[2].x);  // * exp(-2 i pi/3)
    v[0] = a[0] + b[0];
    v[3] = a[0] - b[0];
    v[1] = a[1] + b1;
    v[4] = a[1] - b1;
    v[2] = a[2] + b2;
    v[5] = a[2] - b2;
  }
};

template <typename C, typename T> struct Dft<8, C, T> {
  __device__ __forceinline__ static void run(C* v) {
    const T h = (T)0.70710678118654752440;  // cos(pi/4)
    C e[4] = {v[0], v[2], v[4], v[6]};
    C o[4] = {v[1], v[3], v[5], v[7]};
    Dft<4, C, T>::run(e);
    Dft<4, C, T>::run(o);
    C o1 = mkc(h * (o[1].x + o[1].y), h * (o[1].y - o[1].x));    // * exp(-i pi/4)
    C o2 = mul_mi(o[2]);                                          // * exp(-i pi/2)
    C o3 = mkc(h * (o[3].y - o[3].x), -h * (o[3].x + o[3].y));   // * exp(-3 i pi/4)
    v[0] = e[0] + o[0];
    v[4] = e[0] - o[0];
    v[1] = e[1] + o1;
    v[5] = e[1] - o1;
    v[2] = e[2] + o2;
    v[6] = e[2] - o2;
    v[3] = e[3] + o3;
    v[7] = e[3] - o3;
  }
};

// x * exp(-2 pi i j / 16) for the j = n2 * k1 products of a 4 x 4 split.
template <typename C, typename T> __device__ __forceinline__ C tw16(C a, int j) {
  const T c1 = (T)0.92387953251128675613;  // cos(pi/8)
  const T s1 = (T)0.38268343236508977173;  // sin(pi/8)
  const T h = (T)0.70710678118654752440;
  switch (j) {
    case 1: return cmul(a, mkc(c1, -s1));
    case 2: return cmul(a, mkc(h, -h));
    case 3: return cmul(a, mkc(s1, -c1));
    case 4: return mul_mi(a);
    case 6: return cmul(a, mkc(-h, -h));
    case 9: return cmul(a, mkc(-c1, s1));
    default: return a;  // j == 0
  }
}

template <typename C, typename T> struct Dft<16, C, T> {
  __device__ __forceinline__ static void run(C* v) {
    // n = 4 n1 + n2, k = k1 + 4 k2
    C a[4][4];
#pragma unroll
    for (int n2 = 0; n2 < 4; ++n2) {
      C t[4] = {v[n2], v[4 + n2], v[8 + n2], v[12 + n2]};
      Dft<4, C, T>::run(t);
#pragma unroll
      for (int k1 = 0; k1 < 4; ++k1) a[n2][k1] = tw16<C, T>(t[k1], n2 * k1);
    }
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1) {
      C t[4] = {a[0][k1], a[1][k1], a[2][k1], a[3][k1]};
      Dft<4, C, T>::run(t);
#pragma unroll
      for (int k2 = 0; k2 < 4; ++k2) v[k1 + 4 * k2] = t[k2];
    }
  }
};

// One Stockham stage of radix R over the line `line` (element stride es in
// shared memory).  Ns = product of the radices already applied.  Thread tl of
// the line's tpl threads handles butterflies j = tl + u * tpl, u < nb.
// tw[q * tws] = exp(-2 pi i q / n).
template <typename T, int R, int EMAX>
__device__ __forceinline__ void fft_stage(cplx<T>* line, int es, int n, int Ns, int tl, int tpl, int nb,
                                          const cplx<T>* __restrict__ tw, int tws) {
  using C = cplx<T>;
  constexpr int NBMAX = EMAX / R;
  C v[NBMAX * R];
  const int nr = n / R;
  const int step = (n / (Ns * R)) * tws;
#pragma unroll
  for (int u = 0; u < NBMAX; ++u) {
    if (u < nb) {
      const int j = tl + u * tpl;
      const int jm = j % Ns;
#pragma unroll
      for (int r = 0; r < R; ++r) {
        C a = line[(j + r * nr) * es];
        if (r > 0 && Ns > 1) a = cmul(a, __ldg(&tw[jm * r * step]));
        v[u * R + r] = a;
      }
    }
  }
  __syncthreads();
#pragma unroll
  for (int u = 0; u < NBMAX; ++u) {
    if (u < nb) {
      Dft<R, C, T>::run(&v[u * R]);
      const int j = tl + u * tpl;
      const int jm = j % Ns;
      const int base = (j - jm) * R + jm;
#pragma unroll
      for (int r = 0; r < R; ++r) line[(base + r * Ns) * es] = v[u * R + r];
    }
  }
  __syncthreads();
}

// Calls f(std::integral_constant<int, R>) for the runtime radix R.
template <int EMAX, class F> __device__ __forceinline__ void with_radix(int R, F&& f) {
  if (R == 2) {
    f(std::integral_constant<int, 2>{});
  } else if (R == 4) {
    if constexpr (EMAX % 4 == 0) f(std::integral_constant<int, 4>{});
  } else if (R == 8) {
    if constexpr (EMAX % 8 == 0) f(std::integral_constant<int, 8>{});
  } else if (R == 16) {
    if constexpr (EMAX % 16 == 0) f(std::integral_constant<int, 16>{});
  } else if (R == 3) {
    if constexpr (EMAX % 3 == 0) f(std::integral_constant<int, 3>{});
  }
}

// Radices after the first stage.  Power-of-two lengths are planned as
// [remainder, P, P, ...] with P = EMAX (16 for float, 8 for double), so only
// the first stage needs the small radices; this keeps the inlined stage
// variants, and with them register pressure, down.
template <int EMAX, class F> __device__ __forceinline__ void with_radix_tail(int R, F&& f) {
  if constexpr (EMAX == 16 || EMAX == 8) {
    if (R == EMAX) f(std::integral_constant<int, EMAX>{});
  } else {
    with_radix<EMAX>(R, f);
  }
}

// First stage (no twiddles): ld(i) gives element i of the line; results go
// to shared memory.  No barrier inside: the caller syncs afterwards.
template <typename T, int R, int EMAX, class Ld>
__device__ __forceinline__ void stage_first_to_smem(const Ld& ld, cplx<T>* line, int es, int n, int tl, int tpl,
                                                    int nb) {
  using C = cplx<T>;
  constexpr int NBMAX = EMAX / R;
  C v[NBMAX * R];
  const int nr = n / R;
#pragma unroll
  for (int u = 0; u < NBMAX; ++u)
    if (u < nb) {
      const int j = tl + u * tpl;
#pragma unroll
      for (int r = 0; r < R; ++r) v[u * R + r] = ld(j + r * nr);
    }
#pragma unroll
  for (int u = 0; u < NBMAX; ++u)
    if (u < nb) {
      Dft<R, C, T>::run(&v[u * R]);
      const int j = tl + u * tpl;
#pragma unroll
      for (int r = 0; r < R; ++r) line[(j * R + r) * es] = v[u * R + r];
    }
}

// Last stage: reads shared memory (twiddled), st(i, v) stores output element i.
template <typename T, int R, int EMAX, class St>
__device__ __forceinline__ void stage_last_to_global(const cplx<T>* line, int es, const St& st, int n, int Ns,
                                                     int tl, int tpl, int nb, const cplx<T>* __restrict__ tw,
                                                     int tws) {
  using C = cplx<T>;
  constexpr int NBMAX = EMAX / R;
  C v[NBMAX * R];
  const int nr = n / R;
  const int step = (n / (Ns * R)) * tws;
#pragma unroll
  for (int u = 0; u < NBMAX; ++u)
    if (u < nb) {
      const int j = tl + u * tpl;
      const int jm = j % Ns;
#pragma unroll
      for (int r = 0; r < R; ++r) {
        C a = line[(j + r * nr) * es];
        if (r > 0 && Ns > 1) a = cmul(a, __ldg(&tw[jm * r * step]));
        v[u * R + r] = a;
      }
    }
#pragma unroll
  for (int u = 0; u < NBMAX; ++u)
    if (u < nb) {
      Dft<R, C, T>::run(&v[u * R]);
      const int j = tl + u * tpl;
      const int jm = j % Ns;
      const int base = (j - jm) * R + jm;
#pragma unroll
      for (int r = 0; r < R; ++r) st(base + r * Ns, v[u * R + r]);
    }
}

// Single-stage transform from ld to st; one barrier separates every load of
// the CTA from every store, so ld and st may address the same memory.
template <typename T, int R, int EMAX, class Ld, class St>
__device__ __forceinline__ void stage_only(const Ld& ld, const St& st, int n, int tl, int tpl, int nb) {
  using C = cplx<T>;
  constexpr int NBMAX = EMAX / R;
  C v[NBMAX * R];
  const int nr = n / R;
#pragma unroll
  for (int u = 0; u < NBMAX; ++u)
    if (u < nb) {
      const int j = tl + u * tpl;
#pragma unroll
      for (int r = 0; r < R; ++r) v[u * R + r] = ld(j + r * nr);
    }
  __syncthreads();
#pragma unroll
  for (int u = 0; u < NBMAX; ++u)
    if (u < nb) {
      Dft<R, C, T>::run(&v[u * R]);
      const int j = tl + u * tpl;
#pragma unroll
      for (int r = 0; r < R; ++r) st(j * R + r, v[u * R + r]);
    }
}

// Global -> global transform of one line (shared memory as the exchange
// buffer).  Every load of the CTA happens before its first barrier and every
// store after it, so ld and st may address the same global memory.
template <typename T, int EMAX, class Ld, class St>
__device__ __forceinline__ void fft_line_gg(const Ld& ld, const St& st, cplx<T>* line, int es, const FftAxis& ax,
                                            int tl, int tpl, const cplx<T>* __restrict__ tw, int tws) {
  const int nst = ax.nst;
  if (nst == 0) {
    const cplx<T> v = ld(0);
    __syncthreads();
    st(0, v);
    return;
  }
  if (nst == 1) {
    with_radix<EMAX>(ax.radix[0], [&](auto RC) {
      constexpr int R = decltype(RC)::value;
      stage_only<T, R, EMAX>(ld, st, ax.n, tl, tpl, ax.e / R);
    });
    return;
  }
  with_radix<EMAX>(ax.radix[0], [&](auto RC) {
    constexpr int R = decltype(RC)::value;
    stage_first_to_smem<T, R, EMAX>(ld, line, es, ax.n, tl, tpl, ax.e / R);
  });
  __syncthreads();
  int Ns = ax.radix[0];
  for (int s = 1; s < nst - 1; ++s) {
    const int R0 = ax.radix[s];
    with_radix_tail<EMAX>(R0, [&](auto RC) {
      constexpr int R = decltype(RC)::value;
      fft_stage<T, R, EMAX>(line, es, ax.n, Ns, tl, tpl, ax.e / R, tw, tws);
    });
    Ns *= R0;
  }
  with_radix_tail<EMAX>(ax.radix[nst - 1], [&](auto RC) {
    constexpr int R = decltype(RC)::value;
    stage_last_to_global<T, R, EMAX>(line, es, st, ax.n, Ns, tl, tpl, ax.e / R, tw, tws);
  });
}

// Global -> shared: the transformed line ends in natural order in `line`,
// after a barrier.
template <typename T, int EMAX, class Ld>
__device__ __forceinline__ void fft_line_gs(const Ld& ld, cplx<T>* line, int es, const FftAxis& ax, int tl,
                                            int tpl, const cplx<T>* __restrict__ tw, int tws) {
  const int nst = ax.nst;
  if (nst == 0) {
    line[0] = ld(0);
    __syncthreads();
    return;
  }
  with_radix<EMAX>(ax.radix[0], [&](auto RC) {
    constexpr int R = decltype(RC)::value;
    stage_first_to_smem<T, R, EMAX>(ld, line, es, ax.n, tl, tpl, ax.e / R);
  });
  __syncthreads();
  int Ns = ax.radix[0];
  for (int s = 1; s < nst; ++s) {
    const int R0 = ax.radix[s];
    with_radix_tail<EMAX>(R0, [&](auto RC) {
      constexpr int R = decltype(RC)::value;
      fft_stage<T, R, EMAX>(line, es, ax.n, Ns, tl, tpl, ax.e / R, tw, tws);
    });
    Ns *= R0;
  }
}

// Shared -> global: the line in `line` (complete, after a barrier) is
// transformed and written through st.
template <typename T, int EMAX, class St>
__device__ __forceinline__ void fft_line_sg(cplx<T>* line, const St& st, int es, const FftAxis& ax, int tl,
                                            int tpl, const cplx<T>* __restrict__ tw, int tws) {
  const int nst = ax.nst;
  if (nst == 0) {
    st(0, line[0]);
    return;
  }
  int Ns = 1;
  if (nst == 1) {
    with_radix<EMAX>(ax.radix[0], [&](auto RC) {
      constexpr int R = decltype(RC)::value;
      stage_last_to_global<T, R, EMAX>(line, es, st, ax.n, Ns, tl, tpl, ax.e / R, tw, tws);
    });
    return;
  }
  with_radix<EMAX>(ax.radix[0], [&](auto RC) {
    constexpr int R = decltype(RC)::value;
    fft_stage<T, R, EMAX>(line, es, ax.n, Ns, tl, tpl, ax.e / R, tw, tws);
  });
  Ns = ax.radix[0];
  for (int s = 1; s < nst - 1; ++s) {
    const int R0 = ax.radix[s];
    with_radix_tail<EMAX>(R0, [&](auto RC) {
      constexpr int R = decltype(RC)::value;
      fft_stage<T, R, EMAX>(line, es, ax.n, Ns, tl, tpl, ax.e / R, tw, tws);
    });
    Ns *= R0;
  }
  with_radix_tail<EMAX>(ax.radix[nst - 1], [&](auto RC) {
    constexpr int R = decltype(RC)::value;
    stage_last_to_global<T, R, EMAX>(line, es, st, ax.n, Ns, tl, tpl, ax.e / R, tw, tws);
  });
}

}  // namespace sr3d

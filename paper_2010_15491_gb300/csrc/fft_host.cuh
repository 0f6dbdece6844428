// Host-side helpers shared by the FFT-pass translation units.
#pragma once
#include "internal.h"

namespace sr3d {

// ---------------------------------------------------------------------------
// host launchers
// ---------------------------------------------------------------------------
// Opts a kernel in to more than 48 KB of dynamic shared memory.  The kernels
// launched through it declare no static shared memory, so bytes is their
// whole footprint.
template <typename K> static inline cudaError_t allow_smem(K kernel, size_t bytes) {
  if (bytes <= 48 * 1024) return cudaSuccess;
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

static inline MAxis maxis(const Geometry& g) {
  MAxis a;
  a.M = g.M; a.H = g.M / 2; a.Ml = g.Ml; a.dr = g.dr; a.Ms = g.Ms; a.Mp = g.Mp; a.f = g.fm;
  return a;
}

static inline LAxis laxis(int n, int nl, int dc, const FftAxis& f) {
  LAxis a;
  a.N = n; a.Nl = nl; a.dc = dc; a.f = f;
  return a;
}

static inline bool fam3(const FftAxis& f) { return f.n % 3 == 0; }

// Lines per CTA of the m passes: at most 256 threads (tpl per line); L_req > 0
// (a schedule choice, checked by m_lines_valid) takes fewer lines.
static inline void m_launch_shape(const Geometry& g, size_t csz, int L_req, int& L, int& Hp, int& threads,
                                  size_t& smem) {
  const int H = g.M / 2;
  const int tpl = H / g.fm.e;
  L = tpl >= 256 ? 1 : 256 / tpl;
  if (L_req > 0 && L_req < L) L = L_req;
  Hp = H + (H >= 32 ? (int)(64 / csz) : 0);
  threads = L * tpl;
  smem = (size_t)L * Hp * csz;
}

// A lines-per-CTA value the m-pass kernels take: at most the default, and
// whole warps (the forward pass strides its stores over the CTA's warps).
static inline bool m_lines_valid(const Geometry& g, int L) {
  const int tpl = (g.M / 2) / g.fm.e;
  const int lmax = tpl >= 256 ? 1 : 256 / tpl;
  return L >= 1 && L <= lmax && (L * tpl) % 32 == 0;
}

// lengths with a compile-time plan (FP32 only): 2^a with 16 elements per
// thread, 3 * 2^a with 12, as the runtime plan of the axis has them
template <typename T> static inline int ct_len(int n, const FftAxis& f) {
  if (sizeof(T) != 4) return 0;
  if (f.e == 16) return (n == 32 || n == 64 || n == 128 || n == 256 || n == 512) ? n : 0;
  if (f.e == 12) return (n == 48 || n == 96 || n == 192) ? n : 0;
  return 0;
}

}  // namespace sr3d

// Learned warm start: a 3D U-Net (channels 16 / 32 / 64, 3x3x3 convolutions,
// 2x2x2 max pooling, nearest upsampling, skip concatenation, ReLU, residual
// 1x1x1 head) trained and run with the library's own kernels, plus the
// KKT-consistent initial dual for ADMM started from its output.
//
// Activations and gradients are BF16, channels last ([voxel][channel]);
// master weights, Adam moments and reductions are FP32 / FP64.  Every 3x3x3
// convolution with 16-multiple input channels is an implicit GEMM on the
// tensor cores: rows are voxels, columns output channels, the reduction runs
// over (tap, input channel).  Two kernels compute it: k_conv3 (mma.sync
// m16n8k16 BF16, FP32 accumulation; input brick + halo in shared memory, taps
// read by ldmatrix) and k_conv3_tc (tcgen05.mma with TMEM accumulators, a
// persistent CTA per row marching over s), chosen per layer shape.  The data
// gradient is the same convolution with flipped, transposed weights; the
// weight gradient is a third GEMM (channels x k over voxels) split over voxel
// groups.  The first layer (one input channel) is a plain FP32 stencil.
#include <cuda_bf16.h>
#include <stdio.h>
#include <string.h>

#include <cmath>
#include <string>
#include <vector>

#include "internal.h"
#include "sr3d.h"

namespace sr3d {

typedef __nv_bfloat16 bf16;

struct ConvIn {
  const bf16* src0;  // first source, c0 channels; up0: stored at half size (nearest upsampling)
  const bf16* src1;  // second source at full size, c1 channels (c1 = 0: none)
  int c0, c1, up0;
  int M, N, S;       // full (output) size
};

__device__ __forceinline__ bool vox_of(long long v, const ConvIn& in, int& s, int& n, int& m) {
  const long long P = (long long)in.M * in.N;
  if (v >= P * in.S) return false;
  s = (int)(v / P);
  const long long r = v - (long long)s * P;
  n = (int)(r / in.M);
  m = (int)(r - (long long)n * in.M);
  return true;
}

// 8 consecutive input channels [ci0, ci0+8) at voxel (s, n, m) (zero outside)
__device__ __forceinline__ uint4 load8(const ConvIn& in, int s, int n, int m, int ci0) {
  if (s < 0 || s >= in.S || n < 0 || n >= in.N || m < 0 || m >= in.M) return make_uint4(0, 0, 0, 0);
  const bf16* p;
  if (ci0 < in.c0) {
    long long idx;
    if (in.up0) idx = ((long long)(s >> 1) * (in.N >> 1) + (n >> 1)) * (in.M >> 1) + (m >> 1);
    else idx = ((long long)s * in.N + n) * in.M + m;
    p = in.src0 + idx * in.c0 + ci0;
  } else {
    p = in.src1 + (((long long)s * in.N + n) * in.M + m) * in.c1 + (ci0 - in.c0);
  }
  return __ldg(reinterpret_cast<const uint4*>(p));
}

__device__ __forceinline__ bf16 load1(const ConvIn& in, int s, int n, int m) {
  if (s < 0 || s >= in.S || n < 0 || n >= in.N || m < 0 || m >= in.M) return __float2bfloat16(0.f);
  return in.src0[((long long)s * in.N + n) * in.M + m];
}

// Fills a warp's 16 x 16 slab: rows = voxels v0..v0+15, columns = k in
// [16 kc, 16 kc + 16) of the im2col matrix (k = tap * Cin + ci; with PACKED,
// Cin = 1 and k = tap).
template <bool PACKED>
__device__ __forceinline__ void fill_slab(bf16* slab, const ConvIn& in, long long v0, int kc, int Cin, int lane) {
  if constexpr (!PACKED) {
    const int vi = lane >> 1, h = lane & 1;
    const int k0 = kc * 16;
    const int tap = k0 / Cin, ci0 = k0 - tap * Cin;
    const int ds = tap / 9 - 1, dn = (tap / 3) % 3 - 1, dm = tap % 3 - 1;
    int s, n, m;
    uint4 val = make_uint4(0, 0, 0, 0);
    if (tap < 27 && vox_of(v0 + vi, in, s, n, m)) val = load8(in, s + ds, n + dn, m + dm, ci0 + 8 * h);
    reinterpret_cast<uint4*>(slab + vi * 16)[h] = val;
  } else {
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      const int idx = lane * 8 + e, vi = idx >> 4, j = idx & 15;
      const int tap = kc * 16 + j;
      bf16 val = __float2bfloat16(0.f);
      int s, n, m;
      if (tap < 27 && vox_of(v0 + vi, in, s, n, m)) val = load1(in, s + tap / 9 - 1, n + (tap / 3) % 3 - 1, m + tap % 3 - 1);
      slab[idx] = val;
    }
  }
}

__device__ __forceinline__ void ldsm_x4(uint32_t* r, const bf16* p) {
  const unsigned a = (unsigned)__cvta_generic_to_shared(p);
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(a));
}
__device__ __forceinline__ void ldsm_x4_t(uint32_t* r, const bf16* p) {
  const unsigned a = (unsigned)__cvta_generic_to_shared(p);
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(a));
}
__device__ __forceinline__ void mma16816(float* d, const uint32_t* a, uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// ---------------------------------------------------------------------------
// first layer (one input channel, 16 outputs) as an implicit GEMM on the
// tensor cores: rows = 16 voxels along m, K = the 27 taps (padded to 32, two
// m16n8k16 chunks), N = the 16 output channels.  A 128 x 8 tile of voxels
// per CTA marches over s with a ring of three BF16 x planes (with halo) in
// shared memory; each warp owns one row of 128 voxels, and each lane gathers
// the tap values of its A fragment (voxel rows g, g+8; taps 2t, 2t+1, 2t+8,
// 2t+9 of each chunk) straight from the ring.  The weights are rounded to
// BF16 once per CTA into the lanes' B fragments, as the other layers' are;
// accumulation in FP32.  The next plane is fetched into registers during the
// step's MMAs.
// ---------------------------------------------------------------------------
constexpr int F_TM = 32, F_TN = 8, F_TS = 8, F_VM = 4;  // 128 x 8 voxels per CTA (256 threads), planes per CTA
__global__ void __launch_bounds__(F_TM * F_TN, 2) k_conv_first(const bf16* __restrict__ x, const float* __restrict__ W,
                                                            const float* __restrict__ bias, bf16* __restrict__ out,
                                                            int M, int N, int S) {
  constexpr int TMV = F_TM * F_VM;                // voxels along m per row
  constexpr int HM = TMV + 2, HW = HM + 6, HH = F_TN + 2;  // halo row m0-1 .. m0+128 (padded)
  __shared__ __align__(16) bf16 xs[3][HH * HW];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int g = lane >> 2, t = lane & 3;
  const int m0 = blockIdx.x * TMV, n0 = blockIdx.y * F_TN, s0 = blockIdx.z * F_TS;
  const int s_end = min(S, s0 + F_TS);
  // B fragments: chunk c, n8 tile j: (b0, b1) = W[8j + g][16c + 2t (+1)], W[8j + g][16c + 2t + 8 (+9)]
  uint32_t bw[2][2][2];
  auto wv = [&](int co, int tap) -> float { return tap < 27 ? W[co * 27 + tap] : 0.f; };
  auto pk = [](float a, float b) -> uint32_t {
    const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<const uint32_t*>(&h);
  };
#pragma unroll
  for (int c = 0; c < 2; ++c)
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      const int co = 8 * j + g, k0 = 16 * c + 2 * t;
      bw[c][j][0] = pk(wv(co, k0), wv(co, k0 + 1));
      bw[c][j][1] = pk(wv(co, k0 + 8), wv(co, k0 + 9));
    }
  const float b_lo0 = bias[2 * t], b_lo1 = bias[2 * t + 1], b_hi0 = bias[8 + 2 * t], b_hi1 = bias[9 + 2 * t];
  // the lane's taps: k = 16c + 2t + {0, 1, 8, 9}; offset of tap k from the voxel's
  // (ring row, halo column) and its plane (0..2); taps 27..31 are padding
  int toff[2][4], tpl[2][4];
  bool tok[2][4];
#pragma unroll
  for (int c = 0; c < 2; ++c)
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int k = 16 * c + 2 * t + (q & 1) + 8 * (q >> 1);
      tok[c][q] = k < 27;
      const int kk = k < 27 ? k : 0;
      toff[c][q] = ((kk / 3) % 3) * HW + kk % 3;
      tpl[c][q] = kk / 9;
    }
  // a plane's halo tile is fetched into registers (FP values per thread) one
  // step ahead and stored to its ring slot after the step's MMAs
  constexpr int FP = (HH * HW + F_TM * F_TN - 1) / (F_TM * F_TN);
  bf16 pre[FP];
  auto fetch_plane = [&](int ps) {
#pragma unroll
    for (int k = 0; k < FP; ++k) {
      const int i = tid + k * F_TM * F_TN;
      const int hn = i / HW, hm = i - hn * HW, m = m0 - 1 + hm, n = n0 - 1 + hn;
      bf16 v = __float2bfloat16(0.f);
      if (i < HH * HW && hm < HM && ps >= 0 && ps < S && n >= 0 && n < N && m >= 0 && m < M)
        v = x[((long long)ps * N + n) * M + m];
      pre[k] = v;
    }
  };
  auto store_plane = [&](bf16* buf) {
#pragma unroll
    for (int k = 0; k < FP; ++k) {
      const int i = tid + k * F_TM * F_TN;
      if (i < HH * HW) buf[i] = pre[k];
    }
  };
  fetch_plane(s0 - 1);
  store_plane(xs[0]);
  fetch_plane(s0);
  store_plane(xs[1]);
  fetch_plane(s0 + 1);
  store_plane(xs[2]);
  const int n = n0 + warp;
  int r0 = 0;  // ring slot of plane s-1; s in r0+1, s+1 in r0+2 (mod 3)
  for (int s = s0; s < s_end; ++s) {
    __syncthreads();  // plane s+1 is stored (in the slot that held plane s-2)
    if (s + 2 < s_end + 1) fetch_plane(s + 2);
    // the lane's eight tap pointers for this step (plane of the ring + offset)
    const bf16* tb[2][4];
#pragma unroll
    for (int c = 0; c < 2; ++c)
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int pl = tpl[c][q];
        tb[c][q] = (pl == 0 ? xs[r0] : pl == 1 ? xs[(r0 + 1) % 3] : xs[(r0 + 2) % 3]) + toff[c][q];
      }
#pragma unroll 2
    for (int tile = 0; tile < TMV / 16; ++tile) {
      const int rb = warp * HW + tile * 16;  // ring row warp (voxel row n - 1 + dn with dn = 0), column of voxel 0 - 1
      float acc[2][4] = {{0.f, 0.f, 0.f, 0.f}, {0.f, 0.f, 0.f, 0.f}};
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        uint32_t a[4];
#pragma unroll
        for (int h = 0; h < 2; ++h) {  // a[0], a[1]: rows g, g+8 of taps 2t, 2t+1; a[2], a[3]: taps 2t+8, 2t+9
#pragma unroll
          for (int r = 0; r < 2; ++r) {
            const int row = rb + g + 8 * r;
            const int q0 = 2 * h, q1 = 2 * h + 1;
            const bf16 v0 = tok[c][q0] ? tb[c][q0][row] : __float2bfloat16(0.f);
            const bf16 v1 = tok[c][q1] ? tb[c][q1][row] : __float2bfloat16(0.f);
            __nv_bfloat162 pr;
            pr.x = v0;
            pr.y = v1;
            a[2 * h + r] = *reinterpret_cast<const uint32_t*>(&pr);
          }
        }
        mma16816(acc[0], a, bw[c][0][0], bw[c][0][1]);
        mma16816(acc[1], a, bw[c][1][0], bw[c][1][1]);
      }
      if (n < N) {
#pragma unroll
        for (int r = 0; r < 2; ++r) {
          const int m = m0 + tile * 16 + g + 8 * r;
          if (m < M) {
            bf16* o = out + (((long long)s * N + n) * M + m) * 16;
            *reinterpret_cast<uint32_t*>(o + 2 * t) =
                pk(fmaxf(acc[0][2 * r] + b_lo0, 0.f), fmaxf(acc[0][2 * r + 1] + b_lo1, 0.f));
            *reinterpret_cast<uint32_t*>(o + 8 + 2 * t) =
                pk(fmaxf(acc[1][2 * r] + b_hi0, 0.f), fmaxf(acc[1][2 * r + 1] + b_hi1, 0.f));
          }
        }
      }
    }
    __syncthreads();  // every warp is done with plane s-1's slot
    if (s + 2 < s_end + 1) store_plane(xs[r0]);  // plane s+2 into the slot of plane s-1
    r0 = (r0 + 1) % 3;
  }
}

// ---------------------------------------------------------------------------
// halo-tiled convolution for 16-multiple channel counts (forward and data
// gradient).  A CTA computes a 16 (m) x 4 (n) x 2*MT (s) brick of output
// voxels, 8 warps each owning MT rows of 16 voxels along m.  The input brick
// plus its one-voxel halo is copied once into shared memory (one padded row of
// CIN channels per voxel); the 27 taps then read their shifted A rows straight
// from it with ldmatrix (each lane addresses its own voxel row, so the im2col
// is implicit), while the next tap's weight slice streams in with cp.async.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void cpz16(void* dst, const void* src, bool valid) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  const int n = valid ? 16 : 0;  // 0 source bytes: the 16 bytes are zero-filled
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(d), "l"(src), "r"(n) : "memory");
}
__device__ __forceinline__ void cp_commit_() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait_() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

template <int CIN, int COUT, int MT, int UPC = 0>
struct Conv3Cfg {
  static constexpr int TM = 16, TN = 4, TS = 2 * MT;
  static constexpr int HM = TM + 2, HN = TN + 2, HS = TS + 2;
  static constexpr int HV = HM * HN * HS;
  static constexpr int CH = CIN / 8;           // 16-byte chunks per voxel row
  static constexpr int VST = CIN * 2 + 16;     // padded row: an odd number of chunks, conflict-free ldmatrix
  // UPC > 0: the first UPC input channels are a nearest-upsampled source; its
  // brick (with halo) is kept at the source's own half resolution, and the
  // full-resolution brick holds the other CIN - UPC channels
  static constexpr int CF = CIN - UPC;
  static constexpr int VSTF = CF * 2 + 16;
  static constexpr int HMH = TM / 2 + 2, HNH = TN / 2 + 2, HSH = TS / 2 + 2;
  static constexpr int HVH = UPC > 0 ? HMH * HNH * HSH : 0;
  static constexpr int VSTU = UPC * 2 + 16;
  static constexpr int HALO = HV * VSTF + HVH * VSTU;
  static constexpr int WBYTES = COUT * VST;    // one tap's weights, rows n (out), CIN wide
  static constexpr int SMEM = HALO + 2 * WBYTES;
};

// address of channels [c, c+8) of the (concatenated, possibly upsampled) input at an in-range voxel
__device__ __forceinline__ const bf16* chunk_ptr(const ConvIn& in, int s, int n, int m, int c) {
  if (c < in.c0) {
    long long idx;
    if (in.up0) idx = ((long long)(s >> 1) * (in.N >> 1) + (n >> 1)) * (in.M >> 1) + (m >> 1);
    else idx = ((long long)s * in.N + n) * in.M + m;
    return in.src0 + idx * in.c0 + c;
  }
  return in.src1 + (((long long)s * in.N + n) * in.M + m) * in.c1 + (c - in.c0);
}

template <int CIN, int COUT, int MT>
__device__ __forceinline__ void conv3_load_w(unsigned char* dst, const bf16* __restrict__ wt, int tap) {
  using C = Conv3Cfg<CIN, COUT, MT>;
  const bf16* src = wt + (long long)tap * COUT * CIN;
  for (int i = threadIdx.x; i < COUT * C::CH; i += 256) {
    const int n = i / C::CH, c = i - n * C::CH;
    cpz16(dst + n * C::VST + c * 16, src + n * CIN + c * 8, true);
  }
}

// wt: [27][COUT][CIN] BF16 (tap-major slices, rows = output channel).  With
// UPC > 0 the input is (nearest-upsampled src0 with UPC channels, src1) and
// M, N, S are even: the upsampled channels are read from their half-resolution
// brick, each lane addressing the source voxel of its own voxel row, so the
// products and their order are those of the plain kernel.
template <int CIN, int COUT, int MT, int UPC = 0>
__global__ void __launch_bounds__(256) k_conv3(ConvIn in, const bf16* __restrict__ wt, const float* __restrict__ bias,
                                               int relu, bf16* __restrict__ out) {
  using C = Conv3Cfg<CIN, COUT, MT, UPC>;
  extern __shared__ __align__(16) unsigned char smem[];
  unsigned char* halo = smem;                    // full resolution, channels UPC .. CIN-1
  unsigned char* uhalo = smem + C::HV * C::VSTF;  // UPC > 0: the upsampled source at its resolution
  unsigned char* wbuf = smem + C::HALO;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int g = lane >> 2, t = lane & 3;
  const int tilesM = (in.M + C::TM - 1) / C::TM, tilesN = (in.N + C::TN - 1) / C::TN;
  int b = blockIdx.x;
  const int m0 = (b % tilesM) * C::TM;
  b /= tilesM;
  const int n0 = (b % tilesN) * C::TN;
  const int s0 = (b / tilesN) * C::TS;

  constexpr int CHF = C::CF / 8;
  for (int i = threadIdx.x; i < C::HV * CHF; i += 256) {
    const int hv = i / CHF, c = i - hv * CHF;
    const int hm = hv % C::HM, r = hv / C::HM;
    const int m = m0 + hm - 1, n = n0 + r % C::HN - 1, s = s0 + r / C::HN - 1;
    const bool ok = m >= 0 && m < in.M && n >= 0 && n < in.N && s >= 0 && s < in.S;
    cpz16(halo + hv * C::VSTF + c * 16, ok ? chunk_ptr(in, s, n, m, UPC + c * 8) : in.src0, ok);
  }
  if constexpr (UPC > 0) {
    // source voxels (m0/2 - 1 ..) x (n0/2 - 1 ..) x (s0/2 - 1 ..); zero outside
    constexpr int CHU = UPC / 8;
    const int Mh = in.M >> 1, Nh = in.N >> 1, Sh = in.S >> 1;
    const int mh0 = (m0 >> 1) - 1, nh0 = (n0 >> 1) - 1, sh0 = (s0 >> 1) - 1;
    for (int i = threadIdx.x; i < C::HVH * CHU; i += 256) {
      const int hv = i / CHU, c = i - hv * CHU;
      const int hm = hv % C::HMH, r = hv / C::HMH;
      const int mh = mh0 + hm, nh = nh0 + r % C::HNH, sh = sh0 + r / C::HNH;
      const bool ok = mh >= 0 && mh < Mh && nh >= 0 && nh < Nh && sh >= 0 && sh < Sh;
      cpz16(uhalo + hv * C::VSTU + c * 16, ok ? in.src0 + (((long long)sh * Nh + nh) * Mh + mh) * in.c0 + c * 8 : in.src0,
            ok);
    }
  }
  conv3_load_w<CIN, COUT, MT>(wbuf, wt, 0);
  cp_commit_();

  float acc[MT][COUT / 8][4];
#pragma unroll
  for (int i = 0; i < MT; ++i)
#pragma unroll
    for (int j = 0; j < COUT / 8; ++j)
#pragma unroll
      for (int e = 0; e < 4; ++e) acc[i][j][e] = 0.f;

  const int lr = (lane & 7) + 8 * ((lane >> 3) & 1), lc = 8 * (lane >> 4);  // A: voxel row, channel block
  const int bn = (lane & 7) + 8 * (lane >> 4), bk = 8 * ((lane >> 3) & 1);  // B: out-channel row, k block
#pragma unroll 1
  for (int tap = 0; tap < 27; ++tap) {
    if (tap + 1 < 27) conv3_load_w<CIN, COUT, MT>(wbuf + ((tap + 1) & 1) * C::WBYTES, wt, tap + 1);
    cp_commit_();
    cp_wait_<1>();
    __syncthreads();
    const unsigned char* wb = wbuf + (tap & 1) * C::WBYTES;
    const int dm = tap % 3, dn = (tap / 3) % 3, ds = tap / 9;  // halo offsets (0..2)
    int arow[MT], urow[MT];
#pragma unroll
    for (int i = 0; i < MT; ++i) {
      const int r = warp * MT + i;  // row of 16 voxels: n = r % 4, s = r / 4 within the brick
      const int hs = (r >> 2) + ds, hn = (r & 3) + dn, hm = lr + dm;  // full-resolution halo position
      arow[i] = (hs * C::HN + hn) * C::HM + hm;
      // its source voxel in the half-resolution brick (halo position h -> ((h - 1) >> 1) + 1)
      urow[i] = ((((hs - 1) >> 1) + 1) * C::HNH + (((hn - 1) >> 1) + 1)) * C::HMH + (((hm - 1) >> 1) + 1);
    }
#pragma unroll
    for (int kk = 0; kk < CIN / 16; ++kk) {
      uint32_t bfr[COUT / 16][4];
#pragma unroll
      for (int np = 0; np < COUT / 16; ++np)
        ldsm_x4(bfr[np], reinterpret_cast<const bf16*>(wb + (np * 16 + bn) * C::VST + (kk * 16 + bk) * 2));
#pragma unroll
      for (int i = 0; i < MT; ++i) {
        uint32_t a[4];
        if (kk * 16 < UPC)
          ldsm_x4(a, reinterpret_cast<const bf16*>(uhalo + urow[i] * C::VSTU + (kk * 16 + lc) * 2));
        else
          ldsm_x4(a, reinterpret_cast<const bf16*>(halo + arow[i] * C::VSTF + (kk * 16 - UPC + lc) * 2));
#pragma unroll
        for (int np = 0; np < COUT / 16; ++np) {
          mma16816(acc[i][2 * np], a, bfr[np][0], bfr[np][1]);
          mma16816(acc[i][2 * np + 1], a, bfr[np][2], bfr[np][3]);
        }
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < MT; ++i) {
    const int r = warp * MT + i;
    const int n = n0 + (r & 3), s = s0 + (r >> 2);
    if (n >= in.N || s >= in.S) continue;
#pragma unroll
    for (int half = 0; half < 2; ++half) {
      const int m = m0 + g + 8 * half;
      if (m >= in.M) continue;
      bf16* o = out + (((long long)s * in.N + n) * in.M + m) * COUT;
#pragma unroll
      for (int nt = 0; nt < COUT / 8; ++nt) {
        const int co = nt * 8 + 2 * t;
        float x0 = acc[i][nt][2 * half], x1 = acc[i][nt][2 * half + 1];
        if (bias) {
          x0 += bias[co];
          x1 += bias[co + 1];
        }
        if (relu) {
          x0 = fmaxf(x0, 0.f);
          x1 = fmaxf(x1, 0.f);
        }
        *reinterpret_cast<__nv_bfloat162*>(o + co) = __floats2bfloat162_rn(x0, x1);
      }
    }
  }
}

// Row-stationary variant for layers with 16 full-resolution input channels,
// after UPC channels of a nearest-upsampled source (UPC = 0: none; the
// decoder's 48 -> 16 layer has UPC = 32): a 16 (m) x 4 (n) x 8 (s) output
// brick, each warp the four n rows of one s plane.  The taps run in nine stages (ds, dm); in each, the weight fragments
// of the three dn taps sit in registers and each of the warp's six input rows
// (its four rows and their n halo) is loaded once per channel chunk and feeds
// every output row it reaches (i = n_in - dn): 9 ldmatrix per 24 MMAs where
// the tap-by-tap order takes 15.  The full-resolution brick has unpadded
// 32-byte voxel rows whose two 16-byte chunks are swapped on every other
// group of four voxels (chunk c of voxel v at c ^ ((v >> 2) & 1)), so the
// eight consecutive voxels of an ldmatrix matrix fall on distinct banks and
// three CTAs fit on an SM.  The sums run in another order than k_conv3's.
template <int CIN, int COUT, int UPC>
__global__ void __launch_bounds__(256) k_conv3_rs(ConvIn in, const bf16* __restrict__ wt,
                                                  const float* __restrict__ bias, int relu, bf16* __restrict__ out) {
  static_assert(CIN - UPC == 16 && UPC % 16 == 0 && COUT % 16 == 0, "16 full-resolution channels");
  constexpr int TM = 16, TN = 4, TS = 8, MT = 4;
  constexpr int HM = TM + 2, HN = TN + 2, HS = TS + 2, HV = HM * HN * HS;
  constexpr int HMH = TM / 2 + 2, HNH = TN / 2 + 2, HSH = TS / 2 + 2, HVH = UPC > 0 ? HMH * HNH * HSH : 0;
  constexpr int VSTU = UPC * 2 + 16;  // upsampled source rows (padded)
  constexpr int VST = CIN * 2 + 16;   // weight rows (padded)
  constexpr int WSL = COUT * VST;     // one tap's weights
  constexpr int WST = 3 * WSL;        // one stage: the taps dn = 0, 1, 2
  constexpr int FB = HV * 32, UB = HVH * VSTU;
  extern __shared__ __align__(16) unsigned char smem[];
  unsigned char* halo = smem;        // [HV][2 chunks], swizzled
  unsigned char* uhalo = smem + FB;  // [HVH][VSTU]
  unsigned char* wbuf = smem + FB + UB;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int g = lane >> 2, t = lane & 3;
  const int tilesM = (in.M + TM - 1) / TM, tilesN = (in.N + TN - 1) / TN;
  int b = blockIdx.x;
  const int m0 = (b % tilesM) * TM;
  b /= tilesM;
  const int n0 = (b % tilesN) * TN;
  const int s0 = (b / tilesN) * TS;

  for (int i = threadIdx.x; i < HV * 2; i += 256) {
    const int hv = i >> 1, c = i & 1;
    const int hm = hv % HM, r = hv / HM;
    const int m = m0 + hm - 1, n = n0 + r % HN - 1, s = s0 + r / HN - 1;
    const bool ok = m >= 0 && m < in.M && n >= 0 && n < in.N && s >= 0 && s < in.S;
    cpz16(halo + hv * 32 + (c ^ ((hv >> 2) & 1)) * 16, ok ? chunk_ptr(in, s, n, m, UPC + c * 8) : in.src0, ok);
  }
  if constexpr (UPC > 0) {
    constexpr int CHU = UPC / 8;
    const int Mh = in.M >> 1, Nh = in.N >> 1, Sh = in.S >> 1;
    const int mh0 = (m0 >> 1) - 1, nh0 = (n0 >> 1) - 1, sh0 = (s0 >> 1) - 1;
    for (int i = threadIdx.x; i < HVH * CHU; i += 256) {
      const int hv = i / CHU, c = i - hv * CHU;
      const int hm = hv % HMH, r = hv / HMH;
      const int mh = mh0 + hm, nh = nh0 + r % HNH, sh = sh0 + r / HNH;
      const bool ok = mh >= 0 && mh < Mh && nh >= 0 && nh < Nh && sh >= 0 && sh < Sh;
      cpz16(uhalo + hv * VSTU + c * 16, ok ? in.src0 + (((long long)sh * Nh + nh) * Mh + mh) * in.c0 + c * 8 : in.src0,
            ok);
    }
  }
  // stage st = ds * 3 + dm: the weight slices of taps (ds, dn, dm), dn = 0..2
  auto load_stage = [&](unsigned char* dst, int st) {
    const int ds = st / 3, dm = st - 3 * ds;
    constexpr int CH = CIN / 8;
    for (int i = threadIdx.x; i < 3 * COUT * CH; i += 256) {
      const int dn = i / (COUT * CH), rem = i - dn * (COUT * CH);
      const int n = rem / CH, c = rem - n * CH;
      const int tap = (ds * 3 + dn) * 3 + dm;
      cpz16(dst + dn * WSL + n * VST + c * 16, wt + ((long long)tap * COUT + n) * CIN + c * 8, true);
    }
  };
  load_stage(wbuf, 0);
  cp_commit_();

  float acc[MT][COUT / 8][4];
#pragma unroll
  for (int i = 0; i < MT; ++i)
#pragma unroll
    for (int j = 0; j < COUT / 8; ++j)
#pragma unroll
      for (int e = 0; e < 4; ++e) acc[i][j][e] = 0.f;

  const int lr = (lane & 7) + 8 * ((lane >> 3) & 1), lc = 8 * (lane >> 4);  // A: voxel row, channel block
  const int bn = (lane & 7) + 8 * (lane >> 4), bk = 8 * ((lane >> 3) & 1);  // B: out-channel row, k block
  const int sl = warp;  // the warp's s plane in the brick; its rows i are n = n0 + i
#pragma unroll 1
  for (int st = 0; st < 9; ++st) {
    if (st + 1 < 9) load_stage(wbuf + ((st + 1) & 1) * WST, st + 1);
    cp_commit_();
    cp_wait_<1>();
    __syncthreads();
    const unsigned char* wb = wbuf + (st & 1) * WST;
    const int ds = st / 3, dm = st - 3 * ds;
    const int hs = sl + ds, hm = lr + dm;
    const int ush = ((hs - 1) >> 1) + 1, umh = ((hm - 1) >> 1) + 1;
#pragma unroll
    for (int kk = 0; kk < CIN / 16; ++kk) {
      uint32_t bfr[3][COUT / 16][4];
#pragma unroll
      for (int dn = 0; dn < 3; ++dn)
#pragma unroll
        for (int np = 0; np < COUT / 16; ++np)
          ldsm_x4(bfr[dn][np], reinterpret_cast<const bf16*>(wb + dn * WSL + (np * 16 + bn) * VST + (kk * 16 + bk) * 2));
#pragma unroll
      for (int nin = 0; nin < TN + 2; ++nin) {
        uint32_t a[4];
        if (kk * 16 < UPC) {
          const int urow = (ush * HNH + (((nin - 1) >> 1) + 1)) * HMH + umh;
          ldsm_x4(a, reinterpret_cast<const bf16*>(uhalo + urow * VSTU + (kk * 16 + lc) * 2));
        } else {
          const int hv = (hs * HN + nin) * HM + hm;
          ldsm_x4(a, reinterpret_cast<const bf16*>(halo + hv * 32 + (((lc >> 3) ^ ((hv >> 2) & 1)) * 16)));
        }
#pragma unroll
        for (int dn = 0; dn < 3; ++dn) {
          const int i = nin - dn;  // output row reached through tap dn
          if (i >= 0 && i < MT) {
#pragma unroll
            for (int np = 0; np < COUT / 16; ++np) {
              mma16816(acc[i][2 * np], a, bfr[dn][np][0], bfr[dn][np][1]);
              mma16816(acc[i][2 * np + 1], a, bfr[dn][np][2], bfr[dn][np][3]);
            }
          }
        }
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < MT; ++i) {
    const int n = n0 + i, s = s0 + sl;
    if (n >= in.N || s >= in.S) continue;
#pragma unroll
    for (int half = 0; half < 2; ++half) {
      const int m = m0 + g + 8 * half;
      if (m >= in.M) continue;
      bf16* o = out + (((long long)s * in.N + n) * in.M + m) * COUT;
#pragma unroll
      for (int nt = 0; nt < COUT / 8; ++nt) {
        const int co = nt * 8 + 2 * t;
        float x0 = acc[i][nt][2 * half], x1 = acc[i][nt][2 * half + 1];
        if (bias) {
          x0 += bias[co];
          x1 += bias[co + 1];
        }
        if (relu) {
          x0 = fmaxf(x0, 0.f);
          x1 = fmaxf(x1, 0.f);
        }
        *reinterpret_cast<__nv_bfloat162*>(o + co) = __floats2bfloat162_rn(x0, x1);
      }
    }
  }
}

// ---------------------------------------------------------------------------
// tcgen05 (5th-generation tensor core) convolution for levels whose m extent
// is a multiple of 128 and CIN, COUT in {16, 32, 48}.  A CTA owns one line of
// 128 output voxels along m at row n and marches over a chunk of SC planes in
// s.  The 27 weight slices stay in shared memory for the whole march; input
// planes (the rows n-1, n, n+1 with a one-voxel m halo) stream through a ring
// of 5 planes, so every plane is loaded once per CTA.  For output line s one
// thread issues 27 x CIN/16 MMAs (M = 128 voxels, N = COUT, K = 16 channels)
// into a TMEM accumulator; the A operand of tap (dm, dn, ds) is the ring row of
// plane s+ds-1, row n+dn-1, starting at halo column dm: shared memory is kept
// in the canonical no-swizzle K-major layout (8 voxels x 16 bytes per core
// matrix, 16-byte rows consecutive along m, channel chunks a fixed stride
// apart), so a shifted tap is just a shifted descriptor start address.  Two
// TMEM accumulators alternate: while the tensor core works on line s, warps
// 0-3 drain line s-1 (tcgen05.ld of their TMEM lane quarter, bias, ReLU,
// BF16 stores) and a fifth warp, whose lane 0 issues the MMAs, shares the
// plane loads, so issuing and draining overlap.  Every wait on
// the MMA-completion barrier is bounded (about one second of clock); on
// timeout the CTA sets *err and skips its stores.
// ---------------------------------------------------------------------------
namespace tc {

__device__ __forceinline__ uint32_t su32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// shared-memory matrix descriptor: no swizzle, K-major; lbo = byte distance
// between core matrices along K, sbo = along M/N
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFF);
  d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
  d |= (uint64_t)1 << 46;  // descriptor version of this architecture family
  return d;
}

// instruction descriptor, kind::f16: BF16 A and B, FP32 accumulator, both K-major
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t accum) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(
          d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(accum)
      : "memory");
}
__device__ __forceinline__ void commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(su32(bar))
               : "memory");
}
__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// bounded wait for the completion of phase `parity` of an mbarrier: false
// once `limit` SM clock cycles have passed (the default is about one second)
constexpr long long kWaitLimit = 2000000000LL;
__device__ __forceinline__ bool wait_bar(uint64_t* bar, uint32_t parity, long long limit = kWaitLimit) {
  const long long t0 = clock64();
  while (true) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(su32(bar)), "r"(parity)
        : "memory");
    if (ok) return true;
    if (clock64() - t0 > limit) return false;
  }
}

__device__ __forceinline__ void ld16(uint32_t taddr, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

template <int CIN, int COUT>
struct Cfg {
  static constexpr int CH = CIN / 8;                 // 16-byte channel chunks
  static constexpr int HMP = 130;                    // halo row: m0-1 .. m0+128
  static constexpr int RING = 5;                     // planes in the ring
  static constexpr int LINES = RING * 3;             // rows n-1, n, n+1 of each plane
  static constexpr int HALO = CH * LINES * HMP * 16; // [chunk][line][hm][16 B]
  static constexpr int WB = 27 * CH * COUT * 16;     // [tap][chunk][co][16 B]
  static constexpr int SMEM = HALO + WB + 64;
  static constexpr uint32_t LBO_A = LINES * HMP * 16;
  static constexpr uint32_t IDESC = idesc_bf16(128, COUT);
};

}  // namespace tc

// wu: [27][CIN/8][COUT][8] BF16 (UMMA K-major slices)
constexpr int TC_THREADS = 160;  // four epilogue warps and the MMA-issuing warp
template <int CIN, int COUT>
__global__ void __launch_bounds__(TC_THREADS, 1) k_conv3_tc(ConvIn in, const bf16* __restrict__ wu,
                                                     const float* __restrict__ bias, int relu, bf16* __restrict__ out,
                                                     int SC, int* __restrict__ err) {
  using C = tc::Cfg<CIN, COUT>;
  extern __shared__ __align__(128) unsigned char smem_tc[];
  unsigned char* smem = smem_tc;
  unsigned char* halo = smem;
  unsigned char* wsm = smem + C::HALO;
  uint64_t* bars = reinterpret_cast<uint64_t*>(wsm + C::WB);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(bars + 2);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int MB = in.M / 128;
  int b = blockIdx.x;
  const int m0 = (b % MB) * 128;
  b /= MB;
  const int n = b % in.N;
  const int s0 = (b / in.N) * SC;
  const int s_end = min(in.S, s0 + SC);

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 128;" ::"r"(tc::su32(tslot))
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(tc::su32(&bars[0])) : "memory");
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(tc::su32(&bars[1])) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  // resident weights
  for (int i = tid; i < 27 * C::CH * COUT; i += TC_THREADS) cpz16(wsm + i * 16, wu + (long long)i * 8, true);
  // one input plane (rows n-1..n+1, m0-1..m0+128) into its ring slot; zero outside the volume
  auto load_plane = [&](int ps) {
    const int slot = ((ps % C::RING) + C::RING) % C::RING;
    for (int i = tid; i < 3 * C::HMP * C::CH; i += TC_THREADS) {
      const int c = i % C::CH, rest = i / C::CH, hm = rest % C::HMP, li = rest / C::HMP;
      const int m = m0 - 1 + hm, nn = n - 1 + li;
      const bool ok = ps >= 0 && ps < in.S && nn >= 0 && nn < in.N && m >= 0 && m < in.M;
      unsigned char* dst = halo + ((c * C::LINES + slot * 3 + li) * C::HMP + hm) * 16;
      cpz16(dst, ok ? chunk_ptr(in, ps, nn, m, c * 8) : in.src0, ok);
    }
  };
  load_plane(s0 - 1);
  load_plane(s0);
  load_plane(s0 + 1);
  cp_commit_();
  cp_wait_<0>();
  tc::fence_async_smem();
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tmem = *tslot;
  const uint32_t hbase = tc::su32(halo), wbase = tc::su32(wsm);

  auto epilogue = [&](int jj, int s) {
    if (warp >= 4) return true;  // the MMA-issuing warp holds no TMEM lanes
    if (!tc::wait_bar(&bars[jj & 1], (uint32_t)((jj >> 1) & 1))) return false;
    tc::fence_after();
    const int m = m0 + 32 * warp + lane;
    bf16* o = out + (((long long)s * in.N + n) * in.M + m) * COUT;
#pragma unroll
    for (int c0 = 0; c0 < COUT; c0 += 16) {
      float v[16];
      tc::ld16(tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)((jj & 1) * 64 + c0), v);
      uint32_t pk[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        float a0 = v[2 * q], a1 = v[2 * q + 1];
        if (bias) {
          a0 += bias[c0 + 2 * q];
          a1 += bias[c0 + 2 * q + 1];
        }
        if (relu) {
          a0 = fmaxf(a0, 0.f);
          a1 = fmaxf(a1, 0.f);
        }
        const __nv_bfloat162 h = __floats2bfloat162_rn(a0, a1);
        pk[q] = *reinterpret_cast<const uint32_t*>(&h);
      }
      if (m < in.M) {
        reinterpret_cast<uint4*>(o + c0)[0] = make_uint4(pk[0], pk[1], pk[2], pk[3]);
        reinterpret_cast<uint4*>(o + c0)[1] = make_uint4(pk[4], pk[5], pk[6], pk[7]);
      }
    }
    return true;
  };

  // The failure decision is CTA-wide (__syncthreads_or), so once any thread's
  // completion wait runs out no thread issues further plane loads or MMAs.
  int j = 0, last = -1;  // last = index of the last committed MMA batch
  bool bad = false;
  for (int s = s0; s < s_end; ++s, ++j) {
    if (s + 1 < s_end) load_plane(s + 2);  // needed by line s+1; its slot held plane s-3, drained at step j-1
    cp_commit_();
    if (warp == 4 && lane == 0) {
      // The issuing thread bounds the step (every thread meets it at the
      // step's barrier), so the descriptors are formed from per-step bases
      // with the taps unrolled: the address field of each is
      // one add on the base of its ring plane (or of the weights) plus a
      // compile-time offset, the other fields are constant.
      const uint32_t d = tmem + (uint32_t)((j & 1) * 64);
      const int slot0 = (((s - 1) % C::RING) + C::RING) % C::RING;
      uint32_t abase[3];  // address field (>> 4) of ring row (plane s+ds-1, dn = 0, dm = 0, chunk 0)
#pragma unroll
      for (int ds = 0; ds < 3; ++ds) {
        const int slot = slot0 + ds >= C::RING ? slot0 + ds - C::RING : slot0 + ds;
        abase[ds] = (hbase >> 4) + (uint32_t)(slot * 3 * C::HMP);
      }
      const uint32_t wb4 = wbase >> 4;
      const uint64_t ahi = tc::sdesc(0, C::LBO_A, 128), bhi = tc::sdesc(0, COUT * 16, 128);
#pragma unroll
      for (int tap = 0; tap < 27; ++tap) {
        const int dm = tap % 3, dn = (tap / 3) % 3, ds = tap / 9;
#pragma unroll
        for (int kk = 0; kk < CIN / 16; ++kk) {
          const uint32_t a4 = abase[ds] + (uint32_t)((2 * kk * C::LINES + dn) * C::HMP + dm);
          const uint32_t b4 = wb4 + (uint32_t)((tap * C::CH + 2 * kk) * COUT);
          tc::mma(d, ahi | (uint64_t)(a4 & 0x3FFF), bhi | (uint64_t)(b4 & 0x3FFF), C::IDESC,
                  (tap | kk) != 0 ? 1u : 0u);
        }
      }
      tc::commit(&bars[j & 1]);
    }
    last = j;
    bool mine = true;
    if (j >= 1) mine = epilogue(j - 1, s - 1);
    cp_wait_<0>();
    tc::fence_async_smem();
    tc::fence_before();
    bad = __syncthreads_or(!mine) != 0;
    tc::fence_after();
    if (bad) break;
  }
  if (!bad && j >= 1) {
    const bool mine = epilogue(j - 1, s_end - 1);
    bad = __syncthreads_or(!mine) != 0;
  }
  if (bad) {
    // A completion wait ran out.  Before the accumulator columns are freed,
    // one more bounded wait on the last commit, which covers every MMA this
    // CTA issued; then the flag tells the host to discard this launch's output.
    if (tid == 0 && last >= 0) tc::wait_bar(&bars[last & 1], (uint32_t)((last >> 1) & 1));
    if (tid == 0) atomicExch(err, 1);
  }
  tc::fence_before();
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 128;" ::"r"(tmem) : "memory");
}

// Self-test of the bounded completion wait and of the error path that follows
// it: one CTA allocates TMEM as k_conv3_tc does, waits with the same bounded
// wait, shortened to `limit` cycles, on an mbarrier that nothing arrives on
// (no MMA is issued and none is in flight), sets *err when the wait runs out,
// then frees its TMEM and returns.
__global__ void __launch_bounds__(128, 1) k_wait_selftest(long long limit, int* __restrict__ err) {
  __shared__ __align__(8) uint64_t bar;
  __shared__ uint32_t tslot;
  const int warp = threadIdx.x >> 5;
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 128;" ::"r"(tc::su32(&tslot))
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(tc::su32(&bar)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tmem = tslot;
  if (threadIdx.x == 0 && !tc::wait_bar(&bar, 0u, limit)) atomicExch(err, 1);
  tc::fence_before();
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 128;" ::"r"(tmem) : "memory");
}

// UMMA weight slices: forward wu[tap][c][co][e] = W[co][tap][8c+e] (K = ci);
// data gradient wub[tap][c][ci][e] = W[8c+e][26-tap][ci] (K = co)
__global__ void k_pack_w_umma(const float* __restrict__ W, int Cout, int Cin, bf16* __restrict__ wu,
                              bf16* __restrict__ wub) {
  const int total = 27 * Cout * Cin;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
    {  // forward: i = ((tap * Cin/8 + c) * Cout + co) * 8 + e
      const int e = i % 8, r = i / 8, co = r % Cout, r2 = r / Cout, c = r2 % (Cin / 8), tap = r2 / (Cin / 8);
      wu[i] = __float2bfloat16(W[((long long)co * 27 + tap) * Cin + c * 8 + e]);
    }
    {  // data gradient: i = ((tap * Cout/8 + c) * Cin + ci) * 8 + e
      const int e = i % 8, r = i / 8, ci = r % Cin, r2 = r / Cin, c = r2 % (Cout / 8), tap = r2 / (Cout / 8);
      wub[i] = __float2bfloat16(W[((long long)(c * 8 + e) * 27 + (26 - tap)) * Cin + ci]);
    }
  }
}

// tap-major weight slices for k_conv3: forward wt[tap][co][ci] = W[co][tap][ci];
// data gradient wtb[tap][ci][co] = W[co][26 - tap][ci]
__global__ void k_pack_w3(const float* __restrict__ W, int Cout, int Cin, bf16* __restrict__ wt, bf16* __restrict__ wtb) {
  const int total = 27 * Cout * Cin;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
    const int ci = i % Cin, r = i / Cin, co = r % Cout, tap = r / Cout;
    wt[i] = __float2bfloat16(W[((long long)co * 27 + tap) * Cin + ci]);
    const int cb = i % Cout, rb = i / Cout, cib = rb % Cin, tb = rb / Cin;
    wtb[i] = __float2bfloat16(W[((long long)cb * 27 + (26 - tb)) * Cin + cib]);
  }
}

// ---------------------------------------------------------------------------
// weight gradient: dw[co][k] += sum_v g[v][co] A[v][k] for the k-chunk
// blockIdx.x, over the 16-voxel tiles blockIdx.y*4 + warp (+ stride).
// ---------------------------------------------------------------------------
template <int COUT, bool PACKED>
__global__ void __launch_bounds__(128) k_conv_wgrad(ConvIn in, const bf16* __restrict__ gy, int Kpad, int Cin,
                                                    long long V, float* __restrict__ dw) {
  __shared__ __align__(16) bf16 gs[4][16 * COUT];
  __shared__ __align__(16) bf16 as[4][256];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int g = lane >> 2, t = lane & 3;
  const int kc = blockIdx.x;
  float acc[COUT / 16][2][4];
#pragma unroll
  for (int i = 0; i < COUT / 16; ++i)
#pragma unroll
    for (int j = 0; j < 2; ++j)
#pragma unroll
      for (int e = 0; e < 4; ++e) acc[i][j][e] = 0.f;
  const long long ntiles = (V + 15) / 16;
  const long long stride = (long long)gridDim.y * 4;
  // ldmatrix.trans lanes: voxel row and 8-column block
  const int tv = (lane & 7) + 8 * (lane >> 4), tcb = 8 * ((lane >> 3) & 1);  // G^T: co block varies with lane bit 3
  const int bv = (lane & 7) + 8 * ((lane >> 3) & 1), bcb = 8 * (lane >> 4);  // B: voxel block with lane bit 3
#pragma unroll 1
  for (long long tile = (long long)blockIdx.y * 4 + warp; tile < ntiles; tile += stride) {
    const long long v0 = tile * 16;
    // G slab: 16 voxels x COUT
    for (int i = lane; i < 16 * COUT / 8; i += 32) {
      const int vi = i / (COUT / 8), c8 = i - vi * (COUT / 8);
      uint4 val = make_uint4(0, 0, 0, 0);
      if (v0 + vi < V) val = __ldg(reinterpret_cast<const uint4*>(gy + (v0 + vi) * COUT) + c8);
      reinterpret_cast<uint4*>(gs[warp] + vi * COUT)[c8] = val;
    }
    fill_slab<PACKED>(as[warp], in, v0, kc, Cin, lane);
    __syncwarp();
    uint32_t b[4];
    ldsm_x4_t(b, as[warp] + bv * 16 + bcb);
#pragma unroll
    for (int mt = 0; mt < COUT / 16; ++mt) {
      uint32_t a[4];
      ldsm_x4_t(a, gs[warp] + tv * COUT + mt * 16 + tcb);
      mma16816(acc[mt][0], a, b[0], b[1]);
      mma16816(acc[mt][1], a, b[2], b[3]);
    }
    __syncwarp();
  }
#pragma unroll
  for (int mt = 0; mt < COUT / 16; ++mt)
#pragma unroll
    for (int nt = 0; nt < 2; ++nt)
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int co = mt * 16 + g + 8 * (e >> 1);
        const int k = kc * 16 + nt * 8 + 2 * t + (e & 1);
        atomicAdd(&dw[(long long)co * Kpad + k], acc[mt][nt][e]);
      }
}

// ---------------------------------------------------------------------------
// elementwise helpers
// ---------------------------------------------------------------------------
__global__ void k_to_bf16(const float* __restrict__ x, bf16* __restrict__ y, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    y[i] = __float2bfloat16(x[i]);
}

__global__ void k_relu_mask(bf16* __restrict__ g, const bf16* __restrict__ y, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    if (!(__bfloat162float(y[i]) > 0.f)) g[i] = __float2bfloat16(0.f);
}

// 2x2x2 max pooling of x (full size M, N, S, C channels, C a multiple of 8);
// the first maximum in (s, n, m) order wins.  A thread takes 8 channels of
// one pooled voxel: 16-byte loads of the 8 children, one 16-byte store of the
// maxima and one 8-byte store of their child indices.
__global__ void k_maxpool(const bf16* __restrict__ x, bf16* __restrict__ y, unsigned char* __restrict__ idx, int M,
                          int N, int S, int C) {
  const int CG = C / 8;
  const long long total = (long long)(M / 2) * (N / 2) * (S / 2) * CG;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const int c0 = (int)(i % CG) * 8;
    const long long v = i / CG;
    const int m2 = (int)(v % (M / 2)), n2 = (int)((v / (M / 2)) % (N / 2)), s2 = (int)(v / ((long long)(M / 2) * (N / 2)));
    float best[8];
    int bi[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      best[k] = -INFINITY;
      bi[k] = 0;
    }
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int s = 2 * s2 + (q >> 2), n = 2 * n2 + ((q >> 1) & 1), m = 2 * m2 + (q & 1);
      const uint4 raw = __ldg(reinterpret_cast<const uint4*>(x + (((long long)s * N + n) * M + m) * C + c0));
      const __nv_bfloat162* h = reinterpret_cast<const __nv_bfloat162*>(&raw);
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const float2 f = __bfloat1622float2(h[k]);
        if (f.x > best[2 * k]) { best[2 * k] = f.x; bi[2 * k] = q; }
        if (f.y > best[2 * k + 1]) { best[2 * k + 1] = f.y; bi[2 * k + 1] = q; }
      }
    }
    uint32_t pk[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const __nv_bfloat162 h2 = __floats2bfloat162_rn(best[2 * k], best[2 * k + 1]);
      pk[k] = *reinterpret_cast<const uint32_t*>(&h2);
    }
    *reinterpret_cast<uint4*>(y + v * C + c0) = make_uint4(pk[0], pk[1], pk[2], pk[3]);
    uint32_t ix0 = 0, ix1 = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      ix0 |= (uint32_t)bi[k] << (8 * k);
      ix1 |= (uint32_t)bi[k + 4] << (8 * k);
    }
    *reinterpret_cast<uint2*>(idx + v * C + c0) = make_uint2(ix0, ix1);
  }
}

// g[v][c] = (argmax child of v's block == v ? gp[parent][c] : 0) + skip[v][coff + c]
__global__ void k_unpool_add(const bf16* __restrict__ gp, const unsigned char* __restrict__ idx,
                             const bf16* __restrict__ skip, int Cskip, int coff, bf16* __restrict__ g, int M, int N,
                             int S, int C) {
  const long long total = (long long)M * N * S * C;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const int c = (int)(i % C);
    const long long v = i / C;
    const int m = (int)(v % M), n = (int)((v / M) % N), s = (int)(v / ((long long)M * N));
    const long long par = ((long long)(s >> 1) * (N >> 1) + (n >> 1)) * (M >> 1) + (m >> 1);
    const int child = ((s & 1) << 2) | ((n & 1) << 1) | (m & 1);
    float val = idx[par * C + c] == child ? __bfloat162float(gp[par * C + c]) : 0.f;
    val += __bfloat162float(skip[v * Cskip + coff + c]);
    g[i] = __float2bfloat16(val);
  }
}

// adjoint of nearest upsampling on channels [0, C) of a Ctot-channel tensor
__global__ void k_up_adj(const bf16* __restrict__ gf, int Ctot, bf16* __restrict__ g, int M, int N, int S, int C) {
  const long long total = (long long)(M / 2) * (N / 2) * (S / 2) * C;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const int c = (int)(i % C);
    const long long v = i / C;
    const int m2 = (int)(v % (M / 2)), n2 = (int)((v / (M / 2)) % (N / 2)), s2 = (int)(v / ((long long)(M / 2) * (N / 2)));
    float acc = 0.f;
    for (int q = 0; q < 8; ++q) {
      const int s = 2 * s2 + (q >> 2), n = 2 * n2 + ((q >> 1) & 1), m = 2 * m2 + (q & 1);
      acc += __bfloat162float(gf[(((long long)s * N + n) * M + m) * Ctot + c]);
    }
    g[i] = __float2bfloat16(acc);
  }
}

// out[v] = sum_c wh[c] d1[v][c] + bh + x[v]
template <int C>
__global__ void k_head_fwd(const bf16* __restrict__ d1, const float* __restrict__ wh, const float* __restrict__ x,
                           float* __restrict__ out, long long V) {
  for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < V; v += (long long)gridDim.x * blockDim.x) {
    float acc = wh[C];
#pragma unroll
    for (int c8 = 0; c8 < C; c8 += 8) {
      const uint4 raw = __ldg(reinterpret_cast<const uint4*>(d1 + v * C + c8));
      const __nv_bfloat162* h = reinterpret_cast<const __nv_bfloat162*>(&raw);
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const float2 dv = __bfloat1622float2(h[k]);
        acc += wh[c8 + 2 * k] * dv.x + wh[c8 + 2 * k + 1] * dv.y;
      }
    }
    out[v] = acc + x[v];
  }
}

__device__ __forceinline__ double wsum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// r = out - t; loss += sum r^2 (FP64); gd1[v][c] = (2 r / V) wh[c];
// gwh[c] += sum_v (2 r / V) d1[v][c]; gwh[C] += sum_v 2 r / V
template <int C>
__global__ void k_head_bwd(const float* __restrict__ out, const float* __restrict__ tgt, const bf16* __restrict__ d1,
                           const float* __restrict__ wh, bf16* __restrict__ gd1, float* __restrict__ gwh,
                           double* __restrict__ loss, long long V) {
  double l = 0.0;
  float gw[C + 1];
#pragma unroll
  for (int c = 0; c <= C; ++c) gw[c] = 0.f;
  const float sc = 2.0f / (float)V;
  for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < V; v += (long long)gridDim.x * blockDim.x) {
    const float r = out[v] - tgt[v];
    l += (double)r * r;
    const float go = sc * r;
#pragma unroll
    for (int c = 0; c < C; c += 2) {
      const float2 dv = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(d1 + v * C + c));
      *reinterpret_cast<__nv_bfloat162*>(gd1 + v * C + c) = __floats2bfloat162_rn(go * wh[c], go * wh[c + 1]);
      gw[c] += go * dv.x;
      gw[c + 1] += go * dv.y;
    }
    gw[C] += go;
  }
  l = wsum(l);
  if ((threadIdx.x & 31) == 0) atomicAdd(loss, l);
#pragma unroll
  for (int c = 0; c <= C; ++c) {
    const double t = wsum((double)gw[c]);
    if ((threadIdx.x & 31) == 0) atomicAdd(&gwh[c], (float)t);
  }
}

// gb[c] += sum_v g[v][c]; blockDim and the grid stride are multiples of C,
// so every thread keeps one channel
__global__ void k_bias_grad(const bf16* __restrict__ g, float* __restrict__ gb, long long V, int C) {
  __shared__ float red[256];
  float acc = 0.f;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < V * C; i += (long long)gridDim.x * blockDim.x)
    acc += __bfloat162float(g[i]);
  red[threadIdx.x] = acc;
  __syncthreads();
  if (threadIdx.x < C) {
    float t = 0.f;
    for (int j = threadIdx.x; j < blockDim.x; j += C) t += red[j];
    atomicAdd(&gb[threadIdx.x], t);
  }
}

// copy dw[co][Kpad] (first 27*Cin columns) into the flat gradient (co, 27, ci)
__global__ void k_unpack_dw(const float* __restrict__ dw, int Cout, int Cin, int Kpad, float* __restrict__ gflat) {
  const int total = Cout * 27 * Cin;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
    const int co = i / (27 * Cin), k = i - co * 27 * Cin;
    gflat[i] = dw[(long long)co * Kpad + k];
  }
}

__global__ void k_adam(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m1,
                       float* __restrict__ m2, long long n, float lr, float b1, float b2, float eps, float c1, float c2) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float a = b1 * m1[i] + (1.f - b1) * gi;
    const float b = b2 * m2[i] + (1.f - b2) * gi * gi;
    m1[i] = a;
    m2[i] = b;
    p[i] -= lr * (a / c1) / (sqrtf(b / c2) + eps);
  }
}

// d0_j = t g_j / max(||g_j||, t), g = L x (periodic forward differences), t = lambda / rho
template <typename T>
__global__ void k_dual_init(const T* __restrict__ x, T* __restrict__ d, int M, int N, int S, T thr) {
  const long long V = (long long)M * N * S;
  for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < V; v += (long long)gridDim.x * blockDim.x) {
    const int m = (int)(v % M), n = (int)((v / M) % N), s = (int)(v / ((long long)M * N));
    const T xv = x[v];
    const T g0 = x[v - m + (m + 1) % M] - xv;
    const T g1 = x[v + (long long)(((n + 1) % N) - n) * M] - xv;
    const T g2 = x[v + (long long)(((s + 1) % S) - s) * M * N] - xv;
    const T nrm = sqrt(g0 * g0 + g1 * g1 + g2 * g2);
    const T sc = thr / (nrm > thr ? nrm : thr);
    d[v] = g0 * sc;
    d[V + v] = g1 * sc;
    d[2 * V + v] = g2 * sc;
  }
}

}  // namespace sr3d

using namespace sr3d;

// ---------------------------------------------------------------------------
// host side: the network
// ---------------------------------------------------------------------------
namespace {

constexpr int C1 = 16, C2 = 32, C3 = 64;
struct LayerShape {
  int cout, cin;
};
const LayerShape kLayers[10] = {{C1, 1},       {C1, C1}, {C2, C1}, {C2, C2}, {C3, C2},
                                {C3, C3},      {C2, C3 + C2}, {C2, C2}, {C1, C2 + C1}, {C1, C1}};

int ufail(int code, const char* msg, cudaError_t e = cudaSuccess) {
  char buf[512];
  snprintf(buf, sizeof(buf), "%s%s%s", msg, e != cudaSuccess ? ": " : "", e != cudaSuccess ? cudaGetErrorString(e) : "");
  return record_error(code, buf);
}

}  // namespace

struct sr3d_unet_s {
  cudaStream_t stream = nullptr;
  long long np = 0;
  float* p = nullptr;   // master parameters (flat, oracle order)
  float* g = nullptr;   // gradient (same layout)
  float* m1 = nullptr;  // Adam moments
  float* m2 = nullptr;
  long long step = 0;
  long long off_w[10], off_b[10], off_h;
  int kpad[10];
  bf16* wt[10] = {};    // layers 1..9: tap-major forward slices [27][co][ci]
  bf16* wtb[10] = {};   // layers 1..9: tap-major data-gradient slices [27][ci][co]
  bf16* wu[10] = {};    // layers 1..9: tcgen05 (UMMA K-major) forward slices [27][ci/8][co][8]
  bf16* wub[10] = {};   // layers 1..9: tcgen05 data-gradient slices [27][co/8][ci][8]
  int use_tc = 1;       // tcgen05 path where available
  int* err = nullptr;   // device flag: a bounded wait of the tcgen05 kernel ran out
  float* dw = nullptr;  // weight-gradient scratch [Cout][Kpad]
  size_t dw_cap = 0;
  double* loss = nullptr;
  // activations for the current size
  int M = 0, N = 0, S = 0;
  std::vector<void*> bufs;
  bf16 *xb, *e1a, *e1, *p1, *e2a, *e2, *p2, *e3a, *e3, *d2a, *d2, *d1a, *d1;
  unsigned char *i1, *i2;
  float* out;
  bf16 *ga, *gb, *gc, *gd, *ge;  // gradient scratch
};

static int grid_for(long long n) { return (int)((n + 255) / 256 < 8192 ? (n + 255) / 256 : 8192); }

static int unet_alloc(sr3d_unet_s* u, void** p, size_t bytes) {
  cudaError_t e = cudaMalloc(p, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return ufail(e == cudaErrorMemoryAllocation ? SR3D_ERR_OOM : SR3D_ERR_CUDA, "cudaMalloc", e);
  }
  u->bufs.push_back(*p);
  return SR3D_OK;
}

#define UCK(call)                                                      \
  do {                                                                 \
    cudaError_t e_ = (call);                                           \
    if (e_ != cudaSuccess) return ufail(SR3D_ERR_CUDA, #call, e_);     \
  } while (0)
#define UTRY(call)                      \
  do {                                  \
    int r_ = (call);                    \
    if (r_ != SR3D_OK) return r_;       \
  } while (0)

static int ensure_size(sr3d_unet_s* u, int M, int N, int S) {
  if (u->M == M && u->N == N && u->S == S) return SR3D_OK;
  for (void* b : u->bufs) cudaFree(b);
  u->bufs.clear();
  u->M = M; u->N = N; u->S = S;
  const long long V = (long long)M * N * S, V2 = V / 8, V4 = V / 64;
  auto A = [&](bf16** p, long long n) { return unet_alloc(u, (void**)p, (size_t)n * sizeof(bf16)); };
  UTRY(A(&u->xb, V));
  UTRY(A(&u->e1a, V * C1)); UTRY(A(&u->e1, V * C1));
  UTRY(A(&u->p1, V2 * C1)); UTRY(A(&u->e2a, V2 * C2)); UTRY(A(&u->e2, V2 * C2));
  UTRY(A(&u->p2, V4 * C2)); UTRY(A(&u->e3a, V4 * C3)); UTRY(A(&u->e3, V4 * C3));
  UTRY(A(&u->d2a, V2 * C2)); UTRY(A(&u->d2, V2 * C2));
  UTRY(A(&u->d1a, V * C1)); UTRY(A(&u->d1, V * C1));
  UTRY(unet_alloc(u, (void**)&u->i1, (size_t)V2 * C1));
  UTRY(unet_alloc(u, (void**)&u->i2, (size_t)V4 * C2));
  UTRY(unet_alloc(u, (void**)&u->out, (size_t)V * sizeof(float)));
  const long long gmax = V * (C2 + C1) > V2 * (C3 + C2) ? V * (C2 + C1) : V2 * (C3 + C2);
  UTRY(A(&u->ga, gmax)); UTRY(A(&u->gb, gmax)); UTRY(A(&u->gc, gmax));
  UTRY(A(&u->gd, V * C1)); UTRY(A(&u->ge, V2 * C2));
  return SR3D_OK;
}

// first layer: one input channel, 16 outputs, bias and ReLU
static cudaError_t conv_first(cudaStream_t st, const bf16* x, const float* W, const float* bias, bf16* out, int M,
                              int N, int S) {
  dim3 grid((M + F_TM * F_VM - 1) / (F_TM * F_VM), (N + F_TN - 1) / F_TN, (S + F_TS - 1) / F_TS);
  k_conv_first<<<grid, F_TM * F_TN, 0, st>>>(x, W, bias, out, M, N, S);
  return cudaGetLastError();
}

template <int CIN, int COUT, int MT, int UPC = 0>
static cudaError_t conv3_t(cudaStream_t st, const ConvIn& in, const bf16* wt, const float* bias, int relu, bf16* out) {
  using C = Conv3Cfg<CIN, COUT, MT, UPC>;
  cudaError_t e =
      cudaFuncSetAttribute(k_conv3<CIN, COUT, MT, UPC>, cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM);
  if (e != cudaSuccess) return e;
  const long long blocks = (long long)((in.M + C::TM - 1) / C::TM) * ((in.N + C::TN - 1) / C::TN) *
                           ((in.S + C::TS - 1) / C::TS);
  k_conv3<CIN, COUT, MT, UPC><<<(unsigned)blocks, 256, C::SMEM, st>>>(in, wt, bias, relu, out);
  return cudaGetLastError();
}

template <int CIN, int COUT, int UPC>
static cudaError_t conv3_rs_t(cudaStream_t st, const ConvIn& in, const bf16* wt, const float* bias, int relu,
                              bf16* out) {
  constexpr int HV = 18 * 6 * 10, HVH = UPC > 0 ? 10 * 4 * 6 : 0;
  constexpr int SMEM = HV * 32 + HVH * (UPC * 2 + 16) + 2 * 3 * COUT * (CIN * 2 + 16);
  cudaError_t e = cudaFuncSetAttribute(k_conv3_rs<CIN, COUT, UPC>, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM);
  if (e != cudaSuccess) return e;
  const long long blocks = (long long)((in.M + 15) / 16) * ((in.N + 3) / 4) * ((in.S + 7) / 8);
  k_conv3_rs<CIN, COUT, UPC><<<(unsigned)blocks, 256, SMEM, st>>>(in, wt, bias, relu, out);
  return cudaGetLastError();
}

template <int CIN, int COUT>
static cudaError_t conv3_tc_t(cudaStream_t st, const ConvIn& in, const bf16* wu, const float* bias, int relu,
                              bf16* out, int* err) {
  using C = tc::Cfg<CIN, COUT>;
  cudaError_t e = cudaFuncSetAttribute(k_conv3_tc<CIN, COUT>, cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM);
  if (e != cudaSuccess) return e;
  const long long lines = (long long)(in.M / 128) * in.N * in.S;
  int sc = (int)(lines / (152 * 4));  // about four waves of one CTA per SM
  sc = sc < 8 ? 8 : (sc > 64 ? 64 : sc);
  if (sc > in.S) sc = in.S;
  const long long blocks = (long long)(in.M / 128) * in.N * ((in.S + sc - 1) / sc);
  k_conv3_tc<CIN, COUT><<<(unsigned)blocks, TC_THREADS, C::SMEM, st>>>(in, wu, bias, relu, out, sc, err);
  return cudaGetLastError();
}

// the tcgen05 kernel takes levels whose m extent is a multiple of 128 and
// 16, 32 or 48 input and output channels; returns cudaErrorNotSupported
// otherwise.  With all_shapes false only the shapes where it beats the
// mma.sync kernel are taken: (16, 16) and (16, 32).  Measured in the U-Net
// forward at 256^3 (levels 256^3 and 128^3): (16, 16) 0.70 ms against 1.29 ms,
// (16, 32) 0.16 against 0.23 ms, while the rings of 32 and 48 input channels
// leave one CTA per SM ((32, 32) 0.42 against 0.33 ms, (48, 16) 5.0 against
// 2.9 ms).
static cudaError_t conv3_tc(cudaStream_t st, int cin, int cout, const ConvIn& in, const bf16* wu, const float* bias,
                            int relu, bf16* out, int* err, bool all_shapes) {
  if (in.M % 128 != 0) return cudaErrorNotSupported;
  if (!all_shapes && !(cin == 16 && (cout == 16 || cout == 32))) return cudaErrorNotSupported;
#define SR3D_CONV3_TC(CI, CO) \
  if (cin == CI && cout == CO) return conv3_tc_t<CI, CO>(st, in, wu, bias, relu, out, err);
  SR3D_CONV3_TC(16, 16)
  SR3D_CONV3_TC(16, 32)
  SR3D_CONV3_TC(32, 16)
  SR3D_CONV3_TC(32, 32)
  SR3D_CONV3_TC(16, 48)
  SR3D_CONV3_TC(48, 16)
#undef SR3D_CONV3_TC
  return cudaErrorNotSupported;
}

// 3x3x3 convolution with cin = in.c0 + in.c1 input channels (a multiple of 16)
static cudaError_t conv3(cudaStream_t st, int cin, int cout, const ConvIn& in, const bf16* wt, const float* bias,
                         int relu, bf16* out) {
  // the decoder layers whose first source is upsampled: that source's brick at its own resolution
  if (in.up0 && in.c1 > 0 && in.M % 2 == 0 && in.N % 2 == 0 && in.S % 2 == 0) {
    if (cin == 48 && cout == 16 && in.c0 == 32) return conv3_rs_t<48, 16, 32>(st, in, wt, bias, relu, out);
    if (cin == 96 && cout == 32 && in.c0 == 64) return conv3_t<96, 32, 2, 64>(st, in, wt, bias, relu, out);
  }
  // one full-resolution source of 16 channels: row-stationary
  if (!in.up0 && in.c1 == 0 && cin == 16) {
    if (cout == 16) return conv3_rs_t<16, 16, 0>(st, in, wt, bias, relu, out);
    if (cout == 32) return conv3_rs_t<16, 32, 0>(st, in, wt, bias, relu, out);
  }
#define SR3D_CONV3(CI, CO, MT_) \
  if (cin == CI && cout == CO) return conv3_t<CI, CO, MT_>(st, in, wt, bias, relu, out);
  SR3D_CONV3(16, 16, 2)
  SR3D_CONV3(16, 32, 2)
  SR3D_CONV3(32, 32, 2)
  SR3D_CONV3(32, 64, 2)
  SR3D_CONV3(64, 64, 2)
  SR3D_CONV3(96, 32, 1)
  SR3D_CONV3(48, 16, 2)
  SR3D_CONV3(16, 48, 2)
  SR3D_CONV3(32, 96, 2)
  SR3D_CONV3(64, 32, 2)
  SR3D_CONV3(32, 16, 2)
#undef SR3D_CONV3
  return cudaErrorInvalidValue;
}

template <int COUT>
static cudaError_t conv_wgrad_c(cudaStream_t st, const ConvIn& in, const bf16* gy, int Kpad, int Cin, long long V,
                                float* dw) {
  const long long ntiles = (V + 15) / 16;
  int gy_ = (int)((ntiles + 4 * 64 - 1) / (4 * 64));  // up to 64 tiles per warp
  if (gy_ > 4096) gy_ = 4096;
  if (gy_ < 1) gy_ = 1;
  dim3 grid(Kpad / 16, gy_);
  if (Cin == 1) k_conv_wgrad<COUT, true><<<grid, 128, 0, st>>>(in, gy, Kpad, Cin, V, dw);
  else k_conv_wgrad<COUT, false><<<grid, 128, 0, st>>>(in, gy, Kpad, Cin, V, dw);
  return cudaGetLastError();
}

static cudaError_t conv_wgrad(cudaStream_t st, int Cout, const ConvIn& in, const bf16* gy, int Kpad, int Cin,
                              long long V, float* dw) {
  switch (Cout) {
    case 16: return conv_wgrad_c<16>(st, in, gy, Kpad, Cin, V, dw);
    case 32: return conv_wgrad_c<32>(st, in, gy, Kpad, Cin, V, dw);
    case 64: return conv_wgrad_c<64>(st, in, gy, Kpad, Cin, V, dw);
  }
  return cudaErrorInvalidValue;
}

static ConvIn cin(const bf16* a, int ca, int up, const bf16* b, int cb, int M, int N, int S) {
  ConvIn c;
  c.src0 = a; c.c0 = ca; c.up0 = up; c.src1 = b; c.c1 = cb; c.M = M; c.N = N; c.S = S;
  return c;
}

static int pack_weights(sr3d_unet_s* u) {
  for (int l = 1; l < 10; ++l) {
    const LayerShape& L = kLayers[l];
    k_pack_w3<<<128, 256, 0, u->stream>>>(u->p + u->off_w[l], L.cout, L.cin, u->wt[l], u->wtb[l]);
    UCK(cudaGetLastError());
    k_pack_w_umma<<<128, 256, 0, u->stream>>>(u->p + u->off_w[l], L.cout, L.cin, u->wu[l], u->wub[l]);
    UCK(cudaGetLastError());
  }
  return SR3D_OK;
}

// layer l forward (data gradient with grad = true): tcgen05 where it applies
static cudaError_t conv_layer(sr3d_unet_s* u, int l, bool grad, const ConvIn& in, const float* bias, int relu,
                              bf16* out) {
  const LayerShape& L = kLayers[l];
  const int cin = grad ? L.cout : L.cin, cout = grad ? L.cin : L.cout;
  if (u->use_tc) {
    const cudaError_t e =
        conv3_tc(u->stream, cin, cout, in, grad ? u->wub[l] : u->wu[l], bias, relu, out, u->err, u->use_tc == 2);
    if (e != cudaErrorNotSupported) return e;
  }
  return conv3(u->stream, cin, cout, in, grad ? u->wtb[l] : u->wt[l], bias, relu, out);
}

static int unet_forward(sr3d_unet_s* u, const float* x) {
  const int M = u->M, N = u->N, S = u->S;
  const long long V = (long long)M * N * S, V2 = V / 8, V4 = V / 64;
  cudaStream_t st = u->stream;
  float* b = u->p;
  auto bias = [&](int l) { return b + u->off_b[l]; };
  k_to_bf16<<<grid_for(V), 256, 0, st>>>(x, u->xb, V);
  UCK(cudaGetLastError());
  UCK(conv_first(st, u->xb, u->p + u->off_w[0], bias(0), u->e1a, M, N, S));
  UCK(conv_layer(u, 1, false, cin(u->e1a, C1, 0, nullptr, 0, M, N, S), bias(1), 1, u->e1));
  k_maxpool<<<grid_for(V2 * C1 / 8), 256, 0, st>>>(u->e1, u->p1, u->i1, M, N, S, C1);
  UCK(conv_layer(u, 2, false, cin(u->p1, C1, 0, nullptr, 0, M / 2, N / 2, S / 2), bias(2), 1, u->e2a));
  UCK(conv_layer(u, 3, false, cin(u->e2a, C2, 0, nullptr, 0, M / 2, N / 2, S / 2), bias(3), 1, u->e2));
  k_maxpool<<<grid_for(V4 * C2 / 8), 256, 0, st>>>(u->e2, u->p2, u->i2, M / 2, N / 2, S / 2, C2);
  UCK(conv_layer(u, 4, false, cin(u->p2, C2, 0, nullptr, 0, M / 4, N / 4, S / 4), bias(4), 1, u->e3a));
  UCK(conv_layer(u, 5, false, cin(u->e3a, C3, 0, nullptr, 0, M / 4, N / 4, S / 4), bias(5), 1, u->e3));
  UCK(conv_layer(u, 6, false, cin(u->e3, C3, 1, u->e2, C2, M / 2, N / 2, S / 2), bias(6), 1, u->d2a));
  UCK(conv_layer(u, 7, false, cin(u->d2a, C2, 0, nullptr, 0, M / 2, N / 2, S / 2), bias(7), 1, u->d2));
  UCK(conv_layer(u, 8, false, cin(u->d2, C2, 1, u->e1, C1, M, N, S), bias(8), 1, u->d1a));
  UCK(conv_layer(u, 9, false, cin(u->d1a, C1, 0, nullptr, 0, M, N, S), bias(9), 1, u->d1));
  k_head_fwd<C1><<<grid_for(V), 256, 0, st>>>(u->d1, b + u->off_h, x, u->out, V);
  UCK(cudaGetLastError());
  return SR3D_OK;
}

// gradient of one 3x3x3 layer: gy (gradient of its output, ReLU mask applied
// here) -> weight / bias gradients; if gx, the gradient of its input
static int layer_back(sr3d_unet_s* u, int l, const ConvIn& in, bf16* gy, const bf16* y, long long V, bf16* gx) {
  const LayerShape& L = kLayers[l];
  cudaStream_t st = u->stream;
  k_relu_mask<<<grid_for(V * L.cout), 256, 0, st>>>(gy, y, V * L.cout);
  UCK(cudaGetLastError());
  UCK(cudaMemsetAsync(u->dw, 0, (size_t)L.cout * u->kpad[l] * sizeof(float), st));
  UCK(conv_wgrad(st, L.cout, in, gy, u->kpad[l], L.cin, V, u->dw));
  k_unpack_dw<<<64, 256, 0, st>>>(u->dw, L.cout, L.cin, u->kpad[l], u->g + u->off_w[l]);
  k_bias_grad<<<256, 256, 0, st>>>(gy, u->g + u->off_b[l], V, L.cout);
  UCK(cudaGetLastError());
  if (gx) {
    const ConvIn gi = cin(gy, L.cout, 0, nullptr, 0, in.M, in.N, in.S);
    UCK(conv_layer(u, l, true, gi, nullptr, 0, gx));
  }
  return SR3D_OK;
}

static int unet_backward(sr3d_unet_s* u, const float* tgt) {
  const int M = u->M, N = u->N, S = u->S;
  const long long V = (long long)M * N * S, V2 = V / 8, V4 = V / 64;
  cudaStream_t st = u->stream;
  UCK(cudaMemsetAsync(u->g, 0, (size_t)u->np * sizeof(float), st));
  UCK(cudaMemsetAsync(u->loss, 0, sizeof(double), st));
  // head
  k_head_bwd<C1><<<512, 256, 0, st>>>(u->out, tgt, u->d1, u->p + u->off_h, u->gd, u->g + u->off_h, u->loss, V);
  UCK(cudaGetLastError());
  // decoder level 1
  UTRY(layer_back(u, 9, cin(u->d1a, C1, 0, nullptr, 0, M, N, S), u->gd, u->d1, V, u->ga));  // ga: g d1a (V x 16)
  UTRY(layer_back(u, 8, cin(u->d2, C2, 1, u->e1, C1, M, N, S), u->ga, u->d1a, V, u->gb));    // gb: g c1 (V x 48)
  k_up_adj<<<grid_for(V2 * C2), 256, 0, st>>>(u->gb, C2 + C1, u->ge, M, N, S, C2);             // ge: g d2 (V2 x 32)
  // decoder level 2
  UTRY(layer_back(u, 7, cin(u->d2a, C2, 0, nullptr, 0, M / 2, N / 2, S / 2), u->ge, u->d2, V2, u->ga));  // g d2a
  UTRY(layer_back(u, 6, cin(u->e3, C3, 1, u->e2, C2, M / 2, N / 2, S / 2), u->ga, u->d2a, V2, u->gc));  // g c2 (V2 x 96)
  k_up_adj<<<grid_for(V4 * C3), 256, 0, st>>>(u->gc, C3 + C2, u->ga, M / 2, N / 2, S / 2, C3);  // ga: g e3 (V4 x 64)
  // bottleneck
  UTRY(layer_back(u, 5, cin(u->e3a, C3, 0, nullptr, 0, M / 4, N / 4, S / 4), u->ga, u->e3, V4, u->ge));  // ge: g e3a
  UTRY(layer_back(u, 4, cin(u->p2, C2, 0, nullptr, 0, M / 4, N / 4, S / 4), u->ge, u->e3a, V4, u->ga));  // ga: g p2
  // encoder level 2: g e2 = unpool(g p2) + skip part of g c2
  k_unpool_add<<<grid_for(V2 * C2), 256, 0, st>>>(u->ga, u->i2, u->gc, C3 + C2, C3, u->ge, M / 2, N / 2, S / 2, C2);
  UCK(cudaGetLastError());
  UTRY(layer_back(u, 3, cin(u->e2a, C2, 0, nullptr, 0, M / 2, N / 2, S / 2), u->ge, u->e2, V2, u->ga));  // g e2a
  UTRY(layer_back(u, 2, cin(u->p1, C1, 0, nullptr, 0, M / 2, N / 2, S / 2), u->ga, u->e2a, V2, u->gc));  // gc: g p1
  // encoder level 1: g e1 = unpool(g p1) + skip part of g c1
  k_unpool_add<<<grid_for(V * C1), 256, 0, st>>>(u->gc, u->i1, u->gb, C2 + C1, C2, u->gd, M, N, S, C1);
  UCK(cudaGetLastError());
  UTRY(layer_back(u, 1, cin(u->e1a, C1, 0, nullptr, 0, M, N, S), u->gd, u->e1, V, u->ga));  // g e1a
  UTRY(layer_back(u, 0, cin(u->xb, 1, 0, nullptr, 0, M, N, S), u->ga, u->e1a, V, nullptr));
  return SR3D_OK;
}

extern "C" {

long long sr3d_unet_param_count(void) {
  long long n = 0;
  for (const LayerShape& L : kLayers) n += (long long)L.cout * 27 * L.cin + L.cout;
  return n + C1 + 1;
}

int sr3d_unet_create(sr3d_unet_t* out, void* stream) {
  if (!out) return ufail(SR3D_ERR_INVALID_ARG, "NULL argument");
  *out = nullptr;
  sr3d_unet_s* u = new sr3d_unet_s();
  u->stream = (cudaStream_t)stream;
  u->np = sr3d_unet_param_count();
  long long o = 0;
  for (int l = 0; l < 10; ++l) {
    u->off_w[l] = o;
    o += (long long)kLayers[l].cout * 27 * kLayers[l].cin;
    u->off_b[l] = o;
    o += kLayers[l].cout;
    u->kpad[l] = ((27 * kLayers[l].cin + 15) / 16) * 16;
  }
  u->off_h = o;
  auto fin = [&](int rc) {
    if (rc != SR3D_OK) {
      sr3d_unet_destroy(u);
      return rc;
    }
    *out = u;
    return SR3D_OK;
  };
  cudaError_t e = cudaSuccess;
  if (e == cudaSuccess) e = cudaMalloc(&u->p, u->np * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&u->g, u->np * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&u->m1, u->np * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&u->m2, u->np * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&u->loss, sizeof(double));
  size_t dwmax = 0;
  for (int l = 0; l < 10 && e == cudaSuccess; ++l) {
    const size_t nw = (size_t)27 * kLayers[l].cout * kLayers[l].cin;
    if (l > 0) e = cudaMalloc(&u->wt[l], nw * sizeof(bf16));
    if (e == cudaSuccess && l > 0) e = cudaMalloc(&u->wtb[l], nw * sizeof(bf16));
    if (e == cudaSuccess && l > 0) e = cudaMalloc(&u->wu[l], nw * sizeof(bf16));
    if (e == cudaSuccess && l > 0) e = cudaMalloc(&u->wub[l], nw * sizeof(bf16));
    const size_t dws = (size_t)kLayers[l].cout * u->kpad[l];
    if (dws > dwmax) dwmax = dws;
  }
  if (e == cudaSuccess) e = cudaMalloc(&u->dw, dwmax * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&u->err, sizeof(int));
  if (e == cudaSuccess) e = cudaMemsetAsync(u->err, 0, sizeof(int), u->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(u->p, 0, u->np * sizeof(float), u->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(u->m1, 0, u->np * sizeof(float), u->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(u->m2, 0, u->np * sizeof(float), u->stream);
  if (e != cudaSuccess) return fin(ufail(e == cudaErrorMemoryAllocation ? SR3D_ERR_OOM : SR3D_ERR_CUDA, "unet create", e));
  int rc = pack_weights(u);
  if (rc == SR3D_OK) {
    e = cudaStreamSynchronize(u->stream);
    if (e != cudaSuccess) rc = ufail(SR3D_ERR_CUDA, "unet create", e);
  }
  return fin(rc);
}

int sr3d_unet_destroy(sr3d_unet_t u) {
  if (!u) return SR3D_OK;
  if (u->stream) cudaStreamSynchronize(u->stream);
  for (void* b : u->bufs) cudaFree(b);
  void* ps[] = {u->p, u->g, u->m1, u->m2, u->loss, u->dw};
  for (void* b : ps)
    if (b) cudaFree(b);
  for (int l = 0; l < 10; ++l) {
    if (u->wt[l]) cudaFree(u->wt[l]);
    if (u->wtb[l]) cudaFree(u->wtb[l]);
    if (u->wu[l]) cudaFree(u->wu[l]);
    if (u->wub[l]) cudaFree(u->wub[l]);
  }
  if (u->err) cudaFree(u->err);
  delete u;
  return SR3D_OK;
}

int sr3d_unet_set_params(sr3d_unet_t u, const float* host, long long n) {
  if (!u || !host || n != u->np) return ufail(SR3D_ERR_INVALID_ARG, "parameter count mismatch");
  UCK(cudaMemcpyAsync(u->p, host, n * sizeof(float), cudaMemcpyHostToDevice, u->stream));
  UCK(cudaMemsetAsync(u->m1, 0, n * sizeof(float), u->stream));
  UCK(cudaMemsetAsync(u->m2, 0, n * sizeof(float), u->stream));
  u->step = 0;
  UTRY(pack_weights(u));
  UCK(cudaStreamSynchronize(u->stream));
  return SR3D_OK;
}

int sr3d_unet_get_params(sr3d_unet_t u, float* host, long long n) {
  if (!u || !host || n != u->np) return ufail(SR3D_ERR_INVALID_ARG, "parameter count mismatch");
  UCK(cudaMemcpyAsync(host, u->p, n * sizeof(float), cudaMemcpyDeviceToHost, u->stream));
  UCK(cudaStreamSynchronize(u->stream));
  return SR3D_OK;
}

static int check_dims(int m, int n, int s) {
  if (m <= 0 || n <= 0 || s <= 0 || m % 4 || n % 4 || s % 4)
    return ufail(SR3D_ERR_UNSUPPORTED_SIZE, "U-Net sizes must be positive multiples of 4");
  return SR3D_OK;
}

// waits for the stream; SR3D_ERR_TIMEOUT if a bounded wait of the tcgen05
// kernel ran out (the results of that launch, and of every later launch on the
// stream, are then to be discarded)
static int finish(sr3d_unet_s* u) {
  int h = 0;
  UCK(cudaMemcpyAsync(&h, u->err, sizeof(int), cudaMemcpyDeviceToHost, u->stream));
  UCK(cudaStreamSynchronize(u->stream));
  if (h) {
    cudaMemsetAsync(u->err, 0, sizeof(int), u->stream);
    return ufail(SR3D_ERR_TIMEOUT, "a tensor-core completion wait ran out");
  }
  return SR3D_OK;
}

int sr3d_unet_set_path(sr3d_unet_t u, int path) {
  if (!u || path < SR3D_UNET_PATH_TCGEN05 || path > SR3D_UNET_PATH_TCGEN05_ALL)
    return ufail(SR3D_ERR_INVALID_ARG, "unknown convolution path");
  u->use_tc = path == SR3D_UNET_PATH_TCGEN05 ? 1 : path == SR3D_UNET_PATH_TCGEN05_ALL ? 2 : 0;
  return SR3D_OK;
}

int sr3d_unet_forward(sr3d_unet_t u, int m, int n, int s, const float* x, float* out) {
  if (!u || !x || !out) return ufail(SR3D_ERR_INVALID_ARG, "NULL argument");
  UTRY(check_dims(m, n, s));
  UTRY(ensure_size(u, m, n, s));
  UTRY(unet_forward(u, x));
  UCK(cudaMemcpyAsync(out, u->out, (size_t)m * n * s * sizeof(float), cudaMemcpyDeviceToDevice, u->stream));
  return finish(u);
}

int sr3d_unet_train_step(sr3d_unet_t u, int m, int n, int s, const float* x, const float* target, double lr,
                         double* loss, float* grad_host, int update) {
  if (!u || !x || !target) return ufail(SR3D_ERR_INVALID_ARG, "NULL argument");
  UTRY(check_dims(m, n, s));
  UTRY(ensure_size(u, m, n, s));
  UTRY(unet_forward(u, x));
  UTRY(unet_backward(u, target));
  if (grad_host) UCK(cudaMemcpyAsync(grad_host, u->g, u->np * sizeof(float), cudaMemcpyDeviceToHost, u->stream));
  if (update) {
    u->step += 1;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.f - powf(b1, (float)u->step), c2 = 1.f - powf(b2, (float)u->step);
    k_adam<<<grid_for(u->np), 256, 0, u->stream>>>(u->p, u->g, u->m1, u->m2, u->np, (float)lr, b1, b2, 1e-8f, c1, c2);
    UCK(cudaGetLastError());
    UTRY(pack_weights(u));
  }
  double l = 0;
  UCK(cudaMemcpyAsync(&l, u->loss, sizeof(double), cudaMemcpyDeviceToHost, u->stream));
  UCK(cudaStreamSynchronize(u->stream));
  if (loss) *loss = l / ((double)m * n * s);
  return finish(u);
}

int sr3d_unet_wait_selftest(sr3d_unet_t u, long long limit_cycles) {
  if (!u || limit_cycles < 1 || limit_cycles > tc::kWaitLimit)
    return ufail(SR3D_ERR_INVALID_ARG, "wait limit must be in [1, 2e9] cycles");
  k_wait_selftest<<<1, 128, 0, u->stream>>>(limit_cycles, u->err);
  UCK(cudaGetLastError());
  return finish(u);
}

int sr3d_unet_read(sr3d_unet_t u, int which, void* host, long long bytes) {
  if (!u || !host) return ufail(SR3D_ERR_INVALID_ARG, "NULL argument");
  if (!u->M) return ufail(SR3D_ERR_INVALID_ARG, "no forward pass has run");
  const long long V = (long long)u->M * u->N * u->S, V2 = V / 8, V4 = V / 64;
  const void* src[14] = {u->xb, u->e1a, u->e1, u->p1, u->e2a, u->e2, u->p2,
                         u->e3a, u->e3, u->d2a, u->d2, u->d1a, u->d1, u->out};
  const long long n[14] = {V, V * C1, V * C1, V2 * C1, V2 * C2, V2 * C2, V4 * C2,
                           V4 * C3, V4 * C3, V2 * C2, V2 * C2, V * C1, V * C1, V};
  if (which < 0 || which > 13) return ufail(SR3D_ERR_INVALID_ARG, "activation index out of range");
  const long long need = n[which] * (which == 13 ? 4 : 2);
  if (bytes != need) return ufail(SR3D_ERR_INVALID_ARG, "byte count does not match the activation");
  UCK(cudaMemcpyAsync(host, src[which], need, cudaMemcpyDeviceToHost, u->stream));
  UCK(cudaStreamSynchronize(u->stream));
  return SR3D_OK;
}

}  // extern "C"

// KKT-consistent initial dual (declared in sr3d.h; uses the plan's sizes)
namespace sr3d {
cudaError_t launch_dual_init(const Plan& p, const void* x, double thr, void* d) {
  const Geometry& g = p.hr;
  const int blocks = grid_for(g.V());
  if (p.dtype) k_dual_init<double><<<blocks, 256, 0, p.stream>>>((const double*)x, (double*)d, g.M, g.N, g.S, thr);
  else k_dual_init<float><<<blocks, 256, 0, p.stream>>>((const float*)x, (float*)d, g.M, g.N, g.S, (float)thr);
  return cudaGetLastError();
}
}  // namespace sr3d

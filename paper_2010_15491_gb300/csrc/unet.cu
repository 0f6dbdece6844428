// Learned warm start: a 3D U-Net (channels 16 / 32 / 64, 3x3x3 convolutions,
// 2x2x2 max pooling, nearest upsampling, skip concatenation, ReLU, residual
// 1x1x1 head) trained and run with the library's own kernels, plus the
// KKT-consistent initial dual for ADMM started from its output.
//
// Activations and gradients are BF16, channels last ([voxel][channel]);
// master weights, Adam moments and reductions are FP32 / FP64.  Every 3x3x3
// convolution is an implicit GEMM on the tensor cores (mma.sync m16n8k16 BF16
// with FP32 accumulation): rows are voxels, columns output channels, and the
// reduction runs over (tap, input channel) in chunks of 16 staged per warp in
// shared memory and read with ldmatrix.  The data gradient is the same kernel
// with flipped, transposed weights; the weight gradient is a second GEMM
// (channels x k over voxels) split over voxel groups.
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
// forward convolution: out[v][co] = act(bias[co] + sum_k A[v][k] W[co][k]);
// 4 warps x 32 voxels per CTA.  Also the data gradient (weights flipped and
// transposed, no bias, no activation).
// ---------------------------------------------------------------------------
template <int COUT, bool PACKED>
__global__ void __launch_bounds__(128) k_conv_fwd(ConvIn in, const bf16* __restrict__ w, int Kpad, int Cin,
                                                  const float* __restrict__ bias, int relu, bf16* __restrict__ out,
                                                  long long V) {
  __shared__ __align__(16) bf16 slab[4][2][256];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int g = lane >> 2, t = lane & 3;
  const long long vbase = ((long long)blockIdx.x * 4 + warp) * 32;
  float acc[2][COUT / 8][4];
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < COUT / 8; ++j)
#pragma unroll
      for (int e = 0; e < 4; ++e) acc[i][j][e] = 0.f;
  const int nk = Kpad / 16;
  const int lr = (lane & 7) + 8 * ((lane >> 3) & 1), lc = 8 * (lane >> 4);  // ldmatrix row / column of this lane
#pragma unroll 1
  for (int kc = 0; kc < nk; ++kc) {
    fill_slab<PACKED>(slab[warp][0], in, vbase, kc, Cin, lane);
    fill_slab<PACKED>(slab[warp][1], in, vbase + 16, kc, Cin, lane);
    __syncwarp();
    uint32_t a0[4], a1[4];
    ldsm_x4(a0, slab[warp][0] + lr * 16 + lc);
    ldsm_x4(a1, slab[warp][1] + lr * 16 + lc);
#pragma unroll
    for (int nt = 0; nt < COUT / 8; ++nt) {
      const bf16* wp = w + (long long)(nt * 8 + g) * Kpad + kc * 16 + 2 * t;
      const uint32_t b0 = __ldg(reinterpret_cast<const uint32_t*>(wp));
      const uint32_t b1 = __ldg(reinterpret_cast<const uint32_t*>(wp + 8));
      mma16816(acc[0][nt], a0, b0, b1);
      mma16816(acc[1][nt], a1, b0, b1);
    }
    __syncwarp();
  }
#pragma unroll
  for (int mt = 0; mt < 2; ++mt)
#pragma unroll
    for (int half = 0; half < 2; ++half) {
      const long long v = vbase + mt * 16 + g + 8 * half;
      if (v >= V) continue;
#pragma unroll
      for (int nt = 0; nt < COUT / 8; ++nt) {
        const int co = nt * 8 + 2 * t;
        float x0 = acc[mt][nt][2 * half], x1 = acc[mt][nt][2 * half + 1];
        if (bias) {
          x0 += bias[co];
          x1 += bias[co + 1];
        }
        if (relu) {
          x0 = fmaxf(x0, 0.f);
          x1 = fmaxf(x1, 0.f);
        }
        *reinterpret_cast<__nv_bfloat162*>(out + v * COUT + co) = __floats2bfloat162_rn(x0, x1);
      }
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

template <int CIN, int COUT, int MT>
struct Conv3Cfg {
  static constexpr int TM = 16, TN = 4, TS = 2 * MT;
  static constexpr int HM = TM + 2, HN = TN + 2, HS = TS + 2;
  static constexpr int HV = HM * HN * HS;
  static constexpr int CH = CIN / 8;           // 16-byte chunks per voxel row
  static constexpr int VST = CIN * 2 + 16;     // padded row: an odd number of chunks, conflict-free ldmatrix
  static constexpr int HALO = HV * VST;
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

// wt: [27][COUT][CIN] BF16 (tap-major slices, rows = output channel)
template <int CIN, int COUT, int MT>
__global__ void __launch_bounds__(256) k_conv3(ConvIn in, const bf16* __restrict__ wt, const float* __restrict__ bias,
                                               int relu, bf16* __restrict__ out) {
  using C = Conv3Cfg<CIN, COUT, MT>;
  extern __shared__ __align__(16) unsigned char smem[];
  unsigned char* halo = smem;
  unsigned char* wbuf = smem + C::HALO;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int g = lane >> 2, t = lane & 3;
  const int tilesM = (in.M + C::TM - 1) / C::TM, tilesN = (in.N + C::TN - 1) / C::TN;
  int b = blockIdx.x;
  const int m0 = (b % tilesM) * C::TM;
  b /= tilesM;
  const int n0 = (b % tilesN) * C::TN;
  const int s0 = (b / tilesN) * C::TS;

  for (int i = threadIdx.x; i < C::HV * C::CH; i += 256) {
    const int hv = i / C::CH, c = i - hv * C::CH;
    const int hm = hv % C::HM, r = hv / C::HM;
    const int m = m0 + hm - 1, n = n0 + r % C::HN - 1, s = s0 + r / C::HN - 1;
    const bool ok = m >= 0 && m < in.M && n >= 0 && n < in.N && s >= 0 && s < in.S;
    cpz16(halo + hv * C::VST + c * 16, ok ? chunk_ptr(in, s, n, m, c * 8) : in.src0, ok);
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
    int arow[MT];
#pragma unroll
    for (int i = 0; i < MT; ++i) {
      const int r = warp * MT + i;  // row of 16 voxels: n = r % 4, s = r / 4 within the brick
      arow[i] = (((r >> 2) + ds) * C::HN + (r & 3) + dn) * C::HM + lr + dm;
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
        ldsm_x4(a, reinterpret_cast<const bf16*>(halo + arow[i] * C::VST + (kk * 16 + lc) * 2));
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

// 2x2x2 max pooling of x (full size M, N, S, C channels); the first maximum
// in (s, n, m) order wins
__global__ void k_maxpool(const bf16* __restrict__ x, bf16* __restrict__ y, unsigned char* __restrict__ idx, int M,
                          int N, int S, int C) {
  const long long total = (long long)(M / 2) * (N / 2) * (S / 2) * C;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const int c = (int)(i % C);
    const long long v = i / C;
    const int m2 = (int)(v % (M / 2)), n2 = (int)((v / (M / 2)) % (N / 2)), s2 = (int)(v / ((long long)(M / 2) * (N / 2)));
    float best = -INFINITY;
    int bi = 0;
    for (int q = 0; q < 8; ++q) {
      const int s = 2 * s2 + (q >> 2), n = 2 * n2 + ((q >> 1) & 1), m = 2 * m2 + (q & 1);
      const float val = __bfloat162float(x[(((long long)s * N + n) * M + m) * C + c]);
      if (val > best) { best = val; bi = q; }
    }
    y[i] = __float2bfloat16(best);
    idx[i] = (unsigned char)bi;
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
    for (int c = 0; c < C; c += 2) {
      const float2 dv = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(d1 + v * C + c));
      acc += wh[c] * dv.x + wh[c + 1] * dv.y;
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

// BF16 GEMM weights: wf[co][Kpad] (k = tap*Cin + ci, zero padded) and the
// data-gradient weights wb[ci][27*Cout] with k' = tap'*Cout + co holding
// W[co][26 - tap'][ci]
__global__ void k_pack_w(const float* __restrict__ W, int Cout, int Cin, int Kpad, bf16* __restrict__ wf,
                         bf16* __restrict__ wb) {
  const int total = Cout * Kpad;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
    const int co = i / Kpad, k = i - co * Kpad;
    float val = 0.f;
    if (k < 27 * Cin) val = W[(long long)co * 27 * Cin + k];
    wf[i] = __float2bfloat16(val);
  }
  if (!wb) return;
  const int tb = Cin * 27 * Cout;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < tb; i += gridDim.x * blockDim.x) {
    const int ci = i / (27 * Cout), r = i - ci * 27 * Cout, tap = r / Cout, co = r - tap * Cout;
    wb[i] = __float2bfloat16(W[((long long)co * 27 + (26 - tap)) * Cin + ci]);
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
  bf16* wf0 = nullptr;  // first layer (one input channel): [co][Kpad] im2col weights
  bf16* wt[10] = {};    // layers 1..9: tap-major forward slices [27][co][ci]
  bf16* wtb[10] = {};   // layers 1..9: tap-major data-gradient slices [27][ci][co]
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

// first layer: one input channel, im2col k = tap (27 taps padded to 32)
static cudaError_t conv_first(cudaStream_t st, const ConvIn& in, const bf16* w, int Kpad, const float* bias,
                              bf16* out, long long V) {
  const unsigned blocks = (unsigned)((V + 127) / 128);
  k_conv_fwd<16, true><<<blocks, 128, 0, st>>>(in, w, Kpad, 1, bias, 1, out, V);
  return cudaGetLastError();
}

template <int CIN, int COUT, int MT>
static cudaError_t conv3_t(cudaStream_t st, const ConvIn& in, const bf16* wt, const float* bias, int relu, bf16* out) {
  using C = Conv3Cfg<CIN, COUT, MT>;
  cudaError_t e = cudaFuncSetAttribute(k_conv3<CIN, COUT, MT>, cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM);
  if (e != cudaSuccess) return e;
  const long long blocks = (long long)((in.M + C::TM - 1) / C::TM) * ((in.N + C::TN - 1) / C::TN) *
                           ((in.S + C::TS - 1) / C::TS);
  k_conv3<CIN, COUT, MT><<<(unsigned)blocks, 256, C::SMEM, st>>>(in, wt, bias, relu, out);
  return cudaGetLastError();
}

// 3x3x3 convolution with cin = in.c0 + in.c1 input channels (a multiple of 16)
static cudaError_t conv3(cudaStream_t st, int cin, int cout, const ConvIn& in, const bf16* wt, const float* bias,
                         int relu, bf16* out) {
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
  k_pack_w<<<64, 256, 0, u->stream>>>(u->p + u->off_w[0], kLayers[0].cout, 1, u->kpad[0], u->wf0, nullptr);
  UCK(cudaGetLastError());
  for (int l = 1; l < 10; ++l) {
    const LayerShape& L = kLayers[l];
    k_pack_w3<<<128, 256, 0, u->stream>>>(u->p + u->off_w[l], L.cout, L.cin, u->wt[l], u->wtb[l]);
    UCK(cudaGetLastError());
  }
  return SR3D_OK;
}

static int unet_forward(sr3d_unet_s* u, const float* x) {
  const int M = u->M, N = u->N, S = u->S;
  const long long V = (long long)M * N * S, V2 = V / 8, V4 = V / 64;
  cudaStream_t st = u->stream;
  float* b = u->p;
  auto bias = [&](int l) { return b + u->off_b[l]; };
  k_to_bf16<<<grid_for(V), 256, 0, st>>>(x, u->xb, V);
  UCK(cudaGetLastError());
  UCK(conv_first(st, cin(u->xb, 1, 0, nullptr, 0, M, N, S), u->wf0, u->kpad[0], bias(0), u->e1a, V));
  UCK(conv3(st, C1, C1, cin(u->e1a, C1, 0, nullptr, 0, M, N, S), u->wt[1], bias(1), 1, u->e1));
  k_maxpool<<<grid_for(V2 * C1), 256, 0, st>>>(u->e1, u->p1, u->i1, M, N, S, C1);
  UCK(conv3(st, C1, C2, cin(u->p1, C1, 0, nullptr, 0, M / 2, N / 2, S / 2), u->wt[2], bias(2), 1, u->e2a));
  UCK(conv3(st, C2, C2, cin(u->e2a, C2, 0, nullptr, 0, M / 2, N / 2, S / 2), u->wt[3], bias(3), 1, u->e2));
  k_maxpool<<<grid_for(V4 * C2), 256, 0, st>>>(u->e2, u->p2, u->i2, M / 2, N / 2, S / 2, C2);
  UCK(conv3(st, C2, C3, cin(u->p2, C2, 0, nullptr, 0, M / 4, N / 4, S / 4), u->wt[4], bias(4), 1, u->e3a));
  UCK(conv3(st, C3, C3, cin(u->e3a, C3, 0, nullptr, 0, M / 4, N / 4, S / 4), u->wt[5], bias(5), 1, u->e3));
  UCK(conv3(st, C3 + C2, C2, cin(u->e3, C3, 1, u->e2, C2, M / 2, N / 2, S / 2), u->wt[6], bias(6), 1, u->d2a));
  UCK(conv3(st, C2, C2, cin(u->d2a, C2, 0, nullptr, 0, M / 2, N / 2, S / 2), u->wt[7], bias(7), 1, u->d2));
  UCK(conv3(st, C2 + C1, C1, cin(u->d2, C2, 1, u->e1, C1, M, N, S), u->wt[8], bias(8), 1, u->d1a));
  UCK(conv3(st, C1, C1, cin(u->d1a, C1, 0, nullptr, 0, M, N, S), u->wt[9], bias(9), 1, u->d1));
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
    UCK(conv3(st, L.cout, L.cin, gi, u->wtb[l], nullptr, 0, gx));
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
  if (e == cudaSuccess) e = cudaMalloc(&u->wf0, (size_t)kLayers[0].cout * u->kpad[0] * sizeof(bf16));
  for (int l = 0; l < 10 && e == cudaSuccess; ++l) {
    const size_t nw = (size_t)27 * kLayers[l].cout * kLayers[l].cin;
    if (l > 0) e = cudaMalloc(&u->wt[l], nw * sizeof(bf16));
    if (e == cudaSuccess && l > 0) e = cudaMalloc(&u->wtb[l], nw * sizeof(bf16));
    const size_t dws = (size_t)kLayers[l].cout * u->kpad[l];
    if (dws > dwmax) dwmax = dws;
  }
  if (e == cudaSuccess) e = cudaMalloc(&u->dw, dwmax * sizeof(float));
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
  if (u->wf0) cudaFree(u->wf0);
  for (int l = 0; l < 10; ++l) {
    if (u->wt[l]) cudaFree(u->wt[l]);
    if (u->wtb[l]) cudaFree(u->wtb[l]);
  }
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

int sr3d_unet_forward(sr3d_unet_t u, int m, int n, int s, const float* x, float* out) {
  if (!u || !x || !out) return ufail(SR3D_ERR_INVALID_ARG, "NULL argument");
  UTRY(check_dims(m, n, s));
  UTRY(ensure_size(u, m, n, s));
  UTRY(unet_forward(u, x));
  UCK(cudaMemcpyAsync(out, u->out, (size_t)m * n * s * sizeof(float), cudaMemcpyDeviceToDevice, u->stream));
  UCK(cudaStreamSynchronize(u->stream));
  return SR3D_OK;
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
  return SR3D_OK;
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

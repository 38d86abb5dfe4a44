// Learned second preconditioner stage: a small 3D convolutional network N applied after
// the direct second-order preconditioner M (Eq. 3DAP) inside flexible GMRES,
//
//     z = M^-1 u + c s N((u - A M^-1 u) / s),   s = sqrt(mean |u - A M^-1 u|^2),
//
// with A the sixth-order operator (Eq. scheme).  The paper has no such stage.
//
// Network: 4 layers of zero-padded 3x3x3 cross-correlation, channels 2-16-16-16-2, bias,
// GELU x Phi(x) after layers 1-3.  Channel 0/1 = real/imaginary part.  Parameters are one
// flat FP32 vector (per layer W[c_out][c_in][dz][dy][dx], then b[c_out]); the kernels use
// BF16-rounded weights, BF16 activations between layers, FP32 accumulation, FP32 biases.
//
// Kernels (SIMT, one output point per thread, 32x4x2-point tiles with the input halo and
// all taps of a layer staged in shared memory as FP32):
//   conv_kernel   forward layer; also the input gradient (the transpose of a zero-padded
//                 correlation is the correlation with the flipped, channel-transposed taps)
//   wgrad_kernel  weight and bias gradients, block partials over persistent tiles
//   mse_kernel, adam_kernel, prep_kernel (BF16 taps in both layouts from the master vector)
#include <cuda_bf16.h>

#include <cmath>
#include <cstring>
#include <vector>

#include "helm6_internal.h"

namespace helm6 {

namespace {

constexpr int TXc = 32, TYc = 4, TZc = 2, NT = TXc * TYc * TZc;  // output tile, threads per block
constexpr int HX = TXc + 2, HY = TYc + 2, HZ = TZc + 2, HP = HX * HY * HZ;
constexpr int NL = 4;
// channels entering layer l (l = 0..3) and leaving the last one (l = 4)
__host__ __device__ constexpr int ch(int l) { return (l == 0 || l == NL) ? 2 : 16; }

// halo floats per point (16 channels padded to 20: conflict-free 16-byte shared loads)
template <int C>
struct PStride {
  static constexpr int v = (C == 16) ? 20 : C;
};

enum { IN_F32 = 0, IN_BF16 = 1, IN_PLANAR = 2 };
enum { OUT_HIDDEN = 0, OUT_F32 = 1, OUT_FIELD = 2, OUT_GRAD = 3 };

struct ConvArgs {
  int nb, nz, ny, nx;  // images and their size (x fastest, channel-last)
  int tx, ty, tz;      // tiles per axis
  const void* in;
  int round_in;        // IN_F32: round the input to BF16 first
  const float* w;      // taps [27][CIN][COUT]
  const float* bias;   // [COUT] or null
  float* pre;          // OUT_HIDDEN: FP32 pre-activations written (nullable); OUT_GRAD: read
  void* out;
  const double* sumsq;  // IN_PLANAR and OUT_FIELD: sum of |t|^2 over the input field
  float out_scale;      // OUT_FIELD: c
};

__device__ __forceinline__ float bf16r(float v) { return __bfloat162float(__float2bfloat16_rn(v)); }
__device__ __forceinline__ float gelu_f(float x) { return 0.5f * x * (1.f + erff(x * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_df(float x) {
  return 0.5f * (1.f + erff(x * 0.70710678118654752f)) + x * 0.39894228040143268f * expf(-0.5f * x * x);
}
__device__ __forceinline__ uint32_t pack_bf16(float a, float b) {
  const __nv_bfloat16 lo = __float2bfloat16_rn(a), hi = __float2bfloat16_rn(b);
  uint16_t l, h;
  memcpy(&l, &lo, 2);
  memcpy(&h, &hi, 2);
  return (uint32_t)l | ((uint32_t)h << 16);
}
__device__ __forceinline__ float bf16_lo(uint32_t v) { return __uint_as_float(v << 16); }
__device__ __forceinline__ float bf16_hi(uint32_t v) { return __uint_as_float(v & 0xffff0000u); }

// tile index -> (image, z0, y0, x0) of the output tile
__device__ __forceinline__ void tile_origin(const ConvArgs& a, int64_t tile, int& img, int& z0, int& y0, int& x0) {
  const int bx = (int)(tile % a.tx);
  tile /= a.tx;
  const int by = (int)(tile % a.ty);
  tile /= a.ty;
  const int bz = (int)(tile % a.tz);
  img = (int)(tile / a.tz);
  x0 = bx * TXc;
  y0 = by * TYc;
  z0 = bz * TZc;
}

__device__ __forceinline__ float plane_scale(const ConvArgs& a, int64_t npts) {
  const double ss = *a.sumsq;
  return ss > 0.0 ? (float)(1.0 / sqrt(ss / (double)npts)) : 0.f;
}

// Stage the input halo of one tile into sx (HP points x PStride<CIN> floats).
template <int CIN, int IN>
__device__ __forceinline__ void load_halo(const ConvArgs& a, int img, int z0, int y0, int x0, float sc,
                                          float* sx) {
  constexpr int PS = PStride<CIN>::v;
  const int64_t npts = (int64_t)a.nb * a.nz * a.ny * a.nx;
  for (int i = threadIdx.x; i < HP; i += NT) {
    const int hx = i % HX, r = i / HX, hy = r % HY, hz = r / HY;
    const int gx = x0 + hx - 1, gy = y0 + hy - 1, gz = z0 + hz - 1;
    const bool ok = gx >= 0 && gx < a.nx && gy >= 0 && gy < a.ny && gz >= 0 && gz < a.nz;
    const int64_t p = (((int64_t)img * a.nz + gz) * a.ny + gy) * a.nx + gx;
    float* d = sx + i * PS;
    if constexpr (IN == IN_PLANAR) {
      const float* f = (const float*)a.in;
      d[0] = ok ? bf16r(f[p] * sc) : 0.f;
      d[1] = ok ? bf16r(f[npts + p] * sc) : 0.f;
    } else if constexpr (IN == IN_BF16) {
      static_assert(IN != IN_BF16 || CIN == 16, "BF16 activations carry 16 channels");
      uint4 q0 = make_uint4(0, 0, 0, 0), q1 = q0;
      if (ok) {
        const uint4* s = (const uint4*)a.in + 2 * p;
        q0 = s[0];
        q1 = s[1];
      }
      float4* d4 = (float4*)d;
      d4[0] = make_float4(bf16_lo(q0.x), bf16_hi(q0.x), bf16_lo(q0.y), bf16_hi(q0.y));
      d4[1] = make_float4(bf16_lo(q0.z), bf16_hi(q0.z), bf16_lo(q0.w), bf16_hi(q0.w));
      d4[2] = make_float4(bf16_lo(q1.x), bf16_hi(q1.x), bf16_lo(q1.y), bf16_hi(q1.y));
      d4[3] = make_float4(bf16_lo(q1.z), bf16_hi(q1.z), bf16_lo(q1.w), bf16_hi(q1.w));
    } else {
      const float* f = (const float*)a.in + p * CIN;
      if constexpr (CIN == 16) {
        float4* d4 = (float4*)d;
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          float4 v = ok ? ((const float4*)f)[c] : make_float4(0.f, 0.f, 0.f, 0.f);
          if (a.round_in) v = make_float4(bf16r(v.x), bf16r(v.y), bf16r(v.z), bf16r(v.w));
          d4[c] = v;
        }
      } else {
#pragma unroll
        for (int c = 0; c < CIN; ++c) {
          const float v = ok ? f[c] : 0.f;
          d[c] = a.round_in ? bf16r(v) : v;
        }
      }
    }
  }
}

template <int CIN, int COUT, int IN, int OUT>
__global__ void __launch_bounds__(NT, 2) conv_kernel(ConvArgs a) {
  extern __shared__ __align__(16) float smem[];
  constexpr int PS = PStride<CIN>::v;
  float* sw = smem;                  // 27 * CIN * COUT
  float* sx = smem + 27 * CIN * COUT;  // HP * PS (27*CIN*COUT is a multiple of 4)
  const int tid = threadIdx.x;
  const int64_t npts = (int64_t)a.nb * a.nz * a.ny * a.nx;
  for (int i = tid; i < 27 * CIN * COUT; i += NT) sw[i] = a.w[i];
  int img, z0, y0, x0;
  tile_origin(a, blockIdx.x, img, z0, y0, x0);
  const float sc = (IN == IN_PLANAR) ? plane_scale(a, npts) : 1.f;
  load_halo<CIN, IN>(a, img, z0, y0, x0, sc, sx);
  __syncthreads();

  const int lx = tid % TXc, ly = (tid / TXc) % TYc, lz = tid / (TXc * TYc);
  float acc[COUT];
#pragma unroll
  for (int o = 0; o < COUT; ++o) acc[o] = a.bias ? a.bias[o] : 0.f;
  const int base = (lz * HY + ly) * HX + lx;
#pragma unroll 1
  for (int t = 0; t < 27; ++t) {
    const int dz = t / 9, dy = (t / 3) % 3, dx = t % 3;
    const float* xp = sx + (base + (dz * HY + dy) * HX + dx) * PS;
    const float* wp = sw + t * CIN * COUT;
    float xv[CIN];
    if constexpr (CIN == 16) {
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const float4 v = ((const float4*)xp)[c];
        xv[4 * c] = v.x;
        xv[4 * c + 1] = v.y;
        xv[4 * c + 2] = v.z;
        xv[4 * c + 3] = v.w;
      }
    } else {
#pragma unroll
      for (int c = 0; c < CIN; ++c) xv[c] = xp[c];
    }
#pragma unroll
    for (int ci = 0; ci < CIN; ++ci) {
      if constexpr (COUT == 16) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const float4 w4 = ((const float4*)(wp + ci * COUT))[q];
          acc[4 * q] = fmaf(xv[ci], w4.x, acc[4 * q]);
          acc[4 * q + 1] = fmaf(xv[ci], w4.y, acc[4 * q + 1]);
          acc[4 * q + 2] = fmaf(xv[ci], w4.z, acc[4 * q + 2]);
          acc[4 * q + 3] = fmaf(xv[ci], w4.w, acc[4 * q + 3]);
        }
      } else {
#pragma unroll
        for (int o = 0; o < COUT; ++o) acc[o] = fmaf(xv[ci], wp[ci * COUT + o], acc[o]);
      }
    }
  }

  const int gx = x0 + lx, gy = y0 + ly, gz = z0 + lz;
  if (gx >= a.nx || gy >= a.ny || gz >= a.nz) return;
  const int64_t p = (((int64_t)img * a.nz + gz) * a.ny + gy) * a.nx + gx;
  if constexpr (OUT == OUT_HIDDEN) {
    static_assert(OUT != OUT_HIDDEN || COUT == 16, "hidden layers have 16 channels");
    if (a.pre) {
      float4* pr = (float4*)(a.pre + p * 16);
#pragma unroll
      for (int q = 0; q < 4; ++q) pr[q] = make_float4(acc[4 * q], acc[4 * q + 1], acc[4 * q + 2], acc[4 * q + 3]);
    }
    uint32_t pk[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) pk[q] = pack_bf16(gelu_f(acc[2 * q]), gelu_f(acc[2 * q + 1]));
    uint4* o4 = (uint4*)a.out + 2 * p;
    o4[0] = make_uint4(pk[0], pk[1], pk[2], pk[3]);
    o4[1] = make_uint4(pk[4], pk[5], pk[6], pk[7]);
  } else if constexpr (OUT == OUT_F32) {
    float* o = (float*)a.out + p * COUT;
#pragma unroll
    for (int c = 0; c < COUT; ++c) o[c] = acc[c];
  } else if constexpr (OUT == OUT_GRAD) {
    const float* pr = a.pre + p * COUT;
    float* o = (float*)a.out + p * COUT;
#pragma unroll
    for (int c = 0; c < COUT; ++c) o[c] = acc[c] * gelu_df(pr[c]);
  } else {  // OUT_FIELD: z += c s y on the planar complex field
    static_assert(OUT != OUT_FIELD || COUT == 2, "the field output has 2 channels");
    const double ss = *a.sumsq;
    if (!(ss > 0.0)) return;
    const float cs = a.out_scale * (float)sqrt(ss / (double)npts);
    float* z = (float*)a.out;
    z[p] = fmaf(cs, acc[0], z[p]);
    z[npts + p] = fmaf(cs, acc[1 % COUT], z[npts + p]);
  }
}

// Weight and bias gradients of one layer: dW[t][ci][co] = sum_p in[p + d_t][ci] g[p][co],
// db[co] = sum_p g[p][co].  Persistent blocks over tiles, one partial row per block.
template <int CIN, int COUT, int IN>
__global__ void __launch_bounds__(NT) wgrad_kernel(ConvArgs a, const float* __restrict__ g,
                                                   float* __restrict__ partial, int64_t ntiles) {
  extern __shared__ __align__(16) float smem[];
  constexpr int PS = PStride<CIN>::v;
  constexpr int E = 27 * CIN * COUT;
  constexpr int KE = (E + NT - 1) / NT;
  float* sx = smem;            // HP * PS
  float* sg = smem + HP * PS;  // NT * COUT
  const int tid = threadIdx.x;
  int xo[KE], go[KE];
  float acc[KE];
#pragma unroll
  for (int k = 0; k < KE; ++k) {
    const int e = (tid + k * NT < E) ? tid + k * NT : 0;  // entries past E read entry 0, unused
    const int t = e / (CIN * COUT), r = e % (CIN * COUT);
    const int ci = r / COUT, co = r % COUT;
    const int dz = t / 9, dy = (t / 3) % 3, dx = t % 3;
    xo[k] = ((dz * HY + dy) * HX + dx) * PS + ci;
    go[k] = co;
    acc[k] = 0.f;
  }
  float bacc = 0.f;
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    int img, z0, y0, x0;
    tile_origin(a, tile, img, z0, y0, x0);
    load_halo<CIN, IN>(a, img, z0, y0, x0, 1.f, sx);
    {
      const int lx = tid % TXc, ly = (tid / TXc) % TYc, lz = tid / (TXc * TYc);
      const int gx = x0 + lx, gy = y0 + ly, gz = z0 + lz;
      const bool ok = gx < a.nx && gy < a.ny && gz < a.nz;
      const int64_t p = (((int64_t)img * a.nz + gz) * a.ny + gy) * a.nx + gx;
#pragma unroll
      for (int c = 0; c < COUT; ++c) sg[tid * COUT + c] = ok ? g[p * COUT + c] : 0.f;
    }
    __syncthreads();
#pragma unroll 2
    for (int q = 0; q < NT; ++q) {
      const int hb = ((q / (TXc * TYc)) * HY + (q / TXc) % TYc) * HX + q % TXc;
      const float* xq = sx + hb * PS;
      const float* gq = sg + q * COUT;
#pragma unroll
      for (int k = 0; k < KE; ++k)
        if (KE * NT == E || tid + k * NT < E) acc[k] = fmaf(xq[xo[k]], gq[go[k]], acc[k]);
    }
    if (tid < COUT)
      for (int q = 0; q < NT; ++q) bacc += sg[q * COUT + tid];
    __syncthreads();
  }
  float* row = partial + (int64_t)blockIdx.x * (E + COUT);
#pragma unroll
  for (int k = 0; k < KE; ++k)
    if (tid + k * NT < E) row[tid + k * NT] = acc[k];
  if (tid < COUT) row[E + tid] = bacc;
}

// grad[flat] = sum over blocks of the partial rows, entries mapped from the kernel's
// [t][ci][co] order to the parameter vector's [co][ci][t] order; biases follow.
__global__ void wgrad_reduce_kernel(const float* __restrict__ partial, int nblk, int cin, int cout,
                                    float* __restrict__ grad_w, float* __restrict__ grad_b) {
  const int E = 27 * cin * cout;
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= E + cout) return;
  double s = 0.0;
  for (int b = 0; b < nblk; ++b) s += partial[(int64_t)b * (E + cout) + e];
  if (e < E) {
    const int t = e / (cin * cout), r = e % (cin * cout), ci = r / cout, co = r % cout;
    grad_w[(co * cin + ci) * 27 + t] = (float)s;
  } else {
    grad_b[e - E] = (float)s;
  }
}

// g = 2 (y - t) / n and block partial sums of (y - t)^2.
__global__ void mse_kernel(const float* __restrict__ y, const float* __restrict__ t, int64_t n,
                           float* __restrict__ g, double* __restrict__ partial) {
  __shared__ double sh[32];
  double acc = 0.0;
  const float sc = (float)(2.0 / (double)n);
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const float d = y[i] - t[i];
    g[i] = sc * d;
    acc += (double)d * d;
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x < 32) {
    acc = (threadIdx.x < blockDim.x / 32) ? sh[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (threadIdx.x == 0) partial[blockIdx.x] = acc;
  }
}

// Adam (beta1 0.9, beta2 0.999, eps 1e-8) with bias corrections c1 = 1 - beta1^t, c2 = 1 - beta2^t.
__global__ void adam_kernel(float* __restrict__ theta, float* __restrict__ m, float* __restrict__ v,
                            const float* __restrict__ g, int n, float lr, float c1, float c2) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = g[i];
  const float mi = 0.9f * m[i] + 0.1f * gi;
  const float vi = 0.999f * v[i] + 0.001f * gi * gi;
  m[i] = mi;
  v[i] = vi;
  theta[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + 1e-8f);
}

// Interior 27-point operator on channel-last complex patches [pts][2] with zero values
// outside each image: out = scale * sum over the 27 offsets of w[class] * y[p + d], class
// = number of nonzero offset components (centre, face, edge, corner).  The caller
// conjugates the weights for the adjoint.
struct PatchW {
  float re[4], im[4];
};

__global__ void patch_op_kernel(int nb, int nz, int ny, int nx, const float* __restrict__ y, float* __restrict__ out,
                                PatchW w, float scale) {
  const int64_t npts = (int64_t)nb * nz * ny * nx;
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= npts) return;
  const int x = (int)(p % nx);
  int64_t r = p / nx;
  const int yy = (int)(r % ny);
  r /= ny;
  const int z = (int)(r % nz);
  float ar = 0.f, ai = 0.f;
  for (int dz = -1; dz <= 1; ++dz) {
    if (z + dz < 0 || z + dz >= nz) continue;
    for (int dy = -1; dy <= 1; ++dy) {
      if (yy + dy < 0 || yy + dy >= ny) continue;
      for (int dx = -1; dx <= 1; ++dx) {
        if (x + dx < 0 || x + dx >= nx) continue;
        const int cls = (dz != 0) + (dy != 0) + (dx != 0);
        const float2 v = ((const float2*)y)[p + ((int64_t)dz * ny + dy) * nx + dx];
        ar = fmaf(w.re[cls], v.x, fmaf(-w.im[cls], v.y, ar));
        ai = fmaf(w.re[cls], v.y, fmaf(w.im[cls], v.x, ai));
      }
    }
  }
  ((float2*)out)[p] = make_float2(scale * ar, scale * ai);
}

// R = (Ay - x) at interior points (1 away from every image face), 0 elsewhere, and block
// partial sums of |R|^2.
__global__ void resid_loss_kernel(int nb, int nz, int ny, int nx, const float* __restrict__ Ay,
                                  const float* __restrict__ x, float* __restrict__ R, double* __restrict__ partial) {
  __shared__ double sh[32];
  const int64_t npts = (int64_t)nb * nz * ny * nx;
  double acc = 0.0;
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < npts; p += (int64_t)gridDim.x * blockDim.x) {
    const int xi = (int)(p % nx);
    int64_t r = p / nx;
    const int yi = (int)(r % ny);
    r /= ny;
    const int zi = (int)(r % nz);
    const bool in = xi > 0 && xi < nx - 1 && yi > 0 && yi < ny - 1 && zi > 0 && zi < nz - 1;
    float2 d = make_float2(0.f, 0.f);
    if (in) {
      const float2 a = ((const float2*)Ay)[p], b = ((const float2*)x)[p];
      d = make_float2(a.x - b.x, a.y - b.y);
      acc += (double)d.x * d.x + (double)d.y * d.y;
    }
    ((float2*)R)[p] = d;
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x < 32) {
    acc = (threadIdx.x < blockDim.x / 32) ? sh[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (threadIdx.x == 0) partial[blockIdx.x] = acc;
  }
}

// ---------------------------------------------------------------------------------------
// Tensor-core layer for the field path (tcgen05, BF16 operands, FP32 accumulation in TMEM).
// Implicit GEMM: per 128-point tile, D[128 x 16] = sum over the 27 taps of A_t W_t^T with
// A_t the input rows shifted by the tap's offset (K = 16 input channels) and W_t the
// 16 x 16 taps (layers with 2 channels are zero-padded to 16).  A CTA owns a brick of
// 30 x 8 x 4 output points; its 32 x 10 x 6 input halo sits in shared memory as two
// channel planes (channels 0-7 and 8-15, 16 bytes per point, points x fastest), the
// no-swizzle K-major layout: a core matrix is 8 consecutive points of one plane (128 B),
// the K step between the planes is the plane distance and the step between 8-row groups
// is 128 B, so every tap's A operand is the same descriptor with its start address moved
// by the tap offset.  The 8 tiles (4 halo rows x 32 points each: y rows 1-4 and 5-8 of
// z planes 1-4) accumulate in 8 x 16 TMEM columns; outputs at halo columns are computed
// and dropped.
constexpr int BX = 30, BY = 8, BZ = 4;                       // output points of a brick
constexpr int GX = BX + 2, GY = BY + 2, GZ = BZ + 2, GP = GX * GY * GZ;  // halo (GX = 32)
constexpr int TC_TILES = BZ * BY / 4;                         // 128-point tiles of a brick
constexpr int PLANE_B = (GP + 2) * 16;                        // one point of padding each end
constexpr int TCW_TAP = 512;                                  // bytes of one tap's 16 x 16 BF16
constexpr size_t TC_SMEM = 1024 + 2 * (size_t)PLANE_B + 27 * TCW_TAP + 256;
constexpr int kConvPolls = 1 << 22;

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory descriptor, no swizzle: start, K-direction step (lbo), 8-row step (sbo).
__device__ __forceinline__ uint64_t desc_noswz(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = (uint64_t)((addr & 0x3FFFFu) >> 4);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem, uint64_t a, uint64_t b, uint32_t id, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
      "l"(a), "l"(b), "r"(id), "r"(acc));
}

__device__ __forceinline__ void cp16(uint32_t dst, const void* src, bool ok) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(ok ? 16 : 0) : "memory");
}

struct TcConvArgs {
  int nz, ny, nx;
  int bx, by, bz;        // bricks per axis
  const void* in;        // IN_BF16: [N][16] BF16; IN_PLANAR: planar FP32 complex field
  const uint16_t* w;     // 27 taps of 16 x 16 BF16 in the canonical layout
  const float* bias;     // [c_out] (c_out = 16, or 2 for the field output)
  void* out;             // OUT_HIDDEN: [N][16] BF16; OUT_FIELD: planar FP32 z (updated)
  const double* sumsq;   // IN_PLANAR / OUT_FIELD: sum |t|^2
  float out_scale;
  int* err;              // set if the MMA completion wait timed out
};

template <int IN, int OUT>
__global__ void __launch_bounds__(128) conv_tc_kernel(TcConvArgs a) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* sm = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint8_t* plane0 = sm + 16;               // point -1 at sm, point 0 at sm + 16
  uint8_t* plane1 = plane0 + PLANE_B;
  uint8_t* wts = sm + 2 * PLANE_B;         // 27 x 512 B (1024-aligned base + 2 * PLANE_B: 16-aligned)
  uint64_t* bar = (uint64_t*)(wts + 27 * TCW_TAP);
  uint32_t* tslot = (uint32_t*)(bar + 1);
  int* fail = (int*)(tslot + 1);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int64_t npts = (int64_t)a.nz * a.ny * a.nx;

  int64_t b = blockIdx.x;
  const int ibx = (int)(b % a.bx);
  b /= a.bx;
  const int iby = (int)(b % a.by);
  const int ibz = (int)(b / a.by);
  const int x0 = ibx * BX - 1, y0 = iby * BY - 1, z0 = ibz * BZ - 1;  // global coordinate of halo (0,0,0)

  // weights: 27 x 512 B
  for (int i = tid; i < 27 * TCW_TAP / 16; i += 128) cp16(smem_u32(wts) + 16u * i, (const uint4*)a.w + i, true);
  // halo planes
  float sc = 1.f;
  if constexpr (IN == IN_PLANAR) {
    const double ss = *a.sumsq;
    sc = ss > 0.0 ? (float)(1.0 / sqrt(ss / (double)npts)) : 0.f;
  }
  for (int i = tid; i < GP; i += 128) {
    const int hx = i % GX, r = i / GX, hy = r % GY, hz = r / GY;
    const int gx = x0 + hx, gy = y0 + hy, gz = z0 + hz;
    const bool ok = gx >= 0 && gx < a.nx && gy >= 0 && gy < a.ny && gz >= 0 && gz < a.nz;
    const int64_t p = ok ? ((int64_t)gz * a.ny + gy) * a.nx + gx : 0;
    if constexpr (IN == IN_BF16) {
      const uint4* src = (const uint4*)a.in + 2 * p;
      cp16(smem_u32(plane0) + 16u * i, src, ok);
      cp16(smem_u32(plane1) + 16u * i, src + 1, ok);
    } else {
      const float* f = (const float*)a.in;
      const float re = ok ? f[p] * sc : 0.f, im = ok ? f[npts + p] * sc : 0.f;
      *(uint4*)(plane0 + 16 * i) = make_uint4(pack_bf16(re, im), 0u, 0u, 0u);
      *(uint4*)(plane1 + 16 * i) = make_uint4(0u, 0u, 0u, 0u);
    }
  }
  if (tid < 2) {  // the padding points before and after each plane
    *(uint4*)(sm + tid * PLANE_B) = make_uint4(0u, 0u, 0u, 0u);
    *(uint4*)(plane0 + tid * PLANE_B + 16 * GP) = make_uint4(0u, 0u, 0u, 0u);
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(1));
    asm volatile("fence.mbarrier_init.release.cluster;");
    *fail = 0;
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                 "r"(128));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("cp.async.wait_all;" ::: "memory");
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = *tslot;

  if (tid == 0) {
    // kind::f16, D = F32, A = B = BF16, K-major, M = 128, N = 16
    const uint32_t id = (1u << 4) | (1u << 7) | (1u << 10) | (2u << 17) | (8u << 24);
    const uint32_t p0 = smem_u32(plane0);
    for (int tile = 0; tile < TC_TILES; ++tile) {
      const int hz = 1 + tile / (BY / 4), hy = 1 + 4 * (tile % (BY / 4));
      const int q0 = (hz * GY + hy) * GX;
      for (int t = 0; t < 27; ++t) {
        const int dz = t / 9 - 1, dy = (t / 3) % 3 - 1, dx = t % 3 - 1;
        const int q = q0 + (dz * GY + dy) * GX + dx;  // in [-1, GP - 128]: the padding covers -1 and GP
        const uint64_t ad = desc_noswz(p0 + (uint32_t)(q * 16), PLANE_B, 128);
        const uint64_t bd = desc_noswz(smem_u32(wts) + (uint32_t)(t * TCW_TAP), 128, 256);
        mma_bf16(tmem + 16u * tile, ad, bd, id, t > 0 ? 1u : 0u);
      }
    }
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
  }
  __syncthreads();
  bool ok = false;
  for (int it = 0; it < kConvPolls; ++it) {
    uint32_t r;
    asm volatile(
        "{\n .reg .pred P1;\n mbarrier.try_wait.parity.shared::cta.b64 P1, [%1], %2;\n"
        " selp.b32 %0, 1, 0, P1;\n}\n"
        : "=r"(r)
        : "r"(smem_u32(bar)), "r"(0)
        : "memory");
    if (r) {
      ok = true;
      break;
    }
  }
  asm volatile("tcgen05.fence::after_thread_sync;");
  if (!ok) {
    *fail = 1;
  } else {
    float bias[16];
#pragma unroll
    for (int c = 0; c < 16; ++c) bias[c] = (OUT == OUT_HIDDEN || c < 2) ? a.bias[c] : 0.f;
    float cs = 0.f;
    if constexpr (OUT == OUT_FIELD) {
      const double ss = *a.sumsq;
      cs = ss > 0.0 ? a.out_scale * (float)sqrt(ss / (double)npts) : 0.f;
    }
    for (int tile = 0; tile < TC_TILES; ++tile) {
      uint32_t v[16];
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
          : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
            "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
          : "r"(tmem + ((uint32_t)(32 * warp) << 16) + 16u * tile));
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      const int r = 32 * warp + lane;  // row of the tile: halo x = r % 32, y = hy + r / 32
      const int hx = r % GX, hz = 1 + tile / (BY / 4), hy = 1 + 4 * (tile % (BY / 4)) + r / GX;
      const int gx = x0 + hx, gy = y0 + hy, gz = z0 + hz;
      if (hx < 1 || hx > BX || gx >= a.nx || gy >= a.ny || gz >= a.nz) continue;
      const int64_t p = ((int64_t)gz * a.ny + gy) * a.nx + gx;
      if constexpr (OUT == OUT_HIDDEN) {
        uint32_t pk[8];
#pragma unroll
        for (int q = 0; q < 8; ++q)
          pk[q] = pack_bf16(gelu_f(__uint_as_float(v[2 * q]) + bias[2 * q]),
                            gelu_f(__uint_as_float(v[2 * q + 1]) + bias[2 * q + 1]));
        uint4* o4 = (uint4*)a.out + 2 * p;
        o4[0] = make_uint4(pk[0], pk[1], pk[2], pk[3]);
        o4[1] = make_uint4(pk[4], pk[5], pk[6], pk[7]);
      } else {
        float* z = (float*)a.out;
        z[p] = fmaf(cs, __uint_as_float(v[0]) + bias[0], z[p]);
        z[npts + p] = fmaf(cs, __uint_as_float(v[1]) + bias[1], z[npts + p]);
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(128));
  if (tid == 0 && *fail) atomicExch(a.err, 1);
}

// Canonical tensor-core taps of every layer: layer l, tap t, 16 x 16 BF16 with c_out rows
// and c_in columns zero-padded to 16, stored [c_out / 8][c_in / 8][c_out % 8][c_in % 8].
__global__ void prep_tc_kernel(const float* __restrict__ theta, uint16_t* __restrict__ wtc) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;  // over 4 layers x 27 taps x 256
  if (i >= NL * 27 * 256) return;
  const int l = i / (27 * 256), t = (i / 256) % 27, e = i % 256;
  const int co = e / 16, ci = e % 16;
  int toff = 0;
  for (int q = 0; q < l; ++q) toff += 27 * ch(q) * ch(q + 1) + ch(q + 1);
  const int cin = ch(l), cout = ch(l + 1);
  const float w = (co < cout && ci < cin) ? theta[toff + (co * cin + ci) * 27 + t] : 0.f;
  const __nv_bfloat16 b16 = __float2bfloat16_rn(w);
  uint16_t u;
  memcpy(&u, &b16, 2);
  wtc[(l * 27 + t) * 256 + ((co / 8) * 2 + ci / 8) * 64 + (co % 8) * 8 + (ci % 8)] = u;
}

struct LayerDims {
  int cin[NL], cout[NL], toff[NL], boff[NL], woff[NL];
};

__host__ __device__ inline LayerDims layer_dims() {
  LayerDims d{};
  int t = 0, w = 0;
  for (int l = 0; l < NL; ++l) {
    d.cin[l] = ch(l);
    d.cout[l] = ch(l + 1);
    d.toff[l] = t;
    d.boff[l] = t + 27 * ch(l) * ch(l + 1);
    d.woff[l] = w;
    t = d.boff[l] + ch(l + 1);
    w += 27 * ch(l) * ch(l + 1);
  }
  return d;
}

// BF16-rounded taps of every layer in the forward layout [t][ci][co] (wf) and in the
// input-gradient layout [t'][co][ci] with t' = 26 - t (wb).
__global__ void prep_kernel(const float* __restrict__ theta, float* __restrict__ wf, float* __restrict__ wb) {
  const LayerDims d = layer_dims();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  for (int l = 0; l < NL; ++l) {
    const int n = 27 * d.cin[l] * d.cout[l];
    if (i >= n) continue;
    const int ci_n = d.cin[l], co_n = d.cout[l];
    // forward entry i = (t * cin + ci) * cout + co
    {
      const int t = i / (ci_n * co_n), r = i % (ci_n * co_n), ci = r / co_n, co = r % co_n;
      wf[d.woff[l] + i] = bf16r(theta[d.toff[l] + (co * ci_n + ci) * 27 + t]);
    }
    // input-gradient entry i = (t' * cout + co) * cin + ci
    {
      const int t2 = i / (ci_n * co_n), r = i % (ci_n * co_n), co = r / ci_n, ci = r % ci_n;
      wb[d.woff[l] + i] = bf16r(theta[d.toff[l] + (co * ci_n + ci) * 27 + (26 - t2)]);
    }
  }
}

constexpr int kWeights = 27 * (2 * 16 + 16 * 16 + 16 * 16 + 16 * 2);  // 15552 taps
static_assert(kWeights + 16 + 16 + 16 + 2 == HELM6_CNN_NPARAMS, "parameter count");

template <int CIN, int COUT>
constexpr size_t conv_smem() {
  return sizeof(float) * (27 * CIN * COUT + HP * PStride<CIN>::v);
}
template <int CIN, int COUT>
constexpr size_t wgrad_smem() {
  return sizeof(float) * (HP * PStride<CIN>::v + NT * COUT);
}

template <int CIN, int COUT, int IN, int OUT>
cudaError_t launch_conv(const ConvArgs& a, cudaStream_t s) {
  const size_t sm = conv_smem<CIN, COUT>();
  static bool configured = false;
  if (!configured) {
    cudaError_t e = cudaFuncSetAttribute(conv_kernel<CIN, COUT, IN, OUT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)sm);
    if (e != cudaSuccess) return e;
    configured = true;
  }
  const int64_t tiles = (int64_t)a.tx * a.ty * a.tz * a.nb;
  note_launch();
  conv_kernel<CIN, COUT, IN, OUT><<<(unsigned)tiles, NT, sm, s>>>(a);
  return cudaGetLastError();
}

template <int CIN, int COUT, int IN>
cudaError_t launch_wgrad(const ConvArgs& a, const float* g, float* partial, int nblk, cudaStream_t s) {
  const size_t sm = wgrad_smem<CIN, COUT>();
  static bool configured = false;
  if (!configured) {
    cudaError_t e =
        cudaFuncSetAttribute(wgrad_kernel<CIN, COUT, IN>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    configured = true;
  }
  const int64_t tiles = (int64_t)a.tx * a.ty * a.tz * a.nb;
  note_launch();
  wgrad_kernel<CIN, COUT, IN><<<nblk, NT, sm, s>>>(a, g, partial, tiles);
  return cudaGetLastError();
}

ConvArgs vol_args(int nb, int nz, int ny, int nx) {
  ConvArgs a{};
  a.nb = nb;
  a.nz = nz;
  a.ny = ny;
  a.nx = nx;
  a.tx = (nx + TXc - 1) / TXc;
  a.ty = (ny + TYc - 1) / TYc;
  a.tz = (nz + TZc - 1) / TZc;
  return a;
}

}  // namespace

// ---------------------------------------------------------------------------------------
// Library-internal interface (helm6_internal.h)
// ---------------------------------------------------------------------------------------

int cnn_alloc(CnnNet& net) {
  if (cudaMalloc((void**)&net.wtc, sizeof(uint16_t) * NL * 27 * 256) != cudaSuccess) return HELM6_ERR_NOMEM;
  if (cudaMalloc((void**)&net.theta, sizeof(float) * HELM6_CNN_NPARAMS) != cudaSuccess) return HELM6_ERR_NOMEM;
  if (cudaMalloc((void**)&net.wf, sizeof(float) * kWeights) != cudaSuccess) return HELM6_ERR_NOMEM;
  if (cudaMalloc((void**)&net.wb, sizeof(float) * kWeights) != cudaSuccess) return HELM6_ERR_NOMEM;
  return HELM6_OK;
}

void cnn_free(CnnNet& net) {
  cudaFree(net.theta);
  cudaFree(net.wf);
  cudaFree(net.wb);
  cudaFree(net.wtc);
  net = CnnNet{};
}

int cnn_configure() {
  // the field kernels' shared-memory limits, set once before any launch (and so never
  // inside a stream capture)
  if (cudaFuncSetAttribute(conv_tc_kernel<IN_PLANAR, OUT_HIDDEN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)TC_SMEM) != cudaSuccess ||
      cudaFuncSetAttribute(conv_tc_kernel<IN_BF16, OUT_HIDDEN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)TC_SMEM) != cudaSuccess ||
      cudaFuncSetAttribute(conv_tc_kernel<IN_BF16, OUT_FIELD>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)TC_SMEM) != cudaSuccess)
    return HELM6_ERR_CUDA;
  if (cudaFuncSetAttribute(conv_kernel<2, 16, IN_PLANAR, OUT_HIDDEN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)conv_smem<2, 16>()) != cudaSuccess ||
      cudaFuncSetAttribute(conv_kernel<16, 16, IN_BF16, OUT_HIDDEN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)conv_smem<16, 16>()) != cudaSuccess ||
      cudaFuncSetAttribute(conv_kernel<16, 2, IN_BF16, OUT_FIELD>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)conv_smem<16, 2>()) != cudaSuccess)
    return HELM6_ERR_CUDA;
  return HELM6_OK;
}

void cnn_prepare(const CnnNet& net, cudaStream_t s) {
  note_launch(net.wtc ? 2 : 1);
  prep_kernel<<<(27 * 16 * 16 + 255) / 256, 256, 0, s>>>(net.theta, net.wf, net.wb);
  if (net.wtc) prep_tc_kernel<<<(NL * 27 * 256 + 255) / 256, 256, 0, s>>>(net.theta, net.wtc);
}

int cnn_apply_field(const CnnNet& net, int nz, int ny, int nx, const float* t, const double* sumsq, uint16_t* act0,
                    uint16_t* act1, float out_scale, float* z, int* err, cudaStream_t s) {
  const LayerDims d = layer_dims();
  TcConvArgs a{};
  a.nz = nz;
  a.ny = ny;
  a.nx = nx;
  a.bx = (nx + BX - 1) / BX;
  a.by = (ny + BY - 1) / BY;
  a.bz = (nz + BZ - 1) / BZ;
  a.sumsq = sumsq;
  a.out_scale = out_scale;
  a.err = err;
  const unsigned grid = (unsigned)((int64_t)a.bx * a.by * a.bz);
  const uint16_t* in[4] = {nullptr, act0, act1, act0};
  void* out[4] = {act0, act1, act0, z};
  note_launch(4);
  for (int l = 0; l < NL; ++l) {
    a.in = l == 0 ? (const void*)t : (const void*)in[l];
    a.w = net.wtc + (size_t)l * 27 * 256;
    a.bias = net.theta + d.boff[l];
    a.out = out[l];
    if (l == 0)
      conv_tc_kernel<IN_PLANAR, OUT_HIDDEN><<<grid, 128, TC_SMEM, s>>>(a);
    else if (l < NL - 1)
      conv_tc_kernel<IN_BF16, OUT_HIDDEN><<<grid, 128, TC_SMEM, s>>>(a);
    else
      conv_tc_kernel<IN_BF16, OUT_FIELD><<<grid, 128, TC_SMEM, s>>>(a);
  }
  return cudaGetLastError() == cudaSuccess ? HELM6_OK : HELM6_ERR_CUDA;
}

}  // namespace helm6

// ---------------------------------------------------------------------------------------
// C-ABI: the trainer
// ---------------------------------------------------------------------------------------

using namespace helm6;

struct helm6_cnn_trainer {
  int nb = 0, nz = 0, ny = 0, nx = 0;
  int64_t npts = 0;
  cudaStream_t stream = nullptr;
  CnnNet net;
  float *m = nullptr, *v = nullptr, *grad = nullptr;
  float *pre[3] = {nullptr, nullptr, nullptr};   // FP32 pre-activations of layers 1-3
  uint16_t* act[3] = {nullptr, nullptr, nullptr};  // BF16 activations after layers 1-3
  float *y = nullptr, *g4 = nullptr, *ga = nullptr, *gb = nullptr;
  float* partial = nullptr;
  double *lpart = nullptr, *loss = nullptr;
  double* pinned = nullptr;
  int nblk = 0, nloss = 0;
  long long step = 0;
  bool residual = false;    // loss mean|A_h y - x|^2 over interior points (else MSE)
  PatchW w{}, wconj{};      // interior operator weights and their conjugates
  double loss_div = 1.0;    // normaliser of the summed squares
};

namespace {

int tr_forward(helm6_cnn_trainer* tr, const float* x) {
  const LayerDims d = layer_dims();
  ConvArgs a = vol_args(tr->nb, tr->nz, tr->ny, tr->nx);
  cudaStream_t s = tr->stream;
  a.in = x;
  a.round_in = 1;
  a.w = tr->net.wf + d.woff[0];
  a.bias = tr->net.theta + d.boff[0];
  a.pre = tr->pre[0];
  a.out = tr->act[0];
  if (launch_conv<2, 16, IN_F32, OUT_HIDDEN>(a, s) != cudaSuccess) return HELM6_ERR_CUDA;
  a.round_in = 0;
  for (int l = 1; l < 3; ++l) {
    a.in = tr->act[l - 1];
    a.w = tr->net.wf + d.woff[l];
    a.bias = tr->net.theta + d.boff[l];
    a.pre = tr->pre[l];
    a.out = tr->act[l];
    if (launch_conv<16, 16, IN_BF16, OUT_HIDDEN>(a, s) != cudaSuccess) return HELM6_ERR_CUDA;
  }
  a.in = tr->act[2];
  a.w = tr->net.wf + d.woff[3];
  a.bias = tr->net.theta + d.boff[3];
  a.pre = nullptr;
  a.out = tr->y;
  if (launch_conv<16, 2, IN_BF16, OUT_F32>(a, s) != cudaSuccess) return HELM6_ERR_CUDA;
  return HELM6_OK;
}

// loss, g4 = dL/dy, then every layer's weight/bias gradient into tr->grad
int tr_backward(helm6_cnn_trainer* tr, const float* x, const float* target) {
  const LayerDims d = layer_dims();
  cudaStream_t s = tr->stream;
  const int64_t n = tr->npts * 2;
  if (tr->residual) {
    // R = A y - x (interior), loss = |R|^2 / (2M), g4 = A^H R / M
    const unsigned nb = (unsigned)((tr->npts + 255) / 256);
    const int64_t M = (int64_t)tr->nb * (tr->nz - 2) * (tr->ny - 2) * (tr->nx - 2);
    note_launch(3);
    patch_op_kernel<<<nb, 256, 0, s>>>(tr->nb, tr->nz, tr->ny, tr->nx, tr->y, tr->ga, tr->w, 1.f);
    resid_loss_kernel<<<tr->nloss, 256, 0, s>>>(tr->nb, tr->nz, tr->ny, tr->nx, tr->ga, target, tr->gb, tr->lpart);
    patch_op_kernel<<<nb, 256, 0, s>>>(tr->nb, tr->nz, tr->ny, tr->nx, tr->gb, tr->g4, tr->wconj,
                                       (float)(1.0 / (double)M));
  } else {
    note_launch();
    mse_kernel<<<tr->nloss, 256, 0, s>>>(tr->y, target, n, tr->g4, tr->lpart);
  }
  launch_reduce_sum(tr->lpart, tr->nloss, tr->loss, s);
  ConvArgs a = vol_args(tr->nb, tr->nz, tr->ny, tr->nx);
  auto reduce = [&](int l) {
    note_launch();
    const int ne = 27 * d.cin[l] * d.cout[l] + d.cout[l];
    wgrad_reduce_kernel<<<(ne + 255) / 256, 256, 0, s>>>(tr->partial, tr->nblk, d.cin[l], d.cout[l],
                                                         tr->grad + d.toff[l], tr->grad + d.boff[l]);
  };
  // layer 4: dW from act3 and g4; g3 = (W4^T * g4) gelu'(pre3)
  a.in = tr->act[2];
  if (launch_wgrad<16, 2, IN_BF16>(a, tr->g4, tr->partial, tr->nblk, s) != cudaSuccess) return HELM6_ERR_CUDA;
  reduce(3);
  a.in = tr->g4;
  a.round_in = 0;
  a.w = tr->net.wb + d.woff[3];
  a.bias = nullptr;
  a.pre = tr->pre[2];
  a.out = tr->ga;
  if (launch_conv<2, 16, IN_F32, OUT_GRAD>(a, s) != cudaSuccess) return HELM6_ERR_CUDA;
  // layers 3 and 2
  float* gcur = tr->ga;
  float* gnext = tr->gb;
  for (int l = 2; l >= 1; --l) {
    a.in = tr->act[l - 1];
    if (launch_wgrad<16, 16, IN_BF16>(a, gcur, tr->partial, tr->nblk, s) != cudaSuccess) return HELM6_ERR_CUDA;
    reduce(l);
    a.in = gcur;
    a.w = tr->net.wb + d.woff[l];
    a.pre = tr->pre[l - 1];
    a.out = gnext;
    if (launch_conv<16, 16, IN_F32, OUT_GRAD>(a, s) != cudaSuccess) return HELM6_ERR_CUDA;
    std::swap(gcur, gnext);
  }
  // layer 1: dW from the BF16-rounded input and g1
  a.in = x;
  a.round_in = 1;
  if (launch_wgrad<2, 16, IN_F32>(a, gcur, tr->partial, tr->nblk, s) != cudaSuccess) return HELM6_ERR_CUDA;
  reduce(0);
  return HELM6_OK;
}

int read_loss(helm6_cnn_trainer* tr, double* loss) {
  if (!loss) return HELM6_OK;
  if (cudaMemcpyAsync(tr->pinned, tr->loss, sizeof(double), cudaMemcpyDeviceToHost, tr->stream) != cudaSuccess)
    return HELM6_ERR_CUDA;
  if (cudaStreamSynchronize(tr->stream) != cudaSuccess) return HELM6_ERR_CUDA;
  *loss = tr->pinned[0] / tr->loss_div;
  return HELM6_OK;
}

}  // namespace

extern "C" {

void helm6_cnn_trainer_destroy(helm6_cnn_trainer* tr) {
  if (!tr) return;
  if (tr->stream) cudaStreamSynchronize(tr->stream);
  else cudaDeviceSynchronize();
  cnn_free(tr->net);
  void* bufs[] = {tr->m, tr->v, tr->grad, tr->pre[0], tr->pre[1], tr->pre[2], tr->act[0], tr->act[1],
                  tr->act[2], tr->y, tr->g4, tr->ga, tr->gb, tr->partial, tr->lpart, tr->loss};
  for (void* p : bufs) cudaFree(p);
  if (tr->pinned) cudaFreeHost(tr->pinned);
  delete tr;
}

int helm6_cnn_trainer_create(helm6_cnn_trainer** out, int batch, int nz, int ny, int nx, const float* theta0,
                             void* stream) {
  if (!out || !theta0 || batch < 1 || nz < 1 || ny < 1 || nx < 1) return HELM6_ERR_INVALID;
  *out = nullptr;
  const int64_t npts = (int64_t)batch * nz * ny * nx;
  const int64_t tiles = (int64_t)((nx + TXc - 1) / TXc) * ((ny + TYc - 1) / TYc) * ((nz + TZc - 1) / TZc) * batch;
  if (tiles > INT32_MAX || npts > ((int64_t)1 << 34)) return HELM6_ERR_INVALID;
  auto* tr = new helm6_cnn_trainer();
  tr->nb = batch;
  tr->nz = nz;
  tr->ny = ny;
  tr->nx = nx;
  tr->npts = npts;
  tr->stream = (cudaStream_t)stream;
  tr->loss_div = (double)npts * 2.0;
  tr->nblk = (int)std::min<int64_t>(tiles, 2 * (int64_t)device_sm_count());
  tr->nloss = 4 * device_sm_count();
  auto fail = [&](int rc) {
    helm6_cnn_trainer_destroy(tr);
    return rc;
  };
  auto al = [&](void** p, size_t bytes) { return cudaMalloc(p, bytes) == cudaSuccess; };
  const size_t np = HELM6_CNN_NPARAMS;
  if (cnn_alloc(tr->net) != HELM6_OK) return fail(HELM6_ERR_NOMEM);
  bool ok = al((void**)&tr->m, np * 4) && al((void**)&tr->v, np * 4) && al((void**)&tr->grad, np * 4) &&
            al((void**)&tr->y, npts * 8) && al((void**)&tr->g4, npts * 8) && al((void**)&tr->ga, npts * 64) &&
            al((void**)&tr->gb, npts * 64) && al((void**)&tr->partial, (size_t)tr->nblk * (6912 + 16) * 4) &&
            al((void**)&tr->lpart, (size_t)tr->nloss * 8) && al((void**)&tr->loss, 8);
  for (int l = 0; l < 3 && ok; ++l) ok = al((void**)&tr->pre[l], npts * 64) && al((void**)&tr->act[l], npts * 32);
  if (!ok) return fail(HELM6_ERR_NOMEM);
  if (cudaMallocHost((void**)&tr->pinned, 64) != cudaSuccess) return fail(HELM6_ERR_NOMEM);
  if (cudaMemcpy(tr->net.theta, theta0, np * 4, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemset(tr->m, 0, np * 4) != cudaSuccess || cudaMemset(tr->v, 0, np * 4) != cudaSuccess ||
      cudaMemset(tr->grad, 0, np * 4) != cudaSuccess)
    return fail(HELM6_ERR_CUDA);
  cnn_prepare(tr->net, tr->stream);
  if (cudaStreamSynchronize(tr->stream) != cudaSuccess) return fail(HELM6_ERR_CUDA);
  *out = tr;
  return HELM6_OK;
}

int helm6_cnn_forward(helm6_cnn_trainer* tr, const float* x, float* y) {
  if (!tr || !x || !y) return HELM6_ERR_INVALID;
  int rc = tr_forward(tr, x);
  if (rc) return rc;
  if (cudaMemcpyAsync(y, tr->y, tr->npts * 8, cudaMemcpyDeviceToDevice, tr->stream) != cudaSuccess)
    return HELM6_ERR_CUDA;
  return HELM6_OK;
}

int helm6_cnn_gradient(helm6_cnn_trainer* tr, const float* x, const float* target, float* grad, double* loss) {
  if (!tr || !x || !target || !grad) return HELM6_ERR_INVALID;
  int rc = tr_forward(tr, x);
  if (!rc) rc = tr_backward(tr, x, target);
  if (rc) return rc;
  if (cudaMemcpyAsync(grad, tr->grad, sizeof(float) * HELM6_CNN_NPARAMS, cudaMemcpyDeviceToDevice, tr->stream) !=
      cudaSuccess)
    return HELM6_ERR_CUDA;
  return read_loss(tr, loss);
}

int helm6_cnn_train_step(helm6_cnn_trainer* tr, const float* x, const float* target, float lr, double* loss) {
  if (!tr || !x || !target || !(lr >= 0.f)) return HELM6_ERR_INVALID;
  int rc = tr_forward(tr, x);
  if (!rc) rc = tr_backward(tr, x, target);
  if (rc) return rc;
  tr->step += 1;
  const float c1 = (float)(1.0 - std::pow(0.9, (double)tr->step));
  const float c2 = (float)(1.0 - std::pow(0.999, (double)tr->step));
  note_launch();
  adam_kernel<<<(HELM6_CNN_NPARAMS + 255) / 256, 256, 0, tr->stream>>>(tr->net.theta, tr->m, tr->v, tr->grad,
                                                                     HELM6_CNN_NPARAMS, lr, c1, c2);
  cnn_prepare(tr->net, tr->stream);
  if (cudaGetLastError() != cudaSuccess) return HELM6_ERR_CUDA;
  return read_loss(tr, loss);
}

int helm6_cnn_set_residual_loss(helm6_cnn_trainer* tr, helm6_c64 k, double h) {
  if (!tr || !(h > 0) || !std::isfinite(k.re) || !std::isfinite(k.im)) return HELM6_ERR_INVALID;
  if (tr->nz < 3 || tr->ny < 3 || tr->nx < 3) return HELM6_ERR_INVALID;
  StencilCoef c;
  stencil_coefficients(cd(k.re, k.im), h, c);
  const c64d cls[4] = {c.interior.w[1][0], c.interior.w[1][1], c.interior.w[1][2], c.interior.w[0][2]};
  for (int i = 0; i < 4; ++i) {
    tr->w.re[i] = (float)cls[i].re;
    tr->w.im[i] = (float)cls[i].im;
    tr->wconj.re[i] = (float)cls[i].re;
    tr->wconj.im[i] = -(float)cls[i].im;
  }
  tr->residual = true;
  tr->loss_div = 2.0 * (double)tr->nb * (tr->nz - 2) * (tr->ny - 2) * (tr->nx - 2);
  return HELM6_OK;
}

int helm6_cnn_get_params(helm6_cnn_trainer* tr, float* theta) {
  if (!tr || !theta) return HELM6_ERR_INVALID;
  if (cudaMemcpyAsync(theta, tr->net.theta, sizeof(float) * HELM6_CNN_NPARAMS, cudaMemcpyDeviceToHost,
                      tr->stream) != cudaSuccess ||
      cudaStreamSynchronize(tr->stream) != cudaSuccess)
    return HELM6_ERR_CUDA;
  return HELM6_OK;
}

}  // extern "C"

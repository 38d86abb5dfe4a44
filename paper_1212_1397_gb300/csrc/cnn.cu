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
// Kernels:
//   conv_tc_kernel  a layer as a tensor-core implicit GEMM (tcgen05, TMEM accumulators): the
//                   field path's four layers, the trainer's forward layers (FP32
//                   pre-activations kept) and its input gradients (the transpose of a
//                   zero-padded correlation is the correlation with the flipped,
//                   channel-transposed taps; the FP32 gradient split into BF16 hi + lo)
//   wgrad_kernel    weight and bias gradients (SIMT, 32x4x2-point tiles with the input halo
//                   staged in shared memory), block partials over persistent tiles
//   mse_kernel, adam_kernel, prep_tc_kernel / prep_tcb_kernel (BF16 taps in the layouts the
//   tensor-core kernel reads, from the master vector)
#include <cuda_bf16.h>

#include <cmath>
#include <cstring>
#include <utility>
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

// IN_G32 (tensor-core kernel only): FP32 gradients split into BF16 hi + lo operand copies
enum { IN_F32 = 0, IN_BF16 = 1, IN_PLANAR = 2, IN_G32 = 3 };
enum { OUT_HIDDEN = 0, OUT_F32 = 1, OUT_FIELD = 2, OUT_GRAD = 3 };

// The SIMT weight-gradient kernel's view of a batch of images.
struct ConvArgs {
  int nb, nz, ny, nx;  // images and their size (x fastest, channel-last)
  int tx, ty, tz;      // tiles per axis
  const void* in;      // the layer's input activations: IN_F32 [N][CIN] or IN_BF16 [N][16]
  int round_in;        // IN_F32: round the input to BF16 first
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

// Stage the input halo of one tile into sx (HP points x PStride<CIN> floats).
template <int CIN, int IN>
__device__ __forceinline__ void load_halo(const ConvArgs& a, int img, int z0, int y0, int x0, float* sx) {
  constexpr int PS = PStride<CIN>::v;
  for (int i = threadIdx.x; i < HP; i += NT) {
    const int hx = i % HX, r = i / HX, hy = r % HY, hz = r / HY;
    const int gx = x0 + hx - 1, gy = y0 + hy - 1, gz = z0 + hz - 1;
    const bool ok = gx >= 0 && gx < a.nx && gy >= 0 && gy < a.ny && gz >= 0 && gz < a.nz;
    const int64_t p = (((int64_t)img * a.nz + gz) * a.ny + gy) * a.nx + gx;
    float* d = sx + i * PS;
    if constexpr (IN == IN_BF16) {
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
    load_halo<CIN, IN>(a, img, z0, y0, x0, sx);
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
// 30 x 4 x 4 output points; its 32 x 6 x 6 input halo sits in shared memory as two
// channel planes (channels 0-7 and 8-15, 16 bytes per point, points x fastest), the
// no-swizzle K-major layout: a core matrix is 8 consecutive points of one plane (128 B),
// the K step between the planes is the plane distance and the step between 8-row groups
// is 128 B, so every tap's A operand is the same descriptor with its start address moved
// by the tap offset.  The 4 tiles (4 halo rows x 32 points each: y rows 1-4 of z planes
// 1-4) accumulate in 4 x 16 TMEM columns; outputs at halo columns are computed and dropped.
// Bricks this small (52 KB of shared memory, 64 TMEM columns) let four CTAs share an SM, so
// that one CTA's halo loads overlap another's MMAs and epilogue (measured against 30 x 8 x 4
// bricks, one CTA per SM).  The same kernel serves the trainer on batches of images (zero padding at
// every image face): its forward layers (FP32 pre-activations kept) and the input gradients
// of the backward pass, whose FP32 gradient operand is split into BF16 hi + lo copies (two
// more channel planes; 54 MMAs per tile) so that it keeps FP32-like accuracy.
constexpr int BX = 30, BY = 4, BZ = 4;                       // output points of a brick
constexpr int GX = BX + 2, GY = BY + 2, GZ = BZ + 2, GP = GX * GY * GZ;  // halo (GX = 32)
constexpr int TC_TILES = BZ * BY / 4;                         // 128-point tiles of a brick
constexpr int TC_TMEM = TC_TILES * 16 <= 32 ? 32 : TC_TILES * 16 <= 64 ? 64 : 128;  // TMEM columns
constexpr int PLANE_B = (GP + 2) * 16;                        // one point of padding each end
constexpr int TCW_TAP = 512;                                  // bytes of one tap's 16 x 16 BF16
constexpr size_t TC_SMEM = 1024 + 2 * (size_t)PLANE_B + 27 * TCW_TAP + 256;
constexpr size_t TC_SMEM4 = 1024 + 4 * (size_t)PLANE_B + 27 * TCW_TAP + 256;  // IN_G32: hi and lo planes
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
  int nb;                // images (1 for the field path)
  int nz, ny, nx;        // size of an image
  int bx, by, bz;        // bricks per axis of an image
  const void* in;        // IN_BF16: [N][16] BF16; IN_PLANAR: planar FP32 complex field;
                         // IN_F32 (rounded to BF16) / IN_G32: [N][cin] FP32, channel-last
  int cin;               // IN_F32 / IN_G32: input channels (2 or 16)
  const uint16_t* w;     // 27 taps of 16 x 16 BF16 in the canonical layout
  const float* bias;     // [c_out] (c_out = 16, or 2 for the field output) or null
  float* pre;            // OUT_HIDDEN: FP32 pre-activations [N][16] written (nullable); OUT_GRAD: read
  void* out;             // OUT_HIDDEN: [N][16] BF16; OUT_FIELD: planar FP32 z (updated);
                         // OUT_F32: [N][2] FP32; OUT_GRAD: [N][16] FP32 (times GELU'(pre))
  const double* sumsq;   // IN_PLANAR / OUT_FIELD: sum |t|^2
  float out_scale;
  int* err;              // set if the MMA completion wait timed out
};

template <int IN, int OUT>
__global__ void __launch_bounds__(128) conv_tc_kernel(TcConvArgs a) {
  extern __shared__ uint8_t smem_raw[];
  constexpr int NPL = IN == IN_G32 ? 4 : 2;  // channel planes: 0-7, 8-15 (hi), then lo
  uint8_t* sm = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint8_t* plane0 = sm + 16;               // point -1 at sm, point 0 at sm + 16
  uint8_t* plane1 = plane0 + PLANE_B;
  uint8_t* wts = sm + NPL * PLANE_B;       // 27 x 512 B (1024-aligned base + NPL * PLANE_B: 16-aligned)
  uint64_t* bar = (uint64_t*)(wts + 27 * TCW_TAP);
  uint32_t* tslot = (uint32_t*)(bar + 1);
  int* fail = (int*)(tslot + 1);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int64_t npts = (int64_t)a.nz * a.ny * a.nx;

  int64_t b = blockIdx.x;
  const int ibx = (int)(b % a.bx);
  b /= a.bx;
  const int iby = (int)(b % a.by);
  b /= a.by;
  const int ibz = (int)(b % a.bz);
  const int64_t img = b / a.bz;
  const int x0 = ibx * BX - 1, y0 = iby * BY - 1, z0 = ibz * BZ - 1;  // global coordinate of halo (0,0,0)

  // weights: 27 x 512 B
  for (int i = tid; i < 27 * TCW_TAP / 16; i += 128) cp16(smem_u32(wts) + 16u * i, (const uint4*)a.w + i, true);
  // halo planes
  float sc = 1.f;
  if constexpr (IN == IN_PLANAR) {
    const double ss = *a.sumsq;
    sc = ss > 0.0 ? (float)(1.0 / sqrt(ss / (double)npts)) : 0.f;
  }
  if constexpr (IN == IN_PLANAR) {
    // the planar FP32 field: every load of the thread's halo points issued before any is used
    constexpr int PER = (GP + 127) / 128;
    const float* f = (const float*)a.in;
    float re[PER], im[PER];
#pragma unroll
    for (int k = 0; k < PER; ++k) {
      const int i = tid + 128 * k;
      const int hx = i % GX, r = i / GX, hy = r % GY, hz = r / GY;
      const int gx = x0 + hx, gy = y0 + hy, gz = z0 + hz;
      const bool ok = i < GP && gx >= 0 && gx < a.nx && gy >= 0 && gy < a.ny && gz >= 0 && gz < a.nz;
      const int64_t p = ok ? ((img * a.nz + gz) * a.ny + gy) * a.nx + gx : 0;
      re[k] = ok ? f[p] : 0.f;
      im[k] = ok ? f[npts + p] : 0.f;
    }
#pragma unroll
    for (int k = 0; k < PER; ++k) {
      const int i = tid + 128 * k;
      if (i < GP) {
        *(uint4*)(plane0 + 16 * i) = make_uint4(pack_bf16(re[k] * sc, im[k] * sc), 0u, 0u, 0u);
        *(uint4*)(plane1 + 16 * i) = make_uint4(0u, 0u, 0u, 0u);
      }
    }
  }
  for (int i = tid; i < GP && IN != IN_PLANAR; i += 128) {
    const int hx = i % GX, r = i / GX, hy = r % GY, hz = r / GY;
    const int gx = x0 + hx, gy = y0 + hy, gz = z0 + hz;
    const bool ok = gx >= 0 && gx < a.nx && gy >= 0 && gy < a.ny && gz >= 0 && gz < a.nz;
    const int64_t p = ok ? ((img * a.nz + gz) * a.ny + gy) * a.nx + gx : 0;
    if constexpr (IN == IN_BF16) {
      const uint4* src = (const uint4*)a.in + 2 * p;
      cp16(smem_u32(plane0) + 16u * i, src, ok);
      cp16(smem_u32(plane1) + 16u * i, src + 1, ok);
    } else if constexpr (IN == IN_F32 || IN == IN_G32) {
      // channel-last FP32: BF16 (IN_F32), or BF16 hi + lo = the value to 16 bits (IN_G32)
      const float* f = (const float*)a.in + p * a.cin;
      float v[16];
#pragma unroll
      for (int c = 0; c < 16; ++c) v[c] = (ok && c < a.cin) ? f[c] : 0.f;
      uint32_t hi[8], lo[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        hi[q] = pack_bf16(v[2 * q], v[2 * q + 1]);
        lo[q] = pack_bf16(v[2 * q] - bf16_lo(hi[q]), v[2 * q + 1] - bf16_hi(hi[q]));
      }
      *(uint4*)(plane0 + 16 * i) = make_uint4(hi[0], hi[1], hi[2], hi[3]);
      *(uint4*)(plane1 + 16 * i) = make_uint4(hi[4], hi[5], hi[6], hi[7]);
      if constexpr (IN == IN_G32) {
        *(uint4*)(plane0 + 2 * PLANE_B + 16 * i) = make_uint4(lo[0], lo[1], lo[2], lo[3]);
        *(uint4*)(plane0 + 3 * PLANE_B + 16 * i) = make_uint4(lo[4], lo[5], lo[6], lo[7]);
      }
    }
  }
  if (tid < NPL) {  // the padding points before and after each plane
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
                 "r"(TC_TMEM));
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
        if constexpr (IN == IN_G32)  // the lo copy of the operand
          mma_bf16(tmem + 16u * tile, desc_noswz(p0 + 2u * PLANE_B + (uint32_t)(q * 16), PLANE_B, 128), bd, id, 1u);
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
    for (int c = 0; c < 16; ++c) bias[c] = (a.bias && (OUT == OUT_HIDDEN || c < 2)) ? a.bias[c] : 0.f;
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
      const int64_t p = ((img * a.nz + gz) * a.ny + gy) * a.nx + gx;
      if constexpr (OUT == OUT_HIDDEN) {
        if (a.pre) {
          float4* pr = (float4*)(a.pre + p * 16);
#pragma unroll
          for (int q = 0; q < 4; ++q)
            pr[q] = make_float4(__uint_as_float(v[4 * q]) + bias[4 * q], __uint_as_float(v[4 * q + 1]) + bias[4 * q + 1],
                                __uint_as_float(v[4 * q + 2]) + bias[4 * q + 2],
                                __uint_as_float(v[4 * q + 3]) + bias[4 * q + 3]);
        }
        uint32_t pk[8];
#pragma unroll
        for (int q = 0; q < 8; ++q)
          pk[q] = pack_bf16(gelu_f(__uint_as_float(v[2 * q]) + bias[2 * q]),
                            gelu_f(__uint_as_float(v[2 * q + 1]) + bias[2 * q + 1]));
        uint4* o4 = (uint4*)a.out + 2 * p;
        o4[0] = make_uint4(pk[0], pk[1], pk[2], pk[3]);
        o4[1] = make_uint4(pk[4], pk[5], pk[6], pk[7]);
      } else if constexpr (OUT == OUT_F32) {
        float* o = (float*)a.out + p * 2;
        o[0] = __uint_as_float(v[0]) + bias[0];
        o[1] = __uint_as_float(v[1]) + bias[1];
      } else if constexpr (OUT == OUT_GRAD) {
        const float4* pr = (const float4*)(a.pre + p * 16);
        float4* o = (float4*)((float*)a.out + p * 16);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const float4 pv = pr[q];
          o[q] = make_float4(__uint_as_float(v[4 * q]) * gelu_df(pv.x), __uint_as_float(v[4 * q + 1]) * gelu_df(pv.y),
                             __uint_as_float(v[4 * q + 2]) * gelu_df(pv.z),
                             __uint_as_float(v[4 * q + 3]) * gelu_df(pv.w));
        }
      } else {
        float* z = (float*)a.out;
        z[p] = fmaf(cs, __uint_as_float(v[0]) + bias[0], z[p]);
        z[npts + p] = fmaf(cs, __uint_as_float(v[1]) + bias[1], z[npts + p]);
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TC_TMEM));
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

// The same for the input gradient of every layer (the transpose of a zero-padded correlation
// is the correlation with the flipped, channel-transposed taps): layer l, tap t' = 26 - t,
// c_out' = the layer's c_in rows and c_in' = its c_out columns.
__global__ void prep_tcb_kernel(const float* __restrict__ theta, uint16_t* __restrict__ wtcb) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= NL * 27 * 256) return;
  const int l = i / (27 * 256), t2 = (i / 256) % 27, e = i % 256;
  const int co2 = e / 16, ci2 = e % 16;  // co2: the layer's input channel, ci2: its output channel
  int toff = 0;
  for (int q = 0; q < l; ++q) toff += 27 * ch(q) * ch(q + 1) + ch(q + 1);
  const int cin = ch(l), cout = ch(l + 1);
  const float w = (co2 < cin && ci2 < cout) ? theta[toff + (ci2 * cin + co2) * 27 + (26 - t2)] : 0.f;
  const __nv_bfloat16 b16 = __float2bfloat16_rn(w);
  uint16_t u;
  memcpy(&u, &b16, 2);
  wtcb[(l * 27 + t2) * 256 + ((co2 / 8) * 2 + ci2 / 8) * 64 + (co2 % 8) * 8 + (ci2 % 8)] = u;
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

constexpr int kWeights = 27 * (2 * 16 + 16 * 16 + 16 * 16 + 16 * 2);  // 15552 taps
static_assert(kWeights + 16 + 16 + 16 + 2 == HELM6_CNN_NPARAMS, "parameter count");

template <int CIN, int COUT>
constexpr size_t wgrad_smem() {
  return sizeof(float) * (HP * PStride<CIN>::v + NT * COUT);
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

int cnn_alloc(CnnNet& net, bool backward) {
  if (cudaMalloc((void**)&net.wtc, sizeof(uint16_t) * NL * 27 * 256) != cudaSuccess) return HELM6_ERR_NOMEM;
  if (backward && cudaMalloc((void**)&net.wtcb, sizeof(uint16_t) * NL * 27 * 256) != cudaSuccess)
    return HELM6_ERR_NOMEM;
  if (cudaMalloc((void**)&net.theta, sizeof(float) * HELM6_CNN_NPARAMS) != cudaSuccess) return HELM6_ERR_NOMEM;
  return HELM6_OK;
}

void cnn_free(CnnNet& net) {
  cudaFree(net.theta);
  cudaFree(net.wtc);
  cudaFree(net.wtcb);
  net = CnnNet{};
}

int cnn_configure() {
  // the field kernels' shared-memory limits, set once before any launch (and so never
  // inside a stream capture)
  static bool done = false;
  if (done) return HELM6_OK;
  const std::pair<const void*, size_t> ks[] = {
      {(const void*)conv_tc_kernel<IN_PLANAR, OUT_HIDDEN>, TC_SMEM},
      {(const void*)conv_tc_kernel<IN_BF16, OUT_HIDDEN>, TC_SMEM},
      {(const void*)conv_tc_kernel<IN_BF16, OUT_FIELD>, TC_SMEM},
      // the trainer's layers
      {(const void*)conv_tc_kernel<IN_F32, OUT_HIDDEN>, TC_SMEM},
      {(const void*)conv_tc_kernel<IN_BF16, OUT_F32>, TC_SMEM},
      {(const void*)conv_tc_kernel<IN_G32, OUT_GRAD>, TC_SMEM4}};
  for (const auto& k : ks)
    if (cudaFuncSetAttribute(k.first, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)k.second) != cudaSuccess)
      return HELM6_ERR_CUDA;
  done = true;
  return HELM6_OK;
}

void cnn_prepare(const CnnNet& net, cudaStream_t s) {
  note_launch((net.wtc ? 1 : 0) + (net.wtcb ? 1 : 0));
  if (net.wtc) prep_tc_kernel<<<(NL * 27 * 256 + 255) / 256, 256, 0, s>>>(net.theta, net.wtc);
  if (net.wtcb) prep_tcb_kernel<<<(NL * 27 * 256 + 255) / 256, 256, 0, s>>>(net.theta, net.wtcb);
}

int cnn_apply_field(const CnnNet& net, int nz, int ny, int nx, const float* t, const double* sumsq, uint16_t* act0,
                    uint16_t* act1, float out_scale, float* z, int* err, cudaStream_t s) {
  const LayerDims d = layer_dims();
  TcConvArgs a{};
  a.nb = 1;
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
  int* tcerr = nullptr;     // set by a tensor-core layer whose MMA wait timed out
  int nblk = 0, nloss = 0;
  long long step = 0;
  bool residual = false;    // loss mean|A_h y - x|^2 over interior points (else MSE)
  PatchW w{}, wconj{};      // interior operator weights and their conjugates
  double loss_div = 1.0;    // normaliser of the summed squares
};

namespace {

// A tensor-core layer over the trainer's batch of images.
TcConvArgs tr_tc_args(const helm6_cnn_trainer* tr) {
  TcConvArgs a{};
  a.nb = tr->nb;
  a.nz = tr->nz;
  a.ny = tr->ny;
  a.nx = tr->nx;
  a.bx = (tr->nx + BX - 1) / BX;
  a.by = (tr->ny + BY - 1) / BY;
  a.bz = (tr->nz + BZ - 1) / BZ;
  a.err = tr->tcerr;
  return a;
}

unsigned tr_tc_grid(const TcConvArgs& a) { return (unsigned)((int64_t)a.bx * a.by * a.bz * a.nb); }

// Forward pass on the tensor cores: BF16 input (rounded), BF16 activations, FP32
// pre-activations kept for the backward pass.
int tr_forward(helm6_cnn_trainer* tr, const float* x) {
  const LayerDims d = layer_dims();
  cudaStream_t s = tr->stream;
  TcConvArgs a = tr_tc_args(tr);
  const unsigned grid = tr_tc_grid(a);
  note_launch(NL);
  for (int l = 0; l < NL; ++l) {
    a.w = tr->net.wtc + (size_t)l * 27 * 256;
    a.bias = tr->net.theta + d.boff[l];
    if (l == 0) {
      a.in = x;
      a.cin = 2;
      a.pre = tr->pre[0];
      a.out = tr->act[0];
      conv_tc_kernel<IN_F32, OUT_HIDDEN><<<grid, 128, TC_SMEM, s>>>(a);
    } else if (l < NL - 1) {
      a.in = tr->act[l - 1];
      a.pre = tr->pre[l];
      a.out = tr->act[l];
      conv_tc_kernel<IN_BF16, OUT_HIDDEN><<<grid, 128, TC_SMEM, s>>>(a);
    } else {
      a.in = tr->act[l - 1];
      a.pre = nullptr;
      a.out = tr->y;
      conv_tc_kernel<IN_BF16, OUT_F32><<<grid, 128, TC_SMEM, s>>>(a);
    }
  }
  return cudaGetLastError() == cudaSuccess ? HELM6_OK : HELM6_ERR_CUDA;
}

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
  // input gradients on the tensor cores (the FP32 gradient split into BF16 hi + lo), weight
  // gradients by the SIMT reduction kernel
  TcConvArgs t = tr_tc_args(tr);
  const unsigned tgrid = tr_tc_grid(t);
  t.bias = nullptr;
  // layer 4: dW from act3 and g4; g3 = (W4^T * g4) gelu'(pre3)
  a.in = tr->act[2];
  if (launch_wgrad<16, 2, IN_BF16>(a, tr->g4, tr->partial, tr->nblk, s) != cudaSuccess) return HELM6_ERR_CUDA;
  reduce(3);
  t.in = tr->g4;
  t.cin = 2;
  t.w = tr->net.wtcb + (size_t)3 * 27 * 256;
  t.pre = tr->pre[2];
  t.out = tr->ga;
  note_launch();
  conv_tc_kernel<IN_G32, OUT_GRAD><<<tgrid, 128, TC_SMEM4, s>>>(t);
  // layers 3 and 2
  float* gcur = tr->ga;
  float* gnext = tr->gb;
  for (int l = 2; l >= 1; --l) {
    a.in = tr->act[l - 1];
    if (launch_wgrad<16, 16, IN_BF16>(a, gcur, tr->partial, tr->nblk, s) != cudaSuccess) return HELM6_ERR_CUDA;
    reduce(l);
    t.in = gcur;
    t.cin = 16;
    t.w = tr->net.wtcb + (size_t)l * 27 * 256;
    t.pre = tr->pre[l - 1];
    t.out = gnext;
    note_launch();
    conv_tc_kernel<IN_G32, OUT_GRAD><<<tgrid, 128, TC_SMEM4, s>>>(t);
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
                  tr->act[2], tr->y, tr->g4, tr->ga, tr->gb, tr->partial, tr->lpart, tr->loss, tr->tcerr};
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
  if (cnn_configure() != HELM6_OK) return fail(HELM6_ERR_CUDA);
  if (cnn_alloc(tr->net, true) != HELM6_OK) return fail(HELM6_ERR_NOMEM);
  if (cudaMalloc((void**)&tr->tcerr, sizeof(int)) != cudaSuccess || cudaMemset(tr->tcerr, 0, sizeof(int)) != cudaSuccess)
    return fail(HELM6_ERR_NOMEM);
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

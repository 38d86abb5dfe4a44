// Vector kernels of the Krylov solvers: classical Gram-Schmidt dot products and updates,
// norms, linear combinations, precision conversions, and the FP64 Givens least-squares
// update of GMRES, all on the device.  Dot products accumulate per thread in the vector
// precision and combine block partials in FP64.
#include <cuda_fp16.h>

#include <algorithm>
#include <atomic>
#include <type_traits>

#include "helm6_internal.h"

namespace helm6 {

namespace {

constexpr int RB = 256;  // threads per block of the reduction kernels

__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Sum a per-thread double over the block; result valid in thread 0.
__device__ __forceinline__ double block_sum(double v, double* sh) {
  v = warp_sum(v);
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __syncthreads();
  if (lane == 0) sh[w] = v;
  __syncthreads();
  v = (threadIdx.x < (blockDim.x >> 5)) ? sh[threadIdx.x] : 0.0;
  if (w == 0) v = warp_sum(v);
  return v;
}

// out[c] (+)= sum_b partial[b*ncols + c]; also adds into accum[c] when accum != nullptr.
__global__ void reduce_cols_kernel(const double* __restrict__ partial, int nblocks, int ncols,
                                   double* __restrict__ out, int accumulate, double* accum) {
  __shared__ double sh[RB / 32];
  const int c = blockIdx.x;
  double v = 0.0;
  for (int b = threadIdx.x; b < nblocks; b += blockDim.x) v += partial[(int64_t)b * ncols + c];
  v = block_sum(v, sh);
  if (threadIdx.x == 0) {
    out[c] = accumulate ? out[c] + v : v;
    if (accum) accum[c] += v;
  }
}

template <typename T>
__global__ void __launch_bounds__(RB) sumsq_kernel(const T* __restrict__ x, int64_t N,
                                                   double* __restrict__ partial) {
  __shared__ double sh[RB / 32];
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  T a = T(0);
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < 2 * N; idx += stride) {
    const T v = x[idx];
    a = fmx(v, v, a);
  }
  const double s = block_sum((double)a, sh);
  if (threadIdx.x == 0) partial[blockIdx.x] = s;
}

template <typename T>
__global__ void scale_copy_kernel(const T* __restrict__ x, T* __restrict__ y, int64_t n2,
                                  const double* __restrict__ inv_dev, double host_scale) {
  const T s = (T)(inv_dev ? *inv_dev : host_scale);
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < n2; idx += stride)
    y[idx] = x[idx] * s;
}

template <typename T>
struct V2;
template <>
struct V2<float> {
  using t = float2;
};
template <>
struct V2<double> {
  using t = double2;
};

// out (+)= scale * sum_i V_i y_i, y complex double.  Two points per thread (vector loads
// when the planes allow) and the basis read 8 vectors at a time, so that each thread has
// 16 independent loads in flight; sums in the input precision, widened once.
template <typename TI, typename TO, bool VEC>
__global__ void __launch_bounds__(RB) lincomb_kernel(const TI* __restrict__ V, int64_t vstride, int count,
                                                     const double* __restrict__ y, double scale,
                                                     TO* __restrict__ out, int64_t N, int accumulate,
                                                     const int* __restrict__ count_dev,
                                                     const double* __restrict__ scale_dev) {
  __shared__ TI yr[64], yi[64];
  if (count_dev) count = *count_dev;  // device-driven solves: the cycle's column count
  if (scale_dev) scale = *scale_dev;
  for (int c = threadIdx.x; c < count; c += blockDim.x) {
    yr[c] = (TI)(y[2 * c] * scale);
    yi[c] = (TI)(y[2 * c + 1] * scale);
  }
  __syncthreads();
  constexpr int P = VEC ? 2 : 1;
  constexpr int UB = 8;
  using TV = typename V2<TI>::t;
  const int64_t npts = N / P;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < npts; q += stride) {
    TI sr[P], si[P];
#pragma unroll
    for (int k = 0; k < P; ++k) sr[k] = si[k] = TI(0);
    for (int c0 = 0; c0 < count; c0 += UB) {
      TI vr[UB][P], vi[UB][P];
#pragma unroll
      for (int u = 0; u < UB; ++u) {
        if (c0 + u < count) {
          const TI* v = V + (int64_t)(c0 + u) * vstride;
          if constexpr (VEC) {
            const TV a = ((const TV*)v)[q], b = ((const TV*)(v + N))[q];
            vr[u][0] = a.x;
            vr[u][1 % P] = a.y;
            vi[u][0] = b.x;
            vi[u][1 % P] = b.y;
          } else {
            vr[u][0] = v[q];
            vi[u][0] = v[N + q];
          }
        }
      }
#pragma unroll
      for (int u = 0; u < UB; ++u) {
        if (c0 + u < count) {
          const TI a = yr[c0 + u], b = yi[c0 + u];
#pragma unroll
          for (int k = 0; k < P; ++k) {
            sr[k] = fmx(vr[u][k], a, fmx(-vi[u][k], b, sr[k]));
            si[k] = fmx(vr[u][k], b, fmx(vi[u][k], a, si[k]));
          }
        }
      }
    }
#pragma unroll
    for (int k = 0; k < P; ++k) {
      const int64_t idx = q * P + k;
      if (accumulate) {
        out[idx] += (TO)sr[k];
        out[N + idx] += (TO)si[k];
      } else {
        out[idx] = (TO)sr[k];
        out[N + idx] = (TO)si[k];
      }
    }
  }
}

template <typename TI, typename TO>
__global__ void convert_kernel(const TI* __restrict__ x, TO* __restrict__ y, int64_t n2, double scale,
                               const double* __restrict__ scale_dev) {
  if (scale_dev) scale = *scale_dev;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < n2; idx += stride)
    y[idx] = (TO)((double)x[idx] * scale);
}

__global__ void inter_to_planar_kernel(const double2* __restrict__ z, double* __restrict__ out, int64_t N) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < N; idx += stride) {
    const double2 v = z[idx];
    out[idx] = v.x;
    out[N + idx] = v.y;
  }
}

__global__ void planar_to_inter_kernel(const double* __restrict__ in, double2* __restrict__ z, int64_t N) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < N; idx += stride)
    z[idx] = make_double2(in[idx], in[N + idx]);
}

// Index in the caller's array of the internal point idx when the caller's axis xaxis
// (0 = x, 1 = y) is the internal z axis (and the internal z axis is the caller's xaxis):
// internal (i, j, l) is the caller's (l, j, i) for xaxis 0 and (i, l, j) for xaxis 1.
__device__ __forceinline__ int64_t caller_index(int64_t idx, int mx, int my, int mz, int xaxis) {
  const int64_t i = idx % mx, j = (idx / mx) % my, l = idx / ((int64_t)mx * my);
  return xaxis == 0 ? (i * my + j) * mz + l : (j * mz + l) * mx + i;
}

__global__ void inter_to_planar_x_kernel(const double2* __restrict__ z, double* __restrict__ out, int mx, int my,
                                         int mz, int xaxis) {
  const int64_t N = (int64_t)mx * my * mz, stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < N; idx += stride) {
    const double2 v = z[caller_index(idx, mx, my, mz, xaxis)];
    out[idx] = v.x;
    out[N + idx] = v.y;
  }
}

__global__ void planar_to_inter_x_kernel(const double* __restrict__ in, double2* __restrict__ z, int mx, int my,
                                         int mz, int xaxis) {
  const int64_t N = (int64_t)mx * my * mz, stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < N; idx += stride)
    z[caller_index(idx, mx, my, mz, xaxis)] = make_double2(in[idx], in[N + idx]);
}

__global__ void reduce_sum_kernel(const double* __restrict__ partial, int n, double* __restrict__ out) {
  __shared__ double sh[RB / 32];
  double v = 0.0;
  for (int b = threadIdx.x; b < n; b += blockDim.x) v += partial[b];
  v = block_sum(v, sh);
  if (threadIdx.x == 0) *out = v;
}

// ---- Arnoldi with delayed classical Gram-Schmidt (one reduction + one update per step) ----
// Vector traits for 2-point loads of a planar field.

constexpr int CHD = 8;  // most basis vectors per warp group of the reduction pass (4 accumulators each)

// P consecutive values of one plane, starting at point q * P, widened to the arithmetic
// type T.  S is the storage type: T itself (P = 1, 2, or 4 for float) or __half (P = 1, 2
// or 4).
template <typename T, int P, typename S>
__device__ __forceinline__ void ldpts(const S* p, int64_t q, T* o) {
  if constexpr (std::is_same<S, T>::value) {
    if constexpr (P == 1) {
      o[0] = p[q];
    } else if constexpr (P == 2) {
      const typename V2<T>::t v = ((const typename V2<T>::t*)p)[q];
      o[0] = v.x;
      o[1] = v.y;
    } else if constexpr (P == 4) {
      static_assert(std::is_same<T, float>::value, "4-point loads are FP32 or FP16");
      const float4 v = ((const float4*)p)[q];
      o[0] = v.x;
      o[1] = v.y;
      o[2] = v.z;
      o[3] = v.w;
    } else {
      static_assert(P == 8 && std::is_same<T, float>::value, "8-point loads are FP32 or FP16");
      const float4 a = ((const float4*)p)[2 * q], b = ((const float4*)p)[2 * q + 1];
      o[0] = a.x;
      o[1] = a.y;
      o[2] = a.z;
      o[3] = a.w;
      o[4] = b.x;
      o[5] = b.y;
      o[6] = b.z;
      o[7] = b.w;
    }
  } else {
    static_assert(std::is_same<S, __half>::value && std::is_same<T, float>::value, "FP16 storage, FP32 arithmetic");
    if constexpr (P == 1) {
      o[0] = __half2float(p[q]);
    } else if constexpr (P == 2) {
      const float2 a = __half22float2(((const __half2*)p)[q]);
      o[0] = a.x;
      o[1] = a.y;
    } else {
      static_assert(P == 4, "FP16 loads are 1, 2 or 4 points");
      const uint2 raw = ((const uint2*)p)[q];
      const float2 a = __half22float2(*(const __half2*)&raw.x), b = __half22float2(*(const __half2*)&raw.y);
      o[0] = a.x;
      o[1] = a.y;
      o[2] = b.x;
      o[3] = b.y;
    }
  }
}

// The store matching ldpts: values rounded to S (round to nearest even).
template <typename T, int P, typename S>
__device__ __forceinline__ void stpts(S* p, int64_t q, const T* v) {
  if constexpr (std::is_same<S, T>::value) {
    if constexpr (P == 1) {
      p[q] = v[0];
    } else if constexpr (P == 2) {
      ((typename V2<T>::t*)p)[q] = typename V2<T>::t{v[0], v[1]};
    } else if constexpr (P == 4) {
      ((float4*)p)[q] = float4{v[0], v[1], v[2], v[3]};
    } else {
      static_assert(P == 8, "stores of 1, 2, 4 or 8 points");
      ((float4*)p)[2 * q] = float4{v[0], v[1], v[2], v[3]};
      ((float4*)p)[2 * q + 1] = float4{v[4], v[5], v[6], v[7]};
    }
  } else {
    if constexpr (P == 1) {
      p[q] = __float2half_rn(v[0]);
    } else if constexpr (P == 2) {
      ((__half2*)p)[q] = __floats2half2_rn(v[0], v[1]);
    } else if constexpr (P == 4) {
      const __half2 a = __floats2half2_rn(v[0], v[1]), b = __floats2half2_rn(v[2], v[3]);
      uint2 raw;
      raw.x = *(const uint32_t*)&a;
      raw.y = *(const uint32_t*)&b;
      ((uint2*)p)[q] = raw;
    } else {
      static_assert(P == 8, "stores of 1, 2, 4 or 8 points");
      const __half2 a = __floats2half2_rn(v[0], v[1]), b = __floats2half2_rn(v[2], v[3]);
      const __half2 c = __floats2half2_rn(v[4], v[5]), d = __floats2half2_rn(v[6], v[7]);
      uint4 raw;
      raw.x = *(const uint32_t*)&a;
      raw.y = *(const uint32_t*)&b;
      raw.z = *(const uint32_t*)&c;
      raw.w = *(const uint32_t*)&d;
      ((uint4*)p)[q] = raw;
    }
  }
}

// P points of one plane held in registers as loaded: widened on use (get), so that an FP16
// basis takes one register per two points.
template <typename T, int P, typename S>
struct PtsReg {
  T v[P];
  __device__ __forceinline__ void load(const S* p, int64_t q) { ldpts<T, P, S>(p, q, v); }
  __device__ __forceinline__ T get(int k) const { return v[k]; }
};
template <>
struct PtsReg<float, 1, __half> {
  __half r;
  __device__ __forceinline__ void load(const __half* p, int64_t q) { r = p[q]; }
  __device__ __forceinline__ float get(int) const { return __half2float(r); }
};
template <>
struct PtsReg<float, 4, __half> {
  uint2 r;
  __device__ __forceinline__ void load(const __half* p, int64_t q) { r = ((const uint2*)p)[q]; }
  __device__ __forceinline__ float get(int k) const {
    const __half2 h = *(const __half2*)(k < 2 ? &r.x : &r.y);
    return (k & 1) ? __high2float(h) : __low2float(h);
  }
};
template <>
struct PtsReg<float, 8, __half> {
  uint4 r;
  __device__ __forceinline__ void load(const __half* p, int64_t q) { r = ((const uint4*)p)[q]; }
  __device__ __forceinline__ float get(int k) const {
    const uint32_t w = k < 2 ? r.x : k < 4 ? r.y : k < 6 ? r.z : r.w;
    const __half2 h = *(const __half2*)&w;
    return (k & 1) ? __high2float(h) : __low2float(h);
  }
};
template <>
struct PtsReg<float, 2, __half> {
  __half2 r;
  __device__ __forceinline__ void load(const __half* p, int64_t q) { r = ((const __half2*)p)[q]; }
  __device__ __forceinline__ float get(int k) const { return k == 0 ? __low2float(r) : __high2float(r); }
};

// x rounded to the storage type S and back (x itself when S is the arithmetic type).
template <typename T, typename S>
__device__ __forceinline__ T round_to(T x) {
  if constexpr (std::is_same<S, T>::value)
    return x;
  else
    return __half2float(__float2half_rn(x));
}

// One reduction pass over the basis V_0..V_{count-1}, u and (optionally) w.  Per block:
//   s_i = sum conj(V_i) u,  t_i = sum conj(V_i) w  (i < count),
//   a = sum |u|^2,  b = sum conj(u) w.
// Partial layout per block (ncol = 4 count + 3 doubles): s (2 count), t (2 count), a, b (2).
// The basis is stored in TV (T, or FP16 holding vscale V_i with vscale a power of two), so
// the s and t sums are multiplied by vinv = 1 / vscale in the block epilogue.
// The block's warps form G = 1, 2, 4 or 8 groups (the fewest with at most CH basis vectors
// each); all groups walk the same points, each reducing its own share of the basis, so u
// and w come from DRAM once (the other groups' loads of them hit L1) however many vectors
// there are.  More than G * CH vectors (restarts beyond 32) take further rounds.  At the
// end of a round every accumulator is reduced by warp shuffles and one shared-memory
// exchange.
template <typename T, int PTS, typename TV, int CH>
__global__ void __launch_bounds__(RB, sizeof(T) == 8 ? 1 : 2) dcgs_dot_kernel(const TV* __restrict__ V, int64_t vs, int count,
                                                         const T* __restrict__ u, const T* __restrict__ w,
                                                         int64_t N, double* __restrict__ partial, double vinv) {
  constexpr int NW = RB / 32;
  constexpr int NACC = 4 * CH + 3;
  __shared__ T sh[NW][NACC];
  const int ncol = 4 * count + 3;
  const bool hw = (w != nullptr);
  const int64_t npts = N / PTS;
  double* out = partial + (int64_t)blockIdx.x * ncol;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int G = 1;
  while (G < NW && (count + G - 1) / G > CH) G *= 2;
  const int wpg = NW / G;                     // warps per group
  const int grp = warp / wpg;
  const int tig = (warp % wpg) * 32 + lane;   // thread within the group
  const int64_t tpg = (int64_t)wpg * 32;
  const int64_t stride = (int64_t)gridDim.x * tpg;
  const int nround = count > 0 ? (count + G * CH - 1) / (G * CH) : 1;
  for (int rd = 0; rd < nround; ++rd) {
    const int rbase = rd * G * CH;
    const int rcount = min(G * CH, count - rbase);
    // group g reduces vectors [g rcount / G, (g + 1) rcount / G) of the round: shares
    // differ by at most one, the larger ones last (group 0 also forms a and b)
    const int base = rbase + grp * rcount / G;
    const int nc = rbase + (grp + 1) * rcount / G - base;
    const bool own = (rd == 0 && grp == 0);   // this group also forms a and b
    T acc[NACC];
#pragma unroll
    for (int c = 0; c < NACC; ++c) acc[c] = T(0);
    for (int64_t q = (int64_t)blockIdx.x * tpg + tig; q < npts; q += stride) {
      T ur[PTS], ui[PTS], wr[PTS], wi[PTS];
      ldpts<T, PTS, T>(u, q, ur);
      ldpts<T, PTS, T>(u + N, q, ui);
#pragma unroll
      for (int k = 0; k < PTS; ++k) wr[k] = wi[k] = T(0);
      if (hw) {
        ldpts<T, PTS, T>(w, q, wr);
        ldpts<T, PTS, T>(w + N, q, wi);
      }
      PtsReg<T, PTS, TV> vr[CH], vi[CH];
#pragma unroll
      for (int c = 0; c < CH; ++c) {
        if (c < nc) {
          const TV* v = V + (int64_t)(base + c) * vs;
          vr[c].load(v, q);
          vi[c].load(v + N, q);
        }
      }
      if (own) {
#pragma unroll
        for (int k = 0; k < PTS; ++k) {
          acc[4 * CH] = fmx(ur[k], ur[k], fmx(ui[k], ui[k], acc[4 * CH]));
          acc[4 * CH + 1] = fmx(ur[k], wr[k], fmx(ui[k], wi[k], acc[4 * CH + 1]));
          acc[4 * CH + 2] = fmx(ur[k], wi[k], fmx(-ui[k], wr[k], acc[4 * CH + 2]));
        }
      }
#pragma unroll
      for (int c = 0; c < CH; ++c) {
        if (c < nc) {
#pragma unroll
          for (int k = 0; k < PTS; ++k) {
            const T a = vr[c].get(k), b = vi[c].get(k);
            acc[4 * c] = fmx(a, ur[k], fmx(b, ui[k], acc[4 * c]));
            acc[4 * c + 1] = fmx(a, ui[k], fmx(-b, ur[k], acc[4 * c + 1]));
            acc[4 * c + 2] = fmx(a, wr[k], fmx(b, wi[k], acc[4 * c + 2]));
            acc[4 * c + 3] = fmx(a, wi[k], fmx(-b, wr[k], acc[4 * c + 3]));
          }
        }
      }
    }
#pragma unroll
    for (int c = 0; c < NACC; ++c) {
      T v = acc[c];
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      if (lane == 0) sh[warp][c] = v;
    }
    __syncthreads();
    // group gg's sums over its wpg warps; column c of its accumulators
    for (int e = threadIdx.x; e < G * NACC; e += blockDim.x) {
      const int gg = e / NACC, c = e - gg * NACC;
      double sum = 0.0;
      for (int ww = 0; ww < wpg; ++ww) sum += (double)sh[gg * wpg + ww][c];
      const int gbase = rbase + gg * rcount / G;
      const int gnc = rbase + (gg + 1) * rcount / G - gbase;
      if (c < 4 * CH) {
        const int cc = c >> 2, kind = c & 3;
        if (cc < gnc) out[(kind < 2 ? 0 : 2 * count) + 2 * (gbase + cc) + (kind & 1)] = sum * vinv;
      } else if (rd == 0 && gg == 0) {
        out[4 * count + (c - 4 * CH)] = sum;
      }
    }
    __syncthreads();
  }
}

// One update pass.  coef (complex double unless noted): s[count], t[count], c, inv (real).
//   v_new = (u - sum_i V_i s_i) inv          -> written to v_out (the basis slot `count`)
//   u     = (w - sum_i V_i t_i - v_new c) inv -> written over u (in place)
// With the basis stored in FP16 as vscale V_i, the coefficients are divided by vscale, v_out
// receives vscale v_new rounded to FP16, and the correction of u uses that rounded vector,
// so that u is orthogonalised against the basis as stored.  PTS points per thread; the basis
// is read UB vectors at a time, all loads of a group issued before its FMAs.
template <typename T, int PTS, typename TV, int UB = 8>
__global__ void __launch_bounds__(RB) dcgs_update_kernel(const TV* __restrict__ V, int64_t vs, int count,
                                                         T* u, const T* __restrict__ w, TV* __restrict__ v_out,
                                                         int64_t N, const double* __restrict__ coef, double vscale) {
  __shared__ T s_r[64], s_i[64], t_r[64], t_i[64];
  __shared__ T cc[3];
  const double vinv = 1.0 / vscale;
  for (int c = threadIdx.x; c < count; c += blockDim.x) {
    s_r[c] = (T)(coef[2 * c] * vinv);
    s_i[c] = (T)(coef[2 * c + 1] * vinv);
    t_r[c] = (T)(coef[2 * count + 2 * c] * vinv);
    t_i[c] = (T)(coef[2 * count + 2 * c + 1] * vinv);
  }
  if (threadIdx.x == 0) {
    cc[0] = (T)coef[4 * count];
    cc[1] = (T)coef[4 * count + 1];
    cc[2] = (T)coef[4 * count + 2];
  }
  __syncthreads();
  const T cr = cc[0], ci = cc[1], inv = cc[2];
  const T vsc = (T)vscale, vin = (T)vinv;  // powers of two: exact in T
  const int64_t npts = N / PTS;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < npts; q += stride) {
    T ur[PTS], ui[PTS], wr[PTS], wi[PTS];
    ldpts<T, PTS, T>(u, q, ur);
    ldpts<T, PTS, T>(u + N, q, ui);
    ldpts<T, PTS, T>(w, q, wr);
    ldpts<T, PTS, T>(w + N, q, wi);
    for (int c0 = 0; c0 < count; c0 += UB) {
      PtsReg<T, PTS, TV> vr[UB], vi[UB];
#pragma unroll
      for (int e = 0; e < UB; ++e) {
        if (c0 + e < count) {
          const TV* v = V + (int64_t)(c0 + e) * vs;
          vr[e].load(v, q);
          vi[e].load(v + N, q);
        }
      }
#pragma unroll
      for (int e = 0; e < UB; ++e) {
        if (c0 + e < count) {
          const int c = c0 + e;
#pragma unroll
          for (int k = 0; k < PTS; ++k) {
            const T a = vr[e].get(k), b = vi[e].get(k);
            ur[k] = fmx(-a, s_r[c], fmx(b, s_i[c], ur[k]));
            ui[k] = fmx(-a, s_i[c], fmx(-b, s_r[c], ui[k]));
            wr[k] = fmx(-a, t_r[c], fmx(b, t_i[c], wr[k]));
            wi[k] = fmx(-a, t_i[c], fmx(-b, t_r[c], wi[k]));
          }
        }
      }
    }
    T nr[PTS], ni[PTS];
#pragma unroll
    for (int k = 0; k < PTS; ++k) {
      nr[k] = ur[k] * inv * vsc;
      ni[k] = ui[k] * inv * vsc;
    }
    stpts<T, PTS, TV>(v_out, q, nr);
    stpts<T, PTS, TV>(v_out + N, q, ni);
#pragma unroll
    for (int k = 0; k < PTS; ++k) {
      const T a = round_to<T, TV>(nr[k]) * vin, b = round_to<T, TV>(ni[k]) * vin;
      wr[k] = fmx(-a, cr, fmx(b, ci, wr[k])) * inv;
      wi[k] = fmx(-a, ci, fmx(-b, cr, wi[k])) * inv;
    }
    stpts<T, PTS, T>(u, q, wr);
    stpts<T, PTS, T>(u + N, q, wi);
  }
}

// ---- GMRES least squares (FP64, one thread) ----
struct zc {
  double re, im;
};
__device__ __forceinline__ zc ld(const double* p) { return zc{p[0], p[1]}; }
__device__ __forceinline__ void st(double* p, zc v) { p[0] = v.re; p[1] = v.im; }
__device__ __forceinline__ zc zmul(zc a, zc b) { return zc{a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re}; }
__device__ __forceinline__ zc zadd(zc a, zc b) { return zc{a.re + b.re, a.im + b.im}; }
__device__ __forceinline__ double zabs(zc a) { return hypot(a.re, a.im); }

// Rotation i acts on rows (i, i+1): [c s; -conj(s) c], c real (stored in cs[2i]), s complex.
__global__ void givens_kernel(double* H, int ldh, int j, double* cs, double* sn, double* g, double* res) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double* col = H + 2 * (int64_t)j * ldh;
  for (int i = 0; i < j; ++i) {
    const zc hi = ld(col + 2 * i), hn = ld(col + 2 * (i + 1));
    const double c = cs[2 * i];
    const zc s = ld(sn + 2 * i);
    const zc t = zadd(zc{c * hi.re, c * hi.im}, zmul(s, hn));
    const zc u = zadd(zmul(zc{-s.re, s.im}, hi), zc{c * hn.re, c * hn.im});  // -conj(s) hi + c hn
    st(col + 2 * i, t);
    st(col + 2 * (i + 1), u);
  }
  const zc a = ld(col + 2 * j), b = ld(col + 2 * (j + 1));
  const double aa = zabs(a), bb = zabs(b);
  const double den = hypot(aa, bb);
  double c;
  zc s;
  if (den == 0.0) {
    c = 1.0;
    s = zc{0.0, 0.0};
  } else if (aa == 0.0) {
    c = 0.0;
    s = zc{1.0, 0.0};
  } else {
    c = aa / den;
    const zc ph = zc{a.re / aa, a.im / aa};
    s = zmul(ph, zc{b.re / den, -b.im / den});
  }
  cs[2 * j] = c;
  cs[2 * j + 1] = 0.0;
  st(sn + 2 * j, s);
  st(col + 2 * j, zadd(zc{c * a.re, c * a.im}, zmul(s, b)));
  st(col + 2 * (j + 1), zc{0.0, 0.0});
  const zc gj = ld(g + 2 * j);
  st(g + 2 * (j + 1), zmul(zc{-s.re, s.im}, gj));
  st(g + 2 * j, zc{c * gj.re, c * gj.im});
  *res = zabs(ld(g + 2 * (j + 1)));
}


// Small FP64 algebra of one delayed Gram-Schmidt Arnoldi step j (one thread).
// red: reduced sums s_i = V_i^H u_j, t_i = V_i^H w (i < j), a = ||u_j||^2, b = u_j^H w.
// u_j = V s + alpha v_j with alpha^2 = a - ||s||^2.
//   * column j-1 of the raw Hessenberg Hr gets += s and subdiagonal alpha; it is copied to R
//     and rotated (Givens), giving the residual estimate *est = |g_j| (j = 0: g_0 = alpha);
//   * with w = A M^{-1} u_j (has_w): v_j^H w = (b - s^H t)/alpha = c_j, column j of Hr is
//     ([t; c_j] - Hr[:, 0..j-1] s)/alpha, and T (z_l = sum_i T[i,l] z~_i) gets column
//     (e_j - T s)/alpha;
//   * coef = [s, t, c_j, 1/alpha] for the update pass v_j = (u - V s)/alpha,
//     u_{j+1} = (w - V t - v_j c_j)/alpha.
// *brk = 1 when alpha^2 <= 1e-28 a (u_j in the span of the basis: breakdown).
constexpr int STEP_T = 128;   // threads of the step kernel
constexpr int STEP_MAXJ = 64;  // largest restart length (helm6_opts.max_restart <= 64)

// Sums of three doubles over the block; every thread receives them.
__device__ __forceinline__ void block_sum3(double& a, double& b, double& c, double* sh) {
  a = warp_sum(a);
  b = warp_sum(b);
  c = warp_sum(c);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) {
    sh[3 * w] = a;
    sh[3 * w + 1] = b;
    sh[3 * w + 2] = c;
  }
  __syncthreads();
  a = b = c = 0.0;
  for (int i = 0; i < STEP_T / 32; ++i) {
    a += sh[3 * i];
    b += sh[3 * i + 1];
    c += sh[3 * i + 2];
  }
  __syncthreads();
}

// One block of STEP_T threads; the rotation sweep runs on thread 0 over shared-memory copies
// of the column and of the previous rotations, the O(j^2) products warp per row.
__global__ void __launch_bounds__(STEP_T) dcgs_step_kernel(int j, int has_w, const double* red, double* Hr, double* R,
                                                           int ldh, double* T, int ldt, double* cs, double* sn,
                                                           double* g, double* coef, double* est, int* brk) {
  __shared__ double shr[3 * STEP_T / 32];
  __shared__ double scol[2 * (STEP_MAXJ + 2)], scs[STEP_MAXJ + 1], ssn[2 * (STEP_MAXJ + 1)];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const double* sv = red;
  const double* tv = red + 2 * j;
  const double a = red[4 * j];
  const zc b = zc{red[4 * j + 1], red[4 * j + 2]};
  double s2 = 0.0, pr = 0.0, pi = 0.0;
  for (int i = tid; i < j; i += STEP_T) {
    s2 += sv[2 * i] * sv[2 * i] + sv[2 * i + 1] * sv[2 * i + 1];
    if (has_w) {
      const zc q = zmul(zc{sv[2 * i], -sv[2 * i + 1]}, ld(tv + 2 * i));
      pr += q.re;
      pi += q.im;
    }
  }
  block_sum3(s2, pr, pi, shr);
  const double al2 = a - s2;
  const bool bd = !(al2 > 1e-28 * fmax(a, 1e-300)) || !isfinite(al2);
  const double al = bd ? 0.0 : sqrt(al2);
  const double inv = bd ? 0.0 : 1.0 / al;
  if (tid == 0) *brk = bd ? 1 : 0;
  for (int i = tid; i < j; i += STEP_T) {
    coef[2 * i] = sv[2 * i];
    coef[2 * i + 1] = sv[2 * i + 1];
    coef[2 * j + 2 * i] = tv[2 * i];
    coef[2 * j + 2 * i + 1] = tv[2 * i + 1];
  }
  if (j >= 1) {
    // lagged correction of column j - 1 and its subdiagonal
    double* hc = Hr + 2 * (int64_t)(j - 1) * ldh;
    for (int i = tid; i < j; i += STEP_T) {
      hc[2 * i] += sv[2 * i];
      hc[2 * i + 1] += sv[2 * i + 1];
    }
    if (tid == 0) {
      hc[2 * j] = al;
      hc[2 * j + 1] = 0.0;
    }
    __syncthreads();
    for (int r = tid; r <= 2 * j + 1; r += STEP_T) scol[r] = hc[r];
    for (int i = tid; i < j - 1; i += STEP_T) {
      scs[i] = cs[2 * i];
      ssn[2 * i] = sn[2 * i];
      ssn[2 * i + 1] = sn[2 * i + 1];
    }
    __syncthreads();
    if (tid == 0) {
      // previous rotations on the column, then the rotation that zeroes its subdiagonal
      const int jj = j - 1;
      for (int i = 0; i < jj; ++i) {
        const zc hi = ld(scol + 2 * i), hn = ld(scol + 2 * (i + 1));
        const double c = scs[i];
        const zc s = ld(ssn + 2 * i);
        st(scol + 2 * i, zadd(zc{c * hi.re, c * hi.im}, zmul(s, hn)));
        st(scol + 2 * (i + 1), zadd(zmul(zc{-s.re, s.im}, hi), zc{c * hn.re, c * hn.im}));
      }
      const zc x = ld(scol + 2 * jj), y = ld(scol + 2 * (jj + 1));
      const double ax = zabs(x), ay = zabs(y);
      const double den = hypot(ax, ay);
      double c;
      zc s;
      if (den == 0.0) {
        c = 1.0;
        s = zc{0.0, 0.0};
      } else if (ax == 0.0) {
        c = 0.0;
        s = zc{1.0, 0.0};
      } else {
        c = ax / den;
        s = zmul(zc{x.re / ax, x.im / ax}, zc{y.re / den, -y.im / den});
      }
      cs[2 * jj] = c;
      cs[2 * jj + 1] = 0.0;
      st(sn + 2 * jj, s);
      st(scol + 2 * jj, zadd(zc{c * x.re, c * x.im}, zmul(s, y)));
      st(scol + 2 * (jj + 1), zc{0.0, 0.0});
      const zc gj = ld(g + 2 * jj);
      const zc gn = zmul(zc{-s.re, s.im}, gj);
      st(g + 2 * (jj + 1), gn);
      st(g + 2 * jj, zc{c * gj.re, c * gj.im});
      *est = zabs(gn);
    }
    __syncthreads();
    double* rc = R + 2 * (int64_t)(j - 1) * ldh;
    for (int r = tid; r <= 2 * j + 1; r += STEP_T) rc[r] = scol[r];
  } else if (tid == 0) {
    g[0] = al;
    g[1] = 0.0;
    *est = al;
  }
  if (!has_w || bd) {
    if (tid == 0) {
      coef[4 * j] = 0.0;
      coef[4 * j + 1] = 0.0;
      coef[4 * j + 2] = inv;
    }
    return;
  }
  // c_j = (b - s^H t) / alpha
  const zc cj = zc{(b.re - pr) * inv, (b.im - pi) * inv};
  // column j of Hr: ([t; c_j] - Hr[:, 0..j-1] s) / alpha, rows 0..j (Hessenberg: i >= r - 1)
  double* hj = Hr + 2 * (int64_t)j * ldh;
  for (int r = warp; r <= j; r += STEP_T / 32) {
    double qr = 0.0, qi = 0.0;
    for (int i = (r > 0 ? r - 1 : 0) + lane; i < j; i += 32) {
      const zc q = zmul(ld(Hr + 2 * ((int64_t)i * ldh + r)), ld(sv + 2 * i));
      qr += q.re;
      qi += q.im;
    }
    qr = warp_sum(qr);
    qi = warp_sum(qi);
    if (lane == 0) {
      const zc base = (r < j) ? ld(tv + 2 * r) : cj;
      hj[2 * r] = (base.re - qr) * inv;
      hj[2 * r + 1] = (base.im - qi) * inv;
    }
  }
  // T column j: (e_j - T s) / alpha (T upper triangular)
  if (T) {
    for (int r = warp; r < j; r += STEP_T / 32) {
      double qr = 0.0, qi = 0.0;
      for (int i = r + lane; i < j; i += 32) {
        const zc q = zmul(ld(T + 2 * ((int64_t)i * ldt + r)), ld(sv + 2 * i));
        qr += q.re;
        qi += q.im;
      }
      qr = warp_sum(qr);
      qi = warp_sum(qi);
      if (lane == 0) {
        T[2 * ((int64_t)j * ldt + r)] = -qr * inv;
        T[2 * ((int64_t)j * ldt + r) + 1] = -qi * inv;
      }
    }
    if (tid == 0) {
      T[2 * ((int64_t)j * ldt + j)] = inv;
      T[2 * ((int64_t)j * ldt + j) + 1] = 0.0;
    }
  }
  if (tid == 0) {
    coef[4 * j] = cj.re;
    coef[4 * j + 1] = cj.im;
    coef[4 * j + 2] = inv;
  }
}

// q = T[0..k-1, 0..k-1] y (T upper triangular, column-major, leading dimension ldt).
__global__ void tri_mul_kernel(const double* T, int ldt, int k, const double* y, double* q, const int* k_dev) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  if (k_dev) k = *k_dev;
  for (int r = 0; r < k; ++r) {
    zc acc = zc{0.0, 0.0};
    for (int i = r; i < k; ++i) acc = zadd(acc, zmul(ld(T + 2 * ((int64_t)i * ldt + r)), ld(y + 2 * i)));
    st(q + 2 * r, acc);
  }
}

__global__ void set_subdiag_kernel(double* H, int ldh, int j, const double* sumsq, double* inv) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const double nrm = sqrt(fmax(*sumsq, 0.0));
  double* col = H + 2 * (int64_t)j * ldh;
  col[2 * (j + 1)] = nrm;
  col[2 * (j + 1) + 1] = 0.0;
  *inv = (nrm > 0.0) ? 1.0 / nrm : 0.0;
}

__global__ void backsolve_kernel(const double* H, int ldh, int j, const double* g, double* y, const int* j_dev) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  if (j_dev) j = *j_dev;
  for (int r = j - 1; r >= 0; --r) {
    zc acc = ld(g + 2 * r);
    for (int c = r + 1; c < j; ++c) {
      const zc h = ld(H + 2 * ((int64_t)c * ldh + r));
      const zc yc = ld(y + 2 * c);
      const zc p = zmul(h, yc);
      acc.re -= p.re;
      acc.im -= p.im;
    }
    const zc d = ld(H + 2 * ((int64_t)r * ldh + r));
    const double n2 = d.re * d.re + d.im * d.im;
    zc v = (n2 > 0.0) ? zmul(acc, zc{d.re / n2, -d.im / n2}) : zc{0.0, 0.0};
    st(y + 2 * r, v);
  }
}

// y (+)= alpha * x over 2N reals (accumulate = 0: y = alpha * x)
template <typename TI, typename TO>
__global__ void axpy_kernel(const TI* __restrict__ x, TO* __restrict__ y, int64_t n2, double alpha) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < n2; idx += stride)
    y[idx] += (TO)(alpha * (double)x[idx]);
}

__global__ void set_complex_kernel(double* p, double re, double im) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    p[0] = re;
    p[1] = im;
  }
}

int grid_for(int64_t n, int bs) {
  static int sms = 0;
  if (!sms) sms = device_sm_count();
  int64_t g = (n + bs - 1) / bs;
  const int64_t cap = (int64_t)sms * 8;
  if (g > cap) g = cap;
  if (g < 1) g = 1;
  return (int)g;
}

}  // namespace

static std::atomic<long long> g_launches{0};
void note_launch(int n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
long long launch_total() { return g_launches.load(std::memory_order_relaxed); }

int device_sm_count() {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return sms > 0 ? sms : 1;
}

void launch_reduce_cols(const double* partial, int nblocks, int ncols, double* out, int accumulate,
                        cudaStream_t s) {
  note_launch();
  reduce_cols_kernel<<<ncols, RB, 0, s>>>(partial, nblocks, ncols, out, accumulate, nullptr);
}

template <typename T>
void launch_sumsq(const T* x, int64_t N, double* partial, int nblocks, cudaStream_t s) {
  note_launch();
  sumsq_kernel<T><<<nblocks, RB, 0, s>>>(x, N, partial);
}

template <typename T>
void launch_scale_copy(const T* x, T* y, int64_t N, const double* inv_dev, double host_scale,
                       cudaStream_t s) {
  note_launch();
  scale_copy_kernel<T><<<grid_for(2 * N, RB), RB, 0, s>>>(x, y, 2 * N, inv_dev, host_scale);
}

template <typename TI, typename TO>
void launch_lincomb(const TI* V, int64_t vstride, int count, const double* y, double scale, TO* out,
                    int64_t N, int accumulate, cudaStream_t s, const int* count_dev, const double* scale_dev) {
  note_launch();
  if ((N & 1) == 0 && (vstride & 1) == 0)
    lincomb_kernel<TI, TO, true><<<grid_for(N / 2, RB), RB, 0, s>>>(V, vstride, count, y, scale, out, N, accumulate,
                                                                      count_dev, scale_dev);
  else
    lincomb_kernel<TI, TO, false><<<grid_for(N, RB), RB, 0, s>>>(V, vstride, count, y, scale, out, N, accumulate,
                                                                   count_dev, scale_dev);
}

template <typename TI, typename TO>
void launch_convert(const TI* x, TO* y, int64_t N, double scale, cudaStream_t s, const double* scale_dev) {
  note_launch();
  convert_kernel<TI, TO><<<grid_for(2 * N, RB), RB, 0, s>>>(x, y, 2 * N, scale, scale_dev);
}

void launch_interleaved_to_planar(const double* zin, double* out, int64_t N, cudaStream_t s) {
  note_launch();
  inter_to_planar_kernel<<<grid_for(N, RB), RB, 0, s>>>((const double2*)zin, out, N);
}

void launch_planar_to_interleaved(const double* in, double* zout, int64_t N, cudaStream_t s) {
  note_launch();
  planar_to_inter_kernel<<<grid_for(N, RB), RB, 0, s>>>(in, (double2*)zout, N);
}

void launch_caller_to_planar(const Geom& g, int xaxis, const double* zin, double* out, cudaStream_t s) {
  if (xaxis < 0) {
    launch_interleaved_to_planar(zin, out, g.N, s);
    return;
  }
  note_launch();
  inter_to_planar_x_kernel<<<grid_for(g.N, RB), RB, 0, s>>>((const double2*)zin, out, g.mx, g.my, g.mz, xaxis);
}

void launch_planar_to_caller(const Geom& g, int xaxis, const double* in, double* zout, cudaStream_t s) {
  if (xaxis < 0) {
    launch_planar_to_interleaved(in, zout, g.N, s);
    return;
  }
  note_launch();
  planar_to_inter_x_kernel<<<grid_for(g.N, RB), RB, 0, s>>>(in, (double2*)zout, g.mx, g.my, g.mz, xaxis);
}

void launch_reduce_sum(const double* partial, int n, double* out, cudaStream_t s) {
  note_launch();
  reduce_sum_kernel<<<1, RB, 0, s>>>(partial, n, out);
}

void launch_givens(double* H, int ldh, int j, double* cs, double* sn, double* g, double* res,
                   cudaStream_t s) {
  note_launch();
  givens_kernel<<<1, 32, 0, s>>>(H, ldh, j, cs, sn, g, res);
}

void launch_dcgs_step(int j, int has_w, const double* red, double* Hr, double* R, int ldh, double* T, int ldt,
                      double* cs, double* sn, double* g, double* coef, double* est, int* brk, cudaStream_t s) {
  note_launch();
  dcgs_step_kernel<<<1, STEP_T, 0, s>>>(j, has_w, red, Hr, R, ldh, T, ldt, cs, sn, g, coef, est, brk);
}

void launch_tri_mul(const double* T, int ldt, int k, const double* y, double* q, cudaStream_t s, const int* k_dev) {
  note_launch();
  tri_mul_kernel<<<1, 32, 0, s>>>(T, ldt, k, y, q, k_dev);
}

void launch_set_subdiag(double* H, int ldh, int j, const double* sumsq, double* inv, cudaStream_t s) {
  note_launch();
  set_subdiag_kernel<<<1, 32, 0, s>>>(H, ldh, j, sumsq, inv);
}

void launch_backsolve(const double* H, int ldh, int j, const double* g, double* y, cudaStream_t s, const int* j_dev) {
  note_launch();
  backsolve_kernel<<<1, 32, 0, s>>>(H, ldh, j, g, y, j_dev);
}

__global__ void axpby_kernel(const double* __restrict__ x, double* __restrict__ y, int64_t n, double a, double b) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = fma(a, y[i], b * x[i]);
}

void launch_axpby(const double* x, double* y, int64_t N, double a, double b, cudaStream_t s) {
  note_launch();
  axpby_kernel<<<grid_for(2 * N, RB), RB, 0, s>>>(x, y, 2 * N, a, b);
}

template <typename TI, typename TO>
void launch_axpy(const TI* x, TO* y, int64_t N, double alpha, cudaStream_t s) {
  note_launch();
  axpy_kernel<TI, TO><<<grid_for(2 * N, RB), RB, 0, s>>>(x, y, 2 * N, alpha);
}

void launch_set_complex(double* p, double re, double im, cudaStream_t s) {
  note_launch();
  set_complex_kernel<<<1, 32, 0, s>>>(p, re, im);
}

template void launch_axpy<float, double>(const float*, double*, int64_t, double, cudaStream_t);
template void launch_axpy<double, double>(const double*, double*, int64_t, double, cudaStream_t);

template <typename T>
int cgs_blocks(int64_t N) {
  static int sms = 0;
  if (!sms) sms = device_sm_count();
  int64_t g = (N + RB - 1) / RB;
  const int64_t cap = (int64_t)sms * 8;
  return (int)std::max<int64_t>(1, std::min(g, cap));
}

// Points per thread of the two Gram-Schmidt passes, as many as the planes' alignment allows
// up to 2 for an FP32 or FP64 basis (one 8- or 16-byte load per plane and vector) and 4 for
// an FP16 one (8-byte basis loads; fewer instructions per byte than 2 points).
template <typename TV>
int cgs_pts(int64_t N, int64_t vs) {
  if (std::is_same<TV, __half>::value && N % 4 == 0 && vs % 4 == 0) return 4;
  return (N % 2 == 0 && vs % 2 == 0) ? 2 : 1;
}

// Vectors per warp group of the 8-point FP16 reduction pass for `count` basis vectors: the
// fewest groups G (a power of two, at most 8) that leave at most 6 vectors to a group, and
// the kernel instance compiled for exactly that share (measured at 256 x 258 x 258: an
// instance sized for more vectors than it gets, or a split into more groups, is slower).
int dot_share(int count) {
  int G = 1;
  while (G < 8 && (count + G - 1) / G > 6) G *= 2;
  return std::max(1, std::min(6, (count + G - 1) / G));
}

template <typename T, typename TV>
void launch_dcgs_dot(const TV* V, int64_t vs, int count, const T* u, const T* w, int64_t N, double* partial,
                     int nblocks, double vscale, cudaStream_t s) {
  note_launch();
  const double vinv = 1.0 / vscale;
  if constexpr (std::is_same<TV, __half>::value) {
    if (N % 8 == 0 && vs % 8 == 0) {
      // 8 points per thread: 16-byte basis loads, twice the bytes in flight of 4 points
      switch (dot_share(count)) {
#define DOT8(CH)                                                                                   \
  case CH:                                                                                         \
    dcgs_dot_kernel<T, 8, TV, CH><<<nblocks, RB, 0, s>>>(V, vs, count, u, w, N, partial, vinv); \
    return;
        DOT8(1) DOT8(2) DOT8(3) DOT8(4) DOT8(5) DOT8(6)
#undef DOT8
      }
    }
    if (cgs_pts<TV>(N, vs) == 4) {
      dcgs_dot_kernel<T, 4, TV, CHD><<<nblocks, RB, 0, s>>>(V, vs, count, u, w, N, partial, vinv);
      return;
    }
  }
  if (cgs_pts<TV>(N, vs) == 2)
    dcgs_dot_kernel<T, 2, TV, CHD><<<nblocks, RB, 0, s>>>(V, vs, count, u, w, N, partial, vinv);
  else
    dcgs_dot_kernel<T, 1, TV, CHD><<<nblocks, RB, 0, s>>>(V, vs, count, u, w, N, partial, vinv);
}

// Blocks of the reduction pass: two per SM (its per-block epilogue favours few blocks).
int dot_blocks() { return 2 * device_sm_count(); }

template <typename T, typename TV>
void launch_dcgs_update(const TV* V, int64_t vs, int count, T* u, const T* w, TV* v_out, int64_t N,
                        const double* coef, int nblocks, double vscale, cudaStream_t s) {
  note_launch();
  const int p = cgs_pts<TV>(N, vs);
  if constexpr (std::is_same<TV, __half>::value) {
    if (N % 8 == 0 && vs % 8 == 0) {
      // 8 points per thread, the basis read 4 vectors at a time (measured best at 256 x 258 x 258)
      dcgs_update_kernel<T, 8, TV, 4><<<nblocks, RB, 0, s>>>(V, vs, count, u, w, v_out, N, coef, vscale);
      return;
    }
    if (p == 4) {
      dcgs_update_kernel<T, 4, TV><<<nblocks, RB, 0, s>>>(V, vs, count, u, w, v_out, N, coef, vscale);
      return;
    }
  }
  if (p == 2)
    dcgs_update_kernel<T, 2, TV><<<nblocks, RB, 0, s>>>(V, vs, count, u, w, v_out, N, coef, vscale);
  else
    dcgs_update_kernel<T, 1, TV><<<nblocks, RB, 0, s>>>(V, vs, count, u, w, v_out, N, coef, vscale);
}

template int cgs_blocks<float>(int64_t);
template int cgs_blocks<double>(int64_t);
#define INST_CGS(T, TV)                                                                              \
  template void launch_dcgs_dot<T, TV>(const TV*, int64_t, int, const T*, const T*, int64_t, double*, int, double, \
                                       cudaStream_t);                                                          \
  template void launch_dcgs_update<T, TV>(const TV*, int64_t, int, T*, const T*, TV*, int64_t, const double*, int, \
                                          double, cudaStream_t);
INST_CGS(float, float)
INST_CGS(float, __half)
INST_CGS(double, double)

#define INST_T(T)                                                                              \
  template void launch_sumsq<T>(const T*, int64_t, double*, int, cudaStream_t);                  \
  template void launch_scale_copy<T>(const T*, T*, int64_t, const double*, double, cudaStream_t);
INST_T(float)
INST_T(double)
template void launch_lincomb<float, double>(const float*, int64_t, int, const double*, double, double*,
                                            int64_t, int, cudaStream_t, const int*, const double*);
template void launch_lincomb<double, double>(const double*, int64_t, int, const double*, double,
                                             double*, int64_t, int, cudaStream_t, const int*, const double*);
template void launch_lincomb<float, float>(const float*, int64_t, int, const double*, double, float*,
                                           int64_t, int, cudaStream_t, const int*, const double*);
template void launch_convert<double, float>(const double*, float*, int64_t, double, cudaStream_t, const double*);
template void launch_convert<float, double>(const float*, double*, int64_t, double, cudaStream_t, const double*);
template void launch_convert<double, double>(const double*, double*, int64_t, double, cudaStream_t, const double*);

// ---- control of device-driven solves (graph with conditional nodes) ----
namespace {

// After a true residual: its norm, the solve's status and whether another cycle follows.
__global__ void gctl_residual_kernel(GraphCtl* g, const double* sumsq, const int* zst, const int* tcerr, int first,
                                     cudaGraphConditionalHandle hw) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const double beta = sqrt(fmax(*sumsq, 0.0));
  if (first) {
    g->iters = 0;
    g->outer = 0;
    g->nhist = 0;
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    g->t0 = t;
    if (g->nhist < HELM6_MAX_HIST) g->hist[g->nhist++] = beta / g->normF;
  } else {
    g->outer++;
    if (g->nhist > 0) g->hist[g->nhist - 1] = beta / g->normF;  // the true residual replaces the estimate
  }
  g->beta = beta;
  int st = -1;
  if (!first && *tcerr) st = HELM6_ERR_CUDA;
  else if (!first && *zst == HELM6_BREAKDOWN) st = HELM6_BREAKDOWN;
  else if (!isfinite(beta)) st = HELM6_NONFINITE;
  else if (beta <= g->tol_abs) st = HELM6_OK;
  else if (g->iters >= g->maxit) st = HELM6_NOT_CONVERGED;
  if (st == -1) {
    g->inv_beta = 1.0 / beta;
    g->itol = fmax(g->inner, g->itol_num / beta);
  } else {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    g->t1 = t;
  }
  g->status = st;
  cudaGraphSetConditional(hw, st == -1 ? 1u : 0u);
}

// A cycle starts: step 0 runs, the later steps only when their predecessor enables them.
__global__ void gctl_cycle_kernel(GraphCtl* g, StepHandles ha, int m) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  g->k = 0;
  for (int j = 0; j <= m; ++j) cudaGraphSetConditional(ha.h[j], j == 0 ? 1u : 0u);
}

// After Arnoldi step j (its estimate is that of column j - 1): whether step j + 1 runs.
__global__ void gctl_step_kernel(GraphCtl* g, int j, int m, const double* est, const int* brk,
                                 cudaGraphConditionalHandle next) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const double e = *est;
  const int b = *brk;
  bool stop;
  if (j == 0) {
    stop = b || !isfinite(e);
  } else {
    g->iters++;
    if (g->nhist < HELM6_MAX_HIST) g->hist[g->nhist++] = e * g->beta / g->normF;
    stop = !(e > g->itol) || !isfinite(e) || b || j >= m || g->iters >= g->maxit;
  }
  if (stop) g->k = j;
  if (j < m) cudaGraphSetConditional(next, stop ? 0u : 1u);
}

}  // namespace

void launch_gctl_residual(GraphCtl* g, const double* sumsq, const int* zst, const int* tcerr, int first,
                          cudaGraphConditionalHandle hw, cudaStream_t s) {
  note_launch();
  gctl_residual_kernel<<<1, 32, 0, s>>>(g, sumsq, zst, tcerr, first, hw);
}
void launch_gctl_cycle(GraphCtl* g, const StepHandles& ha, int m, cudaStream_t s) {
  note_launch();
  gctl_cycle_kernel<<<1, 32, 0, s>>>(g, ha, m);
}
void launch_gctl_step(GraphCtl* g, int j, int m, const double* est, const int* brk, cudaGraphConditionalHandle next,
                      cudaStream_t s) {
  note_launch();
  gctl_step_kernel<<<1, 32, 0, s>>>(g, j, m, est, brk, next);
}

}  // namespace helm6

// Vector kernels of the Krylov solvers: classical Gram-Schmidt dot products and updates,
// norms, linear combinations, precision conversions, and the FP64 Givens least-squares
// update of GMRES, all on the device.  Dot products accumulate per thread in the vector
// precision and combine block partials in FP64.
#include <atomic>

#include "helm6_internal.h"

namespace helm6 {

namespace {

constexpr int RB = 256;  // threads per block of the reduction kernels
constexpr int CH = 8;    // basis vectors per pass of the multi-dot kernel

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

// partial[b][2*i + {0,1}] = sum over this block's points of conj(V_i) * w
template <typename T>
__global__ void __launch_bounds__(RB) mdot_kernel(const T* __restrict__ V, int64_t vstride, int count,
                                                  const T* __restrict__ w, int64_t N,
                                                  double* __restrict__ partial) {
  __shared__ double sh[RB / 32];
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t i0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  for (int base = 0; base < count; base += CH) {
    T ar[CH], ai[CH];
#pragma unroll
    for (int c = 0; c < CH; ++c) ar[c] = ai[c] = T(0);
    const int nc = min(CH, count - base);
    for (int64_t idx = i0; idx < N; idx += stride) {
      const T wr = w[idx], wi = w[N + idx];
#pragma unroll
      for (int c = 0; c < CH; ++c) {
        if (c < nc) {
          const T* v = V + (int64_t)(base + c) * vstride;
          const T vr = v[idx], vi = v[N + idx];
          ar[c] = fma(vr, wr, fma(vi, wi, ar[c]));
          ai[c] = fma(vr, wi, fma(-vi, wr, ai[c]));
        }
      }
    }
#pragma unroll
    for (int c = 0; c < CH; ++c) {
      if (c < nc) {
        const double sr = block_sum((double)ar[c], sh);
        const double si = block_sum((double)ai[c], sh);
        if (threadIdx.x == 0) {
          partial[(int64_t)blockIdx.x * 2 * count + 2 * (base + c)] = sr;
          partial[(int64_t)blockIdx.x * 2 * count + 2 * (base + c) + 1] = si;
        }
      }
    }
  }
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

// w -= sum_i V_i h_i   (h complex double, count <= 64)
template <typename T>
__global__ void update_kernel(T* __restrict__ w, const T* __restrict__ V, int64_t vstride, int count,
                              const double* __restrict__ h, int64_t N) {
  __shared__ T hr[64], hi[64];
  if (threadIdx.x < count) {
    hr[threadIdx.x] = (T)h[2 * threadIdx.x];
    hi[threadIdx.x] = (T)h[2 * threadIdx.x + 1];
  }
  __syncthreads();
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < N; idx += stride) {
    T wr = w[idx], wi = w[N + idx];
    for (int c = 0; c < count; ++c) {
      const T* v = V + (int64_t)c * vstride;
      const T vr = v[idx], vi = v[N + idx];
      wr = fma(-vr, hr[c], fma(vi, hi[c], wr));
      wi = fma(-vr, hi[c], fma(-vi, hr[c], wi));
    }
    w[idx] = wr;
    w[N + idx] = wi;
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
    a = fma(v, v, a);
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

// out (+)= scale * sum_i V_i y_i, y complex double
template <typename TI, typename TO>
__global__ void lincomb_kernel(const TI* __restrict__ V, int64_t vstride, int count,
                               const double* __restrict__ y, double scale, TO* __restrict__ out,
                               int64_t N, int accumulate) {
  __shared__ double yr[64], yi[64];
  if (threadIdx.x < count) {
    yr[threadIdx.x] = y[2 * threadIdx.x] * scale;
    yi[threadIdx.x] = y[2 * threadIdx.x + 1] * scale;
  }
  __syncthreads();
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < N; idx += stride) {
    // sum in the input precision, widen once
    TI sr = TI(0), si = TI(0);
    for (int c = 0; c < count; ++c) {
      const TI* v = V + (int64_t)c * vstride;
      const TI vr = v[idx], vi = v[N + idx];
      const TI a = (TI)yr[c], b = (TI)yi[c];
      sr = fma(vr, a, fma(-vi, b, sr));
      si = fma(vr, b, fma(vi, a, si));
    }
    if (accumulate) {
      out[idx] += (TO)sr;
      out[N + idx] += (TO)si;
    } else {
      out[idx] = (TO)sr;
      out[N + idx] = (TO)si;
    }
  }
}

template <typename TI, typename TO>
__global__ void convert_kernel(const TI* __restrict__ x, TO* __restrict__ y, int64_t n2, double scale) {
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

__global__ void reduce_sum_kernel(const double* __restrict__ partial, int n, double* __restrict__ out) {
  __shared__ double sh[RB / 32];
  double v = 0.0;
  for (int b = threadIdx.x; b < n; b += blockDim.x) v += partial[b];
  v = block_sum(v, sh);
  if (threadIdx.x == 0) *out = v;
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

__global__ void set_subdiag_kernel(double* H, int ldh, int j, const double* sumsq, double* inv) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const double nrm = sqrt(fmax(*sumsq, 0.0));
  double* col = H + 2 * (int64_t)j * ldh;
  col[2 * (j + 1)] = nrm;
  col[2 * (j + 1) + 1] = 0.0;
  *inv = (nrm > 0.0) ? 1.0 / nrm : 0.0;
}

__global__ void backsolve_kernel(const double* H, int ldh, int j, const double* g, double* y) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
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

template <typename T>
void launch_mdot(const T* V, int64_t vstride, int count, const T* w, int64_t N, double* partial,
                 int nblocks, cudaStream_t s) {
  note_launch();
  mdot_kernel<T><<<nblocks, RB, 0, s>>>(V, vstride, count, w, N, partial);
}

void launch_reduce_cols(const double* partial, int nblocks, int ncols, double* out, int accumulate,
                        cudaStream_t s) {
  note_launch();
  reduce_cols_kernel<<<ncols, RB, 0, s>>>(partial, nblocks, ncols, out, accumulate, nullptr);
}

void launch_reduce_cols_accum(const double* partial, int nblocks, int ncols, double* out,
                              double* accum, cudaStream_t s) {
  note_launch();
  reduce_cols_kernel<<<ncols, RB, 0, s>>>(partial, nblocks, ncols, out, 0, accum);
}

template <typename T>
void launch_update(T* w, const T* V, int64_t vstride, int count, const double* h, int64_t N,
                   cudaStream_t s) {
  note_launch();
  update_kernel<T><<<grid_for(N, RB), RB, 0, s>>>(w, V, vstride, count, h, N);
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
                    int64_t N, int accumulate, cudaStream_t s) {
  note_launch();
  lincomb_kernel<TI, TO><<<grid_for(N, RB), RB, 0, s>>>(V, vstride, count, y, scale, out, N, accumulate);
}

template <typename TI, typename TO>
void launch_convert(const TI* x, TO* y, int64_t N, double scale, cudaStream_t s) {
  note_launch();
  convert_kernel<TI, TO><<<grid_for(2 * N, RB), RB, 0, s>>>(x, y, 2 * N, scale);
}

void launch_interleaved_to_planar(const double* zin, double* out, int64_t N, cudaStream_t s) {
  note_launch();
  inter_to_planar_kernel<<<grid_for(N, RB), RB, 0, s>>>((const double2*)zin, out, N);
}

void launch_planar_to_interleaved(const double* in, double* zout, int64_t N, cudaStream_t s) {
  note_launch();
  planar_to_inter_kernel<<<grid_for(N, RB), RB, 0, s>>>(in, (double2*)zout, N);
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

void launch_set_subdiag(double* H, int ldh, int j, const double* sumsq, double* inv, cudaStream_t s) {
  note_launch();
  set_subdiag_kernel<<<1, 32, 0, s>>>(H, ldh, j, sumsq, inv);
}

void launch_backsolve(const double* H, int ldh, int j, const double* g, double* y, cudaStream_t s) {
  note_launch();
  backsolve_kernel<<<1, 32, 0, s>>>(H, ldh, j, g, y);
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

#define INST_T(T)                                                                              \
  template void launch_mdot<T>(const T*, int64_t, int, const T*, int64_t, double*, int,         \
                               cudaStream_t);                                                   \
  template void launch_update<T>(T*, const T*, int64_t, int, const double*, int64_t, cudaStream_t); \
  template void launch_sumsq<T>(const T*, int64_t, double*, int, cudaStream_t);                  \
  template void launch_scale_copy<T>(const T*, T*, int64_t, const double*, double, cudaStream_t);
INST_T(float)
INST_T(double)
template void launch_lincomb<float, double>(const float*, int64_t, int, const double*, double, double*,
                                            int64_t, int, cudaStream_t);
template void launch_lincomb<double, double>(const double*, int64_t, int, const double*, double,
                                             double*, int64_t, int, cudaStream_t);
template void launch_lincomb<float, float>(const float*, int64_t, int, const double*, double, float*,
                                           int64_t, int, cudaStream_t);
template void launch_convert<double, float>(const double*, float*, int64_t, double, cudaStream_t);
template void launch_convert<float, double>(const float*, double*, int64_t, double, cudaStream_t);
template void launch_convert<double, double>(const double*, double*, int64_t, double, cudaStream_t);

}  // namespace helm6

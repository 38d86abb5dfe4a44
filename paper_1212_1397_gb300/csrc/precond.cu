// Direct inverse of the 7-point preconditioner A_p (Eq. 3DAP) by separation of variables:
//   X^ = (W_y (x) W_x) X           forward eigen-transforms along x and y (W = V^{-1})
//   (T_z + (lam_p + lam_q) I) U^_pq = X^_pq   for every mode pair (p, q)
//   U  = (V_y (x) V_x) U^          inverse transforms
// This file holds the SIMT pieces: a batched strided real GEMM for the transforms (used
// in FP64, and in FP32 where the tensor-core path is not used) and the batched complex
// Thomas solver for the z lines.
#include <algorithm>

#include "helm6_internal.h"

namespace helm6 {

namespace {

constexpr int BM = 64, BN = 64, BK = 16;

// C(p, n) = sum_k A[p*m + k] B(k, n), one 64 x 64 tile of C per block, 4 x 4 per thread.
template <typename T, bool ALONG_X>
__global__ void __launch_bounds__(256)
    axis_gemm_kernel(const T* __restrict__ A, const T* __restrict__ B, T* __restrict__ C, int m,
                     int ncols, int ld, int64_t bstride) {
  __shared__ T As[BK][BM + 1];
  __shared__ T Bs[BK][BN + 1];
  const int tid = threadIdx.x;
  const int p0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
  const T* Bb = B + (int64_t)blockIdx.z * bstride;
  T* Cb = C + (int64_t)blockIdx.z * bstride;
  // along x the output is contiguous in p: let consecutive threads walk p
  const int tp = ALONG_X ? (tid & 15) : (tid >> 4);
  const int tn = ALONG_X ? (tid >> 4) : (tid & 15);
  T acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = T(0);

  for (int k0 = 0; k0 < m; k0 += BK) {
    for (int e = tid; e < BM * BK; e += 256) {
      const int pp = e / BK, kk = e - pp * BK;
      const int gp = p0 + pp, gk = k0 + kk;
      As[kk][pp] = (gp < m && gk < m) ? A[(int64_t)gp * m + gk] : T(0);
    }
    if (ALONG_X) {
      for (int e = tid; e < BN * BK; e += 256) {
        const int nn = e / BK, kk = e - nn * BK;
        const int gn = n0 + nn, gk = k0 + kk;
        Bs[kk][nn] = (gn < ncols && gk < m) ? Bb[(int64_t)gn * ld + gk] : T(0);
      }
    } else {
      for (int e = tid; e < BN * BK; e += 256) {
        const int kk = e / BN, nn = e - kk * BN;
        const int gn = n0 + nn, gk = k0 + kk;
        Bs[kk][nn] = (gn < ncols && gk < m) ? Bb[(int64_t)gk * ld + gn] : T(0);
      }
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      T av[4], bv[4];
#pragma unroll
      for (int a = 0; a < 4; ++a) av[a] = As[kk][tp + 16 * a];
#pragma unroll
      for (int b = 0; b < 4; ++b) bv[b] = Bs[kk][tn + 16 * b];
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = fmx(av[a], bv[b], acc[a][b]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    const int gp = p0 + tp + 16 * a;
    if (gp >= m) continue;
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const int gn = n0 + tn + 16 * b;
      if (gn >= ncols) continue;
      if (ALONG_X)
        Cb[(int64_t)gn * ld + gp] = acc[a][b];
      else
        Cb[(int64_t)gp * ld + gn] = acc[a][b];
    }
  }
}

// One thread per (p, q) line along z.  Rows of T_z + sigma I in the natural order l:
//   a_l U_{l-1} + d_l U_l + c_l U_{l+1},  a = c = 1 except the corner entries 2 at a
//   Neumann / Sommerfeld-like end (beta = 1), d_l = -2 + k^2h^2 + sigma (+ 2ikh at a
//   Sommerfeld-like end).  Elimination starts at the Sommerfeld-like end when only the top
//   face is one (there the pivots keep a positive imaginary part).
//   xmajor: the plane is stored x-mode-major (index p*my + q, the layout the tensor-core
//   transforms produce) instead of y-major (q*mx + p).
template <typename T>
__global__ void ztri_kernel(Geom g, const double* __restrict__ lamx, const double* __restrict__ lamy,
                            c64d diag0, c64d alpha, const T* __restrict__ x, T* __restrict__ y,
                            T* __restrict__ cw, int* status, int xmajor) {
  const int64_t plane = (int64_t)g.mx * g.my;
  const int64_t pq = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (pq >= plane) return;
  const int p = xmajor ? (int)(pq / g.my) : (int)(pq % g.mx);
  const int q = xmajor ? (int)(pq % g.my) : (int)(pq / g.mx);
  const double sig = lamx[p] + lamy[q];
  const int m = g.mz;
  const bool lo_s = g.face[4] == HELM6_SOMMERFELD, hi_s = g.face[5] == HELM6_SOMMERFELD;
  const T c_lo = (g.face[4] != HELM6_DIRICHLET) ? T(2) : T(1);
  const T a_hi = (g.face[5] != HELM6_DIRICHLET) ? T(2) : T(1);
  const bool rev = (!lo_s && hi_s);
  const cpx<T> dint = mk((T)(diag0.re + sig), (T)diag0.im);
  const cpx<T> al = cast<T>(alpha);
  const int64_t N = g.N;

  // Both sweeps read 8 steps of the line into registers before using them, so that each
  // thread keeps several independent loads in flight.
  constexpr int U = 8;
  cpx<T> cprev = mk(T(0), T(0)), yprev = mk(T(0), T(0));
  bool bad = false;
  for (int r0 = 0; r0 < m; r0 += U) {
    cpx<T> xv[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int r = r0 + u;
      if (r < m) {
        const int l = rev ? (m - 1 - r) : r;
        const int64_t idx = (int64_t)l * plane + pq;
        xv[u] = mk(x[idx], x[N + idx]);
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int r = r0 + u;
      if (r >= m) break;
      const int l = rev ? (m - 1 - r) : r;
      // coefficients in elimination order: sub = towards the previous row, sup = next
      T a_l = (l == m - 1) ? a_hi : T(1);
      T c_l = (l == 0) ? c_lo : T(1);
      if (l == 0) a_l = T(0);
      if (l == m - 1) c_l = T(0);
      const T sub = rev ? c_l : a_l;
      const T sup = rev ? a_l : c_l;
      cpx<T> d = dint;
      if (l == 0 && lo_s) d = d + al;
      if (l == m - 1 && hi_s) d = d + al;
      const cpx<T> den = d - sub * cprev;
      const T n2 = den.re * den.re + den.im * den.im;
      if (!(n2 > T(0))) bad = true;
      const T inv = T(1) / n2;
      const cpx<T> rinv = mk(den.re * inv, -den.im * inv);
      const int64_t idx = (int64_t)l * plane + pq;
      const cpx<T> cp = sup * rinv;
      const cpx<T> yp = (xv[u] - sub * yprev) * rinv;
      cw[idx] = cp.re;
      cw[N + idx] = cp.im;
      y[idx] = yp.re;
      y[N + idx] = yp.im;
      cprev = cp;
      yprev = yp;
    }
  }
  cpx<T> next = mk(T(0), T(0));
  for (int r0 = m - 1; r0 >= 0; r0 -= U) {
    cpx<T> cv[U], yv[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int r = r0 - u;
      if (r >= 0) {
        const int l = rev ? (m - 1 - r) : r;
        const int64_t idx = (int64_t)l * plane + pq;
        cv[u] = mk(cw[idx], cw[N + idx]);
        yv[u] = mk(y[idx], y[N + idx]);
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int r = r0 - u;
      if (r < 0) break;
      const int l = rev ? (m - 1 - r) : r;
      const int64_t idx = (int64_t)l * plane + pq;
      const cpx<T> v = yv[u] - cv[u] * next;
      y[idx] = v.re;
      y[N + idx] = v.im;
      next = v;
    }
  }
  if (bad) atomicExch(status, (int)HELM6_BREAKDOWN);
}

// Line coefficients of the elimination, computed once in FP64 and stored in the working
// precision: for every (p, q) line and step r of the elimination order, the pivot
// reciprocal rinv_r = 1 / (d_r - sub_r c'_{r-1}) and c'_r = sup_r rinv_r.  With them the
// per-apply sweeps are  y'_r = (x_r - sub_r y'_{r-1}) rinv_r  and  x_r = y'_r - c'_r x_{r+1},
// so the rounding of the pivot recursion does not accumulate along ill-conditioned lines.
__device__ __forceinline__ void line_coef(const Geom& g, int l, bool rev, double& sub, double& sup) {
  const int m = g.mz;
  double a_l = (l == m - 1) ? ((g.face[5] != HELM6_DIRICHLET) ? 2.0 : 1.0) : 1.0;
  double c_l = (l == 0) ? ((g.face[4] != HELM6_DIRICHLET) ? 2.0 : 1.0) : 1.0;
  if (l == 0) a_l = 0.0;
  if (l == m - 1) c_l = 0.0;
  sub = rev ? c_l : a_l;
  sup = rev ? a_l : c_l;
}

// Pivot table of the z lines, FP64 arithmetic stored in FP32 (once per context): for each
// (p, q) line (planes x-mode-major with q pitch z.ldq) and step r of the elimination order,
// rinv_r = 1 / (d_r - sub_r c'_{r-1}) with c'_r = sup_r rinv_r.
__global__ void ztri_table_kernel(Geom g, const double* __restrict__ lamx, const double* __restrict__ lamy,
                                  c64d diag0, c64d alpha, ZLines z, int* status) {
  const int64_t plane = (int64_t)g.mx * z.ldq;
  const int64_t pq = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (pq >= plane) return;
  const int p = (int)(pq / z.ldq), q = (int)(pq % z.ldq);
  if (q >= g.my) return;
  const double sig = lamx[p] + lamy[q];
  const int m = g.mz;
  const bool lo_s = g.face[4] == HELM6_SOMMERFELD, hi_s = g.face[5] == HELM6_SOMMERFELD;
  const bool rev = (!lo_s && hi_s);
  const int64_t Np = (int64_t)m * plane;
  double cr = 0.0, ci = 0.0;
  bool bad = false;
  for (int r = 0; r < m; ++r) {
    const int l = rev ? (m - 1 - r) : r;
    double sub, sup;
    line_coef(g, l, rev, sub, sup);
    double dr = diag0.re + sig, di = diag0.im;
    if (l == 0 && lo_s) {
      dr += alpha.re;
      di += alpha.im;
    }
    if (l == m - 1 && hi_s) {
      dr += alpha.re;
      di += alpha.im;
    }
    const double er = dr - sub * cr, ei = di - sub * ci;
    const double n2 = er * er + ei * ei;
    if (!(n2 > 0.0)) bad = true;
    const double ir = er / n2, ii = -ei / n2;
    cr = sup * ir;
    ci = sup * ii;
    const int64_t idx = (int64_t)l * plane + pq;
    z.rinv[idx] = (float)ir;
    z.rinv[Np + idx] = (float)ii;
  }
  if (bad) atomicExch(status, (int)HELM6_BREAKDOWN);
}

// line_coef in FP32 (the coefficients are 0, 1 or 2) for the per-apply sweeps.
__device__ __forceinline__ void line_coef_f(const Geom& g, int l, bool rev, float& sub, float& sup) {
  const int m = g.mz;
  float a_l = (l == m - 1) ? ((g.face[5] != HELM6_DIRICHLET) ? 2.f : 1.f) : 1.f;
  float c_l = (l == 0) ? ((g.face[4] != HELM6_DIRICHLET) ? 2.f : 1.f) : 1.f;
  if (l == 0) a_l = 0.f;
  if (l == m - 1) c_l = 0.f;
  sub = rev ? c_l : a_l;
  sup = rev ? a_l : c_l;
}

// The z-line sweeps: one thread per line (every line in flight), forward then backward,
// the forward results written to y and read back by the backward sweep (which overwrites
// them).  Both sweeps load U steps ahead before using them; c' = sup rinv is formed on the
// fly from the pivot table (sup is 0, 1 or 2: exact).  Measured alternatives that read the
// table only where the pivots have not converged (per line or per warp), or that bound the
// lines in flight so that the forward results stay in L2, were 1.3 to 4 times slower: the
// sweep is bound by the loads in flight, which conditional loads and fewer lines reduce.
template <int U>
__global__ void __launch_bounds__(128) ztri_lines_kernel(Geom g, ZLines z, const float* __restrict__ x,
                                                         float* __restrict__ y) {
  const int64_t plane = (int64_t)g.mx * z.ldq;
  const int64_t pq = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (pq >= plane || (int)(pq % z.ldq) >= g.my) return;
  const int m = g.mz;
  const bool lo_s = g.face[4] == HELM6_SOMMERFELD, hi_s = g.face[5] == HELM6_SOMMERFELD;
  const bool rev = (!lo_s && hi_s);
  const int64_t N = (int64_t)m * plane;
  cpx<float> yprev = mk(0.f, 0.f);
  for (int r0 = 0; r0 < m; r0 += U) {
    cpx<float> xv[U], iv[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int r = r0 + u;
      if (r < m) {
        const int64_t idx = (int64_t)(rev ? m - 1 - r : r) * plane + pq;
        xv[u] = mk(x[idx], x[N + idx]);
        iv[u] = mk(z.rinv[idx], z.rinv[N + idx]);
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int r = r0 + u;
      if (r >= m) break;
      const int l = rev ? m - 1 - r : r;
      float sub, sup;
      line_coef_f(g, l, rev, sub, sup);
      const cpx<float> yp = (xv[u] - sub * yprev) * iv[u];
      const int64_t idx = (int64_t)l * plane + pq;
      y[idx] = yp.re;
      y[N + idx] = yp.im;
      yprev = yp;
    }
  }
  cpx<float> next = mk(0.f, 0.f);
  for (int r0 = m - 1; r0 >= 0; r0 -= U) {
    cpx<float> cv[U], yv[U];
    // loads only here (the multiply by sup stays with the recursion below: measured 1.6x
    // faster than forming c' next to its load)
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int r = r0 - u;
      if (r >= 0) {
        const int l = rev ? m - 1 - r : r;
        const int64_t idx = (int64_t)l * plane + pq;
        cv[u] = mk(z.rinv[idx], z.rinv[N + idx]);
        yv[u] = mk(y[idx], y[N + idx]);
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int r = r0 - u;
      if (r < 0) break;
      const int l = rev ? m - 1 - r : r;
      float sub, sup;
      line_coef_f(g, l, rev, sub, sup);
      const int64_t idx = (int64_t)l * plane + pq;
      const cpx<float> v = yv[u] - (sup * cv[u]) * next;
      y[idx] = v.re;
      y[N + idx] = v.im;
      next = v;
    }
  }
}

}  // namespace

template <typename T>
void launch_axis_gemm(const T* A, const T* B, T* C, int m, int ncols, int ld, int64_t bstride,
                      int nbatch, bool along_x, cudaStream_t s) {
  dim3 grid((ncols + BN - 1) / BN, (m + BM - 1) / BM, nbatch);
  note_launch();
  if (along_x)
    axis_gemm_kernel<T, true><<<grid, 256, 0, s>>>(A, B, C, m, ncols, ld, bstride);
  else
    axis_gemm_kernel<T, false><<<grid, 256, 0, s>>>(A, B, C, m, ncols, ld, bstride);
}

template <typename T>
void launch_ztri(const Geom& g, const double* lamx, const double* lamy, c64d diag0, c64d alpha,
                 const T* x, T* y, T* cw, int* status, cudaStream_t s, int xmajor) {
  const int64_t lines = (int64_t)g.mx * g.my;
  const int bs = 128;
  note_launch();
  ztri_kernel<T><<<(unsigned)((lines + bs - 1) / bs), bs, 0, s>>>(g, lamx, lamy, diag0, alpha, x, y,
                                                                  cw, status, xmajor);
}


void launch_ztri_table(const Geom& g, const double* lamx, const double* lamy, c64d diag0, c64d alpha, ZLines z,
                       int* status, cudaStream_t s) {
  const int64_t lines = (int64_t)g.mx * z.ldq;
  note_launch();
  ztri_table_kernel<<<(unsigned)((lines + 127) / 128), 128, 0, s>>>(g, lamx, lamy, diag0, alpha, z, status);
}

void launch_ztri_apply(const Geom& g, const ZLines& z, const float* x, float* y, cudaStream_t s) {
  const int64_t lines = (int64_t)g.mx * z.ldq;
  note_launch();
  ztri_lines_kernel<8><<<(unsigned)((lines + 127) / 128), 128, 0, s>>>(g, z, x, y);
}

template void launch_axis_gemm<float>(const float*, const float*, float*, int, int, int, int64_t, int,
                                      bool, cudaStream_t);
template void launch_axis_gemm<double>(const double*, const double*, double*, int, int, int, int64_t,
                                       int, bool, cudaStream_t);
template void launch_ztri<float>(const Geom&, const double*, const double*, c64d, c64d, const float*,
                                 float*, float*, int*, cudaStream_t, int);
template void launch_ztri<double>(const Geom&, const double*, const double*, c64d, c64d,
                                  const double*, double*, double*, int*, cudaStream_t, int);

}  // namespace helm6

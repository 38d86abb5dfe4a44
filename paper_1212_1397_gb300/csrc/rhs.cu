// Compact right side F of the sixth-order scheme for separable sources (FP64): sums of
// Gaussian sources, or any f = sum_t c_t X_t(x) Y_t(y) Z_t(z) given by 1D derivative tables.
//
// Interior (Eq. scheme right side, h^2-scaled; the mixed fourth derivatives carry the
// total weight h^4/90 that makes the scheme sixth order):
//   F = h^2 [ cf f + q1 lap f + (h^4/360) sum_a f_aaaa + (h^4/90) sum_{a<b} f_aabb ] + h^2 cf eta
//   cf = 1 - k^2h^2/12 + k^4h^4/360,  q1 = (h^2/12)(1 - k^2h^2/30).
// Neumann face rows (Eq. 3DN, homogeneous data, minus sign on the 7h^5/180 term):
//   F -= D_N,  D_N = dn1 f_n + dn3 f_nnn + dnm (f_ntt + f_nss)
// Sommerfeld-like face rows (Eq. 3DDISCS), fbar = exp(ik n) f in the inward normal n:
//   F -= D_S,  D_S = -e^{ikh} mu3 [ 2h Fbar + mu1 (h^5/3)(fbar_ntt + fbar_nss) ].
// Each separable term contributes products of its factors' 1D derivatives X^(m)(x),
// m = 0..4, tabulated (complex) per axis at the unknown nodes by the host.
#include <algorithm>
#include <cmath>

#include "helm6_internal.h"

#include <climits>

namespace helm6 {

namespace {

struct RhsCoef {
  double h;
  c64d cf, q1;         // interior
  c64d dn1;            // Neumann: coefficient of f_n
  double dn3, dnm;     // Neumann: f_nnn and f_ntt + f_nss
  c64d ik;             // Sommerfeld-like: i k
  c64d a1, a2;         // Fbar = a1 fb_n + a2 fb_nn + a3 (fb_nnn - fb_ntt - fb_nss)
  double a3;
  c64d e1mu3, mu1h5;   // D_S = -e1mu3 (2h Fbar + mu1h5 (fb_ntt + fb_nss))
};

using Z = cpx<double>;

__device__ __forceinline__ Z zc(c64d a) { return Z{a.re, a.im}; }

// Complex table entry: term k, axis a, derivative order m, unknown node p.
__device__ __forceinline__ Z tv(const double* tab, int mmax, int k, int a, int m, int p) {
  const int64_t o = (((int64_t)k * 3 + a) * 5 + m) * mmax + p;
  return Z{tab[2 * o], tab[2 * o + 1]};
}

// Term-summed derivative f^(ox, oy, oz) at node (i, j, l).
__device__ __forceinline__ Z deriv(const double* tab, const double* coef, int nterm, int mmax, int i, int j,
                                   int l, int ox, int oy, int oz) {
  Z s = Z{0.0, 0.0};
  for (int k = 0; k < nterm; ++k) {
    const Z v = tv(tab, mmax, k, 0, ox, i) * tv(tab, mmax, k, 1, oy, j) * tv(tab, mmax, k, 2, oz, l);
    s = s + Z{coef[2 * k], coef[2 * k + 1]} * v;
  }
  return s;
}

__global__ void rhs_kernel(Geom g, RhsCoef c, int nsrc, int mmax, const double* __restrict__ tab,
                           const double* __restrict__ amps, const double* __restrict__ noise,
                           double* __restrict__ F) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= g.N) return;
  const int i = (int)(idx % g.mx);
  const int j = (int)((idx / g.mx) % g.my);
  const int l = (int)(idx / ((int64_t)g.mx * g.my));
  Z S0{0, 0}, S1{0, 0}, S2{0, 0}, S3{0, 0};
  for (int k = 0; k < nsrc; ++k) {
    Z gx[5], gy[5], gz[5];
#pragma unroll
    for (int m = 0; m < 5; ++m) {
      gx[m] = tv(tab, mmax, k, 0, m, i);
      gy[m] = tv(tab, mmax, k, 1, m, j);
      gz[m] = tv(tab, mmax, k, 2, m, l);
    }
    const Z f0 = gx[0] * gy[0] * gz[0];
    const Z lap = gx[2] * gy[0] * gz[0] + gx[0] * gy[2] * gz[0] + gx[0] * gy[0] * gz[2];
    const Z p4 = gx[4] * gy[0] * gz[0] + gx[0] * gy[4] * gz[0] + gx[0] * gy[0] * gz[4];
    const Z m4 = gx[2] * gy[2] * gz[0] + gx[2] * gy[0] * gz[2] + gx[0] * gy[2] * gz[2];
    const Z a = Z{amps[2 * k], amps[2 * k + 1]};
    S0 = S0 + a * f0;
    S1 = S1 + a * lap;
    S2 = S2 + a * p4;
    S3 = S3 + a * m4;
  }
  const double h = c.h, h2 = h * h, h4 = h2 * h2;
  Z Fv = zc(c.cf) * S0 + zc(c.q1) * S1 + (h4 / 360.0) * S2 + (h4 / 90.0) * S3;
  Fv = h2 * Fv;
  if (noise) Fv = Fv + h2 * (zc(c.cf) * Z{noise[2 * idx], noise[2 * idx + 1]});

  // face data terms
  const int pos[3] = {i, j, l};
  const int dimv[3] = {g.mx, g.my, g.mz};
  for (int ax = 0; ax < 3; ++ax) {
    for (int side = 0; side < 2; ++side) {
      const int kind = g.face[2 * ax + side];
      if (kind == HELM6_DIRICHLET) continue;
      if (pos[ax] != (side == 0 ? 0 : dimv[ax] - 1)) continue;
      const double sg = side == 0 ? 1.0 : -1.0;
      const int t1 = (ax == 0) ? 1 : 0, t2 = (ax == 2) ? 1 : 2;
      auto d = [&](int on, int o1, int o2) {
        int o[3] = {0, 0, 0};
        o[ax] = on;
        o[t1] = o1;
        o[t2] = o2;
        Z v = deriv(tab, amps, nsrc, mmax, i, j, l, o[0], o[1], o[2]);
        const double sgn = (on & 1) ? sg : 1.0;
        return sgn * v;
      };
      if (kind == HELM6_NEUMANN) {
        const Z DN = zc(c.dn1) * d(1, 0, 0) + c.dn3 * d(3, 0, 0) + c.dnm * (d(1, 2, 0) + d(1, 0, 2));
        Fv = Fv - DN;
      } else {
        const Z ik = zc(c.ik), ik2 = ik * ik, ik3 = ik2 * ik;
        const Z f0 = d(0, 0, 0), fn = d(1, 0, 0), fnn = d(2, 0, 0), fnnn = d(3, 0, 0);
        const Z ftt = d(0, 2, 0), fss = d(0, 0, 2), fntt = d(1, 2, 0), fnss = d(1, 0, 2);
        const Z fb_n = ik * f0 + fn;
        const Z fb_nn = ik2 * f0 + 2.0 * (ik * fn) + fnn;
        const Z fb_nnn = ik3 * f0 + 3.0 * (ik2 * fn) + 3.0 * (ik * fnn) + fnnn;
        const Z fb_ntt = ik * ftt + fntt;
        const Z fb_nss = ik * fss + fnss;
        const Z Fbar = zc(c.a1) * fb_n + zc(c.a2) * fb_nn + c.a3 * (fb_nnn - fb_ntt - fb_nss);
        const Z DS = Z{0.0, 0.0} - zc(c.e1mu3) * ((2.0 * h) * Fbar + zc(c.mu1h5) * (fb_ntt + fb_nss));
        Fv = Fv - DS;
      }
    }
  }
  F[2 * idx] = Fv.re;
  F[2 * idx + 1] = Fv.im;
}

}  // namespace

// Upload the complex tables [nterm][3][5][mmax] and coefficients, launch, free.
int launch_rhs(const Geom& g, double h, cd k, int nterm, int mmax, const std::vector<double>& tab,
               const double* coef, const double* noise, double* F, cudaStream_t s) {
  double *dtab = nullptr, *dcoef = nullptr;
  if (cudaMallocAsync((void**)&dtab, tab.size() * sizeof(double), s) != cudaSuccess) return HELM6_ERR_NOMEM;
  if (cudaMallocAsync((void**)&dcoef, (size_t)std::max(nterm, 1) * 2 * sizeof(double), s) != cudaSuccess) {
    cudaFreeAsync(dtab, s);
    return HELM6_ERR_NOMEM;
  }
  cudaMemcpyAsync(dtab, tab.data(), tab.size() * sizeof(double), cudaMemcpyHostToDevice, s);
  if (nterm > 0)
    cudaMemcpyAsync(dcoef, coef, (size_t)nterm * 2 * sizeof(double), cudaMemcpyHostToDevice, s);

  RhsCoef c;
  const cd I(0.0, 1.0);
  const cd kh2 = k * k * h * h;
  const double h2 = h * h, h3 = h2 * h, h4 = h2 * h2, h5 = h4 * h;
  c.h = h;
  c.cf = to_pod(1.0 - kh2 / 12.0 + kh2 * kh2 / 360.0);
  c.q1 = to_pod((h2 / 12.0) * (1.0 - kh2 / 30.0));
  c.dn1 = to_pod(-(h3 / 3.0) * (1.0 - kh2 / 20.0));
  c.dn3 = -h5 / 60.0;
  c.dnm = -7.0 * h5 / 180.0;
  const cd ik = I * k;
  c.ik = to_pod(ik);
  const cd mu3 = 1.0 / (1.0 + (2.0 * ik * h / 3.0) * (1.0 + 2.0 * kh2 / 15.0));
  const cd mu1 = (ik * h / 90.0 + (1.0 + kh2 / 30.0) / (6.0 * mu3)) / (1.0 + 2.0 * ik * h / 3.0);
  c.a1 = to_pod(h2 / 6.0 + k * k * h4 / 45.0);
  c.a2 = to_pod(-ik * h4 / 90.0);
  c.a3 = h4 / 120.0;
  c.e1mu3 = to_pod(std::exp(ik * h) * mu3);
  c.mu1h5 = to_pod(mu1 * h5 / 3.0);

  const int bs = 256;
  note_launch();
  rhs_kernel<<<(unsigned)((g.N + bs - 1) / bs), bs, 0, s>>>(g, c, nterm, mmax, dtab, dcoef, noise, F);
  cudaFreeAsync(dtab, s);
  cudaFreeAsync(dcoef, s);
  return cudaGetLastError() == cudaSuccess ? HELM6_OK : HELM6_ERR_CUDA;
}

// Gaussian sources: 1D derivative tables G^(m)(x) = (-1/sigma)^m He_m(t) exp(-t^2/2),
// t = (x-c)/sigma, with He the probabilists' Hermite polynomials, at the unknown nodes of
// each axis (real, stored as complex with zero imaginary part).
int rhs_gaussians(const Geom& g, double h, cd k, int nsrc, const double* centers, const double* amps,
                  double sigma, const double* noise, double* F, cudaStream_t s) {
  const int mmax = std::max(g.mx, std::max(g.my, g.mz));
  const int mdim[3] = {g.mx, g.my, g.mz};
  std::vector<double> tab((size_t)std::max(nsrc, 1) * 15 * mmax * 2, 0.0);
  for (int src = 0; src < nsrc; ++src) {
    for (int ax = 0; ax < 3; ++ax) {
      const int start = (g.face[2 * ax] == HELM6_DIRICHLET) ? 1 : 0;
      for (int p = 0; p < mdim[ax]; ++p) {
        const double x = (start + p) * h;
        const double t = (x - centers[3 * src + ax]) / sigma;
        const double e = std::exp(-0.5 * t * t);
        double he[5];
        he[0] = 1.0;
        he[1] = t;
        for (int m = 1; m < 4; ++m) he[m + 1] = t * he[m] - m * he[m - 1];
        double sc = 1.0;
        for (int m = 0; m < 5; ++m) {
          tab[2 * (((size_t)src * 3 + ax) * 5 + m) * mmax + 2 * (size_t)p] = sc * he[m] * e;
          sc *= -1.0 / sigma;
        }
      }
    }
  }
  return launch_rhs(g, h, k, nsrc, mmax, tab, amps, noise, F, s);
}

// Separable source given by the caller's complex tables [nterm][3][5][mmax] (mmax the
// largest axis length), entry p of an axis = the factor's derivative at its p-th unknown.
int rhs_separable(const Geom& g, double h, cd k, int nterm, const double* coef, const double* tables, double* F,
                  cudaStream_t s) {
  const int mmax = std::max(g.mx, std::max(g.my, g.mz));
  std::vector<double> tab((size_t)std::max(nterm, 1) * 15 * mmax * 2, 0.0);
  if (nterm > 0) std::copy(tables, tables + (size_t)nterm * 15 * mmax * 2, tab.begin());
  return launch_rhs(g, h, k, nterm, mmax, tab, coef, nullptr, F, s);
}

namespace {

// Lifting of inhomogeneous Dirichlet data on a z face: the face's nodes are known, so their
// contribution to the neighbouring plane's rows moves to the right side,
//   F(l, j, i) -= sum over the 3 x 3 face nodes around (i, j) of w(di, dj) u_b,
// w = the interior rows' weights of the z +- 1 plane (centre c1, 4 neighbours c2, 4
// diagonals c3 of Eq. scheme).  ub: (my + 2) x (mx + 2) complex128 values on the face's
// node layer, ring included (the nodes of the neighbouring faces' ghost columns and rows).
// Rows next to a Dirichlet face with known values u_b: the face's nodes enter those rows
// through the 27-point weights of the row (interior, or the Sommerfeld-like face rows on z),
// F -= sum over the face's nodes in the row's 3 x 3 window of w * u_b.  A node's weight is the
// row's class weight for its offset: the plane offset along z and the number of nonzero
// in-plane (x, y) offsets (the interior weights are the same for any axis).  The face data
// holds a ring in the tangential axes that are padded before the face's own axis (x, then y,
// then z), so an edge node belongs to exactly one face: x faces [mz][my], y faces
// [mz][mx + 2], z faces [my + 2][mx + 2].
__global__ void lift_face_kernel(Geom g, RowWeights win, RowWeights wlo, RowWeights whi, int axis, int side,
                                 const double* __restrict__ ub, double* __restrict__ F) {
  const int m[3] = {g.mx, g.my, g.mz};
  const int a1 = axis == 0 ? 1 : 0, a2 = axis == 2 ? 1 : 2;  // tangential axes, a1 < a2
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)m[a1] * m[a2]) return;
  const int u1 = (int)(t % m[a1]), u2 = (int)(t / m[a1]);
  int c[3];
  c[axis] = side ? m[axis] - 1 : 0;
  c[a1] = u1;
  c[a2] = u2;
  const RowWeights& W = (c[2] == 0 && g.face[4] == HELM6_SOMMERFELD)            ? wlo
                        : (c[2] == m[2] - 1 && g.face[5] == HELM6_SOMMERFELD) ? whi
                                                                              : win;
  const int r1 = a1 < axis ? 1 : 0, r2 = a2 < axis ? 1 : 0;
  const int ld = m[a1] + 2 * r1;
  // a node beyond the data along a tangential axis: a Neumann face there reflects the ghost
  // onto the data (U_{-1} = U_1); otherwise it belongs to another face's data or is zero
  auto fold = [&](int q, int a, int ring) -> int {
    if (q >= -ring && q < m[a] + ring) return q;
    if (q < 0) return g.face[2 * a] == HELM6_NEUMANN ? 1 : INT_MIN;
    return g.face[2 * a + 1] == HELM6_NEUMANN ? m[a] - 2 : INT_MIN;
  };
  Z s{0.0, 0.0};
  for (int d2 = -1; d2 <= 1; ++d2)
    for (int d1 = -1; d1 <= 1; ++d1) {
      const int p1 = fold(u1 + d1, a1, r1), p2 = fold(u2 + d2, a2, r2);
      if (p1 == INT_MIN || p2 == INT_MIN) continue;
      int o[3];
      o[axis] = side ? 1 : -1;
      o[a1] = d1;
      o[a2] = d2;
      const int cls = (o[0] != 0) + (o[1] != 0);
      const int64_t q = (int64_t)(p2 + r2) * ld + (p1 + r1);
      s = s + zc(W.w[o[2] + 1][cls]) * Z{ub[2 * q], ub[2 * q + 1]};
    }
  const int64_t o = ((int64_t)c[2] * m[1] + c[1]) * m[0] + c[0];
  F[2 * o] -= s.re;
  F[2 * o + 1] -= s.im;
}

}  // namespace

int lift_dirichlet(const Geom& g, const StencilCoef& coef, int face, const double* ub, double* F, cudaStream_t s) {
  const int axis = face / 2, side = face % 2;
  const int m[3] = {g.mx, g.my, g.mz};
  const int64_t n = (int64_t)m[axis == 0 ? 1 : 0] * m[axis == 2 ? 1 : 2];
  note_launch();
  lift_face_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(g, coef.interior, coef.s_lo, coef.s_hi, axis, side,
                                                                ub, F);
  return cudaGetLastError() == cudaSuccess ? (int)HELM6_OK : (int)HELM6_ERR_CUDA;
}

}  // namespace helm6

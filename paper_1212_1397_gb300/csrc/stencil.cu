// The sixth-order compact 27-point operator (Eq. scheme) with the Neumann (Eq. 3DN) and
// Sommerfeld-like (Eq. 3DDISCS) face rows, applied matrix-free on planar complex data.
//
// Every row is   sum_{dz=-1,0,1}  wc[dz] C(l+dz) + wn[dz] Nb(l+dz) + wd[dz] Dg(l+dz)
// where for z-plane p, C(p) is the value at (i, j), Nb(p) the sum of the 4 in-plane
// neighbours and Dg(p) the sum of the 4 in-plane diagonals.  Interior rows use the four
// class weights c0..c3 of Eq. scheme; a Sommerfeld-like face row has no ghost plane and
// carries G0 on its own plane and G1 on the next plane inward (Eq. 3DDISCS).  Ghost values
// across x/y faces and across Neumann z faces are even reflections (U_{-1} = U_1);
// across Dirichlet faces they are zero.
//
// Thread block: a 32 x 8 (x, y) tile marching over a chunk of 32 z planes.  Each plane
// tile plus a one-point halo is staged in shared memory by asynchronous copies issued
// three planes ahead into a ring of five buffers (one barrier per plane); each thread
// keeps the three plane sums (C, Nb, Dg) of planes l-1, l, l+1 in registers, so every
// input value is read from global memory once per chunk.
#include "helm6_internal.h"

namespace helm6 {

namespace {

constexpr int TX = 32, TY = 8, ZCH = 32;

template <typename T>
struct Sums {
  cpx<T> c, n, d;
};

__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Asynchronous 4- or 8-byte copy global -> shared; src_bytes = 0 zero-fills (ghost = 0).
template <int BYTES>
__device__ __forceinline__ void cp_async(void* dst, const void* src, int src_bytes) {
  const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], %2, %3;\n" ::"r"(d), "l"(src), "n"(BYTES), "r"(src_bytes)
               : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// RW: the interior class weights are real (a real wavenumber); their products with the
// plane sums then take two FMAs instead of four (identical results: the imaginary parts
// that drop out are exact zeros).
template <typename T, int MODE, bool NORM, bool RW>
__global__ void __launch_bounds__(TX* TY)
    stencil_kernel(Geom g, StencilCoef coef, const T* __restrict__ x, T* __restrict__ y,
                   const T* __restrict__ f, double* __restrict__ sumsq) {
  // ring of NBUF staged planes; plane p + DIST is requested while plane p is used
  constexpr int DIST = 3, NBUF = DIST + 2;
  __shared__ T sre[NBUF][TY + 2][TX + 2];
  __shared__ T sim[NBUF][TY + 2][TX + 2];
  __shared__ double red[TX * TY / 32];

  const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * TX + tx;
  const int i = blockIdx.x * TX + tx, j = blockIdx.y * TY + ty;
  const int l0 = blockIdx.z * ZCH;
  const int l1 = min(l0 + ZCH, g.mz);
  const int64_t plane = (int64_t)g.mx * g.my;
  const bool active = (i < g.mx) && (j < g.my);

  const cpx<T> c0 = cast<T>(coef.interior.w[1][0]);
  const cpx<T> c1 = cast<T>(coef.interior.w[1][1]);
  const cpx<T> c2 = cast<T>(coef.interior.w[1][2]);
  const cpx<T> c3 = cast<T>(coef.interior.w[0][2]);

  // Halo tile element t = tid + k * TX*TY (k = 0, 1) of every plane: its in-plane source
  // offset (reflection across Neumann x/y faces) or -1 for a zero ghost, computed once.
  constexpr int HALO = (TX + 2) * (TY + 2);
  int hoff[2];
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    const int t = tid + k * TX * TY;
    hoff[k] = -1;
    if (t < HALO) {
      const int sy = t / (TX + 2), sx = t - sy * (TX + 2);
      int gi = blockIdx.x * TX + sx - 1, gj = blockIdx.y * TY + sy - 1;
      bool ok = true;
      if (gi < 0) {
        if (g.face[0] == HELM6_NEUMANN) gi = 1; else ok = false;
      } else if (gi >= g.mx) {
        if (g.face[1] == HELM6_NEUMANN && gi == g.mx) gi = g.mx - 2; else ok = false;
      }
      if (gj < 0) {
        if (g.face[2] == HELM6_NEUMANN) gj = 1; else ok = false;
      } else if (gj >= g.my) {
        if (g.face[3] == HELM6_NEUMANN && gj == g.my) gj = g.my - 2; else ok = false;
      }
      if (ok) hoff[k] = gj * g.mx + gi;
    }
  }
  T* sre_flat = &sre[0][0][0];
  T* sim_flat = &sim[0][0][0];

  // stage the halo tile of the plane feeding position p (ghost planes: reflection across a
  // Neumann z face, zero otherwise) into ring slot `slot`
  auto stage = [&](int p, int slot) {
    int src = p;
    bool zplane = false;
    if (p < 0) {
      if (g.face[4] == HELM6_NEUMANN) src = 1; else zplane = true;
    } else if (p >= g.mz) {
      if (g.face[5] == HELM6_NEUMANN) src = g.mz - 2; else zplane = true;
    }
    const int64_t pbase = (int64_t)src * plane;
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      const int t = tid + k * TX * TY;
      if (t < HALO) {
        const bool ok = !zplane && hoff[k] >= 0;
        const int64_t idx = ok ? pbase + hoff[k] : 0;
        cp_async<sizeof(T)>(sre_flat + slot * HALO + t, x + idx, ok ? (int)sizeof(T) : 0);
        cp_async<sizeof(T)>(sim_flat + slot * HALO + t, x + g.N + idx, ok ? (int)sizeof(T) : 0);
      }
    }
  };

  Sums<T> P0, P1, P2;  // planes l-1, l, l+1 as the march proceeds
  const cpx<T> zero = {T(0), T(0)};
  P0 = P1 = P2 = Sums<T>{zero, zero, zero};
  double acc = 0.0;

  const int pfirst = l0 - 1;
  for (int d = 0; d < DIST; ++d) {
    if (pfirst + d <= l1) stage(pfirst + d, d);
    cp_commit();
  }
  for (int p = pfirst; p <= l1; ++p) {
    const int k = p - pfirst;
    if (p + DIST <= l1) stage(p + DIST, (k + DIST) % NBUF);
    cp_commit();
    cp_wait<DIST>();  // the group of plane p has landed
    __syncthreads();
    const int buf = k % NBUF;

    // ---- in-plane sums of plane p at (i, j) ----
    Sums<T> cur;
    {
      const int a = ty + 1, b = tx + 1;
      cur.c = mk(sre[buf][a][b], sim[buf][a][b]);
      cur.n = mk(sre[buf][a][b - 1] + sre[buf][a][b + 1] + sre[buf][a - 1][b] + sre[buf][a + 1][b],
                 sim[buf][a][b - 1] + sim[buf][a][b + 1] + sim[buf][a - 1][b] + sim[buf][a + 1][b]);
      cur.d = mk(sre[buf][a - 1][b - 1] + sre[buf][a - 1][b + 1] + sre[buf][a + 1][b - 1] +
                     sre[buf][a + 1][b + 1],
                 sim[buf][a - 1][b - 1] + sim[buf][a - 1][b + 1] + sim[buf][a + 1][b - 1] +
                     sim[buf][a + 1][b + 1]);
    }
    P0 = P1;
    P1 = P2;
    P2 = cur;

    const int l = p - 1;  // row whose three planes are now in P0, P1, P2
    if (l >= l0 && active) {
      cpx<T> out;
      const bool slo = (l == 0) && (g.face[4] == HELM6_SOMMERFELD);
      const bool shi = (l == g.mz - 1) && (g.face[5] == HELM6_SOMMERFELD);
      if (!slo && !shi) {
        // interior class form: c0 C + c1 (Nb + C-+C+) + c2 (Dg + Nb-+Nb+) + c3 (Dg-+Dg+)
        const cpx<T> s1 = P1.n + P0.c + P2.c, s2 = P1.d + P0.n + P2.n, s3 = P0.d + P2.d;
        if constexpr (RW) {
          out.re = fmx(c3.re, s3.re, fmx(c2.re, s2.re, fmx(c1.re, s1.re, c0.re * P1.c.re)));
          out.im = fmx(c3.re, s3.im, fmx(c2.re, s2.im, fmx(c1.re, s1.im, c0.re * P1.c.im)));
        } else {
          out = c0 * P1.c;
          out = cfma(c1, s1, out);
          out = cfma(c2, s2, out);
          out = cfma(c3, s3, out);
        }
      } else {
        const RowWeights& W = slo ? coef.s_lo : coef.s_hi;
        out = zero;
        out = cfma(cast<T>(W.w[0][0]), P0.c, out);
        out = cfma(cast<T>(W.w[0][1]), P0.n, out);
        out = cfma(cast<T>(W.w[0][2]), P0.d, out);
        out = cfma(cast<T>(W.w[1][0]), P1.c, out);
        out = cfma(cast<T>(W.w[1][1]), P1.n, out);
        out = cfma(cast<T>(W.w[1][2]), P1.d, out);
        out = cfma(cast<T>(W.w[2][0]), P2.c, out);
        out = cfma(cast<T>(W.w[2][1]), P2.n, out);
        out = cfma(cast<T>(W.w[2][2]), P2.d, out);
      }
      const int64_t idx = (int64_t)l * plane + (int64_t)j * g.mx + i;
      if (MODE == 1) {
        out = mk(f[idx] - out.re, f[g.N + idx] - out.im);
      } else if (MODE == 2) {
        out = mk(f[idx] + out.re, f[g.N + idx] + out.im);
      }
      y[idx] = out.re;
      y[g.N + idx] = out.im;
      if (NORM) acc += (double)out.re * out.re + (double)out.im * out.im;
    }
  }
  cp_wait<0>();

  if (NORM) {
    acc = warp_sum(acc);
    if ((tid & 31) == 0) red[tid >> 5] = acc;
    __syncthreads();
    if (tid < 32) {
      double v = (tid < TX * TY / 32) ? red[tid] : 0.0;
      v = warp_sum(v);
      if (tid == 0) {
        const int64_t b = ((int64_t)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
        sumsq[b] = v;
      }
    }
  }
}

// FP32 variant for the Krylov bulk: 32 x 16 (x, y) tile, a 32 x 4 thread block, each
// thread computing 4 y-adjacent points from 6 x 3 shared-memory loads per component.  A
// halo row is staged in shared memory as [unused x3 | left ghost | 32 points | right ghost]
// (stride 40 floats) so that the 32-point middle is 16-byte aligned and can be copied in
// 16-byte chunks when mx % 4 == 0; the two edge columns, and everything when a chunk would
// cross the field's x extent, are copied element by element with the ghost rules.
constexpr int T4X = 32, T4Y = 16, T4R = 4, T4ROWS = T4Y + 2, T4LD = 40;
constexpr int Z4CH = 32;  // z planes per block of the FP32 kernel (16 measured slower at 256^3)
constexpr int T4SLOTS = 2 * T4ROWS * 10;  // components x rows x (8 chunks + 2 edges)

__device__ __forceinline__ int ghost_index(int gi, int m, int lo_neumann, int hi_neumann) {
  if (gi < 0) return lo_neumann ? 1 : -1;
  if (gi >= m) return (hi_neumann && gi == m) ? m - 2 : -1;
  return gi;
}

// The FP32 kernel's weights, rounded to FP32 once on the host (a conversion per thread and
// weight would run on the FP64 pipe): the four interior class weights and the two
// Sommerfeld-like face rows.
struct StencilCoef32 {
  cpx<float> c[4];
  cpx<float> lo[3][3], hi[3][3];
};

// NORM: accumulate the block's |y|^2 (FP64) into sumsq; a compile-time flag so that the
// FP32 path carries no FP64 arithmetic when no norm is wanted.
// RW: the interior weights are real (a real wavenumber), so each class term is two real
// FMAs instead of a complex multiply-add.
template <int MODE, bool NORM, bool RW>
__global__ void __launch_bounds__(T4X* T4Y / T4R)
    stencil4_kernel(Geom g, StencilCoef32 coef, const float* __restrict__ x, float* __restrict__ y,
                    const float* __restrict__ f, double* __restrict__ sumsq) {
  constexpr int DIST = 3, NBUF = DIST + 2;
  constexpr int NT = T4X * T4Y / T4R;  // 128 threads
  __shared__ __align__(16) float sbuf[NBUF][2][T4ROWS][T4LD];
  __shared__ double red[NT / 32];

  const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * T4X + tx;
  const int x0 = blockIdx.x * T4X, y0 = blockIdx.y * T4Y;
  const int i = x0 + tx;
  const int l0 = blockIdx.z * Z4CH;
  const int l1 = min(l0 + Z4CH, g.mz);
  const int64_t plane = (int64_t)g.mx * g.my;
  const bool xn0 = g.face[0] == HELM6_NEUMANN, xn1 = g.face[1] == HELM6_NEUMANN;
  const bool yn0 = g.face[2] == HELM6_NEUMANN, yn1 = g.face[3] == HELM6_NEUMANN;
  const bool vec_ok = (g.mx & 3) == 0;

  // per-thread staging slots (fixed for every plane): component, halo row, slot kind
  int soff[3], sdst[3], skind[3];  // skind: 0 none, 1 vector chunk, 2 scalar x4, 3 scalar edge
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const int t = tid + k * NT;
    skind[k] = 0;
    soff[k] = -1;
    sdst[k] = 0;
    if (t < T4SLOTS) {
      const int comp = t / (T4ROWS * 10), rem = t - comp * (T4ROWS * 10);
      const int sy = rem / 10, sl = rem - sy * 10;
      const int gj = ghost_index(y0 + sy - 1, g.my, yn0, yn1);
      sdst[k] = (comp * T4ROWS + sy) * T4LD;  // start of the row in one ring slot
      if (sl < 8) {
        const int xs = x0 + 4 * sl;
        sdst[k] += 4 + 4 * sl;
        skind[k] = (vec_ok && xs + 3 < g.mx) ? 1 : 2;
        soff[k] = (gj < 0) ? -1 : gj * g.mx + xs;  // row offset of the chunk's first point
      } else {
        const int gi = ghost_index(sl == 8 ? x0 - 1 : x0 + T4X, g.mx, xn0, xn1);
        sdst[k] += (sl == 8) ? 3 : 4 + T4X;
        skind[k] = 3;
        soff[k] = (gj < 0 || gi < 0) ? -1 : gj * g.mx + gi;
      }
      soff[k] = (soff[k] < 0) ? -1 : soff[k];
      // component offset in the source is added at staging time
      skind[k] |= comp << 4;
      // for scalar chunks keep the row index for per-element ghost mapping
      if ((skind[k] & 15) == 2) soff[k] = (gj < 0) ? -1 : gj;  // row only
    }
  }

  auto stage = [&](int p, int slot) {
    int src = p;
    bool zplane = false;
    if (p < 0) {
      if (g.face[4] == HELM6_NEUMANN) src = 1; else zplane = true;
    } else if (p >= g.mz) {
      if (g.face[5] == HELM6_NEUMANN) src = g.mz - 2; else zplane = true;
    }
    const int64_t pbase = (int64_t)src * plane;
    float* sl_base = &sbuf[slot][0][0][0];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const int kind = skind[k] & 15;
      if (kind == 0) continue;
      const int comp = skind[k] >> 4;
      const float* xb = x + (comp ? g.N : 0) + pbase;
      float* d = sl_base + sdst[k];
      if (kind == 1) {
        const bool ok = !zplane && soff[k] >= 0;
        const uint32_t da = (uint32_t)__cvta_generic_to_shared(d);
        const float* sp = ok ? xb + soff[k] : x;
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(da), "l"(sp), "r"(ok ? 16 : 0)
                     : "memory");
      } else if (kind == 2) {
        // the 4 points of the chunk one by one (x extent not a multiple of 4, or partial tile)
        const int sl = ((sdst[k] % T4LD) - 4) / 4;
        for (int e = 0; e < 4; ++e) {
          const int gi = ghost_index(x0 + 4 * sl + e, g.mx, xn0, xn1);
          const bool ok = !zplane && soff[k] >= 0 && gi >= 0;
          const float* sp = ok ? xb + (int64_t)soff[k] * g.mx + gi : x;
          cp_async<4>(d + e, sp, ok ? 4 : 0);
        }
      } else {
        const bool ok = !zplane && soff[k] >= 0;
        cp_async<4>(d, ok ? xb + soff[k] : x, ok ? 4 : 0);
      }
    }
  };

  const cpx<float> c0 = coef.c[0], c1 = coef.c[1], c2 = coef.c[2], c3 = coef.c[3];
  const cpx<float> zero = {0.f, 0.f};
  // plane sums of three consecutive planes, rotated by renaming: the loop below is
  // unrolled by three so that no register moves are needed
  Sums<float> SA[T4R], SB[T4R], SC[T4R];
#pragma unroll
  for (int r = 0; r < T4R; ++r) SA[r] = SB[r] = SC[r] = Sums<float>{zero, zero, zero};
  double acc = 0.0;

  const int pfirst = l0 - 1;
  for (int d = 0; d < DIST; ++d) {
    if (pfirst + d <= l1) stage(pfirst + d, d);
    cp_commit();
  }
  // step p: the sums of plane p go to PN; rows of plane p - 1 use P0 (plane p - 2), P1
  // (plane p - 1) and PN (plane p)
  auto step = [&](int p, Sums<float>(&PN)[T4R], Sums<float>(&P0)[T4R], Sums<float>(&P1)[T4R]) {
    const int k = p - pfirst;
    if (p + DIST <= l1) stage(p + DIST, (k + DIST) % NBUF);
    cp_commit();
    cp_wait<DIST>();
    __syncthreads();
    const int buf = k % NBUF;
    // 6 halo rows x 3 columns per component for this thread's 4 points
    float vr[T4R + 2][3], vi[T4R + 2][3];
#pragma unroll
    for (int rr = 0; rr < T4R + 2; ++rr) {
#pragma unroll
      for (int cc = 0; cc < 3; ++cc) {
        vr[rr][cc] = sbuf[buf][0][T4R * ty + rr][tx + 3 + cc];
        vi[rr][cc] = sbuf[buf][1][T4R * ty + rr][tx + 3 + cc];
      }
    }
    // x-neighbour sums of the six halo rows, shared by the four points' face and diagonal sums
    float hr[T4R + 2], hi[T4R + 2];
#pragma unroll
    for (int rr = 0; rr < T4R + 2; ++rr) {
      hr[rr] = vr[rr][0] + vr[rr][2];
      hi[rr] = vi[rr][0] + vi[rr][2];
    }
#pragma unroll
    for (int r = 0; r < T4R; ++r) {
      Sums<float> cur;
      cur.c = mk(vr[r + 1][1], vi[r + 1][1]);
      cur.n = mk(hr[r + 1] + vr[r][1] + vr[r + 2][1], hi[r + 1] + vi[r][1] + vi[r + 2][1]);
      cur.d = mk(hr[r] + hr[r + 2], hi[r] + hi[r + 2]);
      PN[r] = cur;
    }
    const int l = p - 1;
    if (l >= l0 && i < g.mx) {
      const bool slo = (l == 0) && (g.face[4] == HELM6_SOMMERFELD);
      const bool shi = (l == g.mz - 1) && (g.face[5] == HELM6_SOMMERFELD);
#pragma unroll
      for (int r = 0; r < T4R; ++r) {
        const int j = y0 + T4R * ty + r;
        if (j >= g.my) continue;
        cpx<float> out;
        if (!slo && !shi) {
          const cpx<float> s1 = P1[r].n + P0[r].c + PN[r].c, s2 = P1[r].d + P0[r].n + PN[r].n,
                           s3 = P0[r].d + PN[r].d;
          if constexpr (RW) {
            out.re = fmaf(c3.re, s3.re, fmaf(c2.re, s2.re, fmaf(c1.re, s1.re, c0.re * P1[r].c.re)));
            out.im = fmaf(c3.re, s3.im, fmaf(c2.re, s2.im, fmaf(c1.re, s1.im, c0.re * P1[r].c.im)));
          } else {
            out = c0 * P1[r].c;
            out = cfma(c1, s1, out);
            out = cfma(c2, s2, out);
            out = cfma(c3, s3, out);
          }
        } else {
          out = zero;
#pragma unroll
          for (int a = 0; a < 3; ++a) {
            const cpx<float> wc = slo ? coef.lo[0][a] : coef.hi[0][a];
            const cpx<float> wm = slo ? coef.lo[1][a] : coef.hi[1][a];
            const cpx<float> wp = slo ? coef.lo[2][a] : coef.hi[2][a];
            const cpx<float> s0 = (a == 0) ? P0[r].c : (a == 1) ? P0[r].n : P0[r].d;
            const cpx<float> s1 = (a == 0) ? P1[r].c : (a == 1) ? P1[r].n : P1[r].d;
            const cpx<float> s2 = (a == 0) ? PN[r].c : (a == 1) ? PN[r].n : PN[r].d;
            out = cfma(wc, s0, out);
            out = cfma(wm, s1, out);
            out = cfma(wp, s2, out);
          }
        }
        const int64_t idx = (int64_t)l * plane + (int64_t)j * g.mx + i;
        if (MODE == 1) {
          out = mk(f[idx] - out.re, f[g.N + idx] - out.im);
        } else if (MODE == 2) {
          out = mk(f[idx] + out.re, f[g.N + idx] + out.im);
        }
        y[idx] = out.re;
        y[g.N + idx] = out.im;
        if (NORM) acc += (double)out.re * out.re + (double)out.im * out.im;
      }
    }
  };
  for (int p = pfirst; p <= l1; p += 3) {
    step(p, SA, SB, SC);
    if (p + 1 <= l1) step(p + 1, SB, SC, SA);
    if (p + 2 <= l1) step(p + 2, SC, SA, SB);
  }
  cp_wait<0>();
  if (NORM) {
    acc = warp_sum(acc);
    if ((tid & 31) == 0) red[tid >> 5] = acc;
    __syncthreads();
    if (tid < 32) {
      double v = (tid < NT / 32) ? red[tid] : 0.0;
      v = warp_sum(v);
      if (tid == 0) {
        const int64_t b = ((int64_t)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
        sumsq[b] = v;
      }
    }
  }
}

}  // namespace

int stencil_blocks(const Geom& g) {
  // the larger of the two kernels' grids (FP64: 32 x 8 tiles, FP32: 32 x 16 tiles)
  return ((g.mx + TX - 1) / TX) * ((g.my + TY - 1) / TY) * ((g.mz + ZCH - 1) / ZCH);
}

template <typename T>
void launch_stencil(const Geom& g, const StencilCoef& c, const T* x, T* y, const T* f, T* r,
                    int mode, double* sumsq, int* nblk, cudaStream_t s) {
  (void)r;
  if (sizeof(T) == 4) {
    dim3 block(T4X, T4Y / T4R);
    dim3 grid((g.mx + T4X - 1) / T4X, (g.my + T4Y - 1) / T4Y, (g.mz + Z4CH - 1) / Z4CH);
    if (nblk) *nblk = (int)(grid.x * grid.y * grid.z);
    note_launch();
    const float* xf = (const float*)x;
    float* yf = (float*)y;
    const float* ff = (const float*)f;
    StencilCoef32 c32;
    const c64d* cw[4] = {&c.interior.w[1][0], &c.interior.w[1][1], &c.interior.w[1][2], &c.interior.w[0][2]};
    for (int q = 0; q < 4; ++q) c32.c[q] = cpx<float>{(float)cw[q]->re, (float)cw[q]->im};
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) {
        c32.lo[a][b] = cpx<float>{(float)c.s_lo.w[a][b].re, (float)c.s_lo.w[a][b].im};
        c32.hi[a][b] = cpx<float>{(float)c.s_hi.w[a][b].re, (float)c.s_hi.w[a][b].im};
      }
    const bool nrm = sumsq != nullptr;
    const bool rw = c.interior.w[1][0].im == 0.0 && c.interior.w[1][1].im == 0.0 &&
                    c.interior.w[1][2].im == 0.0 && c.interior.w[0][2].im == 0.0;
#define HELM6_S4(M, N)                                                                   \
  do {                                                                                   \
    if (rw)                                                                              \
      stencil4_kernel<M, N, true><<<grid, block, 0, s>>>(g, c32, xf, yf, ff, N ? sumsq : nullptr);  \
    else                                                                                 \
      stencil4_kernel<M, N, false><<<grid, block, 0, s>>>(g, c32, xf, yf, ff, N ? sumsq : nullptr); \
  } while (0)
    if (mode == 0 && !nrm)
      HELM6_S4(0, false);
    else if (mode == 0)
      HELM6_S4(0, true);
    else if (mode == 1 && !nrm)
      HELM6_S4(1, false);
    else if (mode == 1)
      HELM6_S4(1, true);
    else
      HELM6_S4(2, false);
#undef HELM6_S4
    return;
  }
  dim3 block(TX, TY);
  dim3 grid((g.mx + TX - 1) / TX, (g.my + TY - 1) / TY, (g.mz + ZCH - 1) / ZCH);
  if (nblk) *nblk = (int)(grid.x * grid.y * grid.z);
  note_launch();
  const bool nrm = sumsq != nullptr;
  const bool rw = c.interior.w[1][0].im == 0.0 && c.interior.w[1][1].im == 0.0 &&
                  c.interior.w[1][2].im == 0.0 && c.interior.w[0][2].im == 0.0;
#define HELM6_SG(M, N)                                                                        \
  do {                                                                                        \
    if (rw)                                                                                   \
      stencil_kernel<T, M, N, true><<<grid, block, 0, s>>>(g, c, x, y, f, N ? sumsq : nullptr);  \
    else                                                                                      \
      stencil_kernel<T, M, N, false><<<grid, block, 0, s>>>(g, c, x, y, f, N ? sumsq : nullptr); \
  } while (0)
  if (mode == 0 && !nrm)
    HELM6_SG(0, false);
  else if (mode == 0)
    HELM6_SG(0, true);
  else if (mode == 1 && !nrm)
    HELM6_SG(1, false);
  else if (mode == 1)
    HELM6_SG(1, true);
  else
    HELM6_SG(2, false);
#undef HELM6_SG
}

template void launch_stencil<float>(const Geom&, const StencilCoef&, const float*, float*,
                                    const float*, float*, int, double*, int*, cudaStream_t);
template void launch_stencil<double>(const Geom&, const StencilCoef&, const double*, double*,
                                     const double*, double*, int, double*, int*, cudaStream_t);

}  // namespace helm6

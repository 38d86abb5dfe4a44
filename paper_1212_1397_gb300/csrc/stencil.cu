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

template <typename T, int MODE>
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
        out = c0 * P1.c;
        out = cfma(c1, P1.n + P0.c + P2.c, out);
        out = cfma(c2, P1.d + P0.n + P2.n, out);
        out = cfma(c3, P0.d + P2.d, out);
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
      if (sumsq) acc += (double)out.re * out.re + (double)out.im * out.im;
    }
  }
  cp_wait<0>();

  if (sumsq) {
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

}  // namespace

int stencil_blocks(const Geom& g) {
  return ((g.mx + TX - 1) / TX) * ((g.my + TY - 1) / TY) * ((g.mz + ZCH - 1) / ZCH);
}

template <typename T>
void launch_stencil(const Geom& g, const StencilCoef& c, const T* x, T* y, const T* f, T* r,
                    int mode, double* sumsq, int* nblk, cudaStream_t s) {
  (void)r;
  dim3 block(TX, TY);
  dim3 grid((g.mx + TX - 1) / TX, (g.my + TY - 1) / TY, (g.mz + ZCH - 1) / ZCH);
  if (nblk) *nblk = (int)(grid.x * grid.y * grid.z);
  note_launch();
  if (mode == 0)
    stencil_kernel<T, 0><<<grid, block, 0, s>>>(g, c, x, y, f, sumsq);
  else if (mode == 1)
    stencil_kernel<T, 1><<<grid, block, 0, s>>>(g, c, x, y, f, sumsq);
  else
    stencil_kernel<T, 2><<<grid, block, 0, s>>>(g, c, x, y, f, sumsq);
}

template void launch_stencil<float>(const Geom&, const StencilCoef&, const float*, float*,
                                    const float*, float*, int, double*, int*, cudaStream_t);
template void launch_stencil<double>(const Geom&, const StencilCoef&, const double*, double*,
                                     const double*, double*, int, double*, int*, cudaStream_t);

}  // namespace helm6

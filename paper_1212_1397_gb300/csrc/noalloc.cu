// helm6_residual_noalloc: r = F - A u and ||r||^2 without allocating device memory.
//
// For callers that cannot call cudaMalloc (see include/helm6.h): the kernel below is the
// residual variant of the stencil kernel working directly on the boundary's interleaved
// complex128 arrays, and its only scratch -- one FP64 partial sum per thread block -- is
// the file-scope device array g_noalloc_partials instead of library-allocated workspace.
#include <cmath>
#include <mutex>

#include "helm6_internal.h"

namespace helm6 {

namespace {

constexpr int TX = 32, TY = 8, ZCH = 16;
constexpr int kMaxDevices = 64;

// Block partial sums of |r|^2.  Every GPU that loads the library holds this array until
// the process exits.  Each call writes slots [0, nblocks) before reading them.
static __device__ __align__(256) double g_noalloc_partials[HELM6_NOALLOC_MAX_BLOCKS];

// Device address of g_noalloc_partials per device ordinal, looked up once per device.
double* g_partials_ptr[kMaxDevices] = {};
std::mutex g_setup_mutex;

__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Same z-marching tile as the library's stencil kernel: per plane the centre value, the
// sum of the 4 in-plane neighbours and of the 4 diagonals; rows combine three planes with
// the interior class weights or the Sommerfeld-like face weights.  Ghosts: reflection
// across Neumann faces, zero across Dirichlet faces.
__global__ void __launch_bounds__(TX* TY)
    residual_noalloc_kernel(Geom g, StencilCoef coef, const double2* __restrict__ F,
                            const double2* __restrict__ u, double2* __restrict__ r,
                            double* __restrict__ partials) {
  __shared__ double sre[2][TY + 2][TX + 2];
  __shared__ double sim[2][TY + 2][TX + 2];
  __shared__ double red[TX * TY / 32];
  using Z = cpx<double>;

  const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * TX + tx;
  const int i = blockIdx.x * TX + tx, j = blockIdx.y * TY + ty;
  const int l0 = blockIdx.z * ZCH;
  const int l1 = min(l0 + ZCH, g.mz);
  const int64_t plane = (int64_t)g.mx * g.my;
  const bool active = (i < g.mx) && (j < g.my);
  const Z c0 = cast<double>(coef.interior.w[1][0]);
  const Z c1 = cast<double>(coef.interior.w[1][1]);
  const Z c2 = cast<double>(coef.interior.w[1][2]);
  const Z c3 = cast<double>(coef.interior.w[0][2]);
  const Z zero = {0.0, 0.0};
  Z C0 = zero, N0 = zero, D0 = zero, C1 = zero, N1 = zero, D1 = zero, C2 = zero, N2 = zero,
    D2 = zero;
  double acc = 0.0;
  int buf = 0;

  for (int p = l0 - 1; p <= l1; ++p) {
    int src = p;
    bool zplane = false;
    if (p < 0) {
      if (g.face[4] == HELM6_NEUMANN) src = 1; else zplane = true;
    } else if (p >= g.mz) {
      if (g.face[5] == HELM6_NEUMANN) src = g.mz - 2; else zplane = true;
    }
    for (int t = tid; t < (TX + 2) * (TY + 2); t += TX * TY) {
      const int sy = t / (TX + 2), sx = t - sy * (TX + 2);
      int gi = blockIdx.x * TX + sx - 1, gj = blockIdx.y * TY + sy - 1;
      bool ok = !zplane;
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
      double2 v = make_double2(0.0, 0.0);
      if (ok) v = u[(int64_t)src * plane + (int64_t)gj * g.mx + gi];
      sre[buf][sy][sx] = v.x;
      sim[buf][sy][sx] = v.y;
    }
    __syncthreads();
    const int a = ty + 1, b = tx + 1;
    const Z cc = {sre[buf][a][b], sim[buf][a][b]};
    const Z nn = {sre[buf][a][b - 1] + sre[buf][a][b + 1] + sre[buf][a - 1][b] + sre[buf][a + 1][b],
                  sim[buf][a][b - 1] + sim[buf][a][b + 1] + sim[buf][a - 1][b] + sim[buf][a + 1][b]};
    const Z dd = {sre[buf][a - 1][b - 1] + sre[buf][a - 1][b + 1] + sre[buf][a + 1][b - 1] +
                      sre[buf][a + 1][b + 1],
                  sim[buf][a - 1][b - 1] + sim[buf][a - 1][b + 1] + sim[buf][a + 1][b - 1] +
                      sim[buf][a + 1][b + 1]};
    C0 = C1; N0 = N1; D0 = D1;
    C1 = C2; N1 = N2; D1 = D2;
    C2 = cc; N2 = nn; D2 = dd;
    buf ^= 1;

    const int l = p - 1;
    if (l >= l0 && active) {
      Z out;
      const bool slo = (l == 0) && (g.face[4] == HELM6_SOMMERFELD);
      const bool shi = (l == g.mz - 1) && (g.face[5] == HELM6_SOMMERFELD);
      if (!slo && !shi) {
        out = c0 * C1;
        out = cfma(c1, N1 + C0 + C2, out);
        out = cfma(c2, D1 + N0 + N2, out);
        out = cfma(c3, D0 + D2, out);
      } else {
        const RowWeights& W = slo ? coef.s_lo : coef.s_hi;
        out = zero;
        out = cfma(cast<double>(W.w[0][0]), C0, out);
        out = cfma(cast<double>(W.w[0][1]), N0, out);
        out = cfma(cast<double>(W.w[0][2]), D0, out);
        out = cfma(cast<double>(W.w[1][0]), C1, out);
        out = cfma(cast<double>(W.w[1][1]), N1, out);
        out = cfma(cast<double>(W.w[1][2]), D1, out);
        out = cfma(cast<double>(W.w[2][0]), C2, out);
        out = cfma(cast<double>(W.w[2][1]), N2, out);
        out = cfma(cast<double>(W.w[2][2]), D2, out);
      }
      const int64_t idx = (int64_t)l * plane + (int64_t)j * g.mx + i;
      const double2 fv = F[idx];
      const double2 rv = make_double2(fv.x - out.re, fv.y - out.im);
      r[idx] = rv;
      acc += rv.x * rv.x + rv.y * rv.y;
    }
  }
  acc = warp_sum(acc);
  if ((tid & 31) == 0) red[tid >> 5] = acc;
  __syncthreads();
  if (tid < 32) {
    double v = (tid < TX * TY / 32) ? red[tid] : 0.0;
    v = warp_sum(v);
    if (tid == 0)
      partials[((int64_t)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x] = v;
  }
}

__global__ void finish_kernel(const double* __restrict__ partials, int n, double* __restrict__ out) {
  __shared__ double sh[32];
  double v = 0.0;
  for (int b = threadIdx.x; b < n; b += blockDim.x) v += partials[b];
  v = warp_sum(v);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x < 32) {
    v = (threadIdx.x < blockDim.x / 32) ? sh[threadIdx.x] : 0.0;
    v = warp_sum(v);
    if (threadIdx.x == 0) *out = v;
  }
}

// Device address of the scratch array on the current device (looked up once per device).
int scratch_for_current_device(double** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) return HELM6_ERR_CUDA;
  if (dev < 0 || dev >= kMaxDevices) return HELM6_ERR_UNSUPPORTED;
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_partials_ptr[dev]) {
    double* p = nullptr;
    if (cudaGetSymbolAddress((void**)&p, g_noalloc_partials) != cudaSuccess || !p) {
      cudaGetLastError();
      return HELM6_ERR_CUDA;
    }
    g_partials_ptr[dev] = p;
  }
  *out = g_partials_ptr[dev];
  return HELM6_OK;
}

}  // namespace

}  // namespace helm6

using namespace helm6;

extern "C" int helm6_residual_noalloc(int n, double h, helm6_c64 k, const int faces[6], const void* F,
                                      const void* u, void* r, double* sumsq, void* stream) {
  if (!faces || !F || !u || !r || !sumsq || n < 1 || n > 4094) return HELM6_ERR_INVALID;
  for (int a = 0; a < 6; ++a)
    if (faces[a] != HELM6_DIRICHLET && faces[a] != HELM6_NEUMANN && faces[a] != HELM6_SOMMERFELD)
      return HELM6_ERR_INVALID;
  for (int a = 0; a < 4; ++a)
    if (faces[a] == HELM6_SOMMERFELD) return HELM6_ERR_INVALID;
  if (!(std::isfinite(k.re) && std::isfinite(k.im))) return HELM6_ERR_INVALID;
  Geom g;
  for (int a = 0; a < 6; ++a) g.face[a] = faces[a];
  auto cnt = [&](int a) { return n + (faces[2 * a] != HELM6_DIRICHLET) + (faces[2 * a + 1] != HELM6_DIRICHLET); };
  g.mx = cnt(0);
  g.my = cnt(1);
  g.mz = cnt(2);
  g.N = (int64_t)g.mx * g.my * g.mz;
  const dim3 block(TX, TY);
  const dim3 grid((g.mx + TX - 1) / TX, (g.my + TY - 1) / TY, (g.mz + ZCH - 1) / ZCH);
  const int64_t nblocks = (int64_t)grid.x * grid.y * grid.z;
  if (nblocks > HELM6_NOALLOC_MAX_BLOCKS) return HELM6_ERR_INVALID;  // grid too large for the static scratch
  double* scratch = nullptr;
  const int rc = scratch_for_current_device(&scratch);
  if (rc != HELM6_OK) return rc;
  StencilCoef coef;
  stencil_coefficients(cd(k.re, k.im), (h > 0) ? h : 1.0 / (n + 1), coef);
  cudaStream_t s = (cudaStream_t)stream;
  note_launch(2);
  residual_noalloc_kernel<<<grid, block, 0, s>>>(g, coef, (const double2*)F, (const double2*)u, (double2*)r,
                                                 scratch);
  finish_kernel<<<1, 256, 0, s>>>(scratch, (int)nblocks, sumsq);
  return cudaGetLastError() == cudaSuccess ? HELM6_OK : HELM6_ERR_CUDA;
}

// C-ABI entry points of the helm6 library and the host-side drivers of the solvers.
//
// The Krylov loops run on the host thread but keep every vector, the Hessenberg matrix
// and the Givens rotations on the device; one FP64 scalar (the residual estimate) is read
// back per iteration to decide convergence.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <complex>
#include <cstdio>
#include <cstring>
#include <atomic>
#include <limits>
#include <map>
#include <mutex>
#include <thread>
#include <type_traits>
#include <vector>

#include "helm6_internal.h"

using namespace helm6;

struct helm6_ctx {
  Geom g;        // internal geometry: Sommerfeld-like faces, if any, on z
  Geom gu;       // the caller's geometry (its array layout and faces)
  int xaxis = -1;  // the caller's axis (0 = x, 1 = y) carrying Sommerfeld-like faces, exchanged with z
  int n = 0;
  double h = 0;
  cd k;
  helm6_opts opts;
  cudaStream_t stream = nullptr;
  StencilCoef coef;
  c64d diag0, alpha;  // z-line diagonal -2 + k^2h^2 and Sommerfeld-like end term 2ikh
  int mrest = 30;
  int nred = 0;        // blocks of the reduction kernels
  int nsten = 0;       // blocks of the stencil kernel (partials of its fused norm)
  int ncgs = 0;        // blocks of the Gram-Schmidt update kernel
  int ndot = 0;        // blocks of the Gram-Schmidt reduction kernel
  double *Hr = nullptr, *Tm = nullptr, *red = nullptr, *coefv = nullptr, *qv = nullptr;
  int* brk = nullptr;
  double* u64 = nullptr;
  float* u32 = nullptr;
  double last_beta = 0;  // ||F - A U|| after the last FP64 residual
  bool zline_breakdown = false;  // a z line of the precomputed tables had a zero pivot
  // preconditioner tables (device): V, W = V^{-1} row-major m x m, eigenvalues
  double *Vx64 = nullptr, *Wx64 = nullptr, *Vy64 = nullptr, *Wy64 = nullptr;
  float *Vx32 = nullptr, *Wx32 = nullptr, *Vy32 = nullptr, *Wy32 = nullptr;
  double *lamx = nullptr, *lamy = nullptr;
  // MIXED: BF16 hi/lo basis tiles for the tensor-core transforms (null: SIMT FP32 path)
  uint8_t *Wx_tc = nullptr, *Wy_tc = nullptr, *Vx_tc = nullptr, *Vy_tc = nullptr;
  int* tcerr = nullptr;
  ZLines zl;  // z-line pivot tables (tensor-core path)
  // x/y transforms: HELM6_XFORM_DENSE, _FFT or _TENSOR per internal axis, and the FFT plans
  int xform[2] = {HELM6_XFORM_DENSE, HELM6_XFORM_DENSE};
  FftDev fft[2] = {};
  // FP64 vectors (2N doubles each)
  double *F64 = nullptr, *U64 = nullptr, *R64 = nullptr, *E64 = nullptr;
  double* D64 = nullptr;           // Chebyshev direction
  double cheb_lo = 0, cheb_hi = 0;  // spectral interval of A A_p^{-1} (HELM6_CHEB)
  double *V64 = nullptr, *Z64 = nullptr, *w64 = nullptr, *zt64 = nullptr, *tA64 = nullptr,
         *tB64 = nullptr, *cw64 = nullptr;
  // FP32 vectors (MIXED)
  float *V32 = nullptr, *Z32 = nullptr, *w32 = nullptr, *zt32 = nullptr, *tA32 = nullptr,
        *tB32 = nullptr, *cw32 = nullptr;
  __half* V16 = nullptr;  // FP16 basis (HELM6_BASIS_F16) in place of V32, holding vscale V_i
  double vscale = 1.0;
  // small device arrays
  double *partial = nullptr, *spart = nullptr, *H = nullptr, *cs = nullptr, *sn = nullptr,
         *gv = nullptr, *yv = nullptr, *h2 = nullptr, *scal = nullptr;
  int* status = nullptr;
  double* pinned = nullptr;  // host-pinned readback slots
  cudaEvent_t step_ev[2] = {nullptr, nullptr};  // Arnoldi step completion (alternating)
  // learned second stage (helm6_set_cnn)
  CnnNet cnn;
  int cnn_mode = HELM6_CNN_OFF;
  float cnn_scale = 0.f;
  float* cnn_t = nullptr;                          // u - A A_p^{-1} u, planar FP32
  uint16_t *cnn_a0 = nullptr, *cnn_a1 = nullptr;   // BF16 activations, 16 per point
  double* cnn_ss = nullptr;                        // ||u - A A_p^{-1} u||^2
  // AUTO probe: the learned stage preconditions the first cnn_cols columns of a cycle (the
  // rest use the direct preconditioner); probe_est is the cycle's residual estimate after
  // probe_cols columns (relative to its start), probe_rate[1] / [2] the per-column
  // reduction over those columns in cycle 1 (with the stage) and cycle 2 (without)
  int cnn_cols = 1 << 30;
  int probe_cols = 0;
  double probe_est = 0.0;
  double probe_rate[3] = {1.0, 1.0, 1.0};
  // CUDA graphs of the Arnoldi steps (opts.use_graphs): key (j, full, learned stage)
  struct StepGraph {
    cudaGraphExec_t exec;
    int kernels;
  };
  std::map<int, StepGraph> step_graphs;
  cudaStream_t cap_stream = nullptr;  // private stream the step graphs are captured on
  // device-driven solves (opts.use_graphs == 2): control block, its pinned mirror, the
  // whole-solve graph (for restart length solve_m) and two more capture streams
  GraphCtl* gctl = nullptr;
  GraphCtl* gctl_host = nullptr;
  cudaGraphExec_t solve_exec = nullptr;
  int solve_m = 0;
  cudaStream_t cap2 = nullptr, cap3 = nullptr;
  bool own_stream = false;            // `stream` was created by the context
  std::vector<void*> allocs;
  // measurement (helm6_profile_enable)
  struct Pending {
    int ph;
    double bytes;
    cudaEvent_t a, b;
  };
  bool prof_on = false;
  std::vector<cudaEvent_t> ev_pool, ev_all;
  std::vector<Pending> ev_pend;
  int64_t prof_count[HELM6_NPHASE] = {};
  double prof_ms[HELM6_NPHASE] = {};
  double prof_bytes[HELM6_NPHASE] = {};
  long long prof_l0 = 0;
};

namespace {

constexpr int kDiverge = 1000;

// Axis length rounded up to a multiple of 4 (row pitch of the tensor-core intermediates).
inline int pad4(int m) { return (m + 3) & ~3; }  // SKS: relative residual growth that counts as divergence

#define CK(call)                                      \
  do {                                                \
    cudaError_t e_ = (call);                          \
    if (e_ != cudaSuccess) {                          \
      fprintf(stderr, "helm6: %s failed: %s\n", #call, cudaGetErrorString(e_)); \
      return HELM6_ERR_CUDA;                          \
    }                                                 \
  } while (0)

template <typename T>
int dalloc(helm6_ctx* c, T** p, size_t count) {
  void* q = nullptr;
  if (count == 0) count = 1;
  if (cudaMalloc(&q, count * sizeof(T)) != cudaSuccess) {
    cudaGetLastError();
    return HELM6_ERR_NOMEM;
  }
  c->allocs.push_back(q);
  *p = (T*)q;
  return HELM6_OK;
}

// ---- per-phase event timing (measurement only) ----
// Accumulate finished intervals.  blocking = false stops at the first interval whose end
// event has not completed (so that the host does not wait for queued work).
void prof_flush(helm6_ctx* c, bool blocking = true) {
  size_t done = 0;
  for (auto& p : c->ev_pend) {
    if (!blocking && cudaEventQuery(p.b) != cudaSuccess) break;
    float ms = 0.f;
    if (cudaEventSynchronize(p.b) == cudaSuccess && cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) {
      c->prof_count[p.ph] += 1;
      c->prof_ms[p.ph] += ms;
      c->prof_bytes[p.ph] += p.bytes;
    }
    c->ev_pool.push_back(p.a);
    c->ev_pool.push_back(p.b);
    ++done;
  }
  c->ev_pend.erase(c->ev_pend.begin(), c->ev_pend.begin() + done);
  cudaGetLastError();  // a query of an unfinished event is not an error
}

cudaEvent_t prof_start(helm6_ctx* c) {
  if (!c->prof_on) return nullptr;
  if (c->ev_pool.size() < 2) prof_flush(c);
  if (c->ev_pool.size() < 2) return nullptr;
  cudaEvent_t a = c->ev_pool.back();
  c->ev_pool.pop_back();
  cudaEventRecord(a, c->stream);
  return a;
}

// bytes: algorithmic bytes of the interval (0: use the phase's default for one pass over
// a field in the Krylov precision, read + write).
void prof_stop(helm6_ctx* c, int ph, cudaEvent_t a, double bytes = 0.0) {
  if (!a) return;
  cudaEvent_t b = c->ev_pool.back();
  c->ev_pool.pop_back();
  cudaEventRecord(b, c->stream);
  if (bytes == 0.0) {
    const double s = (c->opts.precision == HELM6_FP64) ? 16.0 : 8.0;  // bytes per complex unknown
    bytes = 2.0 * s * (double)c->g.N;
  }
  c->ev_pend.push_back({ph, bytes, a, b});
}

// ---- 1D eigenbases of the x and y second-difference matrices (closed forms) ----
// D-D: nodes 1..n, modes j=1..n, V[l][j] = sin(j l t), t = pi/(n+1), lam = -4 sin^2(j t/2)
// N-N: nodes 0..n+1, modes j=0..n+1, V[l][j] = cos(j l t), V^{-1}[j][l] = (2/(n+1)) w_j w_l cos(j l t)
//      with end weights w = 1/2 at 0 and n+1
// D-N: nodes 1..n+1, th_j = (2j-1) t/2, V[l][j] = sin(l th_j), V^{-1}[j][l] = (2/(n+1)) w_l sin(l th_j),
//      w_{n+1} = 1/2, lam = -4 sin^2(th_j/2);  N-D: nodes 0..n, cos(l th_j), w_0 = 1/2.
void basis(int n, int lo, int hi, std::vector<double>& V, std::vector<double>& W, std::vector<double>& lam) {
  const double t = M_PI / (n + 1);
  const bool nlo = lo != HELM6_DIRICHLET, nhi = hi != HELM6_DIRICHLET;
  const int m = n + (nlo ? 1 : 0) + (nhi ? 1 : 0);
  V.assign((size_t)m * m, 0.0);
  W.assign((size_t)m * m, 0.0);
  lam.assign(m, 0.0);
  const double sc = 2.0 / (n + 1);
  for (int jj = 0; jj < m; ++jj) {
    for (int p = 0; p < m; ++p) {
      double v, wv;
      if (!nlo && !nhi) {
        const int j = jj + 1, l = p + 1;
        v = std::sin(j * l * t);
        wv = sc * v;
        lam[jj] = -4.0 * std::pow(std::sin(j * t / 2), 2);
      } else if (nlo && nhi) {
        const int j = jj, l = p;
        const double wj = (j == 0 || j == n + 1) ? 0.5 : 1.0, wl = (l == 0 || l == n + 1) ? 0.5 : 1.0;
        v = std::cos((double)j * l * t);
        wv = sc * wj * wl * v;
        lam[jj] = -4.0 * std::pow(std::sin(j * t / 2), 2);
      } else if (!nlo && nhi) {
        const int j = jj + 1, l = p + 1;
        const double th = (2 * j - 1) * t / 2, wl = (l == n + 1) ? 0.5 : 1.0;
        v = std::sin(l * th);
        wv = sc * wl * v;
        lam[jj] = -4.0 * std::pow(std::sin(th / 2), 2);
      } else {
        const int j = jj + 1, l = p;
        const double th = (2 * j - 1) * t / 2, wl = (l == 0) ? 0.5 : 1.0;
        v = std::cos(l * th);
        wv = sc * wl * v;
        lam[jj] = -4.0 * std::pow(std::sin(th / 2), 2);
      }
      V[(size_t)p * m + jj] = v;   // row = node p, column = mode jj
      W[(size_t)jj * m + p] = wv;  // row = mode jj, column = node p
    }
  }
}

}  // namespace

// ---- 27-point weights (Eq. scheme, Eq. 3DDISCS) ----
void helm6::stencil_coefficients(cd k, double h, StencilCoef& c) {
  const cd kh2 = k * k * h * h;
  const cd a = (1.0 + kh2 / 30.0) / 6.0;
  const double b = 1.0 / 30.0;
  const cd kappa = kh2 * (1.0 - kh2 / 12.0 + kh2 * kh2 / 360.0);
  // class weights of D_x+D_y+D_z + a(sum D D) + b DDD + kappa on the 27 points
  const cd c0 = -6.0 + 12.0 * a - 8.0 * b + kappa;
  const cd c1 = 1.0 - 4.0 * a + 4.0 * b;
  const cd c2 = a - 2.0 * b;
  const cd c3 = b;
  RowWeights in{};
  in.w[1][0] = to_pod(c0);
  in.w[1][1] = to_pod(c1);
  in.w[1][2] = to_pod(c2);
  for (int dz : {0, 2}) {
    in.w[dz][0] = to_pod(c1);
    in.w[dz][1] = to_pod(c2);
    in.w[dz][2] = to_pod(c3);
  }
  c.interior = in;
  // Sommerfeld-like face: B U_{-1} -> G1 U_1 + G0 U_0,
  // G1 = e2 mu3 [p (Dx+Dy) + DxDy/(30 mu3) + q I], G0 = e1 mu3 [r I - s (Dx+Dy)]
  const cd I(0.0, 1.0), ik = I * k;
  const cd mu3 = 1.0 / (1.0 + (2.0 * ik * h / 3.0) * (1.0 + 2.0 * kh2 / 15.0));
  const cd mu1 = (ik * h / 90.0 + (1.0 + kh2 / 30.0) / (6.0 * mu3)) / (1.0 + 2.0 * ik * h / 3.0);
  const cd e1 = std::exp(ik * h), e2 = std::exp(2.0 * ik * h);
  const cd p = mu1 + (2.0 * ik * h / 3.0) * (1.0 / 60.0 - mu1);
  const cd q = 1.0 - 2.0 * ik * h / 3.0 - 4.0 * ik * kh2 * h / 45.0;
  const cd r = (4.0 * ik * h / 3.0) * (1.0 + 2.0 * kh2 / 15.0);
  const cd s = (4.0 * ik * h / 3.0) * (1.0 / 60.0 - mu1);
  const cd g1c = e2 * mu3 * (-4.0 * p + 4.0 / (30.0 * mu3) + q);
  const cd g1n = e2 * mu3 * (p - 2.0 / (30.0 * mu3));
  const cd g1d = e2 * mu3 / (30.0 * mu3);
  const cd g0c = e1 * mu3 * (r + 4.0 * s);
  const cd g0n = -e1 * mu3 * s;
  RowWeights lo{};
  lo.w[1][0] = to_pod(c0 + g0c);
  lo.w[1][1] = to_pod(c1 + g0n);
  lo.w[1][2] = to_pod(c2);
  lo.w[2][0] = to_pod(c1 + g1c);
  lo.w[2][1] = to_pod(c2 + g1n);
  lo.w[2][2] = to_pod(c3 + g1d);
  RowWeights hi{};
  hi.w[1][0] = lo.w[1][0];
  hi.w[1][1] = lo.w[1][1];
  hi.w[1][2] = lo.w[1][2];
  hi.w[0][0] = lo.w[2][0];
  hi.w[0][1] = lo.w[2][1];
  hi.w[0][2] = lo.w[2][2];
  c.s_lo = lo;
  c.s_hi = hi;
}

namespace {

// ---- preconditioner: x/y forward transforms, z lines, inverse transforms ----
// in -> tA (x fwd) -> tB (y fwd) -> tA (z) -> tB (y inv) -> out (x inv); out may alias in.
template <typename T>
void precond(helm6_ctx* c, const T* in, T* out, T* tA, T* tB, T* cw, const T* Vx, const T* Wx,
             const T* Vy, const T* Wy) {
  const Geom& g = c->g;
  cudaStream_t s = c->stream;
  const int64_t plane = (int64_t)g.mx * g.my;
  const bool fx = c->xform[0] == HELM6_XFORM_FFT, fy = c->xform[1] == HELM6_XFORM_FFT;
  cudaEvent_t e = prof_start(c);
  if (fx)
    launch_fft_axis<T>(c->fft[0], 0, 0, g, in, tA, s);
  else
    launch_axis_gemm<T>(Wx, in, tA, g.mx, 2 * g.my * g.mz, g.mx, 0, 1, true, s);
  prof_stop(c, HELM6_PH_XFWD, e);
  e = prof_start(c);
  if (fy)
    launch_fft_axis<T>(c->fft[1], 1, 0, g, tA, tB, s);
  else
    launch_axis_gemm<T>(Wy, tA, tB, g.my, g.mx, g.mx, plane, 2 * g.mz, false, s);
  prof_stop(c, HELM6_PH_YFWD, e);
  e = prof_start(c);
  launch_ztri<T>(g, c->lamx, c->lamy, c->diag0, c->alpha, tB, tA, cw, c->status, s);
  prof_stop(c, HELM6_PH_ZTRI, e);
  e = prof_start(c);
  if (fy)
    launch_fft_axis<T>(c->fft[1], 1, 1, g, tA, tB, s);
  else
    launch_axis_gemm<T>(Vy, tA, tB, g.my, g.mx, g.mx, plane, 2 * g.mz, false, s);
  prof_stop(c, HELM6_PH_YINV, e);
  e = prof_start(c);
  if (fx)
    launch_fft_axis<T>(c->fft[0], 0, 1, g, tB, out, s);
  else
    launch_axis_gemm<T>(Vx, tB, out, g.mx, 2 * g.my * g.mz, g.mx, 0, 1, true, s);
  prof_stop(c, HELM6_PH_XINV, e);
}

void precond64(helm6_ctx* c, const double* in, double* out) {
  precond<double>(c, in, out, c->tA64, c->tB64, c->cw64, c->Vx64, c->Wx64, c->Vy64, c->Wy64);
}
// Tensor-core path: x forward writes planes x-mode-major ([z][p][y], y pitch Yp); y forward
// contracts the now contiguous y ([z][p][q], pitch Yp); the z lines walk that order; y inverse
// writes [z][y][p] back (p pitch Xp); x inverse restores [z][y][x].  Xp, Yp: the axis lengths
// rounded up to a multiple of 4, so that every intermediate row starts on a 16-byte boundary.
// in -> tA -> tB -> tA -> tB -> out.
void precond_tc(helm6_ctx* c, const float* in, float* out) {
  const Geom& g = c->g;
  cudaStream_t s = c->stream;
  const int terms = c->opts.xform_terms;
  const int rows_x = 2 * g.mz * g.my, rows_y = 2 * g.mz * g.mx;
  const int Xp = pad4(g.mx), Yp = pad4(g.my);
  cudaEvent_t e = prof_start(c);
  launch_xform_tc(in, c->tA32, c->Wx_tc, rows_x, g.mx, g.mx, terms, 1, g.my, c->tcerr, s, g.mx, Yp);
  prof_stop(c, HELM6_PH_XFWD, e);
  e = prof_start(c);
  launch_xform_tc(c->tA32, c->tB32, c->Wy_tc, rows_y, g.my, g.my, terms, 0, 1, c->tcerr, s, Yp, Yp);
  prof_stop(c, HELM6_PH_YFWD, e);
  e = prof_start(c);
  launch_ztri_apply(g, c->zl, c->tB32, c->tA32, s);
  prof_stop(c, HELM6_PH_ZTRI, e);
  e = prof_start(c);
  launch_xform_tc(c->tA32, c->tB32, c->Vy_tc, rows_y, g.my, g.my, terms, 1, g.mx, c->tcerr, s, Yp, Xp);
  prof_stop(c, HELM6_PH_YINV, e);
  e = prof_start(c);
  launch_xform_tc(c->tB32, out, c->Vx_tc, rows_x, g.mx, g.mx, terms, 0, 1, c->tcerr, s, Xp, g.mx);
  prof_stop(c, HELM6_PH_XINV, e);
}

void precond32(helm6_ctx* c, const float* in, float* out) {
  if (c->Wx_tc) {
    precond_tc(c, in, out);
    return;
  }
  precond<float>(c, in, out, c->tA32, c->tB32, c->cw32, c->Vx32, c->Wx32, c->Vy32, c->Wy32);
}

// Two-stage preconditioner: out = A_p^{-1} in + c s N((in - A A_p^{-1} in) / s).
void precond_cnn32(helm6_ctx* c, const float* in, float* out) {
  precond32(c, in, out);
  cudaEvent_t e = prof_start(c);
  int nb = 0;
  launch_stencil<float>(c->g, c->coef, out, c->cnn_t, in, nullptr, 1, c->spart, &nb, c->stream);
  launch_reduce_sum(c->spart, nb, c->cnn_ss, c->stream);
  cnn_apply_field(c->cnn, c->g.mz, c->g.my, c->g.mx, c->cnn_t, c->cnn_ss, c->cnn_a0, c->cnn_a1, c->cnn_scale, out,
                  c->tcerr, c->stream);
  // stencil pass (2 fields in, 1 out) and the four layers (2, 16, 16, 16 channels in; 16,
  // 16, 16 out in BF16; the last layer updates z in place)
  prof_stop(c, HELM6_PH_CNN, e, (double)c->g.N * (24.0 + 8.0 + 3 * 32.0 + 32.0 + 3 * 32.0 + 16.0));
}

// The learned-stage preconditioner of precision T (null for FP64, which has none).
template <typename T>
void (*precond_cnn_ptr())(helm6_ctx*, const T*, T*) {
  return nullptr;
}
template <>
void (*precond_cnn_ptr<float>())(helm6_ctx*, const float*, float*) {
  return precond_cnn32;
}
// The direct preconditioner of precision T (what the learned stage falls back to).
template <typename T>
void (*precond_plain_ptr())(helm6_ctx*, const T*, T*);
template <>
void (*precond_plain_ptr<float>())(helm6_ctx*, const float*, float*) {
  return precond32;
}
template <>
void (*precond_plain_ptr<double>())(helm6_ctx*, const double*, double*) {
  return precond64;
}

// ---- norms ----
template <typename T>
int norm2(helm6_ctx* c, const T* x, double* out) {
  launch_sumsq<T>(x, c->g.N, c->partial, c->nred, c->stream);
  launch_reduce_sum(c->partial, c->nred, c->scal, c->stream);
  CK(cudaMemcpyAsync(c->pinned, c->scal, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  *out = std::sqrt(c->pinned[0]);
  return HELM6_OK;
}

// r = F - A U (FP64) and ||r||
int residual64(helm6_ctx* c, double* beta) {
  int nb = 0;
  cudaEvent_t e = prof_start(c);
  launch_stencil<double>(c->g, c->coef, c->U64, c->R64, c->F64, nullptr, 1, c->spart, &nb, c->stream);
  launch_reduce_sum(c->spart, nb, c->scal, c->stream);
  prof_stop(c, HELM6_PH_RESID64, e, 48.0 * (double)c->g.N);
  CK(cudaMemcpyAsync(c->pinned, c->scal, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  *beta = std::sqrt(c->pinned[0]);
  c->last_beta = *beta;
  return HELM6_OK;
}

void push_hist(helm6_stats* st, double v);

// One Arnoldi cycle with delayed classical Gram-Schmidt.  On entry u holds the starting
// residual (any scale; g_0 = ||u||).  Step j applies the preconditioner and the operator
// to u_j, reduces V^H u_j, V^H w, ||u_j||^2 and u_j^H w in one pass, completes column j-1
// of the Hessenberg matrix (residual estimate |g_j|) and forms column j on the device, and
// writes v_j and u_{j+1} in one update pass.  The cycle ends at m columns (a last reduction
// of u_m completes column m-1), when the estimate of the last completed column is
// <= abs_tol, at a breakdown, or after maxsteps operator applications.  On return y holds
// the least-squares coefficients of its *kout columns and *beta = ||u_0||.
template <typename T, typename TV>
int arnoldi(helm6_ctx* c, TV* V, T* Z, T* u, T* w, T* zt, int m, double abs_tol, int maxsteps, bool flexible,
            void (*prec)(helm6_ctx*, const T*, T*), const StencilCoef& coef, int* kout, double* beta,
            helm6_stats* st) {
  cudaStream_t s = c->stream;  // the stream enqueue() works on (the capture stream while capturing)
  const int64_t N = c->g.N, vs = 2 * N;
  const int ldh = c->mrest + 1;
  CK(cudaMemsetAsync(c->H, 0, sizeof(double) * 2 * ldh * c->mrest, s));
  CK(cudaMemsetAsync(c->Hr, 0, sizeof(double) * 2 * ldh * c->mrest, s));
  CK(cudaMemsetAsync(c->gv, 0, sizeof(double) * 2 * ldh, s));
  if (flexible) CK(cudaMemsetAsync(c->Tm, 0, sizeof(double) * 2 * c->mrest * c->mrest, s));
  int k = 0, applied = 0;
  *beta = 0.0;
  // The host enqueues step j before reading the results of step j - 1 (two pinned slots and
  // events alternate), so the device never waits for the host between steps.  Step s
  // reports the estimate of column s - 1; when that meets the tolerance, the one step
  // queued behind it is wasted work that leaves columns < s untouched.
  auto finish = [&](int sidx, bool* stop) -> int {
    CK(cudaEventSynchronize(c->step_ev[sidx & 1]));
    if (c->prof_on) prof_flush(c, false);
    const double est = c->pinned[8 + (sidx & 1)];
    int brk = 0;
    std::memcpy(&brk, &c->pinned[10 + (sidx & 1)], sizeof(int));
    *stop = false;
    if (sidx == 0) {
      *beta = est;
      if (brk || !std::isfinite(est)) *stop = true;
    } else {
      k = sidx;
      if (st) st->iters++;
      if (sidx == c->probe_cols) c->probe_est = est;
      push_hist(st, est);  // rescaled by the caller
      if (!(est > abs_tol) || !std::isfinite(est) || brk) *stop = true;
    }
    return HELM6_OK;
  };
  // Enqueue step j: preconditioner and operator on u_j (full steps), the reduction pass,
  // the FP64 step algebra, the estimate's readback and event, and the update pass.
  // column j's preconditioner: the learned stage only for the first cnn_cols columns
  auto prec_of = [&](int j) { return (prec == precond_cnn_ptr<T>() && j >= c->cnn_cols) ? precond_plain_ptr<T>() : prec; };
  auto enqueue = [&](int j, bool full) -> int {
    if (full) {
      T* zj = flexible ? Z + (int64_t)j * vs : zt;
      prec_of(j)(c, u, zj);
      cudaEvent_t e = prof_start(c);
      launch_stencil<T>(c->g, coef, zj, w, nullptr, nullptr, 0, nullptr, nullptr, s);
      prof_stop(c, HELM6_PH_STENCIL, e);
    }
    const double vb = 2.0 * sizeof(T) * (double)N;    // one complex field
    const double vbb = 2.0 * sizeof(TV) * (double)N;  // one basis vector
    const double vsc = std::is_same<TV, T>::value ? 1.0 : c->vscale;
    cudaEvent_t e = prof_start(c);
    launch_dcgs_dot<T, TV>(V, vs, j, u, full ? w : nullptr, N, c->partial, c->ndot, vsc, s);
    prof_stop(c, HELM6_PH_DOT, e, vbb * j + vb * (full ? 2 : 1));
    e = prof_start(c);
    launch_reduce_cols(c->partial, c->ndot, 4 * j + 3, c->red, 0, s);
    launch_dcgs_step(j, full ? 1 : 0, c->red, c->Hr, c->H, ldh, flexible ? c->Tm : nullptr, c->mrest, c->cs, c->sn,
                     c->gv, c->coefv, c->scal + 2, c->brk, s);
    prof_stop(c, HELM6_PH_SMALL, e, 8.0 * c->ndot * (4 * j + 3));
    CK(cudaMemcpyAsync(&c->pinned[8 + (j & 1)], c->scal + 2, sizeof(double), cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(&c->pinned[10 + (j & 1)], c->brk, sizeof(int), cudaMemcpyDeviceToHost, s));
    // under stream capture the record must be external to become a graph node the host
    // can wait on (the flag is valid only while capturing)
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    CK(cudaStreamIsCapturing(s, &cap));
    CK(cudaEventRecordWithFlags(c->step_ev[j & 1], s,
                                cap == cudaStreamCaptureStatusActive ? cudaEventRecordExternal : 0u));
    if (full) {
      e = prof_start(c);
      launch_dcgs_update<T, TV>(V, vs, j, u, w, V + (int64_t)j * vs, N, c->coefv, c->ncgs, vsc, s);
      prof_stop(c, HELM6_PH_UPDATE, e, vbb * (j + 1) + vb * 3);
    }
    return HELM6_OK;
  };
  const bool graphs = c->opts.use_graphs && !c->prof_on;
  for (int j = 0;; ++j) {
    const bool full = (j < m) && (applied < maxsteps);
    if (graphs) {
      const int key = (j * 2 + (full ? 1 : 0)) * 2 + (prec_of(j) == precond_cnn_ptr<T>() ? 1 : 0);
      auto it = c->step_graphs.find(key);
      if (it == c->step_graphs.end()) {
        // first use of this step: capture and instantiate it, one thread at a time (the
        // batched solver drives several contexts from several threads; replays run freely)
        static std::mutex capture_mutex;
        std::lock_guard<std::mutex> lock(capture_mutex);
        const long long l0 = launch_total();
        // capture on the context's private stream (never one another context may share);
        // everything enqueue() and the preconditioner launch goes to c->stream, so point it
        // there for the capture
        cudaStream_t home = c->stream;
        c->stream = s = c->cap_stream;
        cudaError_t ce = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
        const int rc0 = ce == cudaSuccess ? enqueue(j, full) : HELM6_ERR_CUDA;
        cudaGraph_t gr = nullptr;
        if (ce == cudaSuccess) ce = cudaStreamEndCapture(s, &gr);
        c->stream = s = home;
        if (rc0 != HELM6_OK || ce != cudaSuccess) {
          if (gr) cudaGraphDestroy(gr);
          return rc0 != HELM6_OK ? rc0 : HELM6_ERR_CUDA;
        }
        cudaGraphExec_t ex = nullptr;
        const cudaError_t ie = cudaGraphInstantiate(&ex, gr, 0);
        cudaGraphDestroy(gr);
        CK(ie);
        const int kern = (int)(launch_total() - l0);
        note_launch(-kern);  // counted when the graph runs
        it = c->step_graphs.emplace(key, helm6_ctx::StepGraph{ex, kern}).first;
      }
      CK(cudaGraphLaunch(it->second.exec, s));
      note_launch(it->second.kernels);
    } else {
      const int rc0 = enqueue(j, full);
      if (rc0 != HELM6_OK) return rc0;
    }
    if (full) ++applied;
    bool stop = false;
    if (j >= 1) {
      int rc2 = finish(j - 1, &stop);
      if (rc2) return rc2;
      if (stop) break;
    }
    if (!full) {
      int rc2 = finish(j, &stop);
      if (rc2) return rc2;
      break;
    }
  }
  *kout = k;
  if (k > 0) launch_backsolve(c->H, ldh, k, c->gv, c->yv, s);
  CK(cudaGetLastError());
  return HELM6_OK;
}

void fix_hist(helm6_stats* st, int from, double scale) {
  if (!st) return;
  for (int i = from; i < st->nhist; ++i) st->hist[i] *= scale;
}

void push_hist(helm6_stats* st, double v) {
  if (st && st->nhist < HELM6_MAX_HIST) st->hist[st->nhist++] = v;
}

// Device status words: z-line breakdown flag, and the tensor-core kernel's timeout flag
// (a timed-out bounded wait is reported as a CUDA error).
int check_status(helm6_ctx* c) {
  int st = 0, te = 0;
  CK(cudaMemcpyAsync(&c->pinned[4], c->status, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaMemcpyAsync(&c->pinned[5], c->tcerr, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  std::memcpy(&st, &c->pinned[4], sizeof(int));
  std::memcpy(&te, &c->pinned[5], sizeof(int));
  if (te) return HELM6_ERR_CUDA;
  if (c->zline_breakdown) return HELM6_BREAKDOWN;
  return st;
}

// FP64 restarted GMRES / FGMRES on U64 with right side F64.
int solve_fp64(helm6_ctx* c, double normF, double tol, int m, int maxit, helm6_stats* st) {
  const bool flex = c->opts.method == HELM6_FGMRES;
  double beta;
  int rc = residual64(c, &beta);
  if (rc) return rc;
  push_hist(st, beta / normF);
  int iters = 0;
  while (true) {
    if (!std::isfinite(beta)) return HELM6_NONFINITE;
    if (beta <= tol * normF) return HELM6_OK;
    if (iters >= maxit) return HELM6_NOT_CONVERGED;
    launch_scale_copy<double>(c->R64, c->u64, c->g.N, nullptr, 1.0, c->stream);
    int k = 0;
    double b0 = 0;
    const int h0 = st ? st->nhist : 0;
    rc = arnoldi<double, double>(c, c->V64, c->Z64, c->u64, c->w64, c->zt64, m, tol * normF, maxit - iters, flex, precond64,
                         c->coef, &k, &b0, st);
    if (rc) return rc;
    fix_hist(st, h0, 1.0 / normF);
    iters += k;
    if (k > 0) {
      if (flex) {
        launch_tri_mul(c->Tm, c->mrest, k, c->yv, c->qv, c->stream);
        launch_lincomb<double, double>(c->Z64, 2 * c->g.N, k, c->qv, 1.0, c->U64, c->g.N, 1, c->stream);
      } else {
        launch_lincomb<double, double>(c->V64, 2 * c->g.N, k, c->yv, 1.0, c->E64, c->g.N, 0, c->stream);
        precond64(c, c->E64, c->E64);
        launch_axpy<double, double>(c->E64, c->U64, c->g.N, 1.0, c->stream);
      }
    }
    if (st) st->outer++;
    rc = residual64(c, &beta);
    if (rc) return rc;
    {
      const int cs = check_status(c);
      if (cs == HELM6_BREAKDOWN || cs < 0) return cs;
    }
  }
}

// MIXED: FP64 refinement around FP32 FGMRES with the FP32 preconditioner.
// Columns of the AUTO probe (cycle 1 preconditions this many columns with the learned stage).
constexpr int kCnnProbe = 2;

// Whether inner cycle `cyc` of a mixed solve uses the learned stage: ON always; AUTO uses
// it for the first kCnnProbe columns of cycle 1 only, of cycles 0-2 (cycle 0, from the
// initial guess, reduces faster than any later one and is not compared), and afterwards
// on every column only if those probe columns reduced the residual estimate per column by
// at least 10 % more, in logarithm, than the same columns of cycle 2 (without the stage).
bool cnn_cycle(const helm6_ctx* c, int cyc) {
  if (c->cnn_mode == HELM6_CNN_ON) return true;
  if (c->cnn_mode != HELM6_CNN_AUTO) return false;
  if (cyc < 3) return cyc == 1;
  const double l1 = std::log(std::max(c->probe_rate[1], 1e-300)), l2 = std::log(std::max(c->probe_rate[2], 1e-300));
  return l2 < 0 && l1 < 1.1 * l2;
}

bool graph_plain_ok(const helm6_ctx* c);
int solve_mixed_graph(helm6_ctx* c, double normF, double tol, int m, int maxit, helm6_stats* st);

int solve_mixed(helm6_ctx* c, double normF, double tol, int m, int maxit, helm6_stats* st) {
  double beta;
  int rc = residual64(c, &beta);
  if (rc) return rc;
  push_hist(st, beta / normF);
  int iters = 0;
  const double inner = c->opts.inner_tol > 0 ? c->opts.inner_tol : 1e-5;
  int cyc = 0;
  // set when a learned-stage cycle produced a non-finite correction: the rest of this
  // solve uses the direct preconditioner alone (the fallback)
  bool cnn_failed = false;
  std::vector<double> qhost;
  while (true) {
    if (!std::isfinite(beta)) return HELM6_NONFINITE;
    if (beta <= tol * normF) return HELM6_OK;
    if (iters >= maxit) return HELM6_NOT_CONVERGED;
    if (cyc >= 3 && (cnn_failed || !cnn_cycle(c, cyc)) && graph_plain_ok(c)) {
      // the learned stage is out for the rest of the solve (AUTO decided against it, or it
      // failed): finish as the plain solve, one device-driven graph launch from the current U
      helm6_stats tail;
      std::memset(&tail, 0, sizeof(tail));
      const int rs = solve_mixed_graph(c, normF, tol, m, maxit - iters, &tail);
      if (st) {
        st->iters += tail.iters;
        st->outer += tail.outer;
        for (int i = 1; i < tail.nhist && st->nhist < HELM6_MAX_HIST; ++i) st->hist[st->nhist++] = tail.hist[i];
      }
      return rs;
    }
    launch_convert<double, float>(c->R64, c->u32, c->g.N, 1.0 / beta, c->stream);
    const double itol = std::max(inner, 0.3 * tol * normF / beta);
    int k = 0;
    double b0 = 0;
    const int h0 = st ? st->nhist : 0;
    const bool use_cnn = !cnn_failed && cnn_cycle(c, cyc);
    auto* prec = use_cnn ? precond_cnn32 : precond32;
    const bool probing = c->cnn_mode == HELM6_CNN_AUTO && (cyc == 1 || cyc == 2);
    c->cnn_cols = (probing && use_cnn) ? kCnnProbe : (1 << 30);
    c->probe_cols = probing ? kCnnProbe : 0;
    c->probe_est = std::numeric_limits<double>::quiet_NaN();
    rc = c->V16 ? arnoldi<float, __half>(c, c->V16, c->Z32, c->u32, c->w32, c->zt32, m, itol, maxit - iters, true,
                                         prec, c->coef, &k, &b0, st)
                : arnoldi<float, float>(c, c->V32, c->Z32, c->u32, c->w32, c->zt32, m, itol, maxit - iters, true,
                                        prec, c->coef, &k, &b0, st);
    if (rc) return rc;
    if (st && use_cnn) st->cnn_cycles++;
    fix_hist(st, h0, beta / normF);
    iters += k;
    bool apply = k > 0;
    if (k > 0) launch_tri_mul(c->Tm, c->mrest, k, c->yv, c->qv, c->stream);
    if (use_cnn) {
      // A network that returns NaN/Inf (corrupt weights, an input far outside its training
      // range) makes the cycle's estimate or coefficients non-finite.  Then U64 keeps the
      // last good iterate and the remaining cycles fall back to the direct preconditioner.
      bool bad = false;
      if (st && st->nhist > h0)
        for (int i = h0; i < st->nhist; ++i) bad = bad || !std::isfinite(st->hist[i]);
      if (k > 0) {
        qhost.resize(2 * (size_t)k);
        CK(cudaMemcpyAsync(qhost.data(), c->qv, sizeof(double) * 2 * k, cudaMemcpyDeviceToHost, c->stream));
        CK(cudaStreamSynchronize(c->stream));
        for (double q : qhost) bad = bad || !std::isfinite(q);
      } else {
        bad = true;  // the cycle stopped before its first column: the stage's first output failed
      }
      if (bad) {
        apply = false;
        cnn_failed = true;
        if (st) st->cnn_fallbacks++;
      }
    }
    if (apply) launch_lincomb<float, double>(c->Z32, 2 * c->g.N, k, c->qv, beta, c->U64, c->g.N, 1, c->stream);
    if (st) st->outer++;
    rc = residual64(c, &beta);
    if (rc) return rc;
    if (st && st->nhist > 0) st->hist[st->nhist - 1] = beta / normF;  // true residual
    {
      const int cs = check_status(c);
      if (cs == HELM6_BREAKDOWN || cs < 0) return cs;
    }
    // per-column reduction over the probe columns (for the AUTO choice of the learned
    // stage); a cycle that ended before them, or failed, gives no reduction
    if (probing)
      c->probe_rate[cyc] = (std::isfinite(c->probe_est) && c->probe_est > 0 && !cnn_failed)
                               ? std::pow(c->probe_est, 1.0 / kCnnProbe)
                               : 1.0;
    c->cnn_cols = 1 << 30;
    c->probe_cols = 0;
    ++cyc;
  }
}

// ---- device-driven solve: the whole mixed FGMRES solve as one CUDA graph ----
// Structure (every decision taken on the device by the control kernels):
//   true residual; control (status, WHILE condition)
//   WHILE (not converged) {
//     u = r / beta; clear H, Hr, g, T; control (cycle starts, IF condition = 1)
//     IF (go) { Arnoldi step 0;  control (estimate, go) }   ...   IF (go) { step m (reduction only) }
//     y = R^-1 g, q = T y, U += beta Z q   (k = the cycle's completed columns, read on the device)
//     true residual; control (status, WHILE condition)
//   }
// The step bodies are the kernels of the host-driven Arnoldi steps without their readbacks.

// Whether a context can run the plain mixed solve (no learned stage) as one device-driven
// graph, and whether it runs its solves (and its part of a batch) that way.
bool graph_plain_ok(const helm6_ctx* c) {
  return c->opts.use_graphs == 2 && c->gctl && c->opts.precision == HELM6_MIXED && c->opts.method == HELM6_FGMRES &&
         !c->prof_on && !c->zline_breakdown;
}
bool graph_solve_ok(const helm6_ctx* c) { return graph_plain_ok(c) && c->cnn_mode == HELM6_CNN_OFF; }

// Add a conditional node (one body) to graph g after deps; *node and *body returned.
int add_conditional(cudaGraph_t g, const cudaGraphNode_t* deps, size_t nd, cudaGraphConditionalHandle h,
                    cudaGraphConditionalNodeType type, cudaGraphNode_t* node, cudaGraph_t* body) {
  cudaGraphNodeParams np = {};
  np.type = cudaGraphNodeTypeConditional;
  np.conditional.handle = h;
  np.conditional.type = type;
  np.conditional.size = 1;
  CK(cudaGraphAddNode(node, g, deps, nullptr, nd, &np));
  *body = np.conditional.phGraph_out[0];
  return HELM6_OK;
}

// Capture what fn enqueues on c's capture stream as a graph and add it to g as a child
// graph node after deps.
template <typename Fn>
int add_segment(helm6_ctx* c, cudaGraph_t g, const cudaGraphNode_t* deps, size_t nd, cudaGraphNode_t* node, Fn fn) {
  cudaStream_t s = c->cap_stream;
  cudaStream_t home = c->stream;
  c->stream = s;
  cudaGraph_t seg = nullptr;
  cudaError_t e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) fn(s);
  cudaError_t e2 = cudaStreamEndCapture(s, &seg);
  c->stream = home;
  if (e != cudaSuccess || e2 != cudaSuccess || !seg) {
    fprintf(stderr, "helm6: graph segment capture failed: %s / %s\n", cudaGetErrorString(e), cudaGetErrorString(e2));
    if (seg) cudaGraphDestroy(seg);
    cudaGetLastError();
    return HELM6_ERR_CUDA;
  }
  e = cudaGraphAddChildGraphNode(node, g, deps, nd, seg);
  cudaGraphDestroy(seg);
  CK(e);
  return HELM6_OK;
}

void enqueue_residual_dev(helm6_ctx* c, cudaStream_t s) {
  int nb = 0;
  launch_stencil<double>(c->g, c->coef, c->U64, c->R64, c->F64, nullptr, 1, c->spart, &nb, s);
  launch_reduce_sum(c->spart, nb, c->scal, s);
}

// Append the context's whole solve to graph G (as an independent branch): the first true
// residual, then a WHILE node whose body is the cycle (pre-cycle segment, m + 1 IF nodes
// holding the Arnoldi steps, post-cycle segment).
template <typename TV>
int append_solve_graph(helm6_ctx* c, TV* V, cudaGraph_t G, int m) {
  const int64_t N = c->g.N, vs = 2 * N;
  const int ldh = c->mrest + 1;
  const double vsc = std::is_same<TV, float>::value ? 1.0 : c->vscale;
  GraphCtl* gc = c->gctl;
  cudaGraphConditionalHandle hw;
  StepHandles ha;
  CK(cudaGraphConditionalHandleCreate(&hw, G, 0, 0));
  cudaGraphNode_t pro, wn;
  int rc = add_segment(c, G, nullptr, 0, &pro, [&](cudaStream_t s) {
    enqueue_residual_dev(c, s);
    launch_gctl_residual(gc, c->scal, c->status, c->tcerr, 1, hw, s);
  });
  if (rc) return rc;
  cudaGraph_t body = nullptr;
  if ((rc = add_conditional(G, &pro, 1, hw, cudaGraphCondTypeWhile, &wn, &body))) return rc;
  for (int j = 0; j <= m; ++j) CK(cudaGraphConditionalHandleCreate(&ha.h[j], body, 0, 0));
  cudaGraphNode_t prev;
  rc = add_segment(c, body, nullptr, 0, &prev, [&](cudaStream_t s) {
    launch_convert<double, float>(c->R64, c->u32, N, 1.0, s, &gc->inv_beta);
    cudaMemsetAsync(c->H, 0, sizeof(double) * 2 * ldh * c->mrest, s);
    cudaMemsetAsync(c->Hr, 0, sizeof(double) * 2 * ldh * c->mrest, s);
    cudaMemsetAsync(c->gv, 0, sizeof(double) * 2 * ldh, s);
    cudaMemsetAsync(c->Tm, 0, sizeof(double) * 2 * c->mrest * c->mrest, s);
    launch_gctl_cycle(gc, ha, m, s);
  });
  if (rc) return rc;
  for (int j = 0; j <= m; ++j) {
    cudaGraphNode_t ifn, inner;
    cudaGraph_t step = nullptr;
    if ((rc = add_conditional(body, &prev, 1, ha.h[j], cudaGraphCondTypeIf, &ifn, &step))) return rc;
    const bool full = j < m;
    rc = add_segment(c, step, nullptr, 0, &inner, [&](cudaStream_t s) {
      if (full) {
        float* zj = c->Z32 + (int64_t)j * vs;
        precond32(c, c->u32, zj);
        launch_stencil<float>(c->g, c->coef, zj, c->w32, nullptr, nullptr, 0, nullptr, nullptr, s);
      }
      launch_dcgs_dot<float, TV>(V, vs, j, c->u32, full ? c->w32 : nullptr, N, c->partial, c->ndot, vsc, s);
      launch_reduce_cols(c->partial, c->ndot, 4 * j + 3, c->red, 0, s);
      launch_dcgs_step(j, full ? 1 : 0, c->red, c->Hr, c->H, ldh, c->Tm, c->mrest, c->cs, c->sn, c->gv, c->coefv,
                       c->scal + 2, c->brk, s);
      if (full)
        launch_dcgs_update<float, TV>(V, vs, j, c->u32, c->w32, V + (int64_t)j * vs, N, c->coefv, c->ncgs, vsc, s);
      launch_gctl_step(gc, j, m, c->scal + 2, c->brk, j < m ? ha.h[j + 1] : ha.h[j], s);
    });
    if (rc) return rc;
    prev = ifn;
  }
  cudaGraphNode_t post;
  return add_segment(c, body, &prev, 1, &post, [&](cudaStream_t s) {
    launch_backsolve(c->H, ldh, 0, c->gv, c->yv, s, &gc->k);
    launch_tri_mul(c->Tm, c->mrest, 0, c->yv, c->qv, s, &gc->k);
    launch_lincomb<float, double>(c->Z32, vs, 0, c->qv, 1.0, c->U64, N, 1, s, &gc->k, &gc->beta);
    enqueue_residual_dev(c, s);
    launch_gctl_residual(gc, c->scal, c->status, c->tcerr, 0, hw, s);
  });
}

int append_solve(helm6_ctx* c, cudaGraph_t G, int m) {
  return c->V16 ? append_solve_graph<__half>(c, c->V16, G, m) : append_solve_graph<float>(c, c->V32, G, m);
}

// Parameters of one solve into the control block (stream-ordered upload from pinned memory).
int graph_params(helm6_ctx* c, double normF, double tol, int m, int maxit) {
  GraphCtl* h = c->gctl_host;
  std::memset(h, 0, sizeof(GraphCtl));
  h->tol_abs = tol * normF;
  h->itol_num = 0.3 * tol * normF;
  h->inner = c->opts.inner_tol > 0 ? c->opts.inner_tol : 1e-5;
  h->normF = normF;
  h->maxit = maxit;
  h->m = m;
  h->status = -1;
  CK(cudaMemcpyAsync(c->gctl, h, offsetof(GraphCtl, hist), cudaMemcpyHostToDevice, c->stream));
  return HELM6_OK;
}

// Statistics and status of a finished device-driven solve (after the control block's readback).
int graph_finish(helm6_ctx* c, helm6_stats* st) {
  const GraphCtl* h = c->gctl_host;
  c->last_beta = h->beta;
  if (st) {
    st->iters = h->iters;
    st->outer = h->outer;
    st->nhist = std::min(h->nhist, (int)HELM6_MAX_HIST);
    std::memcpy(st->hist, h->hist, sizeof(double) * st->nhist);
  }
  return h->status < 0 && h->status != HELM6_ERR_CUDA ? HELM6_ERR_CUDA : h->status;
}

int solve_mixed_graph(helm6_ctx* c, double normF, double tol, int m, int maxit, helm6_stats* st) {
  if (!c->solve_exec || c->solve_m != m) {
    if (c->solve_exec) cudaGraphExecDestroy(c->solve_exec);
    c->solve_exec = nullptr;
    static std::mutex capture_mutex;
    std::lock_guard<std::mutex> lock(capture_mutex);
    cudaGraph_t G;
    CK(cudaGraphCreate(&G, 0));
    const long long l0 = launch_total();
    int rc = append_solve(c, G, m);
    note_launch(-(int)(launch_total() - l0));
    if (rc == HELM6_OK && cudaGraphInstantiate(&c->solve_exec, G, 0) != cudaSuccess) rc = HELM6_ERR_CUDA;
    cudaGraphDestroy(G);
    if (rc) {
      cudaGetLastError();
      return rc;
    }
    c->solve_m = m;
  }
  int rc = graph_params(c, normF, tol, m, maxit);
  if (rc) return rc;
  CK(cudaGraphLaunch(c->solve_exec, c->stream));
  CK(cudaMemcpyAsync(c->gctl_host, c->gctl, sizeof(GraphCtl), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  return graph_finish(c, st);
}

// Batched device-driven solves: one graph holding every problem's whole solve as an
// independent branch, instantiated once per set of contexts and restart length, launched
// once per batch.
struct BatchGraph {
  std::vector<helm6_ctx*> ctxs;
  int m;
  cudaGraphExec_t exec;
};
std::mutex g_batch_mutex;
std::vector<BatchGraph> g_batch_graphs;

void forget_batch_graphs_of(helm6_ctx* c) {
  std::lock_guard<std::mutex> lock(g_batch_mutex);
  for (size_t i = 0; i < g_batch_graphs.size();) {
    const auto& v = g_batch_graphs[i].ctxs;
    if (std::find(v.begin(), v.end(), c) != v.end()) {
      cudaGraphExecDestroy(g_batch_graphs[i].exec);
      g_batch_graphs.erase(g_batch_graphs.begin() + i);
    } else {
      ++i;
    }
  }
}

int batch_exec(const std::vector<helm6_ctx*>& act, int m, cudaGraphExec_t* out) {
  std::lock_guard<std::mutex> lock(g_batch_mutex);
  for (auto& b : g_batch_graphs)
    if (b.m == m && b.ctxs == act) {
      *out = b.exec;
      return HELM6_OK;
    }
  cudaGraph_t G;
  CK(cudaGraphCreate(&G, 0));
  const long long l0 = launch_total();
  int rc = HELM6_OK;
  for (helm6_ctx* c : act)
    if ((rc = append_solve(c, G, m))) break;
  note_launch(-(int)(launch_total() - l0));
  cudaGraphExec_t ex = nullptr;
  if (rc == HELM6_OK && cudaGraphInstantiate(&ex, G, 0) != cudaSuccess) rc = HELM6_ERR_CUDA;
  cudaGraphDestroy(G);
  if (rc) {
    cudaGetLastError();
    return rc;
  }
  g_batch_graphs.push_back(BatchGraph{act, m, ex});
  *out = ex;
  return HELM6_OK;
}

// The whole batch in one launch: right sides and their norms per problem, then the batch
// graph (every problem's device-driven solve as a branch), then the solutions.
int solve_batch_graph(helm6_ctx* const* ctxs, int count, const void* const* F, void* const* u, double tol,
                      int restart, int maxit, helm6_stats* stats) {
  std::vector<double> normF(count, 0.0);
  for (int i = 0; i < count; ++i) {
    helm6_ctx* c = ctxs[i];
    cudaStream_t s = c->stream;
    CK(cudaMemsetAsync(c->status, 0, sizeof(int), s));
    CK(cudaMemsetAsync(c->tcerr, 0, sizeof(int), s));
    launch_caller_to_planar(c->g, c->xaxis, (const double*)F[i], c->F64, s);
    launch_sumsq<double>(c->F64, c->g.N, c->partial, c->nred, s);
    launch_reduce_sum(c->partial, c->nred, c->scal, s);
    CK(cudaMemcpyAsync(c->pinned, c->scal, sizeof(double), cudaMemcpyDeviceToHost, s));
    launch_caller_to_planar(c->g, c->xaxis, (const double*)u[i], c->U64, s);
  }
  std::vector<helm6_ctx*> act;
  std::vector<int> idx, status(count, HELM6_OK);
  for (int i = 0; i < count; ++i) {
    helm6_ctx* c = ctxs[i];
    CK(cudaStreamSynchronize(c->stream));
    normF[i] = std::sqrt(c->pinned[0]);
    if (!std::isfinite(normF[i])) {
      status[i] = HELM6_NONFINITE;
    } else if (normF[i] == 0.0) {
      CK(cudaMemsetAsync(u[i], 0, sizeof(double) * 2 * c->g.N, c->stream));
    } else {
      int rc = graph_params(c, normF[i], tol, restart, maxit);
      if (rc) return rc;
      act.push_back(c);
      idx.push_back(i);
    }
  }
  for (int i = 0; i < count; ++i) CK(cudaStreamSynchronize(ctxs[i]->stream));
  if (!act.empty()) {
    cudaGraphExec_t ex = nullptr;
    int rc = batch_exec(act, restart, &ex);
    if (rc) return rc;
    cudaStream_t s = act[0]->stream;
    CK(cudaGraphLaunch(ex, s));
    for (helm6_ctx* c : act) CK(cudaMemcpyAsync(c->gctl_host, c->gctl, sizeof(GraphCtl), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    for (size_t a = 0; a < act.size(); ++a) {
      helm6_ctx* c = act[a];
      const int i = idx[a];
      helm6_stats local;
      helm6_stats* S = stats ? &stats[i] : &local;
      std::memset(S, 0, sizeof(*S));
      status[i] = graph_finish(c, S);
      if (status[i] < 0) return status[i];
      launch_planar_to_caller(c->g, c->xaxis, c->U64, (double*)u[i], c->stream);
      S->relres = c->last_beta / normF[i];
      S->status = status[i];
      const GraphCtl* h = c->gctl_host;
      S->t_total_ms = h->t1 > h->t0 ? 1e-6 * (double)(h->t1 - h->t0) : 0.0;
    }
  }
  int worst = HELM6_OK;
  for (int i = 0; i < count; ++i) {
    CK(cudaStreamSynchronize(ctxs[i]->stream));
    if (stats && (normF[i] == 0.0 || !std::isfinite(normF[i]))) {
      std::memset(&stats[i], 0, sizeof(helm6_stats));
      stats[i].status = status[i];
    }
    worst = std::max(worst, status[i]);
  }
  return worst;
}

// SKS (Algorithm 1) in its equivalent defect-correction form U <- U + A_p^{-1}(F - A U),
// the residual computed in FP64; MIXED applies A_p^{-1} in FP32 to r/||r||.
int solve_sks(helm6_ctx* c, double normF, double tol, int maxit, helm6_stats* st) {
  double beta;
  int rc = residual64(c, &beta);
  if (rc) return rc;
  const double beta0 = beta;
  int iters = 0;
  while (true) {
    if (!std::isfinite(beta)) return HELM6_NONFINITE;
    if (beta <= tol * normF) return HELM6_OK;
    if (beta > kDiverge * std::max(beta0, normF)) return HELM6_DIVERGED;
    if (iters >= maxit) return HELM6_NOT_CONVERGED;
    if (c->opts.precision == HELM6_FP64) {
      precond64(c, c->R64, c->E64);
      launch_axpy<double, double>(c->E64, c->U64, c->g.N, 1.0, c->stream);
    } else {
      launch_convert<double, float>(c->R64, c->w32, c->g.N, 1.0 / beta, c->stream);
      precond32(c, c->w32, c->zt32);
      launch_axpy<float, double>(c->zt32, c->U64, c->g.N, beta, c->stream);
    }
    ++iters;
    rc = residual64(c, &beta);
    if (rc) return rc;
    if (st) {
      st->iters++;
      push_hist(st, beta / normF);
    }
    {
      const int cs = check_status(c);
      if (cs == HELM6_BREAKDOWN || cs < 0) return cs;
    }
  }
}

// Extremes of the eigenvalues of A A_p^{-1} on the all-Dirichlet cube (real k): both
// operators are diagonal on the sine modes; with c_a = cos(p_a pi h) the 27-point operator's
// eigenvalue is w0 + 2 w1 (cx + cy + cz) + 4 w2 (cx cy + cx cz + cy cz) + 8 w3 cx cy cz
// (w0..w3 its centre, face, edge and corner weights) and the 7-point operator's
// -6 + 2 (cx + cy + cz) + k^2 h^2.  The ratio is symmetric in the three axes, so only
// i <= j <= l are visited.
void dirichlet_ratio_bounds(const helm6_ctx* c, double* lo, double* hi) {
  const int n = c->n;
  const double w0 = c->coef.interior.w[1][0].re, w1 = c->coef.interior.w[1][1].re,
               w2 = c->coef.interior.w[1][2].re, w3 = c->coef.interior.w[0][2].re;
  const double kh2 = (c->k * c->k * c->h * c->h).real();
  std::vector<double> cs(n);
  for (int p = 0; p < n; ++p) cs[p] = std::cos((p + 1) * M_PI * c->h);
  double mn = INFINITY, mx = -INFINITY;
  for (int i = 0; i < n; ++i)
    for (int j = i; j < n; ++j)
      for (int l = j; l < n; ++l) {
        const double x = cs[i], y = cs[j], z = cs[l];
        const double s1 = x + y + z, s2 = x * y + x * z + y * z, s3 = x * y * z;
        const double la = w0 + 2 * w1 * s1 + 4 * w2 * s2 + 8 * w3 * s3;
        const double lp = -6.0 + 2 * s1 + kh2;
        const double r = la / lp;
        mn = std::min(mn, r);
        mx = std::max(mx, r);
      }
  *lo = mn;
  *hi = mx;
}

// Chebyshev acceleration on A A_p^{-1} for the interval [lo, hi] (the theorem of Section 2):
// d_0 = A_p^{-1} r_0 / theta, U += d_n, r = F - A U (FP64), rho_{n+1} = 1/(2 theta/delta - rho_n),
// d_{n+1} = rho_{n+1} rho_n d_n + (2 rho_{n+1}/delta) A_p^{-1} r; MIXED applies A_p^{-1} in FP32
// to r/||r||.  Divergence as for SKS.
int solve_cheb(helm6_ctx* c, double normF, double tol, int maxit, helm6_stats* st) {
  const double theta = 0.5 * (c->cheb_hi + c->cheb_lo), delta = 0.5 * (c->cheb_hi - c->cheb_lo);
  const int64_t N = c->g.N;
  cudaStream_t s = c->stream;
  double beta;
  int rc = residual64(c, &beta);
  if (rc) return rc;
  const double beta0 = beta;
  // E = A_p^{-1} r (FP64 result in both precisions)
  auto prec_r = [&]() {
    if (c->opts.precision == HELM6_FP64) {
      precond64(c, c->R64, c->E64);
    } else {
      launch_convert<double, float>(c->R64, c->w32, N, 1.0 / beta, s);
      precond32(c, c->w32, c->zt32);
      launch_convert<float, double>(c->zt32, c->E64, N, beta, s);
    }
  };
  if (!std::isfinite(beta)) return HELM6_NONFINITE;
  if (beta <= tol * normF) return HELM6_OK;
  double rho = delta / theta;
  prec_r();
  CK(cudaMemsetAsync(c->D64, 0, sizeof(double) * 2 * N, s));
  launch_axpby(c->E64, c->D64, N, 0.0, 1.0 / theta, s);
  int iters = 0;
  while (true) {
    if (iters >= maxit) return HELM6_NOT_CONVERGED;
    launch_axpy<double, double>(c->D64, c->U64, N, 1.0, s);
    ++iters;
    rc = residual64(c, &beta);
    if (rc) return rc;
    if (st) {
      st->iters++;
      push_hist(st, beta / normF);
    }
    {
      const int cs = check_status(c);
      if (cs == HELM6_BREAKDOWN || cs < 0) return cs;
    }
    if (!std::isfinite(beta)) return HELM6_NONFINITE;
    if (beta <= tol * normF) return HELM6_OK;
    if (beta > kDiverge * std::max(beta0, normF)) return HELM6_DIVERGED;
    const double rho_new = 1.0 / (2.0 * theta / delta - rho);
    prec_r();
    launch_axpby(c->E64, c->D64, N, rho_new * rho, 2.0 * rho_new / delta, s);
    rho = rho_new;
  }
}

bool valid_face(int f) { return f == HELM6_DIRICHLET || f == HELM6_NEUMANN || f == HELM6_SOMMERFELD; }

}  // namespace

extern "C" {

void helm6_opts_default(helm6_opts* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->precision = HELM6_FP64;
  o->method = HELM6_GMRES;
  o->xform_terms = 3;
  o->max_restart = 30;
  o->inner_tol = 1e-5;
  o->stream = nullptr;
}

const char* helm6_status_string(int code) {
  switch (code) {
    case HELM6_OK: return "ok";
    case HELM6_NOT_CONVERGED: return "not converged (maxit reached)";
    case HELM6_DIVERGED: return "diverged";
    case HELM6_BREAKDOWN: return "breakdown (zero pivot in a z-line solve)";
    case HELM6_NONFINITE: return "non-finite value in the input or the iteration";
    case HELM6_ERR_INVALID: return "invalid argument";
    case HELM6_ERR_NOMEM: return "device allocation failed";
    case HELM6_ERR_CUDA: return "CUDA error";
    case HELM6_ERR_UNSUPPORTED: return "unsupported";
    default: return "unknown status";
  }
}

void helm6_destroy(helm6_ctx* c) {
  if (!c) return;
  if (c->stream) cudaStreamSynchronize(c->stream); else cudaDeviceSynchronize();
  for (auto& kv : c->step_graphs) cudaGraphExecDestroy(kv.second.exec);
  if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
  forget_batch_graphs_of(c);
  if (c->solve_exec) cudaGraphExecDestroy(c->solve_exec);
  if (c->cap2) cudaStreamDestroy(c->cap2);
  if (c->cap3) cudaStreamDestroy(c->cap3);
  if (c->gctl_host) cudaFreeHost(c->gctl_host);
  for (void* p : c->allocs) cudaFree(p);
  cnn_free(c->cnn);
  for (cudaEvent_t e : c->ev_all) cudaEventDestroy(e);
  for (cudaEvent_t e : c->step_ev)
    if (e) cudaEventDestroy(e);
  if (c->pinned) cudaFreeHost(c->pinned);
  if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
  delete c;
}

int helm6_create(helm6_ctx** out, int n, double h, helm6_c64 k, const int faces[6], const helm6_opts* opts) {
  if (!out || !faces || n < 1 || n > 4094) return HELM6_ERR_INVALID;
  for (int i = 0; i < 6; ++i)
    if (!valid_face(faces[i])) return HELM6_ERR_INVALID;
  // Sommerfeld-like faces on one axis pair at most.  The face rows of Eq. 3DDISCS are
  // written for z and the scheme is symmetric under exchanging axes, so an x or y pair is
  // solved as the z pair of the problem with that axis exchanged with z: the internal
  // geometry carries it on z, and only the conversions at the boundary see the exchange.
  int s_axes = 0, xaxis = -1;
  for (int a = 0; a < 3; ++a)
    if (faces[2 * a] == HELM6_SOMMERFELD || faces[2 * a + 1] == HELM6_SOMMERFELD) {
      ++s_axes;
      if (a < 2) xaxis = a;
    }
  if (s_axes > 1) return HELM6_ERR_INVALID;
  int fint[6];
  for (int i = 0; i < 6; ++i) fint[i] = faces[i];
  if (xaxis >= 0) {
    std::swap(fint[2 * xaxis], fint[4]);
    std::swap(fint[2 * xaxis + 1], fint[5]);
  }
  helm6_opts o;
  helm6_opts_default(&o);
  if (opts) o = *opts;
  if (o.precision != HELM6_FP64 && o.precision != HELM6_MIXED) return HELM6_ERR_INVALID;
  if (o.method < HELM6_GMRES || o.method > HELM6_CHEB) return HELM6_ERR_INVALID;
  if (o.method == HELM6_CHEB) {
    const bool given = o.cheb_lo != 0.0 || o.cheb_hi != 0.0;
    if (given && !(o.cheb_lo > 0.0 && o.cheb_hi > o.cheb_lo && std::isfinite(o.cheb_hi))) return HELM6_ERR_INVALID;
    if (!given) {
      for (int i = 0; i < 6; ++i)
        if (faces[i] != HELM6_DIRICHLET) return HELM6_ERR_UNSUPPORTED;
      if (k.im != 0.0) return HELM6_ERR_UNSUPPORTED;
    }
  }
  if (o.basis < HELM6_BASIS_AUTO || o.basis > HELM6_BASIS_F16) return HELM6_ERR_INVALID;
  if (o.basis == HELM6_BASIS_F16 && o.precision != HELM6_MIXED) return HELM6_ERR_INVALID;
  if (o.transform < HELM6_XFORM_AUTO || o.transform > HELM6_XFORM_FFT) return HELM6_ERR_INVALID;
  if (o.xform_terms == 0) o.xform_terms = 3;
  if (o.xform_terms < 1 || o.xform_terms > 3) return HELM6_ERR_INVALID;
  if (o.max_restart == 0) o.max_restart = 30;
  if (o.max_restart < 1 || o.max_restart > 64) return HELM6_ERR_INVALID;
  if (o.inner_tol == 0) o.inner_tol = 1e-5;
  if (!(o.inner_tol > 0 && o.inner_tol < 1)) return HELM6_ERR_INVALID;
  if (o.dot_blocks < 0 || o.dot_blocks > 64 * 1024 || o.update_blocks < 0 || o.update_blocks > 64 * 1024)
    return HELM6_ERR_INVALID;
  if (!(std::isfinite(k.re) && std::isfinite(k.im))) return HELM6_ERR_INVALID;

  helm6_ctx* c = new helm6_ctx();
  c->n = n;
  c->h = (h > 0) ? h : 1.0 / (n + 1);
  c->k = cd(k.re, k.im);
  c->opts = o;
  c->stream = (cudaStream_t)o.stream;
  c->mrest = o.max_restart;
  auto geom = [&](const int* f, Geom& g) {
    for (int i = 0; i < 6; ++i) g.face[i] = f[i];
    auto cnt = [&](int a) { return n + (f[2 * a] != HELM6_DIRICHLET) + (f[2 * a + 1] != HELM6_DIRICHLET); };
    g.mx = cnt(0);
    g.my = cnt(1);
    g.mz = cnt(2);
    g.N = (int64_t)g.mx * g.my * g.mz;
  };
  geom(fint, c->g);
  geom(faces, c->gu);
  c->xaxis = xaxis;
  stencil_coefficients(c->k, c->h, c->coef);
  const cd I(0.0, 1.0);
  c->diag0 = to_pod(-2.0 + c->k * c->k * c->h * c->h);
  c->alpha = to_pod(2.0 * I * c->k * c->h);

  int rc = HELM6_OK;
  auto fail = [&](int code) {
    helm6_destroy(c);
    return code;
  };
  if (o.own_stream) {
    c->stream = nullptr;
    if (cudaStreamCreate(&c->stream) != cudaSuccess) return fail(HELM6_ERR_CUDA);
    c->own_stream = true;
  }
  if (o.use_graphs && cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking) != cudaSuccess)
    return fail(HELM6_ERR_CUDA);
  if (o.use_graphs == 2) {
    if (cudaStreamCreateWithFlags(&c->cap2, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&c->cap3, cudaStreamNonBlocking) != cudaSuccess ||
        cudaMallocHost(&c->gctl_host, sizeof(GraphCtl)) != cudaSuccess)
      return fail(HELM6_ERR_CUDA);
    if ((rc = dalloc(c, &c->gctl, 1))) return fail(rc);
  }
  // bases
  std::vector<double> Vx, Wx, lx, Vy, Wy, ly;
  basis(n, c->g.face[0], c->g.face[1], Vx, Wx, lx);  // the internal x and y faces
  basis(n, c->g.face[2], c->g.face[3], Vy, Wy, ly);
  const size_t mx2 = (size_t)c->g.mx * c->g.mx, my2 = (size_t)c->g.my * c->g.my;
  if ((rc = dalloc(c, &c->Vx64, mx2)) || (rc = dalloc(c, &c->Wx64, mx2)) || (rc = dalloc(c, &c->Vy64, my2)) ||
      (rc = dalloc(c, &c->Wy64, my2)) || (rc = dalloc(c, &c->Vx32, mx2)) || (rc = dalloc(c, &c->Wx32, mx2)) ||
      (rc = dalloc(c, &c->Vy32, my2)) || (rc = dalloc(c, &c->Wy32, my2)) ||
      (rc = dalloc(c, &c->lamx, (size_t)c->g.mx)) || (rc = dalloc(c, &c->lamy, (size_t)c->g.my)))
    return fail(rc);
  auto up64 = [&](double* d, const std::vector<double>& h_) {
    return cudaMemcpy(d, h_.data(), h_.size() * sizeof(double), cudaMemcpyHostToDevice);
  };
  auto up32 = [&](float* d, const std::vector<double>& h_) {
    std::vector<float> f(h_.begin(), h_.end());
    return cudaMemcpy(d, f.data(), f.size() * sizeof(float), cudaMemcpyHostToDevice);
  };
  if (up64(c->Vx64, Vx) || up64(c->Wx64, Wx) || up64(c->Vy64, Vy) || up64(c->Wy64, Wy) || up64(c->lamx, lx) ||
      up64(c->lamy, ly) || up32(c->Vx32, Vx) || up32(c->Wx32, Wx) || up32(c->Vy32, Vy) || up32(c->Wy32, Wy))
    return fail(HELM6_ERR_CUDA);
  // transforms: dense on tensor cores (MIXED, both axes fit, not FFT-forced), else the FFT
  // form where the axis length has one (unless dense is asked for), else dense
  const bool use_tc = o.precision == HELM6_MIXED && o.transform != HELM6_XFORM_FFT && c->g.mx <= tc_max_axis() &&
                      c->g.my <= tc_max_axis();
  for (int a = 0; a < 2; ++a) {
    c->xform[a] = use_tc ? HELM6_XFORM_TENSOR : HELM6_XFORM_DENSE;
    FftHostPlan fp;
    // FP64: the half-length sine/cosine form (the FP64 pipe bounds the kernel); FP32: the
    // extension form, whose rounding costs the mixed solve fewer iterations
    if (use_tc || o.transform == HELM6_XFORM_DENSE ||
        !fft_make_plan(n, c->g.face[2 * a], c->g.face[2 * a + 1], o.precision == HELM6_FP64, fp))
      continue;
    double2* t64 = nullptr;
    float2* t32 = nullptr;
    int* gi = nullptr;
    const size_t nt = fp.tw.size() / 2;
    if ((rc = dalloc(c, &t64, nt)) || (rc = dalloc(c, &t32, nt)) || (rc = dalloc(c, &gi, std::max<size_t>(1, fp.gidx.size()))))
      return fail(rc);
    std::vector<float> f32(fp.tw.begin(), fp.tw.end());
    if (cudaMemcpy(t64, fp.tw.data(), fp.tw.size() * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(t32, f32.data(), f32.size() * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess ||
        (!fp.gidx.empty() &&
         cudaMemcpy(gi, fp.gidx.data(), fp.gidx.size() * sizeof(int), cudaMemcpyHostToDevice) != cudaSuccess))
      return fail(HELM6_ERR_CUDA);
    fp.d.tw64 = t64;
    fp.d.tw32 = t32;
    fp.d.gidx = gi;
    c->fft[a] = fp.d;
    c->xform[a] = HELM6_XFORM_FFT;
    fft_configure();
  }

  // workspace
  const int64_t N = c->g.N;
  const size_t v = (size_t)(2 * N);
  const int m = c->mrest;
  if ((rc = dalloc(c, &c->F64, v)) || (rc = dalloc(c, &c->U64, v)) || (rc = dalloc(c, &c->R64, v)) ||
      (rc = dalloc(c, &c->E64, v)))
    return fail(rc);
  if (o.precision == HELM6_FP64) {
    const bool needZ = o.method == HELM6_FGMRES;
    const bool krylov = o.method == HELM6_GMRES || o.method == HELM6_FGMRES;
    if (krylov && (rc = dalloc(c, &c->V64, v * (m + 1)))) return fail(rc);
    if (needZ && (rc = dalloc(c, &c->Z64, v * m))) return fail(rc);
    if (krylov && (rc = dalloc(c, &c->u64, v))) return fail(rc);
    if ((rc = dalloc(c, &c->w64, v)) || (rc = dalloc(c, &c->zt64, v)) || (rc = dalloc(c, &c->tA64, v)) ||
        (rc = dalloc(c, &c->tB64, v)) || (rc = dalloc(c, &c->cw64, v)))
      return fail(rc);
  } else {
    const bool krylov = o.method == HELM6_GMRES || o.method == HELM6_FGMRES;
    // AUTO: FP16 from 2^23 unknowns, where the Gram-Schmidt passes are the bulk of a step;
    // below, an easy problem's inner cycles converge deep enough that the rounded basis can
    // cost an extra refinement step, more than the halved basis traffic saves
    if (o.basis == HELM6_BASIS_AUTO) o.basis = (krylov && N >= (int64_t(1) << 23)) ? HELM6_BASIS_F16 : HELM6_BASIS_F32;
    c->opts.basis = o.basis;
    const bool f16 = o.basis == HELM6_BASIS_F16;
    if (krylov && ((rc = f16 ? dalloc(c, &c->V16, v * (m + 1)) : dalloc(c, &c->V32, v * (m + 1))) ||
                   (rc = dalloc(c, &c->Z32, v * m)) || (rc = dalloc(c, &c->u32, v))))
      return fail(rc);
    // 2^e near sqrt(N)/4: a unit vector's entries stay below 2^e <= sqrt(N)/2 (far inside the
    // FP16 range up to N = 2^32) while its mean square is 2^(2e)/N, about 1/16
    c->vscale = std::ldexp(1.0, std::max(0, std::min(14, (int)std::floor(0.5 * std::log2((double)N)) - 2)));
    // the tensor-core path's intermediates have rows padded to a multiple of 4 floats
    const size_t vpad = std::max(v, (size_t)2 * c->g.mz *
                                        std::max((size_t)c->g.mx * pad4(c->g.my), (size_t)c->g.my * pad4(c->g.mx)));
    if ((rc = dalloc(c, &c->w32, v)) || (rc = dalloc(c, &c->zt32, v)) || (rc = dalloc(c, &c->tA32, vpad)) ||
        (rc = dalloc(c, &c->tB32, vpad)) || (rc = dalloc(c, &c->cw32, v)))
      return fail(rc);
    // FP64 scratch used by apply_Pinv in FP64 layout conversions
    if ((rc = dalloc(c, &c->tA64, v))) return fail(rc);
  }
  if (o.method == HELM6_CHEB) {
    if ((rc = dalloc(c, &c->D64, v))) return fail(rc);
    if (o.cheb_lo != 0.0 || o.cheb_hi != 0.0) {
      c->cheb_lo = o.cheb_lo;
      c->cheb_hi = o.cheb_hi;
    } else {
      dirichlet_ratio_bounds(c, &c->cheb_lo, &c->cheb_hi);
      if (!(c->cheb_lo > 0.0 && c->cheb_hi > c->cheb_lo)) return fail(HELM6_ERR_UNSUPPORTED);  // indefinite
    }
  }
  c->nred = std::max(1, device_sm_count() * 4);
  c->nsten = stencil_blocks(c->g);
  c->ncgs = (o.precision == HELM6_FP64) ? cgs_blocks<double>(N) : cgs_blocks<float>(N);
  c->ndot = dot_blocks();
  if (o.dot_blocks > 0) c->ndot = o.dot_blocks;
  if (o.update_blocks > 0) c->ncgs = o.update_blocks;
  const int npart = std::max(c->nred, std::max(c->ncgs, c->ndot));
  const size_t ncol = (size_t)4 * (m + 1) + 3;
  if ((rc = dalloc(c, &c->partial, (size_t)npart * ncol)) || (rc = dalloc(c, &c->red, ncol)) ||
      (rc = dalloc(c, &c->coefv, ncol)) || (rc = dalloc(c, &c->Hr, (size_t)2 * (m + 1) * m)) ||
      (rc = dalloc(c, &c->Tm, (size_t)2 * m * m)) || (rc = dalloc(c, &c->qv, (size_t)2 * (m + 1))) ||
      (rc = dalloc(c, &c->brk, 1)) || (rc = dalloc(c, &c->spart, (size_t)c->nsten)) ||
      (rc = dalloc(c, &c->H, (size_t)2 * (m + 1) * m)) || (rc = dalloc(c, &c->cs, (size_t)2 * (m + 1))) ||
      (rc = dalloc(c, &c->sn, (size_t)2 * (m + 1))) || (rc = dalloc(c, &c->gv, (size_t)2 * (m + 1))) ||
      (rc = dalloc(c, &c->yv, (size_t)2 * (m + 1))) || (rc = dalloc(c, &c->h2, (size_t)2 * (m + 1))) ||
      (rc = dalloc(c, &c->scal, 8)) || (rc = dalloc(c, &c->status, 1)))
    return fail(rc);
  if ((rc = dalloc(c, &c->tcerr, 1))) return fail(rc);
  if (cudaMemset(c->tcerr, 0, sizeof(int)) != cudaSuccess) return fail(HELM6_ERR_CUDA);
  if (use_tc) {
    if (tc_configure() != HELM6_OK) return fail(HELM6_ERR_CUDA);
    std::vector<uint8_t> t;
    auto upt = [&](uint8_t** d, const std::vector<double>& B, int m) -> int {
      tc_prepare_basis(B, m, m, t);
      int r2 = dalloc(c, d, t.size());
      if (r2) return r2;
      return cudaMemcpy(*d, t.data(), t.size(), cudaMemcpyHostToDevice) == cudaSuccess ? (int)HELM6_OK
                                                                                      : (int)HELM6_ERR_CUDA;
    };
    if ((rc = upt(&c->Wx_tc, Wx, c->g.mx)) || (rc = upt(&c->Vx_tc, Vx, c->g.mx)) ||
        (rc = upt(&c->Wy_tc, Wy, c->g.my)) || (rc = upt(&c->Vy_tc, Vy, c->g.my)))
      return fail(rc);
    c->zl.ldq = pad4(c->g.my);
    if ((rc = dalloc(c, &c->zl.rinv, (size_t)2 * c->g.mz * c->g.mx * c->zl.ldq))) return fail(rc);
    if (cudaMemset(c->status, 0, sizeof(int)) != cudaSuccess) return fail(HELM6_ERR_CUDA);
    launch_ztri_table(c->g, c->lamx, c->lamy, c->diag0, c->alpha, c->zl, c->status, 0);
    if (cudaDeviceSynchronize() != cudaSuccess) return fail(HELM6_ERR_CUDA);
    int zst = 0;
    if (cudaMemcpy(&zst, c->status, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return fail(HELM6_ERR_CUDA);
    c->zline_breakdown = zst != 0;
  }
  if (cudaMallocHost((void**)&c->pinned, 16 * sizeof(double)) != cudaSuccess) return fail(HELM6_ERR_NOMEM);
  for (int i = 0; i < 2; ++i)
    if (cudaEventCreateWithFlags(&c->step_ev[i], cudaEventDisableTiming) != cudaSuccess) return fail(HELM6_ERR_CUDA);
  if (cudaMemset(c->status, 0, sizeof(int)) != cudaSuccess) return fail(HELM6_ERR_CUDA);
  if (cudaDeviceSynchronize() != cudaSuccess) return fail(HELM6_ERR_CUDA);
  *out = c;
  return HELM6_OK;
}

int helm6_dims(const helm6_ctx* c, int64_t dims[3]) {
  if (!c || !dims) return HELM6_ERR_INVALID;
  dims[0] = c->gu.mx;
  dims[1] = c->gu.my;
  dims[2] = c->gu.mz;
  return HELM6_OK;
}

int helm6_transform(const helm6_ctx* c, int axis) {
  if (!c || axis < 0 || axis > 1) return HELM6_ERR_INVALID;
  return c->xform[axis];
}

int helm6_basis(const helm6_ctx* c) {
  if (!c) return HELM6_ERR_INVALID;
  if (c->opts.precision != HELM6_MIXED || !(c->V16 || c->V32)) return HELM6_BASIS_AUTO;
  return c->V16 ? HELM6_BASIS_F16 : HELM6_BASIS_F32;
}

int helm6_apply_A(helm6_ctx* c, const void* x, void* y) {
  if (!c || !x || !y) return HELM6_ERR_INVALID;
  cudaStream_t s = c->stream;
  const int64_t N = c->g.N;
  launch_caller_to_planar(c->g, c->xaxis, (const double*)x, c->R64, s);
  if (c->opts.precision == HELM6_FP64) {
    cudaEvent_t e = prof_start(c);
    launch_stencil<double>(c->g, c->coef, c->R64, c->E64, nullptr, nullptr, 0, nullptr, nullptr, s);
    prof_stop(c, HELM6_PH_STENCIL, e);
  } else {
    launch_convert<double, float>(c->R64, c->w32, N, 1.0, s);
    cudaEvent_t e = prof_start(c);
    launch_stencil<float>(c->g, c->coef, c->w32, c->zt32, nullptr, nullptr, 0, nullptr, nullptr, s);
    prof_stop(c, HELM6_PH_STENCIL, e);
    launch_convert<float, double>(c->zt32, c->E64, N, 1.0, s);
  }
  launch_planar_to_caller(c->g, c->xaxis, c->E64, (double*)y, s);
  CK(cudaGetLastError());
  return HELM6_OK;
}

int helm6_apply_Pinv(helm6_ctx* c, const void* x, void* y) {
  if (!c || !x || !y) return HELM6_ERR_INVALID;
  cudaStream_t s = c->stream;
  const int64_t N = c->g.N;
  CK(cudaMemsetAsync(c->status, 0, sizeof(int), s));
  CK(cudaMemsetAsync(c->tcerr, 0, sizeof(int), s));
  launch_caller_to_planar(c->g, c->xaxis, (const double*)x, c->R64, s);
  if (c->opts.precision == HELM6_FP64) {
    precond64(c, c->R64, c->E64);
  } else {
    launch_convert<double, float>(c->R64, c->w32, N, 1.0, s);
    precond32(c, c->w32, c->zt32);
    launch_convert<float, double>(c->zt32, c->E64, N, 1.0, s);
  }
  launch_planar_to_caller(c->g, c->xaxis, c->E64, (double*)y, s);
  CK(cudaGetLastError());
  const int st = check_status(c);
  return (st == HELM6_BREAKDOWN || st < 0) ? st : HELM6_OK;
}

int helm6_set_cnn(helm6_ctx* c, const float* theta, double out_scale, int mode) {
  if (!c) return HELM6_ERR_INVALID;
  if (mode == HELM6_CNN_OFF) {
    c->cnn_mode = HELM6_CNN_OFF;
    return HELM6_OK;
  }
  if (mode != HELM6_CNN_ON && mode != HELM6_CNN_AUTO) return HELM6_ERR_INVALID;
  if (!theta || !std::isfinite(out_scale)) return HELM6_ERR_INVALID;
  if (c->opts.precision != HELM6_MIXED || c->opts.method != HELM6_FGMRES) return HELM6_ERR_UNSUPPORTED;
  cudaStream_t s = c->stream;
  if (s) CK(cudaStreamSynchronize(s)); else CK(cudaDeviceSynchronize());
  if (!c->cnn.theta) {
    if (cnn_alloc(c->cnn) != HELM6_OK) {
      cnn_free(c->cnn);
      return HELM6_ERR_NOMEM;
    }
    const size_t N = (size_t)c->g.N;
    int rc;
    if ((rc = dalloc(c, &c->cnn_t, 2 * N)) || (rc = dalloc(c, &c->cnn_a0, 16 * N)) ||
        (rc = dalloc(c, &c->cnn_a1, 16 * N)) || (rc = dalloc(c, &c->cnn_ss, 1)))
      return rc;
  }
  if (cnn_configure() != HELM6_OK) return HELM6_ERR_CUDA;
  CK(cudaMemcpy(c->cnn.theta, theta, sizeof(float) * HELM6_CNN_NPARAMS, cudaMemcpyHostToDevice));
  cnn_prepare(c->cnn, s);
  if (s) CK(cudaStreamSynchronize(s)); else CK(cudaDeviceSynchronize());
  c->cnn_scale = (float)out_scale;
  c->cnn_mode = mode;
  return HELM6_OK;
}

int helm6_apply_stage2(helm6_ctx* c, const void* x, void* y) {
  if (!c || !x || !y) return HELM6_ERR_INVALID;
  if (c->cnn_mode == HELM6_CNN_OFF || !c->cnn.theta) return HELM6_ERR_UNSUPPORTED;
  cudaStream_t s = c->stream;
  const int64_t N = c->g.N;
  CK(cudaMemsetAsync(c->status, 0, sizeof(int), s));
  CK(cudaMemsetAsync(c->tcerr, 0, sizeof(int), s));
  launch_caller_to_planar(c->g, c->xaxis, (const double*)x, c->R64, s);
  launch_convert<double, float>(c->R64, c->w32, N, 1.0, s);
  precond_cnn32(c, c->w32, c->zt32);
  launch_convert<float, double>(c->zt32, c->E64, N, 1.0, s);
  launch_planar_to_caller(c->g, c->xaxis, c->E64, (double*)y, s);
  CK(cudaGetLastError());
  const int st = check_status(c);
  return (st == HELM6_BREAKDOWN || st < 0) ? st : HELM6_OK;
}

int helm6_solve(helm6_ctx* c, const void* F, void* u, double tol, int restart, int maxit, helm6_stats* st) {
  if (!c || !F || !u || !(tol > 0) || maxit < 0) return HELM6_ERR_INVALID;
  const bool krylov = c->opts.method == HELM6_GMRES || c->opts.method == HELM6_FGMRES;
  if (krylov && (restart < 1 || restart > c->mrest)) return HELM6_ERR_INVALID;
  const auto t0 = std::chrono::steady_clock::now();
  helm6_stats local;
  helm6_stats* S = st ? st : &local;
  std::memset(S, 0, sizeof(*S));
  cudaStream_t s = c->stream;
  const int64_t N = c->g.N;
  CK(cudaMemsetAsync(c->status, 0, sizeof(int), s));
  CK(cudaMemsetAsync(c->tcerr, 0, sizeof(int), s));
  launch_caller_to_planar(c->g, c->xaxis, (const double*)F, c->F64, s);
  double normF = 0;
  int rc = norm2<double>(c, c->F64, &normF);
  if (rc) return rc;
  int status;
  if (!std::isfinite(normF)) {
    status = HELM6_NONFINITE;
  } else if (normF == 0.0) {
    CK(cudaMemsetAsync(u, 0, sizeof(double) * 2 * N, s));
    CK(cudaStreamSynchronize(s));
    status = HELM6_OK;
  } else {
    launch_caller_to_planar(c->g, c->xaxis, (const double*)u, c->U64, s);
    if (c->opts.method == HELM6_SKS)
      status = solve_sks(c, normF, tol, maxit, S);
    else if (c->opts.method == HELM6_CHEB)
      status = solve_cheb(c, normF, tol, maxit, S);
    else if (c->opts.precision == HELM6_FP64)
      status = solve_fp64(c, normF, tol, restart, maxit, S);
    else if (graph_solve_ok(c))
      status = solve_mixed_graph(c, normF, tol, restart, maxit, S);
    else
      status = solve_mixed(c, normF, tol, restart, maxit, S);
    if (status < 0) return status;
    launch_planar_to_caller(c->g, c->xaxis, c->U64, (double*)u, s);
    S->relres = c->last_beta / normF;
  }
  CK(cudaStreamSynchronize(s));
  S->status = status;
  S->t_total_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  return status;
}

int helm6_solve_batch(helm6_ctx* const* ctxs, int count, const void* const* F, void* const* u, double tol,
                      int restart, int maxit, int nthreads, helm6_stats* stats) {
  if (count < 0 || (count > 0 && (!ctxs || !F || !u)) || nthreads < 1 || nthreads > 256) return HELM6_ERR_INVALID;
  for (int i = 0; i < count; ++i)
    if (!ctxs[i] || !F[i] || !u[i]) return HELM6_ERR_INVALID;
  int dev = 0;
  CK(cudaGetDevice(&dev));
  std::vector<int> rc(count, HELM6_OK);
  bool all_graph = count > 0;
  for (int i = 0; i < count; ++i)
    all_graph = all_graph && graph_solve_ok(ctxs[i]) && restart >= 1 && restart <= ctxs[i]->mrest;
  if (all_graph && tol > 0 && maxit >= 0) return solve_batch_graph(ctxs, count, F, u, tol, restart, maxit, stats);
  std::atomic<int> next{0};
  auto worker = [&]() {
    if (cudaSetDevice(dev) != cudaSuccess) return;
    for (int i = next.fetch_add(1); i < count; i = next.fetch_add(1))
      rc[i] = helm6_solve(ctxs[i], F[i], u[i], tol, restart, maxit, stats ? &stats[i] : nullptr);
  };
  const int nt = std::min(nthreads, std::max(count, 1));
  std::vector<std::thread> pool;
  for (int t = 1; t < nt; ++t) pool.emplace_back(worker);
  worker();
  for (auto& t : pool) t.join();
  if (next.load() < count) return HELM6_ERR_CUDA;  // no worker could select the device
  int worst = HELM6_OK;
  for (int i = 0; i < count; ++i) {
    if (rc[i] < 0) return rc[i];
    worst = std::max(worst, rc[i]);
  }
  return worst;
}

int helm6_profile_enable(helm6_ctx* c, int enable) {
  if (!c) return HELM6_ERR_INVALID;
  if (c->stream) cudaStreamSynchronize(c->stream); else cudaDeviceSynchronize();
  prof_flush(c);
  if (c->ev_all.empty()) {
    for (int i = 0; i < 512; ++i) {
      cudaEvent_t e;
      CK(cudaEventCreate(&e));
      c->ev_all.push_back(e);
      c->ev_pool.push_back(e);
    }
  }
  c->prof_on = enable != 0;
  for (int i = 0; i < HELM6_NPHASE; ++i) {
    c->prof_count[i] = 0;
    c->prof_ms[i] = 0.0;
    c->prof_bytes[i] = 0.0;
  }
  c->prof_l0 = launch_total();
  return HELM6_OK;
}

int helm6_profile_read(helm6_ctx* c, helm6_profile* out) {
  if (!c || !out) return HELM6_ERR_INVALID;
  CK(cudaStreamSynchronize(c->stream));
  prof_flush(c);
  out->launches = launch_total() - c->prof_l0;
  for (int i = 0; i < HELM6_NPHASE; ++i) {
    out->count[i] = c->prof_count[i];
    out->ms[i] = c->prof_ms[i];
    out->bytes[i] = c->prof_bytes[i];
  }
  return HELM6_OK;
}

int helm6_rhs_gaussians(helm6_ctx* c, int nsrc, const double* centers, const helm6_c64* amps, double sigma,
                        const void* noise, void* F) {
  if (!c || !F || nsrc < 0 || nsrc > 4096 || !(sigma > 0)) return HELM6_ERR_INVALID;
  if (nsrc > 0 && (!centers || !amps)) return HELM6_ERR_INVALID;
  return rhs_gaussians(c->gu, c->h, c->k, nsrc, centers, (const double*)amps, sigma, (const double*)noise,
                       (double*)F, c->stream);
}

int helm6_rhs_separable(helm6_ctx* c, int nterms, const helm6_c64* coef, const helm6_c64* tables, void* F) {
  if (!c || !F || nterms < 0 || nterms > 4096) return HELM6_ERR_INVALID;
  if (nterms > 0 && (!coef || !tables)) return HELM6_ERR_INVALID;
  return rhs_separable(c->gu, c->h, c->k, nterms, (const double*)coef, (const double*)tables, (double*)F, c->stream);
}

int helm6_lift_dirichlet(helm6_ctx* c, int face, const void* data, void* F) {
  if (!c || !data || !F) return HELM6_ERR_INVALID;
  if (face < 0 || face > 5) return HELM6_ERR_INVALID;
  if (c->xaxis >= 0) return HELM6_ERR_UNSUPPORTED;
  if (c->gu.face[face] != HELM6_DIRICHLET) return HELM6_ERR_INVALID;
  return lift_dirichlet(c->gu, c->coef, face, (const double*)data, (double*)F, c->stream);
}

}  // extern "C"

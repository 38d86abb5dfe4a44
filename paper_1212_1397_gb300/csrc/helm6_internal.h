// Internal declarations of the helm6 library (not part of the C-ABI).
//
// Vectors inside the library are "planar": a complex field of N = mx*my*mz points is a
// real array of 2N elements, the real plane [0, N) then the imaginary plane [N, 2N), each
// indexed (l*my + j)*mx + i with x fastest.  FP64 vectors are double, MIXED-precision
// Krylov vectors are float.
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <complex>
#include <vector>

#include "../../include/helm6.h"

namespace helm6 {

using cd = std::complex<double>;

// ---------------------------------------------------------------------------------------
// Small complex type usable in device code.
// ---------------------------------------------------------------------------------------
// Fused multiply-add in the operands' own precision (fmaf for float, fma for double).
__host__ __device__ __forceinline__ float fmx(float a, float b, float c) { return fmaf(a, b, c); }
__host__ __device__ __forceinline__ double fmx(double a, double b, double c) { return fma(a, b, c); }

template <typename T>
struct cpx {
  T re, im;
};

template <typename T>
__host__ __device__ __forceinline__ cpx<T> mk(T r, T i) { return cpx<T>{r, i}; }
template <typename T>
__host__ __device__ __forceinline__ cpx<T> operator+(cpx<T> a, cpx<T> b) { return {a.re + b.re, a.im + b.im}; }
template <typename T>
__host__ __device__ __forceinline__ cpx<T> operator-(cpx<T> a, cpx<T> b) { return {a.re - b.re, a.im - b.im}; }
template <typename T>
__host__ __device__ __forceinline__ cpx<T> operator*(cpx<T> a, cpx<T> b) {
  return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}
template <typename T>
__host__ __device__ __forceinline__ cpx<T> operator*(T s, cpx<T> a) { return {s * a.re, s * a.im}; }
// a + w * s  (complex fused multiply-add)
template <typename T>
__host__ __device__ __forceinline__ cpx<T> cfma(cpx<T> w, cpx<T> s, cpx<T> a) {
  a.re = fmx(w.re, s.re, a.re);
  a.re = fmx(-w.im, s.im, a.re);
  a.im = fmx(w.re, s.im, a.im);
  a.im = fmx(w.im, s.re, a.im);
  return a;
}

struct c64d {  // plain-old-data complex double for kernel parameters
  double re, im;
};
inline c64d to_pod(cd z) { return c64d{z.real(), z.imag()}; }
template <typename T>
__host__ __device__ __forceinline__ cpx<T> cast(c64d z) { return cpx<T>{(T)z.re, (T)z.im}; }

// ---------------------------------------------------------------------------------------
// Geometry and the scheme's coefficients.
// ---------------------------------------------------------------------------------------
struct Geom {
  int mx, my, mz;       // unknowns per axis
  int64_t N;            // mx*my*mz
  int face[6];          // helm6_bc per face x0 x1 y0 y1 z0 z1
};

// Weights of one row type of the 27-point operator, per z-plane offset dz = -1, 0, +1:
// w[dz+1][0] centre of that plane, [1] its 4 in-plane neighbours, [2] its 4 diagonals.
struct RowWeights {
  c64d w[3][3];
};

struct StencilCoef {
  RowWeights interior;  // Eq. scheme
  RowWeights s_lo;      // z = 0 Sommerfeld-like face row (Eq. 3DDISCS)
  RowWeights s_hi;      // z = top face row, mirrored
};

// Class weights of the interior rows and the Sommerfeld-like face rows for wavenumber k
// and grid step h (host, FP64).
void stencil_coefficients(cd k, double h, StencilCoef& c);

// ---------------------------------------------------------------------------------------
// Kernel launchers (stream-ordered).  Defined in the .cu files.
// ---------------------------------------------------------------------------------------

// y = A x (mode 0);  y = f - A x (mode 1);  y = f + A x (mode 2, no norm), A given by its row
// weights.
// sumsq (nullable): per-block partial sums of |y|^2, nblk entries written, reduced by
// reduce_sum.
template <typename T>
void launch_stencil(const Geom& g, const StencilCoef& c, const T* x, T* y, const T* f, T* r,
                    int mode, double* sumsq, int* nblk, cudaStream_t s);

// Number of blocks (and fused-norm partials) of launch_stencil for this geometry.
int stencil_blocks(const Geom& g);

// Batched strided real GEMM on planar data, C = A * B per batch:
//  along_x = true : B(k, n) = B[b*bstride + n*ld + k], C(p, n) = C[b*bstride + n*ld + p]
//  along_x = false: B(k, n) = B[b*bstride + k*ld + n], C(p, n) = C[b*bstride + p*ld + n]
// A is P x K row-major (P = K = the axis length m).
template <typename T>
void launch_axis_gemm(const T* A, const T* B, T* C, int m, int ncols, int ld, int64_t bstride,
                      int nbatch, bool along_x, cudaStream_t s);

// Tensor-core (tcgen05) BF16-split transform along the contiguous axis of each row:
// out(row, p) = sum_k in(row, k) B(p, k), rows of length K, M_total rows, P <= tc_max_axis().
// W: tc_prepare_basis(B).  transposed = 0: out[row*P + p]; 1: out[(row/R)*R*P + p*R + row%R].
// terms: 1 (hi*hi), 2 (+ lo*hi), 3 (+ hi*lo).  *err is set if a bounded wait timed out.
// Persistent: one CTA per SM (all of its shared memory and tensor memory).
int tc_npad(int P);
int tc_nk(int K);
int tc_max_axis();
int tc_configure();
void tc_prepare_basis(const std::vector<double>& B, int P, int K, std::vector<uint8_t>& out);
// ldin: input row pitch (0: K); ldo: output row pitch (row-major, 0: P) or pitch of the
// transposed rows of a plane (0: R): out[(row/R)*ldo*P + p*ldo + row%R].
void launch_xform_tc(const float* in, float* out, const uint8_t* W, int M_total, int K, int P, int terms,
                     int transposed, int R, int* err, cudaStream_t s, int ldin = 0, int ldo = 0);

// Tridiagonal solve along z for every (x, y) mode pair, Thomas algorithm started at the
// Sommerfeld-like end (if any).  x: input, y: output (may alias x), cw: scratch of 2N T.
// xmajor: planes stored x-mode-major (p*my + q) rather than y-major (q*mx + p).
template <typename T>
void launch_ztri(const Geom& g, const double* lamx, const double* lamy, c64d diag0, c64d alpha,
                 const T* x, T* y, T* cw, int* status, cudaStream_t s, int xmajor = 0);

// The same z-line solve with the elimination's pivots precomputed in FP64 (once per
// context) and stored in FP32 (tensor-core path): rinv holds the pivot reciprocal of every
// step of every line, planar (re then im), indexed like the field; the planes are
// x-mode-major with q pitch ldq >= my (the padded layout of the transforms' intermediates).
struct ZLines {
  float* rinv = nullptr;
  int ldq = 0;
};
void launch_ztri_table(const Geom& g, const double* lamx, const double* lamy, c64d diag0, c64d alpha, ZLines z,
                       int* status, cudaStream_t s);
// y = the z-line solve of x (planar FP32 in that layout; y may not alias x).
void launch_ztri_apply(const Geom& g, const ZLines& z, const float* x, float* y, cudaStream_t s);

// FFT-type x/y transforms (fft.cu): the closed-form 1D eigenbasis of one axis applied through
// one complex DFT of length L = P * Q per line: of the line's odd or even extension, L = 2(n+1)
// (sine, cosine) or 4(n+1) (quarter-wave), or, in the half-length form of the sine and cosine
// axes, L = n + 1 with pre- and post-processing.
struct FftDev {
  int kind;        // 0 D-D (sine), 1 N-N (cosine), 2 D-N, 3 N-D (quarter-wave)
  int half;        // half-length form (kinds 0, 1)
  int N;           // intervals n + 1
  int m;           // unknowns on the axis
  int L, P, Q, M;  // L = P Q, P a power of two, Q = 1 or a prime with M = Q - 1 a power of two
  int logP, logM;
  const double2* tw64;  // [w_P^k: P/2][w_M^k: M/2][kernel spectrum / M: M][w_L^t: L if Q > 1]
                        // [(cos, sin)(pi j / N), j = 0..N: sine and cosine axes]
  const float2* tw32;   // the same in FP32
  const int* gidx;      // [g^q mod Q: M][g^-q mod Q: M]
};
struct FftHostPlan {
  FftDev d;                // sizes; device pointers null
  std::vector<double> tw;  // the complex tables, interleaved
  std::vector<int> gidx;
};
// Plan for n interior nodes and the axis' faces lo, hi (helm6_bc), in the half-length form
// where `half` asks for it and the faces allow it; false when L has no
// factorisation of the form above or a line does not fit in shared memory.
bool fft_make_plan(int n, int lo, int hi, bool half, FftHostPlan& plan);
void fft_configure();  // once per process: the kernels' dynamic shared memory limit
// out = W in (inv = 0, forward) or V in (inv = 1) along axis 0 (x) or 1 (y) of the planar
// field (same layout in and out; out may not alias in).
template <typename T>
void launch_fft_axis(const FftDev& f, int axis, int inv, const Geom& g, const T* in, T* out, cudaStream_t s);

// BLAS-1 style kernels on planar complex vectors of N points.
void launch_reduce_cols(const double* partial, int nblocks, int ncols, double* out, int accumulate,
                        cudaStream_t s);  // out[i] (+)= sum_b partial[b][i], complex double
template <typename T>
void launch_sumsq(const T* x, int64_t N, double* partial, int nblocks, cudaStream_t s);
template <typename T>
void launch_scale_copy(const T* x, T* y, int64_t N, const double* inv_scale_dev, double host_scale,
                       cudaStream_t s);  // y = x * (host_scale or 1/(*dev))
// out (+)= scale*sum V_i y_i; count_dev / scale_dev (nullable): read count / scale on the
// device instead (device-driven solves)
template <typename TI, typename TO>
void launch_lincomb(const TI* V, int64_t vstride, int count, const double* y, double scale, TO* out,
                    int64_t N, int accumulate, cudaStream_t s, const int* count_dev = nullptr,
                    const double* scale_dev = nullptr);
template <typename TI, typename TO>
void launch_convert(const TI* x, TO* y, int64_t N, double scale, cudaStream_t s,
                    const double* scale_dev = nullptr);  // planar, y = scale x
void launch_interleaved_to_planar(const double* zin, double* out, int64_t N, cudaStream_t s);
void launch_planar_to_interleaved(const double* in, double* zout, int64_t N, cudaStream_t s);
// The same between the caller's interleaved array and the internal planar layout of
// geometry g when the caller's axis xaxis (0 = x, 1 = y) is the internal z axis (Sommerfeld-
// like faces on that axis); xaxis < 0: no exchange.
void launch_caller_to_planar(const Geom& g, int xaxis, const double* zin, double* out, cudaStream_t s);
void launch_planar_to_caller(const Geom& g, int xaxis, const double* in, double* zout, cudaStream_t s);
void launch_reduce_sum(const double* partial, int n, double* out, cudaStream_t s);  // one double

// Givens update of Hessenberg column j on the device (single thread, FP64):
// applies the j previous rotations to H[:, j], makes rotation j, updates g; writes
// |g_{j+1}| to *res.  H column-major with leading dimension ldh, complex double.
void launch_givens(double* H, int ldh, int j, double* cs, double* sn, double* g, double* res,
                   cudaStream_t s);
// H[j+1, j] = sqrt(*sumsq); inv = 1/that (0 if zero).
void launch_set_subdiag(double* H, int ldh, int j, const double* sumsq, double* inv, cudaStream_t s);
// Solve the j x j upper triangular system R y = g (complex double) on the device.
void launch_backsolve(const double* H, int ldh, int j, const double* g, double* y, cudaStream_t s,
                      const int* j_dev = nullptr);

// Compact right side for Gaussian sources (FP64, complex128 interleaved output F).
// centers: host nsrc*3, amps: host nsrc*2 (re, im); noise: device complex128 or nullptr.
int rhs_gaussians(const Geom& g, double h, cd k, int nsrc, const double* centers, const double* amps,
                  double sigma, const double* noise, double* F, cudaStream_t s);
// Compact right side for f = sum_t coef_t X_t Y_t Z_t from complex host tables
// [nterm][3][5][max(mx, my, mz)] of the factors' derivatives 0..4 at the unknown nodes.
int rhs_separable(const Geom& g, double h, cd k, int nterm, const double* coef, const double* tables, double* F,
                  cudaStream_t s);

// F -= the contribution of known Dirichlet values ub on face `face` (0..5 = x0 x1 y0 y1 z0 z1)
// to the rows next to it; ub complex128, the face's node layer x fastest with a ring in the
// tangential axes padded before the face's own (x faces [mz][my], y faces [mz][mx + 2], z faces
// [my + 2][mx + 2]); F complex128 interleaved in geometry g.
int lift_dirichlet(const Geom& g, const StencilCoef& coef, int face, const double* ub, double* F, cudaStream_t s);

// y += alpha x (planar, 2N reals), mixed input/output precision.
template <typename TI, typename TO>
void launch_axpy(const TI* x, TO* y, int64_t N, double alpha, cudaStream_t s);
// y = a y + b x (planar FP64, 2N reals).
void launch_axpby(const double* x, double* y, int64_t N, double a, double b, cudaStream_t s);
// p[0] = re, p[1] = im on the device (stream-ordered).
void launch_set_complex(double* p, double re, double im, cudaStream_t s);

// Arnoldi by delayed classical Gram-Schmidt (one reduction and one update pass per step):
//   launch_dcgs_dot:    block partials of V_i^H u, V_i^H w (i < count), ||u||^2, u^H w
//                       (w may be null: the last step of a cycle has no new vector)
//   launch_dcgs_step:   FP64 small algebra of step j (see krylov.cu)
//   launch_dcgs_update: v_out = (u - V s)/alpha,  u = (w - V t - v_out c)/alpha
//   launch_tri_mul:     q = T y for the flexible solution update
template <typename T>
int cgs_blocks(int64_t N);
int dot_blocks();
// The basis is stored in TV: T, or __half for T = float holding vscale V_i (vscale a power
// of two chosen so that unit vectors stay well inside the FP16 range).
template <typename T, typename TV>
void launch_dcgs_dot(const TV* V, int64_t vs, int count, const T* u, const T* w, int64_t N, double* partial,
                     int nblocks, double vscale, cudaStream_t s);
template <typename T, typename TV>
void launch_dcgs_update(const TV* V, int64_t vs, int count, T* u, const T* w, TV* v_out, int64_t N,
                        const double* coef, int nblocks, double vscale, cudaStream_t s);
void launch_dcgs_step(int j, int has_w, const double* red, double* Hr, double* R, int ldh, double* T, int ldt,
                      double* cs, double* sn, double* g, double* coef, double* est, int* brk, cudaStream_t s);
void launch_tri_mul(const double* T, int ldt, int k, const double* y, double* q, cudaStream_t s,
                    const int* k_dev = nullptr);

// Learned second preconditioner stage (cnn.cu).  theta: HELM6_CNN_NPARAMS master
// parameters; wf / wb: BF16-rounded taps of every layer in the forward layout
// [t][c_in][c_out] and in the input-gradient layout [26 - t][c_out][c_in].
struct CnnNet {
  float* theta = nullptr;
  uint16_t* wtc = nullptr;   // BF16 taps of every layer for the tensor-core layers
  uint16_t* wtcb = nullptr;  // the flipped, channel-transposed taps (input gradients; trainer)
};
int cnn_alloc(CnnNet& net, bool backward = false);
void cnn_free(CnnNet& net);
void cnn_prepare(const CnnNet& net, cudaStream_t s);  // the tensor-core taps from theta
int cnn_configure();  // kernel attributes of the field path (before any capture)
// z += c s N(t / s) on planar complex FP32 fields of nz*ny*nx points, s = sqrt(*sumsq / N)
// (z unchanged when *sumsq is 0); act0/act1: scratch of 16 BF16 per point each.  The four
// layers run on the tensor cores; *err is set if a bounded wait timed out.
int cnn_apply_field(const CnnNet& net, int nz, int ny, int nx, const float* t, const double* sumsq,
                    uint16_t* act0, uint16_t* act1, float out_scale, float* z, int* err, cudaStream_t s);

int device_sm_count();

// Device-driven solve (one CUDA graph per solve, convergence decided on the device through
// conditional nodes): parameters written by the host before the launch, state kept by the
// control kernels and read back after it.
struct GraphCtl {
  double tol_abs;   // tol ||F||
  double itol_num;  // 0.3 tol ||F||: a cycle's inner tolerance is max(inner, itol_num / beta)
  double inner;
  double normF;
  int maxit, m;
  double beta, inv_beta, itol;  // current true residual norm, its inverse, inner tolerance
  int iters, outer, k, status;  // status: -1 running, else a HELM6 return code
  int nhist, pad;
  unsigned long long t0, t1;    // %globaltimer at the start and the end of the solve
  double hist[HELM6_MAX_HIST];
};
void launch_gctl_residual(GraphCtl* g, const double* sumsq, const int* zst, const int* tcerr, int first,
                          cudaGraphConditionalHandle hw, cudaStream_t s);
// One conditional handle per IF node (a handle belongs to exactly one conditional node):
// step j's control kernel enables step j + 1, the cycle's first kernel resets them all.
struct StepHandles {
  cudaGraphConditionalHandle h[65];
};
void launch_gctl_cycle(GraphCtl* g, const StepHandles& ha, int m, cudaStream_t s);
void launch_gctl_step(GraphCtl* g, int j, int m, const double* est, const int* brk, cudaGraphConditionalHandle next,
                      cudaStream_t s);

// Kernels launched by the library so far (process-wide counter, for measurement).
void note_launch(int n = 1);
long long launch_total();

}  // namespace helm6

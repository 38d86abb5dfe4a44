/*
 * helm6 -- sixth-order compact 3D Helmholtz solver on one GB300 (sm_103a).
 *
 * Solves  laplacian(u) + k^2 u = f  on the cube [0, a]^3, h = a/(n+1), with complex k and
 * per-face Dirichlet (u = 0), Neumann (u_n = 0) or Sommerfeld-like (u_n - i k u = 0)
 * conditions (Gryazin, "Preconditioned Krylov subspace methods for sixth order compact
 * approximations of the Helmholtz equation", Eq. problem and Eq. bc).  The discrete system
 * is the 27-point sixth-order compact scheme (Eq. scheme) with the paper's explicit
 * sixth-order Neumann (Eq. 3DN) and Sommerfeld-like (Eq. 3DDISCS) face eliminations; it is
 * solved by right-preconditioned restarted GMRES (Eq. AAP) or the SKS iteration
 * (Algorithm 1), preconditioned by the second-order 7-point operator (Eq. 3DAP) inverted
 * directly: eigen-transforms in x and y, complex tridiagonal solves in z.
 *
 * Grid and unknowns.  Nodes are x_i = i h, i = 0..n+1.  A Dirichlet face's nodes are known
 * (zero) and carry no unknown; a Neumann or Sommerfeld-like face's nodes are unknowns, so
 * an axis has n + (number of its non-Dirichlet faces) unknowns (Section 3.3, N_z chosen so
 * that h is equal in all directions).  Sommerfeld-like faces are accepted on one axis pair
 * (the preconditioner of Section 3.3 diagonalises the other two axes).  The paper writes
 * them on z; a pair on x or y is solved as the z pair of the problem with that axis
 * exchanged with z (the scheme is symmetric under exchanging axes), invisibly to the caller:
 * arrays keep the caller's layout.  Two axes with such faces are not supported.
 *
 * Data at the boundary.  Every vector argument is a DEVICE pointer to complex128
 * (interleaved re, im doubles), x fastest: element (i, j, l) at index (l*my + j)*mx + i
 * with (mx, my, mz) from helm6_dims.  The caller owns these buffers; the library never
 * frees or retains them.  The library owns its workspace (allocated in helm6_create,
 * released in helm6_destroy).  All work is ordered on the stream given in the options
 * (NULL: the legacy default stream); calls return after the work has been enqueued, except
 * helm6_solve, which reads convergence scalars back and returns when the solve is done.
 *
 * Errors.  Functions return HELM6_OK (0) on success, a negative HELM6_ERR_* code on
 * failure (nothing was written), or for helm6_solve a positive warning (u then holds the
 * last iterate and the stats are filled in).  helm6_status_string names every code.
 * A context is not thread-safe: one host thread at a time.
 */
#ifndef HELM6_H
#define HELM6_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct helm6_ctx helm6_ctx;  /* opaque, library-owned */

typedef enum { HELM6_DIRICHLET = 0, HELM6_NEUMANN = 1, HELM6_SOMMERFELD = 2 } helm6_bc;

typedef struct { double re, im; } helm6_c64;

/* precision */
enum { HELM6_FP64 = 0,   /* everything in FP64 complex */
       HELM6_MIXED = 1   /* FP32 complex Krylov bulk, BF16-split tensor-core x/y transforms
                            accumulated in FP32, inside FP64 iterative refinement whose true
                            residual F - A U and Givens least squares stay FP64 */ };

/* method */
enum { HELM6_GMRES = 0,  /* right-preconditioned GMRES(m): U += A_p^{-1}(V y) per cycle */
       HELM6_FGMRES = 1, /* flexible GMRES(m): keeps Z_j = A_p^{-1} v_j, U += Z y */
       HELM6_SKS = 2,    /* Algorithm 1 (no inner products except the residual norm) */
       HELM6_CHEB = 3    /* Chebyshev acceleration (the theorem of Section 2) on the real
                            interval [cheb_lo, cheb_hi] holding the spectrum of A A_p^{-1}:
                            no inner products except the residual norm */ };

/* storage of the Krylov basis V_0..V_m of the MIXED inner solve (its arithmetic stays FP32
   and its reductions FP64) */
enum { HELM6_BASIS_AUTO = 0, /* the default below */
       HELM6_BASIS_F32 = 1,  /* FP32 complex, 8 bytes per unknown and vector */
       HELM6_BASIS_F16 = 2   /* FP16 complex holding 2^e V_i (2^e the power of two near
                                sqrt(N)/4, so unit vectors stay inside the FP16 range), 4 bytes
                                per unknown and vector: the Gram-Schmidt passes read half the
                                bytes; each v_i is rounded once, when written, and later steps
                                orthogonalise against the rounded vectors */ };

/* x/y transforms of the preconditioner (Section 3.3: the direct solver of A_p is FFT-type).
   The FFT form applies an axis' closed-form sine/cosine eigenbasis through one complex DFT
   per line, of length L = n+1 (D-D, N-N faces: the sine and cosine transforms with pre- and
   post-processing) or 4(n+1) (D-N, N-D: the line's odd or even extension); it exists when
   n + 1 = 2^a * Q with Q = 1 or a prime with Q - 1 a power of two (Q <= 257): n + 1 a power
   of two, or 257, 17, 5, 3 times a power of two. */
enum { HELM6_XFORM_AUTO = 0,   /* FP64: FFT on every axis that has one, else dense.  MIXED:
                                  dense on tensor cores while both axes fit them (<= 264
                                  unknowns), else FFT where it exists, else dense FP32 */
       HELM6_XFORM_DENSE = 1,  /* the dense m x m basis matrices (tensor cores where MIXED and
                                  the axes fit them) */
       HELM6_XFORM_FFT = 2,    /* FFT on every axis that has one (MIXED: FP32, no tensor
                                  cores), dense on the others */
       HELM6_XFORM_TENSOR = 3  /* reported by helm6_transform only: dense on tensor cores */ };

/* return codes */
enum {
  HELM6_OK = 0,
  HELM6_NOT_CONVERGED = 1,  /* maxit reached above tol */
  HELM6_DIVERGED = 2,       /* residual grew by more than 1e3 (SKS; Table 4 "div") */
  HELM6_BREAKDOWN = 3,      /* zero pivot in a z-line solve or a GMRES breakdown */
  HELM6_NONFINITE = 4,      /* NaN/Inf in F or in the iteration */
  HELM6_ERR_INVALID = -1,   /* bad argument (sizes, faces, pointers, options) */
  HELM6_ERR_NOMEM = -2,     /* device allocation failed */
  HELM6_ERR_CUDA = -3,      /* a CUDA call failed; the context should be destroyed */
  HELM6_ERR_UNSUPPORTED = -4
};

typedef struct {
  int precision;     /* HELM6_FP64 (default) or HELM6_MIXED */
  int method;        /* HELM6_GMRES (default), HELM6_FGMRES or HELM6_SKS */
  int xform_terms;   /* MIXED only: BF16 split terms of the x/y transforms (1, 2 or 3;
                        0 = default 3: hi*hi + hi*lo + lo*hi) */
  int max_restart;   /* largest restart length helm6_solve will be asked for (0 = 30);
                        sizes the Krylov workspace */
  double inner_tol;  /* MIXED only: relative reduction asked of each FP32 inner solve
                        (0 = default 1e-5) */
  void* stream;      /* cudaStream_t; NULL = default stream */
  int use_graphs;    /* 1: each Arnoldi step is captured once as a CUDA graph (per step
                        index, on a private stream of the context) and replayed on the
                        context's stream, one graph launch instead of about 15 kernel
                        launches per step; results are identical to the eager path; no
                        per-phase profiling while on.
                        2: as 1, and a MIXED FGMRES solve without a learned stage runs as ONE
                        graph launch: the whole solve (true residuals, cycles, Arnoldi steps,
                        least squares, updates) is captured once per restart length, and
                        every convergence decision is taken on the device through
                        conditional graph nodes (a WHILE node over refinement cycles, IF
                        nodes over the Arnoldi steps), so the host only launches it and
                        reads the statistics back; helm6_solve_batch with such contexts
                        launches all of its problems as one graph.  Results are identical
                        to the host-driven path. */
  int dot_blocks;    /* thread blocks of the Gram-Schmidt reduction pass (0 = 2 per SM) */
  int update_blocks; /* thread blocks of the Gram-Schmidt update pass (0 = up to 8 per SM) */
  double cheb_lo, cheb_hi;  /* HELM6_CHEB: 0 < cheb_lo < cheb_hi bounding the (real) eigenvalues
                               of A A_p^{-1}; both 0 = the exact bounds, computed on the sine
                               modes, for a real k on the all-Dirichlet cube (Eq. 3DEGV), else
                               UNSUPPORTED */
  int own_stream;    /* nonzero: ignore `stream`; the context creates (and destroys) its own
                        stream, ordered with the legacy default stream like any blocking
                        stream, so that contexts driven from several threads run
                        concurrently while staying ordered with default-stream work */
  int basis;         /* MIXED Krylov methods: HELM6_BASIS_*; AUTO = F16 from 2^23 unknowns
                        (mx*my*mz), F32 below.  F16 with FP64 is INVALID */
  int transform;     /* x/y transforms of the preconditioner: HELM6_XFORM_* (AUTO default) */
} helm6_opts;

#define HELM6_MAX_HIST 1024

typedef struct {
  int iters;          /* Krylov (or SKS) iterations, summed over restarts and refinements */
  int outer;          /* GMRES cycles (FP64) or FP64 refinement steps (MIXED) */
  int status;         /* same value helm6_solve returns */
  double relres;      /* final true relative residual ||F - A U||_2 / ||F||_2, FP64 */
  double t_total_ms;  /* wall time of helm6_solve */
  int nhist;          /* entries in hist */
  double hist[HELM6_MAX_HIST];  /* relative residual after each iteration (estimates for
                                   GMRES, true residuals for SKS and refinement steps) */
  int cnn_cycles;     /* MIXED FGMRES with a learned stage attached: inner cycles that used
                         it (the others used the direct preconditioner alone) */
  int cnn_fallbacks;  /* learned-stage cycles whose correction was non-finite: discarded
                         (U kept its last iterate) and the rest of the solve used the
                         direct preconditioner alone */
} helm6_stats;

/* Fill opts with the defaults listed above. */
void helm6_opts_default(helm6_opts* opts);

/* Create a solver for n interior nodes per side (1 <= n <= 4094), grid step h (h <= 0 means
 * the unit cube, h = 1/(n+1)), wavenumber k and faces[6] = {x0, x1, y0, y1, z0, z1} of
 * helm6_bc.  Builds the 1D eigenbases (closed forms, FP64 host arithmetic), uploads them
 * and allocates the workspace.  opts may be NULL (defaults).  *out is set only on success.
 * Errors: INVALID (n out of range, Sommerfeld-like faces on more than one axis pair, bad
 * option values), NOMEM, CUDA. */
int helm6_create(helm6_ctx** out, int n, double h, helm6_c64 k, const int faces[6],
                 const helm6_opts* opts);

/* Unknowns per axis: dims = {mx, my, mz}. */
int helm6_dims(const helm6_ctx* ctx, int64_t dims[3]);

/* The transform the context applies along axis 0 (internal x) or 1 (internal y):
 * HELM6_XFORM_DENSE, HELM6_XFORM_FFT or HELM6_XFORM_TENSOR; INVALID for a null context or
 * another axis.  With Sommerfeld-like faces on x or y the internal axes are the exchanged
 * ones (that pair becomes the internal z). */
int helm6_transform(const helm6_ctx* ctx, int axis);

/* Storage of the context's Krylov basis as resolved at creation: HELM6_BASIS_F32 or
 * HELM6_BASIS_F16 for a MIXED GMRES/FGMRES context, HELM6_BASIS_AUTO (0) where the basis is
 * FP64 or there is none (SKS, Chebyshev); INVALID if ctx is NULL. */
int helm6_basis(const helm6_ctx* ctx);

/* y = A x, the h^2-scaled sixth-order compact operator (Eq. scheme; face rows per Eq. 3DN
 * with the ghost eliminated by even reflection, and Eq. 3DDISCS).  x and y are device
 * complex128 arrays of mx*my*mz elements and must not overlap.  In MIXED precision the
 * product is computed by the FP32 kernel (inputs rounded to FP32, result widened). */
int helm6_apply_A(helm6_ctx* ctx, const void* x, void* y);

/* y = A_p^{-1} x, the direct inverse of the 7-point preconditioner (Eq. 3DAP): forward x
 * and y eigen-transforms, a tridiagonal solve along z for every (x, y) mode pair, inverse
 * transforms.  FP64: FP64 transforms and Thomas; MIXED: BF16-split tensor-core
 * transforms and FP32 Thomas.  x and y may alias.  Returns BREAKDOWN if a z-line pivot is
 * exactly zero (y is then undefined). */
int helm6_apply_Pinv(helm6_ctx* ctx, const void* x, void* y);

/* Solve A u = F to ||F - A u||_2 / ||F||_2 <= tol (true residual, FP64), starting from
 * the u passed in (in/out).  restart = m of GMRES(m) (1 <= m <= opts.max_restart; ignored
 * by SKS), maxit = cap on iterations (summed).  stats may be NULL.  Returns OK or a
 * positive warning; u holds the final iterate either way.  F must be finite (NONFINITE
 * otherwise, u untouched).  F = 0 returns u = 0. */
int helm6_solve(helm6_ctx* ctx, const void* F, void* u, double tol, int restart, int maxit,
                helm6_stats* stats);

/* Assemble the compact right side F (Eq. scheme right side, h^2-scaled, with the face data
 * terms of Eq. 3DN and Eq. 3DDISCS) for f = sum_s amps[s] exp(-|x - c_s|^2 / (2 sigma^2))
 * plus an optional noise field eta (no derivatives; enters as h^2 cf eta with
 * cf = 1 - k^2h^2/12 + k^4h^4/360).  centers: HOST array of nsrc*3 doubles (x, y, z);
 * amps: HOST array of nsrc helm6_c64; noise: DEVICE complex128 array of the grid's size
 * or NULL; F: DEVICE complex128 output.  0 <= nsrc <= 4096, sigma > 0. */
int helm6_rhs_gaussians(helm6_ctx* ctx, int nsrc, const double* centers,
                        const helm6_c64* amps, double sigma, const void* noise, void* F);

/* Compact right side F (Eq. scheme right side with the Eq. 3DN / Eq. 3DDISCS face terms of
 * homogeneous face data, as helm6_rhs_gaussians) for a separable source
 *     f(x, y, z) = sum_t coef[t] X_t(x) Y_t(y) Z_t(z),
 * given by its factors' derivatives of order 0..4 at the unknown nodes: tables is a HOST
 * array of complex values [nterms][3 axes x, y, z][5 orders][mmax], mmax = the largest of
 * the three unknown counts of helm6_dims; entry p of an axis is the factor's derivative at
 * that axis' p-th unknown, which lies at x = (p + 1) h if the axis' lower face is
 * Dirichlet and at x = p h otherwise (entries beyond the axis length are ignored).  F:
 * DEVICE complex128 output.  0 <= nterms <= 4096.  Returns OK, INVALID, NOMEM or CUDA. */
int helm6_rhs_separable(helm6_ctx* ctx, int nterms, const helm6_c64* coef, const helm6_c64* tables,
                        void* F);

/* Inhomogeneous Dirichlet data on a face (Section 4.2: u = u_b at z = 1 with the Neumann
 * face at z = 0, Tables 5 and 6): the face's nodes are known, so their contribution to the
 * rows next to the face moves to the right side,
 *     F(row) -= sum over the face's nodes in the row's 3 x 3 window of w * u_b(node),
 * w the row's 27-point weight for the node's offset (Eq. scheme's class weights; on a
 * Sommerfeld-like z face row, that row's weights, Eq. 3DDISCS).  face: 0..5 = x0 x1 y0 y1 z0
 * z1, a Dirichlet face of the context.  data: DEVICE complex128 node layer of the face, x
 * fastest, with a one-node ring in the tangential axes that come before the face's own in the
 * order x, y, z (so that a node on an edge belongs to one face only; where a neighbouring
 * face without a ring entry is Neumann, the ghost node is its reflection, U_-1 = U_1, and its
 * value is read from the data):
 *     x faces  [mz][my]            entry (l, j): the node beside unknown row (j, l)
 *     y faces  [mz][mx + 2]        entry (l, i + 1): beside unknown (i, l); ring in x
 *     z faces  [my + 2][mx + 2]    entry (j + 1, i + 1): beside unknown (i, j); ring in x, y
 * F: DEVICE complex128, updated in place.  Stream-ordered.  Returns OK, INVALID (NULL
 * argument, face out of range or not Dirichlet), UNSUPPORTED (a context with
 * Sommerfeld-like faces on x or y) or CUDA. */
int helm6_lift_dirichlet(helm6_ctx* ctx, int face, const void* data, void* F);

/* ---- Measurement (not part of the method) ----
 * Per-phase device time of helm6_solve / helm6_apply_* measured with CUDA events on the
 * context's stream, and the number of kernels the library launched.  Off by default;
 * enabling it resets the counters.  Phases: */
enum {
  HELM6_PH_STENCIL = 0,  /* 27-point operator in the Krylov precision */
  HELM6_PH_XFWD = 1,     /* preconditioner x forward transform */
  HELM6_PH_YFWD = 2,     /* y forward transform */
  HELM6_PH_ZTRI = 3,     /* z tridiagonal lines */
  HELM6_PH_YINV = 4,     /* y inverse transform */
  HELM6_PH_XINV = 5,     /* x inverse transform */
  HELM6_PH_DOT = 6,      /* Gram-Schmidt reduction pass (basis inner products) */
  HELM6_PH_UPDATE = 7,   /* Gram-Schmidt update pass (new basis vector) */
  HELM6_PH_SMALL = 8,    /* partial-sum reduction, FP64 step algebra and Givens */
  HELM6_PH_RESID64 = 9,  /* FP64 true residual F - A U and its norm */
  HELM6_PH_OTHER = 10,   /* conversions, solution updates */
  HELM6_PH_CNN = 11,     /* learned stage: residual of the direct preconditioner and network */
  HELM6_NPHASE = 12
};

typedef struct {
  int64_t launches;              /* kernels launched by the library since enabling */
  int64_t count[HELM6_NPHASE];   /* timed intervals per phase */
  double ms[HELM6_NPHASE];       /* summed device milliseconds per phase */
  double bytes[HELM6_NPHASE];    /* summed algorithmic bytes per phase: one read of each
                                    input and one write of each output, in the phase's
                                    working precision */
} helm6_profile;

/* enable != 0 starts (and resets) measurement, 0 stops it.  INVALID if ctx is NULL. */
int helm6_profile_enable(helm6_ctx* ctx, int enable);

/* Copy the counters accumulated so far into *out (synchronises the stream). */
int helm6_profile_read(helm6_ctx* ctx, helm6_profile* out);

/* ---- Residual without device allocation (the paper has no counterpart) ----
 * r = F - A u for the sixth-order operator of helm6_apply_A, and *sumsq = ||r||_2^2, for
 * callers that cannot call cudaMalloc: a custom device allocator or memory pool that must
 * not re-enter cudaMalloc, an embedding runtime that owns every byte of device memory, or a
 * real-time loop that must never block on the allocator.  It takes the problem description
 * instead of a context (a context allocates workspace), allocates nothing and calls no
 * allocating routine.  It enqueues two kernels on `stream`, so it must be called from
 * ordinary host code: not from a CUDA host function or stream callback, where no CUDA call
 * is allowed at all.
 *
 * Its only scratch is a file-scope device array of HELM6_NOALLOC_MAX_BLOCKS doubles
 * (512 KiB) that every GPU which loads the library holds until the process exits.  Sizes
 * whose stencil grid needs more than HELM6_NOALLOC_MAX_BLOCKS thread blocks --
 * ceil(mx/32) * ceil(my/8) * ceil(mz/16): a cube up to n = 640 with Dirichlet faces, up to
 * n = 638 with non-Dirichlet faces on every axis -- are rejected with HELM6_ERR_INVALID
 * before any device work.  The first call on each device looks up the array's device
 * address with that device current (cudaGetSymbolAddress); with CUDA's lazy module
 * loading that first call may also load the library's device code and back the array with
 * device memory.  So make one warm-up call per device from ordinary code, before any
 * stream capture and before entering a context where allocation is forbidden; only the
 * later calls are guaranteed to allocate nothing.  Every call shares the array and leaves
 * its partial sums there; each call writes every slot it reads, so nothing needs clearing,
 * but calls that overlap on the GPU (several streams, or several host threads on one
 * device) race on it and must be serialised by the caller.
 *
 * n, h, k, faces: as helm6_create, except that Sommerfeld-like faces are accepted on z only
 * here (INVALID otherwise).  F, u, r: DEVICE complex128 arrays (layout as above), r must not
 * overlap u.  sumsq: DEVICE pointer to one double.  stream: cudaStream_t or
 * NULL.  Work is enqueued on the stream; the call returns without synchronising.
 * Returns OK, INVALID (arguments, or grid too large), UNSUPPORTED (device ordinal >= 64)
 * or CUDA. */
#define HELM6_NOALLOC_MAX_BLOCKS 65536
int helm6_residual_noalloc(int n, double h, helm6_c64 k, const int faces[6], const void* F,
                           const void* u, void* r, double* sumsq, void* stream);

/* ---- Learned second preconditioner stage (the paper has no counterpart) ----
 * A small 3D convolutional network N (4 layers of zero-padded 3x3x3 cross-correlation,
 * channels 2 -> 16 -> 16 -> 16 -> 2, bias, GELU x*Phi(x) after layers 1-3; channel 0/1 =
 * real/imaginary part) corrects what the direct preconditioner of Eq. 3DAP leaves:
 *
 *     z = A_p^{-1} u + c s N((u - A A_p^{-1} u) / s),   s = sqrt(mean |u - A A_p^{-1} u|^2),
 *
 * used as the preconditioner of MIXED FGMRES (flexible GMRES accepts any map per column).
 * Parameters: one flat vector of HELM6_CNN_NPARAMS floats, per layer W[c_out][c_in][dz][dy][dx]
 * (C order) then b[c_out].  Arithmetic: BF16-rounded weights and network input, BF16
 * activations between layers, FP32 accumulation, FP32 biases and output. */
#define HELM6_CNN_NPARAMS 15602
enum { HELM6_CNN_OFF = 0,   /* detach: the direct preconditioner alone */
       HELM6_CNN_ON = 1,    /* every inner cycle uses the learned stage */
       HELM6_CNN_AUTO = 2   /* a probe: of inner cycles 0-2 only cycle 1 uses it, and only for
                               its first 2 columns (flexible GMRES allows a different map per
                               column); the later cycles use it on every column only if those
                               2 columns reduced the residual estimate per column at least
                               10 % more (in logarithm) than the first 2 columns of cycle 2
                               did without it; otherwise the direct preconditioner alone (the
                               fallback), run as one device-driven graph where the context
                               solves that way (use_graphs = 2).  In every mode a learned-stage cycle whose
                               correction is non-finite is discarded and the rest of the solve
                               falls back (helm6_stats.cnn_fallbacks) */ };

/* Attach (or with HELM6_CNN_OFF detach) a network to a MIXED FGMRES context.  theta: HOST
 * array of HELM6_CNN_NPARAMS floats (copied); out_scale: c above.  Allocates two BF16
 * activation fields (32 B per unknown each) and one FP32 complex field.  Synchronises the
 * context's stream.  Returns OK, INVALID (NULL ctx or theta, bad mode, non-finite scale),
 * UNSUPPORTED (precision not MIXED or method not FGMRES), NOMEM or CUDA. */
int helm6_set_cnn(helm6_ctx* ctx, const float* theta, double out_scale, int mode);

/* y = the two-stage preconditioner above applied to x (DEVICE complex128 arrays as for
 * helm6_apply_A; y may equal x).  Requires an attached network (else UNSUPPORTED). */
int helm6_apply_stage2(helm6_ctx* ctx, const void* x, void* y);

/* Trainer: the network's forward pass, mean-squared-error gradient and Adam steps
 * (beta1 0.9, beta2 0.999, eps 1e-8) on batches of `batch` images of nz x ny x nx points,
 * stored channel-last as DEVICE float arrays [batch][nz][ny][nx][2].  Zero padding at every
 * image's border.  The gradient is that of the rounded network with each rounding taken
 * as the identity (straight-through) and the GELU differentiated at its FP32 input.
 * theta0: HOST initial parameters.  All work is on `stream` (NULL = default). */
typedef struct helm6_cnn_trainer helm6_cnn_trainer;
int helm6_cnn_trainer_create(helm6_cnn_trainer** out, int batch, int nz, int ny, int nx,
                             const float* theta0, void* stream);
/* y (DEVICE, same layout as x) = N(x).  Stream-ordered, no synchronisation. */
int helm6_cnn_forward(helm6_cnn_trainer* tr, const float* x, float* y);
/* grad (DEVICE, HELM6_CNN_NPARAMS floats) = d/dtheta mean((N(x) - target)^2) over every
 * element; *loss (HOST, nullable) = that mean (then the call synchronises). */
int helm6_cnn_gradient(helm6_cnn_trainer* tr, const float* x, const float* target, float* grad,
                       double* loss);
/* One Adam step of learning rate lr on that gradient; *loss (nullable) as above. */
int helm6_cnn_train_step(helm6_cnn_trainer* tr, const float* x, const float* target, float lr,
                         double* loss);
/* Switch the trainer's loss (for helm6_cnn_gradient and helm6_cnn_train_step) to the
 * residual form  sum |A_h N(x) - target|^2 / (2M)  over the M interior points of the images
 * (at least one point from every face), A_h the interior 27-point operator of Eq. scheme
 * for wavenumber k and step h, with zero values outside each image; target = x makes N a
 * local approximate inverse of A_h.  INVALID for non-finite k, h <= 0 or an image side < 3. */
int helm6_cnn_set_residual_loss(helm6_cnn_trainer* tr, helm6_c64 k, double h);
/* Copy the current FP32 parameters to theta (HOST, HELM6_CNN_NPARAMS floats). */
int helm6_cnn_get_params(helm6_cnn_trainer* tr, float* theta);
void helm6_cnn_trainer_destroy(helm6_cnn_trainer* tr);

/* ---- Batched solve (the paper has no counterpart) ----
 * Solve count independent problems, ctxs[i] with right side F[i] and initial guess /
 * solution u[i] (DEVICE complex128 arrays as for helm6_solve), to the same tol, restart
 * and maxit.  If every context runs device-driven solves (use_graphs = 2, MIXED FGMRES, no
 * learned stage), the batch is ONE graph launch holding every problem's whole solve as an
 * independent branch (built and instantiated on the first call for this set of contexts and
 * restart length, reused afterwards; stats[i].t_total_ms is then problem i's device time,
 * start to convergence); otherwise nthreads host threads (1 <= nthreads <= 256) each take
 * the next unsolved problem and run helm6_solve on its context.  Problems run concurrently on the
 * GPU when their contexts have distinct non-NULL streams; contexts may differ in size,
 * wavenumber, faces and options.  stats: HOST array of count (nullable); stats[i].t_total_ms
 * is problem i's own wall time.  Returns a negative error of any problem (the others still
 * finish), else the largest warning code (OK if every problem converged). */
int helm6_solve_batch(helm6_ctx* const* ctxs, int count, const void* const* F, void* const* u,
                      double tol, int restart, int maxit, int nthreads, helm6_stats* stats);

/* Release the workspace and the context (NULL is allowed).  Synchronises its stream. */
void helm6_destroy(helm6_ctx* ctx);

/* Static string naming a return code. */
const char* helm6_status_string(int code);

#ifdef __cplusplus
}
#endif

#endif /* HELM6_H */

"""Python binding of the helm6 C-ABI (ctypes; argument marshalling only).

Every step of the solver runs in the CUDA library libhelm6.so; this module only turns
torch tensors into device pointers and structs into ctypes.  Importing it does not need a
GPU; opening the library does, and a missing library raises instead of falling back.
"""
from __future__ import annotations

import ctypes as C
import os

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libhelm6.so")

DIRICHLET, NEUMANN, SOMMERFELD = 0, 1, 2
FP64, MIXED = 0, 1
GMRES, FGMRES, SKS, CHEB = 0, 1, 2, 3
MAX_HIST = 1024
CNN_NPARAMS = 15602
CNN_OFF, CNN_ON, CNN_AUTO = 0, 1, 2
BASIS_AUTO, BASIS_F32, BASIS_F16 = 0, 1, 2
XFORM_AUTO, XFORM_DENSE, XFORM_FFT, XFORM_TENSOR = 0, 1, 2, 3
_XFORM_CODE = {"auto": XFORM_AUTO, "dense": XFORM_DENSE, "fft": XFORM_FFT}
_XFORM_NAME = {XFORM_DENSE: "dense", XFORM_FFT: "fft", XFORM_TENSOR: "tensor"}

STATUS = {0: "OK", 1: "NOT_CONVERGED", 2: "DIVERGED", 3: "BREAKDOWN", 4: "NONFINITE",
          -1: "ERR_INVALID", -2: "ERR_NOMEM", -3: "ERR_CUDA", -4: "ERR_UNSUPPORTED"}

_FACE_CODE = {"D": DIRICHLET, "N": NEUMANN, "S": SOMMERFELD}

# every symbol declared in include/helm6.h
EXPORTS = ("helm6_opts_default", "helm6_create", "helm6_dims", "helm6_basis", "helm6_apply_A", "helm6_apply_Pinv",
           "helm6_solve", "helm6_rhs_gaussians", "helm6_destroy", "helm6_status_string",
           "helm6_profile_enable", "helm6_profile_read", "helm6_residual_noalloc", "helm6_set_cnn",
           "helm6_apply_stage2", "helm6_cnn_trainer_create", "helm6_cnn_forward", "helm6_cnn_gradient",
           "helm6_cnn_train_step", "helm6_cnn_set_residual_loss", "helm6_cnn_get_params",
           "helm6_cnn_trainer_destroy", "helm6_solve_batch", "helm6_rhs_separable",
           "helm6_lift_dirichlet", "helm6_transform")

PHASES = ("stencil", "xform_x_fwd", "xform_y_fwd", "ztri", "xform_y_inv", "xform_x_inv", "gs_dot",
          "gs_update", "gs_small", "resid64", "other", "cnn")


class C64(C.Structure):
    _fields_ = [("re", C.c_double), ("im", C.c_double)]


class Opts(C.Structure):
    _fields_ = [("precision", C.c_int), ("method", C.c_int), ("xform_terms", C.c_int),
                ("max_restart", C.c_int), ("inner_tol", C.c_double), ("stream", C.c_void_p),
                ("use_graphs", C.c_int), ("dot_blocks", C.c_int), ("update_blocks", C.c_int),
                ("cheb_lo", C.c_double), ("cheb_hi", C.c_double), ("own_stream", C.c_int),
                ("basis", C.c_int), ("transform", C.c_int)]


class Stats(C.Structure):
    _fields_ = [("iters", C.c_int), ("outer", C.c_int), ("status", C.c_int),
                ("relres", C.c_double), ("t_total_ms", C.c_double), ("nhist", C.c_int),
                ("hist", C.c_double * MAX_HIST), ("cnn_cycles", C.c_int),
                ("cnn_fallbacks", C.c_int)]

    def to_dict(self):
        return dict(iters=self.iters, outer=self.outer, status=STATUS.get(self.status, self.status),
                    relres=self.relres, t_total_ms=self.t_total_ms,
                    history=list(self.hist[: self.nhist]), cnn_cycles=self.cnn_cycles,
                    cnn_fallbacks=self.cnn_fallbacks)


class Profile(C.Structure):
    _fields_ = [("launches", C.c_int64), ("count", C.c_int64 * len(PHASES)),
                ("ms", C.c_double * len(PHASES)), ("bytes", C.c_double * len(PHASES))]

    def to_dict(self):
        return dict(launches=self.launches,
                    phases={PHASES[i]: dict(count=self.count[i], ms=self.ms[i], bytes=self.bytes[i])
                            for i in range(len(PHASES))})


_lib = None


def load(path: str = LIB_PATH):
    """Open libhelm6.so and declare its signatures (raises if it is missing)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with paper_1212_1397_gb300.build.build()")
    lib = C.CDLL(path)
    P, I, D = C.c_void_p, C.c_int, C.c_double
    lib.helm6_opts_default.argtypes = [C.POINTER(Opts)]
    lib.helm6_opts_default.restype = None
    lib.helm6_create.argtypes = [C.POINTER(P), I, D, C64, C.POINTER(C.c_int), C.POINTER(Opts)]
    lib.helm6_create.restype = I
    lib.helm6_dims.argtypes = [P, C.POINTER(C.c_int64)]
    lib.helm6_dims.restype = I
    lib.helm6_basis.argtypes = [P]
    lib.helm6_basis.restype = I
    lib.helm6_transform.argtypes = [P, I]
    lib.helm6_transform.restype = I
    lib.helm6_apply_A.argtypes = [P, P, P]
    lib.helm6_apply_A.restype = I
    lib.helm6_apply_Pinv.argtypes = [P, P, P]
    lib.helm6_apply_Pinv.restype = I
    lib.helm6_solve.argtypes = [P, P, P, D, I, I, C.POINTER(Stats)]
    lib.helm6_solve.restype = I
    lib.helm6_rhs_gaussians.argtypes = [P, I, C.POINTER(C.c_double), C.POINTER(C64), D, P, P]
    lib.helm6_rhs_gaussians.restype = I
    lib.helm6_destroy.argtypes = [P]
    lib.helm6_destroy.restype = None
    lib.helm6_profile_enable.argtypes = [P, I]
    lib.helm6_profile_enable.restype = I
    lib.helm6_profile_read.argtypes = [P, C.POINTER(Profile)]
    lib.helm6_profile_read.restype = I
    lib.helm6_residual_noalloc.argtypes = [I, D, C64, C.POINTER(C.c_int), P, P, P, P, P]
    lib.helm6_residual_noalloc.restype = I
    F32P = C.POINTER(C.c_float)
    lib.helm6_set_cnn.argtypes = [P, F32P, D, I]
    lib.helm6_set_cnn.restype = I
    lib.helm6_apply_stage2.argtypes = [P, P, P]
    lib.helm6_apply_stage2.restype = I
    lib.helm6_cnn_trainer_create.argtypes = [C.POINTER(P), I, I, I, I, F32P, P]
    lib.helm6_cnn_trainer_create.restype = I
    lib.helm6_cnn_forward.argtypes = [P, P, P]
    lib.helm6_cnn_forward.restype = I
    lib.helm6_cnn_gradient.argtypes = [P, P, P, P, C.POINTER(D)]
    lib.helm6_cnn_gradient.restype = I
    lib.helm6_cnn_train_step.argtypes = [P, P, P, C.c_float, C.POINTER(D)]
    lib.helm6_cnn_train_step.restype = I
    lib.helm6_cnn_set_residual_loss.argtypes = [P, C64, D]
    lib.helm6_cnn_set_residual_loss.restype = I
    lib.helm6_cnn_get_params.argtypes = [P, F32P]
    lib.helm6_cnn_get_params.restype = I
    lib.helm6_cnn_trainer_destroy.argtypes = [P]
    lib.helm6_cnn_trainer_destroy.restype = None
    lib.helm6_rhs_separable.argtypes = [P, I, C.POINTER(C64), C.POINTER(C64), P]
    lib.helm6_rhs_separable.restype = I
    lib.helm6_lift_dirichlet.argtypes = [P, I, P, P]
    lib.helm6_lift_dirichlet.restype = I
    lib.helm6_solve_batch.argtypes = [C.POINTER(P), I, C.POINTER(P), C.POINTER(P), D, I, I, I,
                                      C.POINTER(Stats)]
    lib.helm6_solve_batch.restype = I
    lib.helm6_status_string.argtypes = [I]
    lib.helm6_status_string.restype = C.c_char_p
    _lib = lib
    return lib


class Helm6Error(RuntimeError):
    pass


def _check(rc, what):
    if rc < 0:
        msg = load().helm6_status_string(rc).decode()
        raise Helm6Error(f"{what}: {msg} ({rc})")
    return rc


def _ptr(t):
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError("expected a CUDA tensor")
    if t.dtype != torch.complex128 or not t.is_contiguous():
        raise TypeError("expected a contiguous complex128 tensor")
    return C.c_void_p(t.data_ptr())


def residual_noalloc(n, k, faces, F, u, r, sumsq, h=0.0, stream=None):
    """r = F - A u and sumsq[0] = ||r||^2 through helm6_residual_noalloc (no allocation).

    F, u, r: complex128 CUDA tensors of the grid's shape; sumsq: float64 CUDA tensor of one
    element.  Returns the library's return code (raises on errors)."""
    import torch
    if len(faces) != 6 or any(ch not in _FACE_CODE for ch in faces):
        raise ValueError(f"faces must be 6 letters over D, N, S, got {faces!r}")
    # unknowns per axis: n plus one per non-Dirichlet face of that axis
    mx, my, mz = (int(n) + (faces[2 * a] != "D") + (faces[2 * a + 1] != "D") for a in range(3))
    npts = mx * my * mz
    for name, t in (("F", F), ("u", u), ("r", r)):
        if not isinstance(t, torch.Tensor) or t.numel() != npts:
            got = t.numel() if isinstance(t, torch.Tensor) else type(t).__name__
            raise ValueError(f"{name} must hold mx*my*mz = {mx}*{my}*{mz} = {npts} elements, got {got}")
    if not (isinstance(sumsq, torch.Tensor) and sumsq.is_cuda and sumsq.dtype == torch.float64
            and sumsq.numel() >= 1):
        raise TypeError("sumsq must be a float64 CUDA tensor of at least one element")
    lib = load()
    f = (C.c_int * 6)(*[_FACE_CODE[ch] for ch in faces])
    kk = complex(k)
    s = None
    if stream is not None:
        s = C.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))
    return _check(lib.helm6_residual_noalloc(int(n), float(h), C64(kk.real, kk.imag), f, _ptr(F),
                                             _ptr(u), _ptr(r), C.c_void_p(sumsq.data_ptr()), s),
                  "helm6_residual_noalloc")


class Solver:
    """One helm6 context: grid, wavenumber, faces and options fixed at construction.

    faces: 6 letters 'x0 x1 y0 y1 z0 z1' over D (Dirichlet), N (Neumann), S (Sommerfeld-like).
    Vectors are complex128 CUDA tensors of shape (mz, my, mx).
    """

    def __init__(self, n, k, faces="DDDDDD", h=0.0, precision=FP64, method=GMRES,
                 max_restart=30, inner_tol=1e-5, xform_terms=3, stream=None, use_graphs=False,
                 dot_blocks=0, update_blocks=0, own_stream=False, cheb_bounds=(0.0, 0.0), basis=BASIS_AUTO,
                 transform="auto"):
        lib = load()
        self._lib = lib
        o = Opts()
        lib.helm6_opts_default(C.byref(o))
        o.precision, o.method, o.max_restart = precision, method, max_restart
        o.inner_tol, o.xform_terms = inner_tol, xform_terms
        o.use_graphs = 2 if (use_graphs == 2 or use_graphs == "solve") else int(bool(use_graphs))
        o.dot_blocks, o.update_blocks = int(dot_blocks), int(update_blocks)
        o.own_stream = int(bool(own_stream))
        o.basis = int(basis)
        o.transform = _XFORM_CODE[transform] if isinstance(transform, str) else int(transform)
        o.cheb_lo, o.cheb_hi = float(cheb_bounds[0]), float(cheb_bounds[1])
        if stream is not None:
            o.stream = C.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))
        self.stream = stream
        f = (C.c_int * 6)(*[_FACE_CODE[ch] for ch in faces])
        kk = complex(k)
        ctx = C.c_void_p()
        _check(lib.helm6_create(C.byref(ctx), int(n), float(h), C64(kk.real, kk.imag), f, C.byref(o)),
               "helm6_create")
        self._ctx = ctx
        d = (C.c_int64 * 3)()
        _check(lib.helm6_dims(ctx, d), "helm6_dims")
        self.dims = (d[0], d[1], d[2])
        self.shape = (d[2], d[1], d[0])
        self.n, self.k, self.faces = n, kk, faces
        self.h = h if h > 0 else 1.0 / (n + 1)

    @property
    def basis(self):
        """Storage of the Krylov basis as resolved at creation: BASIS_F32 or BASIS_F16 (MIXED
        GMRES/FGMRES), BASIS_AUTO where it is FP64 or there is none."""
        return _check(self._lib.helm6_basis(self._ctx), "helm6_basis")

    @property
    def transforms(self):
        """The x/y transforms as resolved at creation, per internal axis: "dense", "fft" or
        "tensor" (dense on tensor cores)."""
        return tuple(_XFORM_NAME[_check(self._lib.helm6_transform(self._ctx, a), "helm6_transform")]
                     for a in (0, 1))

    def close(self):
        if getattr(self, "_ctx", None):
            self._lib.helm6_destroy(self._ctx)
            self._ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def empty(self):
        import torch
        return torch.zeros(self.shape, dtype=torch.complex128, device="cuda")

    def apply_A(self, x, y=None):
        y = self.empty() if y is None else y
        _check(self._lib.helm6_apply_A(self._ctx, _ptr(x), _ptr(y)), "helm6_apply_A")
        return y

    def apply_Pinv(self, x, y=None):
        y = self.empty() if y is None else y
        rc = _check(self._lib.helm6_apply_Pinv(self._ctx, _ptr(x), _ptr(y)), "helm6_apply_Pinv")
        if rc != 0:
            raise Helm6Error(f"helm6_apply_Pinv: {STATUS.get(rc)}")
        return y

    def set_cnn(self, theta, out_scale, mode=CNN_ON):
        """Attach the learned second stage (theta: CNN_NPARAMS floats, host) or detach it."""
        import numpy as np
        th = np.ascontiguousarray(np.asarray(theta, dtype=np.float32).ravel())
        if th.size != CNN_NPARAMS:
            raise ValueError(f"expected {CNN_NPARAMS} parameters, got {th.size}")
        _check(self._lib.helm6_set_cnn(self._ctx, th.ctypes.data_as(C.POINTER(C.c_float)), float(out_scale),
                                       int(mode)), "helm6_set_cnn")

    def apply_stage2(self, x, y=None):
        y = self.empty() if y is None else y
        rc = _check(self._lib.helm6_apply_stage2(self._ctx, _ptr(x), _ptr(y)), "helm6_apply_stage2")
        if rc != 0:
            raise Helm6Error(f"helm6_apply_stage2: {STATUS.get(rc)}")
        return y

    def solve(self, F, u=None, tol=1e-8, restart=30, maxit=500):
        """Solve A u = F (u in/out, zero if None).  Returns (u, stats dict)."""
        u = self.empty() if u is None else u
        st = Stats()
        rc = _check(self._lib.helm6_solve(self._ctx, _ptr(F), _ptr(u), float(tol), int(restart),
                                          int(maxit), C.byref(st)), "helm6_solve")
        d = st.to_dict()
        d["rc"] = rc
        return u, d

    def profile(self, enable=True):
        """Start (and reset) or stop per-phase event timing inside the library."""
        _check(self._lib.helm6_profile_enable(self._ctx, int(bool(enable))), "helm6_profile_enable")

    def profile_read(self):
        p = Profile()
        _check(self._lib.helm6_profile_read(self._ctx, C.byref(p)), "helm6_profile_read")
        return p.to_dict()

    def rhs_separable(self, coef, tables, F=None):
        """Compact right side of f = sum_t coef[t] X_t Y_t Z_t; tables: complex array
        [nterms, 3, 5, max(dims)] of the factors' derivatives 0..4 at the unknown nodes."""
        import numpy as np
        F = self.empty() if F is None else F
        cf = np.ascontiguousarray(np.asarray(coef, dtype=np.complex128).ravel())
        tb = np.ascontiguousarray(np.asarray(tables, dtype=np.complex128))
        nt = cf.size
        if tb.shape != (nt, 3, 5, max(self.dims)):
            raise ValueError(f"tables must have shape {(nt, 3, 5, max(self.dims))}, got {tb.shape}")
        _check(self._lib.helm6_rhs_separable(self._ctx, nt, cf.ctypes.data_as(C.POINTER(C64)),
                                             tb.ctypes.data_as(C.POINTER(C64)), _ptr(F)), "helm6_rhs_separable")
        return F

    def lift_dirichlet(self, face, data, F):
        """F -= the contribution of Dirichlet values `data` (complex128 CUDA tensor, the face's
        node layer: x faces (mz, my), y faces (mz, mx+2), z faces (my+2, mx+2)) on face
        `face` ("x0", "x1", "y0", "y1", "z0" or "z1")."""
        import torch
        fi = {"x0": 0, "x1": 1, "y0": 2, "y1": 3, "z0": 4, "z1": 5}[face]
        mx, my, mz = self.dims
        shape = [(mz, my), (mz, mx + 2), (my + 2, mx + 2)][fi // 2]
        if not isinstance(data, torch.Tensor) or tuple(data.shape) != shape:
            raise ValueError(f"data must have shape {shape}")
        _check(self._lib.helm6_lift_dirichlet(self._ctx, fi, _ptr(data), _ptr(F)), "helm6_lift_dirichlet")
        return F

    def rhs_gaussians(self, sources, noise=None, F=None):
        """Compact right side for helm6_inputs.GaussianSources (+ optional noise tensor)."""
        F = self.empty() if F is None else F
        ns = len(sources)
        cen = (C.c_double * max(3 * ns, 1))(*sources.centers.ravel().tolist())
        amps = (C64 * max(ns, 1))(*[C64(a.real, a.imag) for a in sources.amps])
        nptr = _ptr(noise) if noise is not None else None
        _check(self._lib.helm6_rhs_gaussians(self._ctx, ns, cen, amps, float(sources.sigma), nptr,
                                             _ptr(F)), "helm6_rhs_gaussians")
        return F


def _fptr(t, numel=None):
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != torch.float32 or not t.is_contiguous():
        raise TypeError("expected a contiguous float32 CUDA tensor")
    if numel is not None and t.numel() != numel:
        raise ValueError(f"expected {numel} elements, got {t.numel()}")
    return C.c_void_p(t.data_ptr())


class Trainer:
    """helm6_cnn_trainer: forward, MSE gradient and Adam steps of the learned stage's network
    on batches of channel-last float32 CUDA tensors of shape (batch, nz, ny, nx, 2)."""

    def __init__(self, batch, nz, ny, nx, theta0, stream=None):
        import numpy as np
        lib = load()
        self._lib = lib
        th = np.ascontiguousarray(np.asarray(theta0, dtype=np.float32).ravel())
        if th.size != CNN_NPARAMS:
            raise ValueError(f"expected {CNN_NPARAMS} parameters, got {th.size}")
        s = None
        if stream is not None:
            s = C.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))
        tr = C.c_void_p()
        _check(lib.helm6_cnn_trainer_create(C.byref(tr), int(batch), int(nz), int(ny), int(nx),
                                            th.ctypes.data_as(C.POINTER(C.c_float)), s),
               "helm6_cnn_trainer_create")
        self._tr = tr
        self.shape = (batch, nz, ny, nx, 2)
        self.numel = batch * nz * ny * nx * 2

    def close(self):
        if getattr(self, "_tr", None):
            self._lib.helm6_cnn_trainer_destroy(self._tr)
            self._tr = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def forward(self, x, y=None):
        import torch
        y = torch.empty(self.shape, dtype=torch.float32, device="cuda") if y is None else y
        _check(self._lib.helm6_cnn_forward(self._tr, _fptr(x, self.numel), _fptr(y, self.numel)),
               "helm6_cnn_forward")
        return y

    def gradient(self, x, target):
        """(loss, grad tensor of CNN_NPARAMS floats)."""
        import torch
        g = torch.empty(CNN_NPARAMS, dtype=torch.float32, device="cuda")
        loss = C.c_double()
        _check(self._lib.helm6_cnn_gradient(self._tr, _fptr(x, self.numel), _fptr(target, self.numel),
                                            _fptr(g), C.byref(loss)), "helm6_cnn_gradient")
        return loss.value, g

    def step(self, x, target, lr, want_loss=True):
        loss = C.c_double()
        _check(self._lib.helm6_cnn_train_step(self._tr, _fptr(x, self.numel), _fptr(target, self.numel),
                                              float(lr), C.byref(loss) if want_loss else None),
               "helm6_cnn_train_step")
        return loss.value if want_loss else None

    def set_residual_loss(self, k, h):
        """Loss mean |A_h N(x) - target|^2 over interior points (A_h: interior operator for k, h)."""
        kk = complex(k)
        _check(self._lib.helm6_cnn_set_residual_loss(self._tr, C64(kk.real, kk.imag), float(h)),
               "helm6_cnn_set_residual_loss")

    def params(self):
        import numpy as np
        th = np.empty(CNN_NPARAMS, dtype=np.float32)
        _check(self._lib.helm6_cnn_get_params(self._tr, th.ctypes.data_as(C.POINTER(C.c_float))),
               "helm6_cnn_get_params")
        return th


def solve_batch(solvers, Fs, us, tol=1e-8, restart=30, maxit=300, nthreads=8):
    """helm6_solve_batch over Solver objects (each ideally on its own stream).  Returns
    (return code, [stats dict per problem])."""
    lib = load()
    cnt = len(solvers)
    if not (len(Fs) == cnt and len(us) == cnt):
        raise ValueError("solvers, Fs and us must have the same length")
    ctxs = (C.c_void_p * cnt)(*[s._ctx.value for s in solvers])
    fp = (C.c_void_p * cnt)(*[_ptr(f).value for f in Fs])
    up = (C.c_void_p * cnt)(*[_ptr(u).value for u in us])
    st = (Stats * cnt)()
    rc = _check(lib.helm6_solve_batch(ctxs, cnt, fp, up, float(tol), int(restart), int(maxit), int(nthreads), st),
                "helm6_solve_batch")
    return rc, [st[i].to_dict() for i in range(cnt)]

"""Plain FP64 CPU oracle for the sixth-order compact Helmholtz method (Gryazin).

TEST INFRASTRUCTURE ONLY.  This is the independent CPU statement of what the CUDA path
computes.  Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg may import
or run it; the product library never does, and it shares no code with the CUDA path
(only the seeded draws of helm6_inputs serve both).

Everything is complex128, arrays indexed [z, y, x] (x fastest), one entry per unknown.
The grid is the unit cube with h = 1/(n+1); a Dirichlet face's nodes are known (zero),
a Neumann or Sommerfeld-like face's nodes are unknowns (Section 3.3: N_x = N_y = N_z - 1
or N_z - 2 when the z faces carry unknowns).  Faces are given as a 6-letter string
'x0 x1 y0 y1 z0 z1' over {D, N, S}.

Readings of the paper taken here where it is garbled or silent:
  * RHS of Eq. scheme: the mixed fourth derivatives enter with total weight h^4/90 and the
    pure ones with h^4/360 (the printed "nabla^4 f" plus an extra h^4/90 mixed term is only
    fourth order).
  * Eq. 3DN: the 7h^5/180 (f_zxx + f_zyy) term enters with a minus sign (the printed plus
    sign leaves an O(h^5) ghost error; the minus sign gives O(h^7)).
  * Eq. 3DDISCS: mu1's "1/6mu3" is 1/(6 mu3); the formula is used as printed.
  * The top faces mirror the bottom-face formulas in the inward normal coordinate.
  * Edges and corners: a homogeneous Neumann face is an even reflection of the unknowns
    for every ghost value needed anywhere (including the in-plane differences of another
    face's elimination); its data term is added to that face's own rows only.
  * Sommerfeld-like faces are allowed on one axis pair.  The paper writes the face rows for
    the z faces only and the scheme is symmetric under exchanging axes, so Sommerfeld-like
    faces on the x (or y) pair are the z-face problem with the x and z (or y and z) axes
    exchanged; the operator and the preconditioner are applied that way (the right side's
    face terms are written per axis and need no exchange).  Two axes with Sommerfeld-like
    faces would need a complex eigenbasis in x or y and are not supported.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import scipy.linalg.lapack as lapack

FACES = "DNS"


# ======================================================================================
# Problem description
# ======================================================================================

@dataclass
class Problem:
    n: int
    k: complex
    faces: str = "DDDDDD"

    def __post_init__(self):
        self.k = complex(self.k)
        assert len(self.faces) == 6 and all(c in FACES for c in self.faces)
        s_axes = [a for a in range(3) if "S" in self.faces[2 * a:2 * a + 2]]
        assert len(s_axes) <= 1, "Sommerfeld-like faces on one axis pair only"
        self.s_axis = s_axes[0] if s_axes else None
        self.h = 1.0 / (self.n + 1)

    def exchanged(self) -> "Problem":
        """The same problem with the Sommerfeld-like axis exchanged with z."""
        f = self.faces
        if self.s_axis == 0:
            return Problem(self.n, self.k, f[4:6] + f[2:4] + f[0:2])
        if self.s_axis == 1:
            return Problem(self.n, self.k, f[0:2] + f[4:6] + f[2:4])
        return self

    def face(self, axis: int, side: int) -> str:
        return self.faces[2 * axis + side]

    def nodes(self, axis: int) -> np.ndarray:
        lo, hi = self.face(axis, 0), self.face(axis, 1)
        start = 1 if lo == "D" else 0
        stop = self.n if hi == "D" else self.n + 1
        return np.arange(start, stop + 1)

    @property
    def dims(self):
        """Unknowns per axis (mx, my, mz)."""
        return tuple(len(self.nodes(a)) for a in range(3))

    @property
    def shape(self):
        """Array shape (mz, my, mx)."""
        mx, my, mz = self.dims
        return (mz, my, mx)

    def coords(self):
        """Broadcastable node coordinates Z, Y, X for arrays of `shape`."""
        h = self.h
        X = (self.nodes(0) * h)[None, None, :]
        Y = (self.nodes(1) * h)[None, :, None]
        Z = (self.nodes(2) * h)[:, None, None]
        return Z, Y, X


# ======================================================================================
# Coefficients of the scheme (Eq. scheme, Eq. 3DDISCS)
# ======================================================================================

def scheme_coefficients(k: complex, h: float) -> dict:
    """Coefficients of the h^2-scaled compact scheme, Eq. scheme.

    With D_a = h^2 delta_a^2 = [1, -2, 1] along axis a the left side is
        (D_x + D_y + D_z) + a (D_xD_y + D_xD_z + D_yD_z) + b D_xD_yD_z + kappa,
    a = (1 + k^2h^2/30)/6, b = 1/30, kappa = k^2h^2 (1 - k^2h^2/12 + k^4h^4/360);
    cf = 1 - k^2h^2/12 + k^4h^4/360 multiplies f on the right side.
    """
    kh2 = (k * h) ** 2
    cf = 1 - kh2 / 12 + kh2 * kh2 / 360
    return dict(a=(1 + kh2 / 30) / 6, b=1.0 / 30, kappa=kh2 * cf, cf=cf)


def sommerfeld_coefficients(k: complex, h: float) -> dict:
    """mu_3, mu_1 and the plane operators' scalars of Eq. 3DDISCS."""
    ik = 1j * k
    kh2 = (k * h) ** 2
    mu3 = 1 / (1 + (2 * ik * h / 3) * (1 + 2 * kh2 / 15))
    mu1 = (ik * h / 90 + (1 + kh2 / 30) / (6 * mu3)) / (1 + 2 * ik * h / 3)
    return dict(
        mu1=mu1, mu3=mu3,
        e1=np.exp(ik * h), e2=np.exp(2 * ik * h),
        # G1 = e2 mu3 [ p (Dx+Dy) + DxDy/(30 mu3) + q I ]
        p=mu1 + (2 * ik * h / 3) * (1.0 / 60 - mu1),
        q=1 - 2 * ik * h / 3 - 4 * ik * (k * h) ** 2 * h / 45,
        # G0 = e1 mu3 [ r I - s (Dx+Dy) ]
        r=(4 * ik * h / 3) * (1 + 2 * kh2 / 15),
        s=(4 * ik * h / 3) * (1.0 / 60 - mu1),
    )


# ======================================================================================
# Finite-difference building blocks on ghost-padded arrays
# ======================================================================================

def exchange(U: np.ndarray, s_axis: int) -> np.ndarray:
    """Array [z, y, x] of a problem with Sommerfeld-like faces on axis s_axis (0 = x, 1 = y)
    as the array of its exchanged problem, and back (the exchange is its own inverse)."""
    return np.ascontiguousarray(np.swapaxes(U, 0, 2 - s_axis))


def _second_difference(P: np.ndarray, axis: int) -> np.ndarray:
    """[1, -2, 1] along `axis`; the result is two shorter along that axis."""
    n = P.shape[axis]
    sl = lambda a, b: tuple(slice(a, b) if ax == axis else slice(None) for ax in range(P.ndim))
    return P[sl(2, n)] - 2 * P[sl(1, n - 1)] + P[sl(0, n - 2)]


def _crop(P: np.ndarray, *axes) -> np.ndarray:
    sl = [slice(None)] * P.ndim
    for ax in axes:
        sl[ax] = slice(1, -1)
    return P[tuple(sl)]


def _pad_ghosts(prob: Problem, U: np.ndarray, boundary=None) -> np.ndarray:
    """Pad U by one ghost layer per side and axis.

    Dirichlet: the boundary node's value (0, or given data for lifting).
    Neumann: even reflection about the face node, U_{-1} = U_{1}.
    Sommerfeld-like: 0 (its rows are completed by the elimination of Eq. 3DDISCS).
    Axes are padded x, then y, then z, so corner ghosts are consistent.
    boundary: optional {(axis, side): array} of Dirichlet data on that ghost layer
    (shape of the padded layer at the time that axis is padded).
    """
    P = U
    for axis in (0, 1, 2):                      # x, y, z
        npax = 2 - axis
        layers = []
        for side in (0, 1):
            kind = prob.face(axis, side)
            idx = 1 if side == 0 else P.shape[npax] - 2
            if kind == "N":
                g = np.take(P, [idx], axis=npax)
            else:
                g = np.zeros_like(np.take(P, [0], axis=npax))
                if kind == "D" and boundary is not None and (axis, side) in boundary:
                    g = g + np.expand_dims(boundary[(axis, side)], npax)
            layers.append(g)
        P = np.concatenate([layers[0], P, layers[1]], axis=npax)
    return P


# ======================================================================================
# The sixth-order operator A (Eq. scheme + Eq. 3DN + Eq. 3DDISCS)
# ======================================================================================

def apply_A(prob: Problem, U: np.ndarray, boundary=None) -> np.ndarray:
    """h^2-scaled sixth-order compact operator applied to U (Eq. scheme, Eq. 3DN, Eq. 3DDISCS).

    Interior rows follow Eq. scheme literally in operator form.  At a Neumann face the
    ghost layer is the even reflection (Eq. 3DN with homogeneous data; the f terms of
    Eq. 3DN go to the right side).  At a Sommerfeld-like face the ghost plane's
    contribution B U_{-1} is replaced by G1 U_1 + G0 U_0 (Eq. 3DDISCS; its data term goes
    to the right side).  Sommerfeld-like faces on x or y: the z-face rows on the exchanged
    problem (see the header).
    """
    if prob.s_axis in (0, 1):
        assert boundary is None, "face data with Sommerfeld-like faces on x or y"
        return exchange(apply_A(prob.exchanged(), exchange(U, prob.s_axis)), prob.s_axis)
    h, k = prob.h, prob.k
    c = scheme_coefficients(k, h)
    P = _pad_ghosts(prob, U, boundary)
    Dx = _second_difference(P, 2)
    Dy = _second_difference(P, 1)
    Dz = _second_difference(P, 0)
    DxDy = _second_difference(Dx, 1)
    DxDz = _second_difference(Dx, 0)
    DyDz = _second_difference(Dy, 0)
    DxDyDz = _second_difference(DxDy, 0)
    out = (_crop(Dx, 0, 1) + _crop(Dy, 0, 2) + _crop(Dz, 1, 2)
           + c["a"] * (_crop(DxDy, 0) + _crop(DxDz, 1) + _crop(DyDz, 2))
           + c["b"] * DxDyDz)
    if boundary is None:
        out = out + c["kappa"] * U
    for side in (0, 1):
        if prob.face(2, side) == "S":
            _add_sommerfeld_rows(prob, P, out, side)
    return out


def _inplane(Pl: np.ndarray):
    """D_x, D_y, D_xD_y of one ghost-padded z-plane (shape (my+2, mx+2))."""
    Dx = _second_difference(Pl, 1)
    Dy = _second_difference(Pl, 0)
    DxDy = _second_difference(Dx, 0)
    return Dx[1:-1, :], Dy[:, 1:-1], DxDy


def _add_sommerfeld_rows(prob: Problem, P: np.ndarray, out: np.ndarray, side: int):
    """Add G1 U_1 + G0 U_0 to the rows of the z face `side` (Eq. 3DDISCS).

    U_0 is the face plane, U_1 the next plane inward (mirrored for the top face).
    """
    s = sommerfeld_coefficients(prob.k, prob.h)
    if side == 0:
        P0, P1, row = P[1], P[2], 0
    else:
        P0, P1, row = P[-2], P[-3], out.shape[0] - 1
    Dx1, Dy1, DxDy1 = _inplane(P1)
    Dx0, Dy0, _ = _inplane(P0)
    U1 = P1[1:-1, 1:-1]
    U0 = P0[1:-1, 1:-1]
    G1U1 = s["e2"] * s["mu3"] * (s["p"] * (Dx1 + Dy1) + DxDy1 / (30 * s["mu3"]) + s["q"] * U1)
    G0U0 = s["e1"] * s["mu3"] * (s["r"] * U0 - s["s"] * (Dx0 + Dy0))
    out[row] += G1U1 + G0U0


# ======================================================================================
# Right-hand side (Eq. scheme right side, Eq. 3DN and Eq. 3DDISCS data terms)
# ======================================================================================

def _face_derivs(prob: Problem, src, axis: int, side: int):
    """Derivatives of f on a face in the face's inward normal coordinate.

    Returns d(nn, t1, t2) on the face plane: nn derivatives along the inward normal,
    t1/t2 along the two tangential axes (in x, y, z order).  The high face uses
    n = 1 - x_axis, so odd normal derivatives change sign.
    """
    Z, Y, X = prob.coords()
    coords = [X, Y, Z]
    npax = 2 - axis
    idx = 0 if side == 0 else prob.shape[npax] - 1
    face_coords = [np.take(cc, [idx], axis=npax) if cc.shape[npax] > 1 else cc for cc in coords]
    tang = [a for a in range(3) if a != axis]
    sign = 1.0 if side == 0 else -1.0

    def d(nn, t1, t2):
        orders = [0, 0, 0]
        orders[axis] = nn
        orders[tang[0]] = t1
        orders[tang[1]] = t2
        val = src.deriv(orders[0], orders[1], orders[2], face_coords[0], face_coords[1],
                        face_coords[2])
        shape = list(prob.shape)
        shape[npax] = 1
        return np.broadcast_to(val, shape) * sign ** nn

    return d, npax, idx


def rhs(prob: Problem, src, noise=None) -> np.ndarray:
    """Right side F of A U = F for a source f given with exact derivatives.

    Interior (Eq. scheme, h^2-scaled, mixed-derivative reading as in the header):
        F = h^2 [ cf f + (h^2/12)(1 - k^2h^2/30) lap f + (h^4/360) sum f_aaaa
                  + (h^4/90) sum_{a<b} f_aabb ]
    A noise field eta (no derivatives) enters as h^2 cf eta.
    Neumann face (homogeneous, Eq. 3DN): F -= D_N on the face rows with
        D_N = -(h^3/3)(1 - h^2k^2/20) f_n - (h^5/60) f_nnn - (7h^5/180)(f_ntt + f_nss).
    Sommerfeld-like face (Eq. 3DDISCS): F -= D_S with fbar = e^{ik n} f,
        Fbar = (h^2/6 + k^2h^4/45) fbar_n - (ikh^4/90) fbar_nn
               + (h^4/120)(fbar_nnn - fbar_ntt - fbar_nss),
        D_S = -e^{ikh} mu3 [ 2h Fbar + mu1 (h^5/3)(fbar_ntt + fbar_nss) ].
    """
    h, k = prob.h, prob.k
    c = scheme_coefficients(k, h)
    Z, Y, X = prob.coords()
    d = lambda a, b, cc: src.deriv(a, b, cc, X, Y, Z)
    f = d(0, 0, 0)
    lap = d(2, 0, 0) + d(0, 2, 0) + d(0, 0, 2)
    pure4 = d(4, 0, 0) + d(0, 4, 0) + d(0, 0, 4)
    mixed4 = d(2, 2, 0) + d(2, 0, 2) + d(0, 2, 2)
    F = h * h * (c["cf"] * f + (h * h / 12) * (1 - (k * h) ** 2 / 30) * lap
                 + (h ** 4 / 360) * pure4 + (h ** 4 / 90) * mixed4)
    F = np.broadcast_to(F, prob.shape).astype(np.complex128).copy()
    if noise is not None:
        F += h * h * c["cf"] * noise
    for axis in range(3):
        for side in (0, 1):
            kind = prob.face(axis, side)
            if kind == "D":
                continue
            fd, npax, idx = _face_derivs(prob, src, axis, side)
            sl = [slice(None)] * 3
            sl[npax] = slice(idx, idx + 1)
            if kind == "N":
                DN = (-(h ** 3 / 3) * (1 - (h * k) ** 2 / 20) * fd(1, 0, 0)
                      - (h ** 5 / 60) * fd(3, 0, 0)
                      - (7 * h ** 5 / 180) * (fd(1, 2, 0) + fd(1, 0, 2)))
                F[tuple(sl)] -= DN
            else:
                F[tuple(sl)] -= _sommerfeld_data(prob, fd)
    return F


def _sommerfeld_data(prob: Problem, fd):
    """D_S of Eq. 3DDISCS from derivatives of f in the inward normal coordinate."""
    h, k = prob.h, prob.k
    ik = 1j * k
    s = sommerfeld_coefficients(k, h)
    f0, fn, fnn, fnnn = fd(0, 0, 0), fd(1, 0, 0), fd(2, 0, 0), fd(3, 0, 0)
    ftt, fss = fd(0, 2, 0), fd(0, 0, 2)
    fntt, fnss = fd(1, 2, 0), fd(1, 0, 2)
    # fbar = exp(ik n) f at n = 0, derivatives by the product rule
    fb_n = ik * f0 + fn
    fb_nn = ik * ik * f0 + 2 * ik * fn + fnn
    fb_nnn = ik ** 3 * f0 + 3 * ik * ik * fn + 3 * ik * fnn + fnnn
    fb_ntt = ik * ftt + fntt
    fb_nss = ik * fss + fnss
    Fbar = ((h * h / 6 + k * k * h ** 4 / 45) * fb_n - (ik * h ** 4 / 90) * fb_nn
            + (h ** 4 / 120) * (fb_nnn - fb_ntt - fb_nss))
    return -s["e1"] * s["mu3"] * (2 * h * Fbar + s["mu1"] * (h ** 5 / 3) * (fb_ntt + fb_nss))


def lift_dirichlet(prob: Problem, F: np.ndarray, boundary) -> np.ndarray:
    """Move known inhomogeneous Dirichlet face values into the right side.

    boundary: {(axis, side): values on the ghost layer}.  Returns F - A(0; boundary),
    i.e. subtracts the boundary nodes' contribution to the neighbouring rows.
    """
    return F - apply_A(prob, np.zeros(prob.shape, dtype=np.complex128), boundary)


# ======================================================================================
# The second-order preconditioner A_p and its direct inverse (Eq. 3DAP)
# ======================================================================================

def axis_matrix(prob: Problem, axis: int) -> np.ndarray:
    """1D second-order matrix of one axis, Eq. 3DAP.

    x, y: A^0 = Lambda^beta - 2I; z: Lambda^beta - (2 - k^2h^2) I + D^alpha.
    beta = 1 at a Neumann or Sommerfeld-like end (corner entry 2), alpha = 2ikh at a
    Sommerfeld-like end.
    """
    m = prob.dims[axis]
    T = np.zeros((m, m), dtype=np.complex128)
    for i in range(m):
        T[i, i] = -2.0
        if i > 0:
            T[i, i - 1] = 1.0
        if i < m - 1:
            T[i, i + 1] = 1.0
    lo, hi = prob.face(axis, 0), prob.face(axis, 1)
    if lo in "NS" and m > 1:
        T[0, 1] = 2.0
    if hi in "NS" and m > 1:
        T[m - 1, m - 2] = 2.0
    if axis == 2:
        T += (prob.k * prob.h) ** 2 * np.eye(m)
        if lo == "S":
            T[0, 0] += 2j * prob.k * prob.h
        if hi == "S":
            T[m - 1, m - 1] += 2j * prob.k * prob.h
    return T


def apply_Ap(prob: Problem, U: np.ndarray) -> np.ndarray:
    """A_p U = (T_x (+) T_y (+) T_z) U, the 7-point operator of Eq. 3DAP (Sommerfeld-like
    faces on x or y: on the exchanged problem)."""
    if prob.s_axis in (0, 1):
        return exchange(apply_Ap(prob.exchanged(), exchange(U, prob.s_axis)), prob.s_axis)
    Tx, Ty, Tz = (axis_matrix(prob, a) for a in range(3))
    return (np.einsum("xi,zyi->zyx", Tx, U) + np.einsum("yi,zix->zyx", Ty, U)
            + np.einsum("zi,iyx->zyx", Tz, U))


class Preconditioner:
    """Direct solve of A_p U = Y by separation of variables (Section 3.3).

    x and y: eigen-decomposition T = V diag(lam) V^{-1} of the real 1D matrices (LAPACK
    eigensolver, inverse by LU).  z: for each pair of x/y modes (p, q) a tridiagonal
    system (T_z + (lam_p + lam_q) I) u = y, solved by LAPACK's pivoted zgtsv.
    """

    def __init__(self, prob: Problem):
        self.prob = prob
        # Sommerfeld-like faces on x or y: the preconditioner of the exchanged problem
        self.inner = Preconditioner(prob.exchanged()) if prob.s_axis in (0, 1) else None
        if self.inner is not None:
            return
        self.lam, self.V, self.W = [], [], []
        for axis in (0, 1):
            T = axis_matrix(prob, axis).real
            lam, V = np.linalg.eig(T)
            order = np.argsort(lam.real)
            lam, V = lam[order].real, V[:, order].real
            self.lam.append(lam)
            self.V.append(V)
            self.W.append(np.linalg.inv(V))
        Tz = axis_matrix(prob, 2)
        self.dl = np.diag(Tz, -1).copy()
        self.du = np.diag(Tz, 1).copy()
        self.d = np.diag(Tz).copy()

    def __call__(self, Y: np.ndarray) -> np.ndarray:
        if self.inner is not None:
            return exchange(self.inner(exchange(np.asarray(Y, dtype=np.complex128), self.prob.s_axis)),
                            self.prob.s_axis)
        Wx, Wy = self.W
        Vx, Vy = self.V
        lx, ly = self.lam
        Y = np.asarray(Y, dtype=np.complex128)
        Yh = Y @ Wx.T          # Yh[z, y, p] = sum_x Wx[p, x] Y[z, y, x]
        Yh = Wy @ Yh           # Yh[z, q, p] = sum_y Wy[q, y] Yh[z, y, p]
        Uh = np.empty_like(Yh)
        mz = Yh.shape[0]
        for q in range(Yh.shape[1]):
            for p in range(Yh.shape[2]):
                sigma = lx[p] + ly[q]
                if mz == 1:
                    Uh[0, q, p] = Yh[0, q, p] / (self.d[0] + sigma)
                    continue
                _, _, _, x, info = lapack.zgtsv(self.dl, self.d + sigma, self.du,
                                                Yh[:, q, p].copy())
                if info != 0:
                    raise np.linalg.LinAlgError(f"singular z-line ({p},{q})")
                Uh[:, q, p] = x
        U = Vy @ Uh            # U[z, y, p] = sum_q Vy[y, q] Uh[z, q, p]
        return U @ Vx.T        # U[z, y, x] = sum_p Vx[x, p] U[z, y, p]


# ======================================================================================
# Krylov solvers: right-preconditioned GMRES (Eq. AAP) and SKS (Algorithm 1)
# ======================================================================================

def _dot(a, b):
    return np.vdot(a.ravel(), b.ravel())


def _norm(a):
    return float(np.linalg.norm(a.ravel()))


def gmres(A, M, F, tol=1e-10, restart=20, maxit=200, U0=None, flexible=False):
    """Restarted right-preconditioned GMRES on A M^{-1} Y = F, U = M^{-1} Y (Eq. AAP).

    Arnoldi by modified Gram-Schmidt, Givens rotations on the Hessenberg matrix.  An
    inner cycle stops when the residual estimate |g_{j+1}| <= tol ||F||; the solution is
    then formed and accepted only if the true residual ||F - A U|| / ||F|| <= tol,
    otherwise the method restarts from it.  `flexible` keeps Z_j = M^{-1} v_j (FGMRES);
    otherwise U += M^{-1}(V y).  Returns U and a dict with the iteration count, the
    true relative residual and the history of residual estimates.
    """
    U = np.zeros_like(F) if U0 is None else U0.copy()
    nF = _norm(F)
    if nF == 0:
        return U, dict(iters=0, relres=0.0, converged=True, history=[0.0])
    r = F - A(U)
    beta = _norm(r)
    hist = [beta / nF]
    iters = 0
    converged = beta / nF <= tol
    while not converged and iters < maxit:
        V = [r / beta]
        Z = []
        H = np.zeros((restart + 1, restart), dtype=np.complex128)
        cs = np.zeros(restart, dtype=np.complex128)
        sn = np.zeros(restart, dtype=np.complex128)
        g = np.zeros(restart + 1, dtype=np.complex128)
        g[0] = beta
        j_used = 0
        for j in range(restart):
            z = M(V[j])
            if flexible:
                Z.append(z)
            w = A(z)
            for i in range(j + 1):
                H[i, j] = _dot(V[i], w)
                w = w - H[i, j] * V[i]
            hn = _norm(w)
            H[j + 1, j] = hn
            # apply previous rotations to the new column
            for i in range(j):
                t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
                H[i + 1, j] = -np.conj(sn[i]) * H[i, j] + cs[i] * H[i + 1, j]
                H[i, j] = t
            a, b = H[j, j], H[j + 1, j]
            den = np.sqrt(abs(a) ** 2 + abs(b) ** 2)
            if den == 0:
                cs[j], sn[j] = 1.0, 0.0
            else:
                cs[j] = abs(a) / den if a != 0 else 0.0
                sn[j] = (a / abs(a)) * np.conj(b) / den if a != 0 else 1.0
            H[j, j] = cs[j] * a + sn[j] * b
            H[j + 1, j] = 0.0
            g[j + 1] = -np.conj(sn[j]) * g[j]
            g[j] = cs[j] * g[j]
            iters += 1
            j_used = j + 1
            hist.append(abs(g[j + 1]) / nF)
            if abs(g[j + 1]) <= tol * nF or iters >= maxit or hn == 0:
                break
            V.append(w / hn)
        y = np.linalg.solve(np.triu(H[:j_used, :j_used]), g[:j_used])
        if flexible:
            U = U + sum(y[i] * Z[i] for i in range(j_used))
        else:
            U = U + M(sum(y[i] * V[i] for i in range(j_used)))
        r = F - A(U)
        beta = _norm(r)
        converged = beta / nF <= tol
        if beta == 0:
            break
    return U, dict(iters=iters, relres=beta / nF, converged=converged, history=hist)


def sks(A, M, F, tol=1e-10, maxit=100, diverge=1e3):
    """Simplified Krylov Subspace iteration, Algorithm 1.

    r_0 = F, Y = r_0, delta_0 = ||r_0||; while j < maxit and eps > tol:
    U = M^{-1} Y, w = A U, r = r_0 - w, eps = ||r|| / delta_0, Y = Y + r.
    (The printed loop test "eps < tol" is read as "eps > tol"; eps starts above tol.)
    Stops early, flagged diverged, if eps exceeds `diverge` or is not finite.
    """
    r0 = F
    Y = r0.copy()
    d0 = _norm(r0)
    eps = np.inf
    j = 1
    U = np.zeros_like(F)
    hist = []
    diverged = False
    while j < maxit + 1 and eps > tol:
        U = M(Y)
        w = A(U)
        r = r0 - w
        eps = _norm(r) / d0
        hist.append(eps)
        Y = Y + r
        j += 1
        if not np.isfinite(eps) or eps > diverge:
            diverged = True
            break
    return U, dict(iters=j - 1, relres=eps, converged=eps <= tol, diverged=diverged,
                   history=hist)


def chebyshev(A, M, F, lo, hi, tol=1e-10, maxit=100, diverge=1e3):
    """Chebyshev acceleration on A M^{-1} Y = F, U = M^{-1} Y, for a spectrum of A M^{-1} in
    the real interval [lo, hi], 0 < lo < hi (the theorem of Section 2 with the exact bounds
    of Eq. 1DEGV / Eq. 3DEGV).  With theta = (hi + lo)/2, delta = (hi - lo)/2 the residual
    after n steps is T_n((theta - A M^{-1})/delta) r_0 / T_n(theta/delta), built by the
    three-term recurrence of the Chebyshev polynomials:
        d_0 = M^{-1} r_0 / theta,  rho_0 = delta/theta;  U += d_n;  r = F - A U;
        rho_{n+1} = 1 / (2 theta/delta - rho_n),  d_{n+1} = rho_{n+1} rho_n d_n + (2 rho_{n+1}/delta) M^{-1} r.
    Stops when ||F - A U|| / ||F|| <= tol (or flags divergence like `sks`)."""
    theta, delta = 0.5 * (hi + lo), 0.5 * (hi - lo)
    nF = _norm(F)
    U = np.zeros_like(F)
    r = F.copy()
    rho = delta / theta
    d = M(r) / theta
    hist = []
    eps, it, diverged = np.inf, 0, False
    while it < maxit:
        U = U + d
        r = F - A(U)
        it += 1
        eps = _norm(r) / nF
        hist.append(eps)
        if eps <= tol:
            break
        if not np.isfinite(eps) or eps > diverge:
            diverged = True
            break
        rho_new = 1.0 / (2.0 * theta / delta - rho)
        d = rho_new * rho * d + (2.0 * rho_new / delta) * M(r)
        rho = rho_new
    return U, dict(iters=it, relres=eps, converged=eps <= tol, diverged=diverged, history=hist)


def dirichlet_ratio_bounds(prob: Problem):
    """Smallest and largest eigenvalue of A A_p^{-1} on the all-Dirichlet cube (real k).

    Both operators are diagonal on the sine modes (i, j, l): with D_a = -4 sin^2(p_a pi h / 2)
    the eigenvalue of the sixth-order operator (Eq. scheme in operator form) is
    sum D_a + a sum_{a<b} D_a D_b + b D_x D_y D_z + kappa, that of the 7-point operator
    sum D_a + k^2 h^2 (Section 3.4, Eq. 3DEGV)."""
    assert prob.faces == "DDDDDD" and prob.k.imag == 0.0
    h, k = prob.h, prob.k.real
    c = scheme_coefficients(k, h)
    D = -4.0 * np.sin(np.arange(1, prob.n + 1) * np.pi * h / 2) ** 2
    Dx, Dy, Dz = D[None, None, :], D[None, :, None], D[:, None, None]
    lam_a = (Dx + Dy + Dz) + c["a"].real * (Dx * Dy + Dx * Dz + Dy * Dz) + c["b"] * Dx * Dy * Dz + c["kappa"].real
    lam_p = (Dx + Dy + Dz) + (k * h) ** 2
    ratio = lam_a / lam_p
    return float(ratio.min()), float(ratio.max())


def psi_order(eps_h: float, eps_gh: float, gamma: float) -> float:
    """Order of the preconditioned matrix from SKS residual ratios on two grids, Eq. PSI.

    eps_h = ||r_2|| / ||r_1|| on the grid of step h, eps_gh the same on step gamma h.
    """
    return (np.log(eps_gh) - np.log(eps_h)) / np.log(gamma)


# ======================================================================================
# Dense matrices for tiny grids
# ======================================================================================

def dense_matrix(apply, shape) -> np.ndarray:
    """Assemble the matrix of a linear map by applying it to unit vectors."""
    N = int(np.prod(shape))
    M = np.zeros((N, N), dtype=np.complex128)
    e = np.zeros(N, dtype=np.complex128)
    for i in range(N):
        e[:] = 0
        e[i] = 1
        M[:, i] = apply(e.reshape(shape)).ravel()
    return M


def solve_dense(prob: Problem, F: np.ndarray) -> np.ndarray:
    """U* = A^{-1} F by dense LU (numpy.linalg.solve), for grids of a few hundred unknowns."""
    Amat = dense_matrix(lambda U: apply_A(prob, U), prob.shape)
    return np.linalg.solve(Amat, F.ravel()).reshape(prob.shape)


def solve(prob: Problem, F: np.ndarray, tol=1e-12, restart=30, maxit=500, method="gmres"):
    """Reference discrete solution of A U = F (GMRES, SKS or, on the all-Dirichlet cube,
    Chebyshev acceleration with the exact bounds, all with the direct A_p^{-1})."""
    M = Preconditioner(prob)
    A = lambda U: apply_A(prob, U)
    if method == "sks":
        return sks(A, M, F, tol=tol, maxit=maxit)
    if method == "cheb":
        lo, hi = dirichlet_ratio_bounds(prob)
        return chebyshev(A, M, F, lo, hi, tol=tol, maxit=maxit)
    return gmres(A, M, F, tol=tol, restart=restart, maxit=maxit)

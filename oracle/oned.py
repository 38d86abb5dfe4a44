"""1D sixth-order compact scheme and its second-order preconditioner (Section 2).

TEST INFRASTRUCTURE: part of the CPU oracle (used to pin the Krylov solvers against the
paper's Table 2).  Only tests/ may use it.

Dirichlet problem u'' + k^2 u = f on [0, 1], x_i = i h, h = 1/(N+1):
    d1 U_{i-1} + d2 U_i + d1 U_{i+1} = F_i,
    d1 = 1 - k^4h^4/360,  d2 = -2 + k^2h^2 - 7k^4h^4/90          (A = d1 Lambda + d2 I)
    F_i = h^2 (1 - 7k^2h^2/90) f_i - (k^2h^4/360)(f_{i-1} + f_{i+1})
          + (7h^4/90) f''_i + (h^4/360)(f''_{i-1} + f''_{i+1}).
The printed right side carries k^4 where k^2 belongs (eliminating u'''' and u^(6) with
u'' = f - k^2 u gives the k^2 form); this module uses the k^2 form.
Preconditioner (Eq. 1DAP): A_p = Lambda - (2 - k^2h^2) I.
Eigenvalues (Theorem 3): lambda^p_j = -4 sin^2(j pi h/2) + h^2k^2,
lambda_j = lambda^p_j - h^4k^4 (14 + cos(j pi h))/180.
"""
from __future__ import annotations

import numpy as np


def matrices(N: int, k: complex):
    h = 1.0 / (N + 1)
    Lam = np.diag(np.ones(N - 1), 1) + np.diag(np.ones(N - 1), -1)
    k2h2 = (k * h) ** 2
    d1 = 1 - k2h2 ** 2 / 360
    d2 = -2 + k2h2 - 7 * k2h2 ** 2 / 90
    A = d1 * Lam + d2 * np.eye(N)
    Ap = Lam - (2 - k2h2) * np.eye(N)
    return A.astype(np.complex128), Ap.astype(np.complex128), h


def rhs(N: int, k: complex, f, f2):
    """Compact right side from f and f'' sampled on x_0..x_{N+1} (callables)."""
    h = 1.0 / (N + 1)
    x = np.arange(N + 2) * h
    fv, f2v = f(x), f2(x)
    k2h2 = (k * h) ** 2
    return (h * h * (1 - 7 * k2h2 / 90) * fv[1:-1]
            - (k * k * h ** 4 / 360) * (fv[:-2] + fv[2:])
            + (7 * h ** 4 / 90) * f2v[1:-1]
            + (h ** 4 / 360) * (f2v[:-2] + f2v[2:]))


def eigenvalues(N: int, k: complex):
    """(lambda^p_j, lambda_j), j = 1..N, Theorem 3."""
    h = 1.0 / (N + 1)
    j = np.arange(1, N + 1)
    lp = -4 * np.sin(j * np.pi * h / 2) ** 2 + (h * k) ** 2
    la = lp - (h * k) ** 4 * (14 + np.cos(j * np.pi * h)) / 180
    return lp, la

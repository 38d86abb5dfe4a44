"""Analytic functions with exact derivatives, for the oracle's right-hand sides.

TEST INFRASTRUCTURE: part of the CPU oracle.  Only tests/, __graft_entry__.smoke() and
bench.py's CPU-baseline leg may use it.

The compact sixth-order right-hand side (Eq. scheme) and the face data terms (Eq. 3DN,
Eq. 3DDISCS) need derivatives of f up to fourth order.  They are supplied analytically:
every function here is a sum of separable products phi_x(x) phi_y(y) phi_z(z), and each
1D factor knows its own derivatives of any order.
"""
from __future__ import annotations

from math import comb

import numpy as np


class Fn1D:
    """A 1D function t -> phi(t) with derivatives of any order: d(order, t)."""

    def d(self, order: int, t):
        raise NotImplementedError

    def __call__(self, t):
        return self.d(0, t)


class PolyExp(Fn1D):
    """P(t) * exp(beta t) with P a polynomial (coefficients in increasing degree).

    d^n/dt^n = sum_j C(n, j) P^(j)(t) beta^(n-j) exp(beta t)  (Leibniz rule).
    """

    def __init__(self, coeffs, beta=0.0):
        self.p = np.polynomial.Polynomial(np.asarray(coeffs, dtype=np.complex128))
        self.beta = complex(beta)

    def d(self, order, t):
        t = np.asarray(t, dtype=np.float64)
        e = np.exp(self.beta * t)
        out = np.zeros(t.shape, dtype=np.complex128)
        pj = self.p
        for j in range(order + 1):
            if j > 0:
                pj = pj.deriv()
            out = out + comb(order, j) * pj(t) * self.beta ** (order - j)
        return out * e


class Sum1D(Fn1D):
    def __init__(self, *terms):
        self.terms = terms

    def d(self, order, t):
        return sum(f.d(order, t) for f in self.terms)


class Scaled1D(Fn1D):
    def __init__(self, c, f):
        self.c, self.f = complex(c), f

    def d(self, order, t):
        return self.c * self.f.d(order, t)


class Shifted1D(Fn1D):
    """The m-th derivative of another function, as a function."""

    def __init__(self, f, m):
        self.f, self.m = f, m

    def d(self, order, t):
        return self.f.d(order + self.m, t)


class Gauss1D(Fn1D):
    """exp(-(t-c)^2/(2 s^2)); d^n = (-1/s)^n He_n((t-c)/s) exp(-(t-c)^2/(2 s^2)).

    He_n are the probabilists' Hermite polynomials, He_{n+1} = u He_n - n He_{n-1}.
    """

    def __init__(self, c, s):
        self.c, self.s = float(c), float(s)

    def d(self, order, t):
        u = (np.asarray(t, dtype=np.float64) - self.c) / self.s
        he_prev, he = np.zeros_like(u), np.ones_like(u)
        for m in range(order):
            he_prev, he = he, u * he - m * he_prev
        return ((-1.0 / self.s) ** order) * he * np.exp(-0.5 * u * u) + 0j


def sin1d(a, phase=0.0):
    """sin(a t + phase) as a sum of exponentials."""
    return Sum1D(PolyExp([np.exp(1j * phase) / 2j], 1j * a),
                 PolyExp([-np.exp(-1j * phase) / 2j], -1j * a))


def cos1d(a, phase=0.0):
    """cos(a t + phase) as a sum of exponentials."""
    return Sum1D(PolyExp([np.exp(1j * phase) / 2], 1j * a), PolyExp([np.exp(-1j * phase) / 2], -1j * a))


def poly_times(coeffs, f: Fn1D):
    """P(t) * f(t) where f is a sum of PolyExp terms."""
    terms = f.terms if isinstance(f, Sum1D) else (f,)
    out = []
    for term in terms:
        assert isinstance(term, PolyExp)
        out.append(PolyExp((np.polynomial.Polynomial(coeffs) * term.p).coef, term.beta))
    return Sum1D(*out)


class Separable:
    """sum_t c_t * fx_t(x) fy_t(y) fz_t(z), with mixed partial derivatives."""

    def __init__(self, terms):
        self.terms = list(terms)   # (coef, fx, fy, fz)

    def deriv(self, a, b, c, X, Y, Z):
        """d^(a+b+c) / dx^a dy^b dz^c on broadcastable coordinate arrays."""
        out = 0
        for coef, fx, fy, fz in self.terms:
            out = out + complex(coef) * fx.d(a, X) * fy.d(b, Y) * fz.d(c, Z)
        return out

    def __call__(self, X, Y, Z):
        return self.deriv(0, 0, 0, X, Y, Z)


def helmholtz_source(u: Separable, k) -> Separable:
    """f = laplacian(u) + k^2 u for a product u = phi1(x) phi2(y) phi3(z) (Eq. problem)."""
    assert len(u.terms) == 1
    c, p1, p2, p3 = u.terms[0]
    k2 = complex(k) ** 2
    return Separable([
        (c, Shifted1D(p1, 2), p2, p3),
        (c, p1, Shifted1D(p2, 2), p3),
        (c, p1, p2, Shifted1D(p3, 2)),
        (c * k2, p1, p2, p3),
    ])


def gaussians(src) -> Separable:
    """Separable form of a helm6_inputs.GaussianSources sum."""
    terms = []
    for (cx, cy, cz), amp in zip(src.centers, src.amps):
        terms.append((amp, Gauss1D(cx, src.sigma), Gauss1D(cy, src.sigma), Gauss1D(cz, src.sigma)))
    return Separable(terms)

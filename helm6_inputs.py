"""Seeded synthetic inputs for the sixth-order compact Helmholtz solver.

This module is the one piece shared by the CUDA path's callers (tests, bench.py) and
the CPU oracle: it draws random numbers and describes workloads, and holds none of the
method's arithmetic (no scheme weights, no right-hand-side assembly, no derivatives).

Random numbers come from SplitMix64 (Steele, Lea, Flood, "Fast splittable pseudorandom
number generators", OOPSLA 2014): state_i = seed + (i+1)*0x9E3779B97F4A7C15, followed by
the published 64-bit finaliser.  Uniforms take the top 53 bits; normals use the
Box-Muller transform.

The workloads follow the paper's test problems (Section 4: manufactured solutions on the
unit cube with Dirichlet, Neumann and Sommerfeld-like faces) scaled to the sizes the
solver is benchmarked on.  Sources are Gaussians of width sigma = 2h placed at least 16h
from every face, standing in for the paper's smooth right-hand sides.
"""
from __future__ import annotations

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, count: int) -> np.ndarray:
    """Return `count` SplitMix64 outputs for the stream started at `seed` (uint64)."""
    with np.errstate(over="ignore"):
        i = np.arange(1, count + 1, dtype=np.uint64)
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + i * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform01(seed: int, count: int) -> np.ndarray:
    """Uniform doubles in [0, 1) from the top 53 bits of SplitMix64."""
    return (splitmix64(seed, count) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def standard_normal(seed: int, count: int) -> np.ndarray:
    """N(0,1) doubles by Box-Muller on consecutive uniform pairs."""
    m = (count + 1) // 2
    u = uniform01(seed, 2 * m)
    u1 = 1.0 - u[0::2]          # in (0, 1]
    u2 = u[1::2]
    r = np.sqrt(-2.0 * np.log(u1))
    z = np.empty(2 * m)
    z[0::2] = r * np.cos(2.0 * np.pi * u2)
    z[1::2] = r * np.sin(2.0 * np.pi * u2)
    return z[:count]


def complex_normal(seed: int, shape) -> np.ndarray:
    """Circular complex normal CN(0,1): real and imaginary parts N(0, 1/2)."""
    cnt = int(np.prod(shape))
    z = standard_normal(seed, 2 * cnt) / np.sqrt(2.0)
    return (z[0::2] + 1j * z[1::2]).reshape(shape)


# --------------------------------------------------------------------------------------
# Grid description (no arithmetic of the method: only which nodes carry unknowns)
# --------------------------------------------------------------------------------------

def axis_nodes(n: int, lo: str, hi: str) -> np.ndarray:
    """Node indices (0..n+1, h = 1/(n+1)) that carry unknowns along one axis.

    A Dirichlet face's node is known, so it is excluded; a Neumann or Sommerfeld-like
    face's node is an unknown.
    """
    start = 1 if lo == "D" else 0
    stop = n if hi == "D" else n + 1
    return np.arange(start, stop + 1)


def dims(n: int, faces: str):
    """Unknowns per axis (mx, my, mz) for faces 'x0x1y0y1z0z1' in {D,N,S}."""
    return tuple(len(axis_nodes(n, faces[2 * a], faces[2 * a + 1])) for a in range(3))


# --------------------------------------------------------------------------------------
# Gaussian point sources
# --------------------------------------------------------------------------------------

class GaussianSources:
    """Sum of isotropic Gaussians f(x) = sum_s A_s exp(-|x - c_s|^2 / (2 sigma^2)).

    centers: (S, 3) float64 coordinates (x, y, z) on grid nodes.
    amps:    (S,) complex128 amplitudes.
    sigma:   width (2h).
    """

    def __init__(self, centers, amps, sigma):
        self.centers = np.ascontiguousarray(centers, dtype=np.float64).reshape(-1, 3)
        self.amps = np.ascontiguousarray(amps, dtype=np.complex128).reshape(-1)
        self.sigma = float(sigma)

    def __len__(self):
        return len(self.amps)


def gaussian_sources(seed: int, n: int, count: int, margin_h: int = 16,
                     random_phase: bool = True) -> GaussianSources:
    """Draw `count` Gaussian sources on nodes at least `margin_h` nodes from every face."""
    h = 1.0 / (n + 1)
    lo, hi = margin_h, n + 1 - margin_h
    if hi < lo:
        lo = hi = (n + 1) // 2
    u = uniform01(seed, 4 * count).reshape(count, 4)
    idx = lo + np.minimum((u[:, :3] * (hi - lo + 1)).astype(np.int64), hi - lo)
    centers = idx * h
    if random_phase:
        amps = np.exp(2j * np.pi * u[:, 3])
    else:
        amps = np.ones(count, dtype=np.complex128)
    return GaussianSources(centers, amps, 2.0 * h)


# --------------------------------------------------------------------------------------
# Workloads (shapes of the paper's test problems at benchmark sizes)
# --------------------------------------------------------------------------------------

WORKLOADS = {
    # Dirichlet cube with a closed-form manufactured solution (oracle-scale case).
    "dirichlet_n32_k10": dict(n=32, k=10.0, faces="DDDDDD", restart=20, tol=1e-10),
    # Mixed faces: Dirichlet x, Neumann y, Sommerfeld-like z; one source + CN noise.
    "mixed_n128_k40": dict(n=128, k=40.0, faces="DDNNSS", restart=20, tol=1e-8,
                           nsrc=1, noise=1e-3),
    # Large mixed-face run: 256 interior points per side, k = 80, eight sources.
    "mixed_n256_k80": dict(n=256, k=80.0, faces="DDNNSS", restart=30, tol=1e-8,
                           nsrc=8, noise=0.0),
    "mixed_n256_k80c": dict(n=256, k=80.0 * (1 + 0.01j), faces="DDNNSS", restart=30,
                            tol=1e-8, nsrc=8, noise=0.0),
    # Mid-size run used for the learned second stage.
    "mixed_n192_k60": dict(n=192, k=60.0, faces="DDNNSS", restart=30, tol=1e-8,
                           nsrc=1, noise=1e-3),
}


# Batched workload: independent problems of uneven size, wavenumber and faces.
BATCH_SIZES = (48, 64, 96, 128, 160)


def batch_problems(seed: int = 0, count: int = 64):
    """`count` problem descriptions drawn from SplitMix64, one stream per attribute
    (seed 16 seed + 1 ... + 8): n uniform over BATCH_SIZES, Re k uniform in [5, 60] with
    Im k = 0.01 Re k, x faces and y faces each from {D, N}^2, z faces from {D, N, S}^2
    (Sommerfeld-like faces on z only), one Gaussian source drawn with seed `src_seed`."""
    u = [uniform01(16 * seed + 1 + a, count) for a in range(8)]
    out = []
    for i in range(count):
        n = BATCH_SIZES[min(int(u[0][i] * len(BATCH_SIZES)), len(BATCH_SIZES) - 1)]
        kr = 5.0 + 55.0 * float(u[1][i])
        xy = "".join("DN"[min(int(u[2 + a][i] * 2), 1)] for a in range(4))
        z = "".join("DNS"[min(int(u[6 + a][i] * 3), 2)] for a in range(2))
        out.append(dict(n=n, k=complex(kr, 0.01 * kr), faces=xy + z, src_seed=1000 * seed + 17 * i + 5))
    return out

"""The large workloads at full size, in the configuration bench.py times.

256 x 258 x 258 = 17,040,384 unknowns, k = 80 and k = 80 (1 + 0.01 i), Dirichlet x faces,
Neumann y faces, Sommerfeld-like z faces, eight Gaussian sources of unit modulus and random
phase (the seed of bench.py's rank 0), solved through the C-ABI by MIXED FGMRES(30) to a
relative residual of 1e-8, the Krylov basis resolved by AUTO to FP16 at this size.  The
oracle's own solve at this size would take hours on the host, so the solution is checked
through what the oracle computes in seconds here:

* the right side assembled on the GPU equals the oracle's assembly (relative max 1e-12);
* the true relative residual ||F - A U|| / ||F|| of the GPU solution, recomputed on the host
  with the oracle's FP64 operator, is at most 1e-8 (times 1.05 for the two evaluation
  orders of a residual that has cancelled eight digits);
* the residual the library reports agrees with that recomputation (relative 1e-3).

The solution itself is compared with the oracle's (test_full_size_solution_matches_the_oracle,
marked slow: minutes of host time): the oracle's FP64 GMRES(30), with its own operator and
preconditioner, continues from the GPU's solution until its true relative residual is
1e-10, which pins the discrete solution U* to far better than the tolerance below whatever
the starting guess; the GPU's solution must lie within 1e-6 relative L2 of it.  The
128 x 130 x 130 mixed workload is compared with the oracle's own solve from zero.
"""
import time

import numpy as np
import pytest

import helm6_inputs as inputs
import oracle as O

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

SRC_SEED = 1000  # bench.py's rank-0 source seed


@pytest.fixture(scope="module")
def H():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1212_1397_gb300 import build, helm6
    build.build()
    return helm6


def relmax(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


@pytest.mark.parametrize("workload", ["mixed_n256_k80", "mixed_n256_k80c"])
def test_full_size_workload(H, workload):
    cfg = inputs.WORKLOADS[workload]
    n, k, faces, m, tol = cfg["n"], cfg["k"], cfg["faces"], cfg["restart"], cfg["tol"]
    src = inputs.gaussian_sources(SRC_SEED, n, cfg["nsrc"])
    with H.Solver(n, k, faces, precision=H.MIXED, method=H.FGMRES, max_restart=m) as s:
        assert s.basis == H.BASIS_F16
        F = s.rhs_gaussians(src)
        u, st = s.solve(F, tol=tol, restart=m, maxit=1000)
        Fg = F.cpu().numpy()
        U = u.cpu().numpy()
    assert st["rc"] == 0, st["status"]
    prob = O.Problem(n, k, faces)
    assert U.shape == prob.shape
    Fo = O.rhs(prob, O.sources.gaussians(src))
    assert relmax(Fg, Fo) < 1e-12
    rel = float(np.linalg.norm(Fo - O.apply_A(prob, U)) / np.linalg.norm(Fo))
    assert rel <= 1.05 * tol, rel
    assert abs(rel - st["relres"]) <= 1e-3 * rel, (rel, st["relres"])


def rel2(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.slow
def test_full_size_solution_matches_the_oracle(H, capsys):
    """256^3, k = 80: the GPU's mixed-precision solution (relative residual 1e-8) against the
    oracle's FP64 solution (relative residual 1e-10): relative L2 below 1e-6."""
    cfg = inputs.WORKLOADS["mixed_n256_k80"]
    n, k, faces, m, tol = cfg["n"], cfg["k"], cfg["faces"], cfg["restart"], cfg["tol"]
    src = inputs.gaussian_sources(SRC_SEED, n, cfg["nsrc"])
    with H.Solver(n, k, faces, precision=H.MIXED, method=H.FGMRES, max_restart=m) as s:
        F = s.rhs_gaussians(src)
        u, st = s.solve(F, tol=tol, restart=m, maxit=1000)
        U = u.cpu().numpy()
    assert st["rc"] == 0, st["status"]
    prob = O.Problem(n, k, faces)
    Fo = O.rhs(prob, O.sources.gaussians(src))
    t0 = time.perf_counter()
    M = O.Preconditioner(prob)
    Uo, info = O.gmres(lambda v: O.apply_A(prob, v), M, Fo, tol=1e-10, restart=30, maxit=600, U0=U)
    t1 = time.perf_counter()
    assert info["converged"], info["relres"]
    err = rel2(U, Uo)
    with capsys.disabled():
        print(f"\nfull-size oracle parity mixed_n256_k80: rel-L2(GPU mixed, oracle) = {err:.3e}; oracle "
              f"continued {info['iters']} iterations to {info['relres']:.2e} in {t1 - t0:.0f} s")
    assert err < 1e-6, err


def test_mixed_n128_solution_matches_the_oracle(H, capsys):
    """128 x 130 x 130, k = 40, one Gaussian source plus 1e-3 complex normal noise (the
    mixed workload of the GMRES-versus-SKS comparison, seeds of bench.py's rank 0): the
    GPU's mixed FGMRES(20) solution at relative residual 1e-8 against the oracle's GMRES(20)
    solve from zero to 1e-10."""
    cfg = inputs.WORKLOADS["mixed_n128_k40"]
    n, k, faces, m, tol = cfg["n"], cfg["k"], cfg["faces"], cfg["restart"], cfg["tol"]
    src = inputs.gaussian_sources(SRC_SEED, n, cfg["nsrc"])
    prob = O.Problem(n, k, faces)
    eta = cfg["noise"] * inputs.complex_normal(2000, prob.shape)
    Fo = O.rhs(prob, O.sources.gaussians(src), noise=eta)
    with H.Solver(n, k, faces, precision=H.MIXED, method=H.FGMRES, max_restart=m) as s:
        F = s.rhs_gaussians(src, noise=torch.from_numpy(eta).cuda())
        assert relmax(F.cpu().numpy(), Fo) < 1e-12
        u, st = s.solve(F, tol=tol, restart=m, maxit=2000)
        U = u.cpu().numpy()
    assert st["rc"] == 0, st["status"]
    t0 = time.perf_counter()
    Uo, info = O.solve(prob, Fo, tol=1e-10, restart=m, maxit=3000)
    t1 = time.perf_counter()
    assert info["converged"], info["relres"]
    err = rel2(U, Uo)
    with capsys.disabled():
        print(f"\noracle parity mixed_n128_k40: rel-L2(GPU mixed, oracle) = {err:.3e}; GPU {st['iters']} "
              f"iterations, oracle {info['iters']} iterations in {t1 - t0:.0f} s")
    assert err < 1e-6, err

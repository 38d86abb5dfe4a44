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

The solution itself is compared with the oracle's element by element at smaller sizes
(test_gpu_parity.py, test_gpu_basis16.py).
"""
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

"""MIXED FGMRES with the Krylov basis stored in FP16 (HELM6_BASIS_F16), through the C-ABI.

Only the storage of V_0..V_m changes (FP16 holding a power of two times each unit vector;
the arithmetic stays FP32 with FP64 block sums).  The FP64 refinement around the inner
solves still drives the true residual to the requested tolerance, so the bar is the mixed
path's: relative residual <= 1e-8 and the oracle's solution within 1e-6 (relative L2).
Cases cover an even unknown count (two points per thread in the Gram-Schmidt passes) and
odd ones (one point), more than 16 basis vectors (two chunks of the reduction pass), graph
replay, and the iteration count against the FP32 basis.
"""
import numpy as np
import pytest

import helm6_inputs as inputs
import oracle as O

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def H():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1212_1397_gb300 import build, helm6
    build.build()
    return helm6


def rel2(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _problem(n, k, faces, seed, nsrc=2):
    prob = O.Problem(n, k, faces)
    src = inputs.gaussian_sources(seed, n, nsrc, margin_h=3)
    return prob, O.rhs(prob, O.sources.gaussians(src))


@pytest.mark.parametrize("n,k,faces,restart", [(45, 14.0, "DDNNSS", 30),      # N odd
                                               (44, 13.0 + 0.2j, "NNDDSS", 30),  # N even
                                               (30, 9.0, "DNNDSN", 20),
                                               (17, 6.5 + 0.1j, "NNNNNN", 8)])
def test_f16_basis_matches_oracle(H, n, k, faces, restart):
    prob, F = _problem(n, k, faces, 300 + n)
    Uref, _ = O.solve(prob, F, tol=1e-13)
    with H.Solver(n, k, faces, precision=H.MIXED, method=H.FGMRES, max_restart=restart,
                  basis=H.BASIS_F16) as s:
        u, st = s.solve(torch.from_numpy(F).cuda(), tol=1e-8, restart=restart, maxit=600)
    assert st["rc"] == 0 and st["relres"] <= 1e-8, st["status"]
    assert rel2(u.cpu().numpy(), Uref) < 1e-6


def test_f16_basis_iterations_near_f32(H):
    """Rounding each basis vector once to FP16 (unit roundoff 2^-11) costs few iterations:
    every inner cycle of this problem reduces the residual by far less than 2^-11."""
    n, k, faces = 64, 22.0 + 0.22j, "DDNNSS"
    _, F = _problem(n, k, faces, 11, nsrc=4)
    its = {}
    for basis in ("BASIS_F32", "BASIS_F16"):
        with H.Solver(n, k, faces, precision=H.MIXED, method=H.FGMRES, max_restart=30,
                      basis=getattr(H, basis)) as s:
            _, st = s.solve(torch.from_numpy(F).cuda(), tol=1e-8, restart=30, maxit=2000)
        assert st["rc"] == 0
        its[basis] = st["iters"]
    assert its["BASIS_F16"] <= 1.15 * its["BASIS_F32"] + 2, its


def test_f16_basis_graph_replay_equals_eager(H):
    n, k, faces = 26, 8.0 + 0.08j, "NDDNSS"
    _, F = _problem(n, k, faces, 5)
    out = {}
    for graphs in (False, True):
        with H.Solver(n, k, faces, precision=H.MIXED, method=H.FGMRES, max_restart=12,
                      stream=torch.cuda.Stream(), use_graphs=graphs, basis=H.BASIS_F16) as s:
            Fd = torch.from_numpy(F).cuda()
            torch.cuda.synchronize()
            u, st = s.solve(Fd, tol=1e-9, restart=12, maxit=400)
            out[graphs] = (u.cpu().numpy(), st["iters"])
    assert out[False][1] == out[True][1]
    assert np.array_equal(out[False][0], out[True][0])


def test_basis_option_is_checked(H):
    with pytest.raises(H.Helm6Error):
        H.Solver(8, 3.0, "DDDDDD", precision=H.FP64, method=H.GMRES, basis=H.BASIS_F16)
    with pytest.raises(H.Helm6Error):
        H.Solver(8, 3.0, "DDDDDD", precision=H.MIXED, method=H.FGMRES, basis=3)


def test_auto_basis_resolution(H):
    """AUTO stores the basis in FP16 from 2^23 unknowns (n = 203: 203 x 205 x 205 with
    Neumann y and z faces), in FP32 below; FP64 and non-Krylov contexts report AUTO."""
    with H.Solver(203, 20.0, "DDNNNN", precision=H.MIXED, method=H.FGMRES, max_restart=4) as s:
        assert s.dims[0] * s.dims[1] * s.dims[2] >= 1 << 23
        assert s.basis == H.BASIS_F16
    with H.Solver(200, 20.0, "DDDDDD", precision=H.MIXED, method=H.FGMRES, max_restart=4) as s:
        assert s.basis == H.BASIS_F32
    with H.Solver(64, 20.0, "DDDDDD", precision=H.MIXED, method=H.FGMRES, basis=H.BASIS_F16) as s:
        assert s.basis == H.BASIS_F16
    with H.Solver(64, 20.0, "DDDDDD", precision=H.FP64, method=H.GMRES) as s:
        assert s.basis == H.BASIS_AUTO
    with H.Solver(64, 20.0, "DDDDDD", precision=H.MIXED, method=H.SKS) as s:
        assert s.basis == H.BASIS_AUTO


@pytest.mark.parametrize("precision,method,basis", [("MIXED", "FGMRES", "BASIS_F16"), ("MIXED", "FGMRES", "BASIS_F32"),
                                                    ("FP64", "GMRES", "BASIS_AUTO")])
def test_restart_beyond_32_vectors(H, precision, method, basis):
    """Restart 40: the reduction pass covers more than 32 basis vectors in two rounds of its
    warp groups (at most 8 vectors per group, 4 groups per round)."""
    n, k, faces = 24, 26.0, "DDNNSS"  # about 110 GMRES(40) iterations
    prob, F = _problem(n, k, faces, 77, nsrc=3)
    Uref, info = O.solve(prob, F, tol=1e-12, restart=40, maxit=1000)
    assert info["converged"]
    tol = 1e-8 if precision == "MIXED" else 1e-10
    with H.Solver(n, k, faces, precision=getattr(H, precision), method=getattr(H, method), max_restart=40,
                  basis=getattr(H, basis)) as s:
        u, st = s.solve(torch.from_numpy(F).cuda(), tol=tol, restart=40, maxit=1000)
    assert st["rc"] == 0 and st["relres"] <= tol, st["status"]
    assert st["iters"] > 32  # the last cycle reached more than 32 vectors
    assert rel2(u.cpu().numpy(), Uref) < (1e-6 if precision == "MIXED" else 1e-8)

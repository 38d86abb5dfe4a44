"""GPU parity: the CUDA path (through the C-ABI) against the CPU oracle.

Sizes span several stencil tiles (32 x 8 x 16) and transform tiles (64) with ragged tails.
Tolerances: FP64 stencil 1e-12 relative (max-norm); FP64 preconditioner 1e-10 (its z-line
solves amplify rounding by the line's condition number); FP32 stencil 2e-6; MIXED
preconditioner 1e-4 (BF16-split transforms, FP32 accumulation); converged solutions
1e-6 relative L2 at relative residual 1e-8 (the MIXED target) and 1e-8 at 1e-10 (FP64).
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


def relmax(a, b):
    return np.abs(a - b).max() / np.abs(b).max()


def rel2(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


CASES = [(37, 9.0 + 0.3j, "DDNNSS"), (33, 12.0, "DDDDDD"), (21, 7.5, "NNDNNS"),
         (19, 6.0 + 1.0j, "NDNNDN"), (40, 15.0, "DNDDSD"), (5, 3.0, "NNNNNN"), (1, 2.0, "DDDDDD")]


@pytest.mark.parametrize("n,k,faces", CASES)
def test_apply_A_fp64(H, n, k, faces):
    prob = O.Problem(n, k, faces)
    x = inputs.complex_normal(100 + n, prob.shape)
    with H.Solver(n, k, faces, precision=H.FP64) as s:
        assert s.shape == prob.shape
        y = s.apply_A(torch.from_numpy(x).cuda()).cpu().numpy()
    assert relmax(y, O.apply_A(prob, x)) < 1e-12


@pytest.mark.parametrize("n,k,faces", CASES[:4])
def test_apply_A_fp32(H, n, k, faces):
    prob = O.Problem(n, k, faces)
    x = inputs.complex_normal(200 + n, prob.shape)
    with H.Solver(n, k, faces, precision=H.MIXED, method=H.FGMRES) as s:
        y = s.apply_A(torch.from_numpy(x).cuda()).cpu().numpy()
    assert relmax(y, O.apply_A(prob, x)) < 2e-6


@pytest.mark.parametrize("n,k,faces", CASES)
def test_apply_Pinv_fp64(H, n, k, faces):
    prob = O.Problem(n, k, faces)
    x = inputs.complex_normal(300 + n, prob.shape)
    with H.Solver(n, k, faces, precision=H.FP64) as s:
        y = s.apply_Pinv(torch.from_numpy(x).cuda()).cpu().numpy()
    assert relmax(y, O.Preconditioner(prob)(x)) < 1e-10


@pytest.mark.parametrize("n,k,faces", CASES[:5])
def test_apply_Pinv_mixed(H, n, k, faces):
    prob = O.Problem(n, k, faces)
    x = inputs.complex_normal(400 + n, prob.shape)
    with H.Solver(n, k, faces, precision=H.MIXED, method=H.FGMRES) as s:
        y = s.apply_Pinv(torch.from_numpy(x).cuda()).cpu().numpy()
    ref = O.Preconditioner(prob)(x)
    assert rel2(y, ref) < 1e-4


@pytest.mark.parametrize("n,faces", [(257, "DDDDDD"), (256, "NNNNDD"), (300, "DDDDDD")])
def test_apply_Pinv_mixed_long_axes(H, n, faces):
    """Axes longer than 256 points: up to 288 the tensor-core transform computes 256 output
    columns and an FP32 tail kernel the rest (257 and 258 points here); beyond, the
    columns are split into two tensor-core groups (300 points)."""
    k = 30.0 + 0.3j
    prob = O.Problem(n, k, faces)
    x = inputs.complex_normal(401, prob.shape)
    with H.Solver(n, k, faces, precision=H.MIXED, method=H.FGMRES) as s:
        y = s.apply_Pinv(torch.from_numpy(x).cuda()).cpu().numpy()
    ref = O.Preconditioner(prob)(x)
    assert rel2(y, ref) < 1e-4


@pytest.mark.parametrize("n,k,faces", [(37, 9.0 + 0.3j, "DDNNSS"), (30, 11.0, "NNNNNN"),
                                       (26, 8.0, "DNNDSN")])
def test_rhs_gaussians(H, n, k, faces):
    prob = O.Problem(n, k, faces)
    # margin 2 nodes: sources near faces exercise the face data terms
    src = inputs.gaussian_sources(7, n, 3, margin_h=2)
    noise = inputs.complex_normal(8, prob.shape)
    with H.Solver(n, k, faces) as s:
        F = s.rhs_gaussians(src, noise=torch.from_numpy(noise).cuda()).cpu().numpy()
    ref = O.rhs(prob, O.sources.gaussians(src), noise=noise)
    assert relmax(F, ref) < 1e-12


def _gauss_problem(n, k, faces, seed=3, nsrc=2):
    prob = O.Problem(n, k, faces)
    src = inputs.gaussian_sources(seed, n, nsrc, margin_h=4)
    F = O.rhs(prob, O.sources.gaussians(src))
    return prob, F


@pytest.mark.parametrize("method", ["GMRES", "FGMRES"])
def test_solve_fp64_matches_oracle(H, method):
    n, k, faces = 29, 10.0 + 0.1j, "DDNNSS"
    prob, F = _gauss_problem(n, k, faces)
    Uref, _ = O.solve(prob, F, tol=1e-13)
    with H.Solver(n, k, faces, precision=H.FP64, method=getattr(H, method), max_restart=20) as s:
        u, st = s.solve(torch.from_numpy(F).cuda(), tol=1e-10, restart=20, maxit=300)
    assert st["rc"] == 0 and st["relres"] <= 1e-10
    assert rel2(u.cpu().numpy(), Uref) < 1e-8


def test_solve_fp64_iterations_match_oracle_gmres(H):
    """Same restart length, same tolerance: iteration counts agree within one."""
    n, k, faces = 23, 8.0, "DDDDSS"
    prob, F = _gauss_problem(n, k, faces)
    _, info = O.gmres(lambda U: O.apply_A(prob, U), O.Preconditioner(prob), F, tol=1e-10,
                      restart=10, maxit=300)
    with H.Solver(n, k, faces, precision=H.FP64, method=H.GMRES, max_restart=10) as s:
        _, st = s.solve(torch.from_numpy(F).cuda(), tol=1e-10, restart=10, maxit=300)
    assert abs(st["iters"] - info["iters"]) <= 1, (st["iters"], info["iters"])


def test_solve_mixed_matches_oracle(H):
    n, k, faces = 45, 14.0, "DDNNSS"
    prob, F = _gauss_problem(n, k, faces, nsrc=3)
    Uref, _ = O.solve(prob, F, tol=1e-13)
    with H.Solver(n, k, faces, precision=H.MIXED, method=H.FGMRES, max_restart=30) as s:
        u, st = s.solve(torch.from_numpy(F).cuda(), tol=1e-8, restart=30, maxit=300)
    assert st["rc"] == 0 and st["relres"] <= 1e-8
    assert rel2(u.cpu().numpy(), Uref) < 1e-6


def test_sks_fp64_matches_oracle_count(H):
    """SKS (Algorithm 1) on the GPU takes the oracle's iteration count exactly."""
    n, k, faces = 31, 6.0, "DDDDNN"
    prob, F = _gauss_problem(n, k, faces)
    Uo, info = O.solve(prob, F, tol=1e-10, method="sks", maxit=100)
    with H.Solver(n, k, faces, precision=H.FP64, method=H.SKS) as s:
        u, st = s.solve(torch.from_numpy(F).cuda(), tol=1e-10, maxit=100)
    assert st["rc"] == 0
    assert st["iters"] == info["iters"]
    assert rel2(u.cpu().numpy(), Uo) < 1e-8


def test_sks_mixed_converges(H):
    n, k, faces = 31, 6.0, "DDNNSS"
    prob, F = _gauss_problem(n, k, faces)
    Uref, _ = O.solve(prob, F, tol=1e-13)
    with H.Solver(n, k, faces, precision=H.MIXED, method=H.SKS) as s:
        u, st = s.solve(torch.from_numpy(F).cuda(), tol=1e-8, maxit=200)
    assert st["rc"] == 0 and st["relres"] <= 1e-8
    assert rel2(u.cpu().numpy(), Uref) < 1e-6


def test_edge_cases(H):
    n, k, faces = 9, 5.0, "DDNNSS"
    prob = O.Problem(n, k, faces)
    with H.Solver(n, k, faces) as s:
        z = s.empty()
        u, st = s.solve(z, tol=1e-8, restart=10)
        assert st["rc"] == 0 and float(u.abs().max()) == 0.0
        F = torch.from_numpy(inputs.complex_normal(5, prob.shape)).cuda()
        F[0, 0, 0] = float("nan")
        _, st = s.solve(F, tol=1e-8, restart=10)
        assert st["rc"] == 4   # NONFINITE
        F = torch.from_numpy(inputs.complex_normal(5, prob.shape)).cuda()
        _, st = s.solve(F, tol=1e-14, restart=10, maxit=1)
        assert st["rc"] == 1 and st["iters"] == 1   # NOT_CONVERGED
        with pytest.raises(H.Helm6Error):
            s.solve(F, tol=1e-8, restart=100)       # restart above max_restart
    with pytest.raises(H.Helm6Error):
        H.Solver(8, 3.0, "SDDDDS")  # Sommerfeld-like faces on two axis pairs


def test_initial_guess_is_used(H):
    n, k, faces = 17, 7.0, "DDNNSS"
    prob, F = _gauss_problem(n, k, faces)
    Uref, _ = O.solve(prob, F, tol=1e-13)
    with H.Solver(n, k, faces, precision=H.FP64) as s:
        u0 = torch.from_numpy(Uref).cuda().clone()
        u, st = s.solve(torch.from_numpy(F).cuda(), u=u0, tol=1e-10, restart=10)
    assert st["iters"] == 0 and st["relres"] < 1e-10


def test_chebyshev_matches_oracle(H):
    """Chebyshev acceleration with the library's exact bounds (all-Dirichlet cube, real k):
    the oracle's iteration count (within one) and solution; the mixed variant converges to
    the same solution."""
    n, k, faces = 23, 8.0, "DDDDDD"
    prob, F = _gauss_problem(n, k, faces)
    Uref, info = O.solve(prob, F, tol=1e-10, maxit=200, method="cheb")
    lo, hi = O.dirichlet_ratio_bounds(prob)
    for prec in (H.FP64, H.MIXED):
        with H.Solver(n, k, faces, precision=prec, method=H.CHEB) as s:
            u, st = s.solve(torch.from_numpy(F).cuda(), tol=1e-10, maxit=200)
        assert st["rc"] == 0 and st["relres"] <= 1e-10
        assert rel2(u.cpu().numpy(), Uref) < 1e-7
        if prec == H.FP64:
            assert abs(st["iters"] - info["iters"]) <= 1, (st["iters"], info["iters"])
    # the same bounds given explicitly: the same iterations
    with H.Solver(n, k, faces, precision=H.FP64, method=H.CHEB, cheb_bounds=(lo, hi)) as s:
        _, st2 = s.solve(torch.from_numpy(F).cuda(), tol=1e-10, maxit=200)
    assert abs(st2["iters"] - info["iters"]) <= 1


def test_chebyshev_arguments(H):
    with pytest.raises(H.Helm6Error):  # no exact bounds for Neumann faces
        H.Solver(10, 5.0, "DDNNDD", method=H.CHEB)
    with pytest.raises(H.Helm6Error):  # complex k
        H.Solver(10, 5.0 + 1j, "DDDDDD", method=H.CHEB)
    with pytest.raises(H.Helm6Error):  # bad interval
        H.Solver(10, 5.0, "DDNNDD", method=H.CHEB, cheb_bounds=(1.5, 0.5))
    with H.Solver(10, 5.0, "DDNNDD", method=H.CHEB, cheb_bounds=(0.5, 1.5)) as s:
        assert s.dims == (10, 12, 10)

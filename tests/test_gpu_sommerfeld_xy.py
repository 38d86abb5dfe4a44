"""Sommerfeld-like faces on the x or y pair, through the C-ABI, against the CPU oracle.

The library solves such a problem as the z-face problem with that axis exchanged with z; the
caller's arrays keep their own layout.  The oracle states the same problem directly in the
caller's layout (its face rows on the exchanged problem, its right side's face terms per
axis), pinned by the face rows' truncation order and the sixth-order error decay.
Tolerances as in test_gpu_parity.py.
"""
import numpy as np
import pytest

import helm6_inputs as inputs
import oracle as O

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

CASES = [(21, 7.0 + 0.3j, "SSNNDD"), (18, 6.0, "DNSSND"), (17, 5.0 + 0.2j, "SSDDNN"), (20, 8.0, "NDSSDD")]


@pytest.fixture(scope="module")
def H():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1212_1397_gb300 import build, helm6
    build.build()
    return helm6


def relmax(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


def rel2(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("n,k,faces", CASES)
def test_dims_apply_A_and_Pinv(H, n, k, faces):
    prob = O.Problem(n, k, faces)
    x = inputs.complex_normal(500 + n, prob.shape)
    with H.Solver(n, k, faces, precision=H.FP64) as s:
        assert s.shape == prob.shape
        xd = torch.from_numpy(x).cuda()
        y = s.apply_A(xd).cpu().numpy()
        z = s.apply_Pinv(xd).cpu().numpy()
    assert relmax(y, O.apply_A(prob, x)) < 1e-12
    assert relmax(z, O.Preconditioner(prob)(x)) < 1e-10
    with H.Solver(n, k, faces, precision=H.MIXED, method=H.FGMRES) as s:
        zm = s.apply_Pinv(torch.from_numpy(x).cuda()).cpu().numpy()
    assert relmax(zm, O.Preconditioner(prob)(x)) < 1e-4


@pytest.mark.parametrize("n,k,faces", CASES[:2])
def test_rhs_gaussians(H, n, k, faces):
    prob = O.Problem(n, k, faces)
    # sources 2 nodes from the faces (the Sommerfeld-like faces' data terms) and a noise field
    # (read in the caller's layout)
    src = inputs.gaussian_sources(600 + n, n, 3, margin_h=2)
    noise = inputs.complex_normal(601 + n, prob.shape)
    with H.Solver(n, k, faces, precision=H.FP64) as s:
        F = s.rhs_gaussians(src, noise=torch.from_numpy(noise).cuda()).cpu().numpy()
    assert relmax(F, O.rhs(prob, O.sources.gaussians(src), noise=noise)) < 1e-12


@pytest.mark.parametrize("n,k,faces", CASES)
def test_solves_match_oracle(H, n, k, faces):
    prob = O.Problem(n, k, faces)
    src = inputs.gaussian_sources(700 + n, n, 2, margin_h=3)
    F = O.rhs(prob, O.sources.gaussians(src))
    Uref, info = O.solve(prob, F, tol=1e-13, restart=40, maxit=1000)
    assert info["converged"]
    with H.Solver(n, k, faces, precision=H.FP64, method=H.GMRES, max_restart=30) as s:
        u, st = s.solve(torch.from_numpy(F).cuda(), tol=1e-10, restart=30, maxit=1000)
    assert st["rc"] == 0 and rel2(u.cpu().numpy(), Uref) < 1e-8
    with H.Solver(n, k, faces, precision=H.MIXED, method=H.FGMRES, max_restart=30) as s:
        u, st = s.solve(torch.from_numpy(F).cuda(), tol=1e-8, restart=30, maxit=1000)
    assert st["rc"] == 0 and st["relres"] <= 1e-8 and rel2(u.cpu().numpy(), Uref) < 1e-6


def test_two_sommerfeld_pairs_are_rejected(H):
    with pytest.raises(H.Helm6Error):
        H.Solver(8, 3.0, "SSDDSS")

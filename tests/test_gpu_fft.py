"""The FFT-type x/y transforms of the preconditioner (Section 3.3, Eq. 3DAP: the direct solver
of A_p is "FFT-type"; Section 1: O(N^2 N_z log N) per application), through the C-ABI.

Each axis' closed-form sine/cosine eigenbasis is applied as one complex DFT per line: of the
line's odd or even extension, of length L = 2(n+1) for D-D and N-N and 4(n+1) for D-N and
N-D (FP32), or, for D-D and N-N in FP64, of length n+1 (the sine and cosine transforms
through pre- and post-processing and a prefix sum), split as
L = P * Q with P a power of two and Q = 1 or a prime with Q - 1 a power of two (Rader's
convolution).  The cases below cover every such Q the grids meet (1, 3, 5, 17, 257), the four
face pairs of an axis, both internal axes, and a problem whose Sommerfeld-like pair is on x
(the internal axes are exchanged).  The oracle's preconditioner is independent of the FFT: its
eigenbases come from LAPACK's eigensolver and its z lines from LAPACK's pivoted tridiagonal
solver.  Tolerances as for the dense path: FP64 1e-10 relative (max-norm; the z-line solves
amplify rounding by the line's condition number), FP32 1e-4 relative L2.
"""
import time

import numpy as np
import pytest

import helm6_inputs as inputs
import oracle as O
from oracle import sources as S

from test_gpu_paper_tables import source_tables
from test_oracle_pins import table_u

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


# (n, faces): the FP64 DFT lengths of the internal x and y axes in the comments (FP32: D-D and
# N-N twice as long)
FFT_CASES = [
    (1, "DNNDSS"),     # 8, 8 (P = 8)
    (2, "DDNNSS"),     # 3, 3 (Q = 3, P = 1)
    (4, "DNNDDD"),     # 20, 20 (Q = 5, P = 4)
    (15, "NNDDSN"),    # 16, 16
    (16, "DDNNSS"),    # 17, 17 (Q = 17)
    (16, "NDDNNN"),    # 68, 68 (Q = 17, P = 4)
    (31, "SSDDNN"),    # Sommerfeld-like x pair: internal x = the N-N pair, y = D-D: 32, 32
    (33, "NNDDSS"),    # 34, 34 (Q = 17, P = 2)
    (63, "DDDDSS"),    # 64, 64
    (127, "NNNNDD"),   # 128, 128
    (256, "DDNNSS"),   # 257, 257 (Q = 257): the 256 x 258 x 258 grid
]


@pytest.mark.parametrize("n,faces", FFT_CASES)
def test_fft_apply_Pinv_fp64(H, n, faces):
    k = 9.0 + 0.3j
    prob = O.Problem(n, k, faces)
    x = inputs.complex_normal(500 + n, prob.shape)
    with H.Solver(n, k, faces, precision=H.FP64) as s:
        assert s.transforms == ("fft", "fft")
        y = s.apply_Pinv(torch.from_numpy(x).cuda()).cpu().numpy()
    assert relmax(y, O.Preconditioner(prob)(x)) < 1e-10


@pytest.mark.parametrize("n,faces", [FFT_CASES[i] for i in (1, 2, 4, 5, 7, 9, 10)])
def test_fft_apply_Pinv_fp32(H, n, faces):
    """MIXED with the FFT asked for: FP32 DFTs in place of the tensor-core transforms."""
    k = 9.0 + 0.3j
    prob = O.Problem(n, k, faces)
    x = inputs.complex_normal(600 + n, prob.shape)
    with H.Solver(n, k, faces, precision=H.MIXED, method=H.FGMRES, transform="fft") as s:
        assert s.transforms == ("fft", "fft")
        y = s.apply_Pinv(torch.from_numpy(x).cuda()).cpu().numpy()
    assert rel2(y, O.Preconditioner(prob)(x)) < 1e-4


def test_transform_selection(H):
    """AUTO takes the FFT in FP64 where the length factors (n = 16: L = 17), dense where it
    does not (n = 20: L = 21 = 3 * 7); MIXED AUTO keeps the tensor-core transform while
    the axes fit it; DENSE keeps the matrices."""
    with H.Solver(16, 5.0, "DDNNSS") as s:
        assert s.transforms == ("fft", "fft")
    with H.Solver(20, 5.0, "DDNNSS") as s:
        assert s.transforms == ("dense", "dense")
    with H.Solver(18, 5.0, "DDDNSS") as s:     # x: L = 19 (no plan), y: D-N, L = 76 = 4 * 19
        assert s.transforms == ("dense", "dense")
    with H.Solver(15, 5.0, "DDDNSS") as s:     # x: 16, y: D-N 64
        assert s.transforms == ("fft", "fft")
    with H.Solver(16, 5.0, "DDNNSS", transform="dense") as s:
        assert s.transforms == ("dense", "dense")
    with H.Solver(16, 5.0, "DDNNSS", precision=H.MIXED, method=H.FGMRES) as s:
        assert s.transforms == ("tensor", "tensor")


def test_fft_and_dense_solves_agree(H):
    """The same FP64 GMRES solve with FFT and with dense transforms: the iteration counts
    match and both solutions meet the oracle's to 1e-8 (relative residual 1e-10)."""
    n, k, faces = 16, 7.0 + 0.2j, "DDNNSS"
    prob = O.Problem(n, k, faces)
    F = inputs.complex_normal(77, prob.shape)
    Uref, _ = O.solve(prob, F, tol=1e-13)
    res = {}
    for tr in ("fft", "dense"):
        with H.Solver(n, k, faces, precision=H.FP64, transform=tr) as s:
            assert s.transforms == (tr, tr)
            u, st = s.solve(torch.from_numpy(F).cuda(), tol=1e-10, restart=20, maxit=300)
        assert st["rc"] == 0 and st["relres"] <= 1e-10
        assert rel2(u.cpu().numpy(), Uref) < 1e-8
        res[tr] = st["iters"]
    assert res["fft"] == res["dense"], res


def test_fft_1024_point_axes(H, capsys):
    """h = 1/1024: 1023 x 1023 x 1025 = 1.07e9 unknowns with Sommerfeld-like z faces, k = 20,
    the corrected Table 7/8 test function; the x/y axes (1023 points) go through FP32 DFTs of
    length 2048.  MIXED SKS (Algorithm 1) to a relative residual of 1e-10; the error against the exact
    solution at the nodes is reported and must stay below 1e-6 (the sixth-order truncation error
    at this step is far smaller, so this bounds the algebraic error)."""
    n, k = 1023, 20.0
    prob = O.Problem(n, k, "DDDDSS")
    c = 1j * k / (1 - 1j * k)
    u = table_u(k, S.PolyExp([1, 0, c], -1j * k))
    src = S.helmholtz_source(u, k)
    with H.Solver(n, k, prob.faces, precision=H.MIXED, method=H.SKS) as s:
        assert s.transforms == ("fft", "fft")
        assert s.shape == prob.shape
        coef, tab = source_tables(prob, src, max(s.dims))
        F = s.rhs_separable(coef, tab)
        t0 = time.perf_counter()
        U, st = s.solve(F, tol=1e-10, maxit=100)
        torch.cuda.synchronize()
        sec = time.perf_counter() - t0
        del F
        # exact solution, one z plane at a time (the full field would be another 17 GB)
        terms = [(complex(cf), *(torch.from_numpy(np.asarray(f.d(0, prob.nodes(a) * prob.h),
                                                             dtype=np.complex128)).cuda()
                                 for a, f in enumerate((fx, fy, fz))))
                 for cf, fx, fy, fz in u.terms]
        err = 0.0
        for iz in range(U.shape[0]):
            ex = sum(cf * vz[iz] * vy[:, None] * vx[None, :] for cf, vx, vy, vz in terms)
            err = max(err, float((U[iz] - ex).abs().max()))
    with capsys.disabled():
        print(f"\n[fft 1023^2 x 1025] SKS iters {st['iters']} status {st['status']} relres {st['relres']:.2e} "
              f"solve {sec:.1f} s err {err:.3e}")
    assert st["rc"] == 0 and st["relres"] <= 1e-10
    assert err < 1e-6, err

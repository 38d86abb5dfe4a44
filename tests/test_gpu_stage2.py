"""GPU parity of the learned second preconditioner stage against oracle/cnn.py.

The network's forward pass and its mean-squared-error gradient (helm6_cnn_forward /
helm6_cnn_gradient through the C-ABI) are compared with the FP64 oracle that rounds the
same quantities to BF16 (network input, weights, hidden activations).  Both sides then
differ only by the GPU's FP32 sums, plus the rare element whose FP32 and FP64
pre-activations round to neighbouring BF16 values (one BF16 step, 2^-8 relative); the
tolerances below (relative L2 1e-3, per-layer gradient blocks 3e-3) leave room for those
and fail on any wrong tap, channel, layout or layer.  Sizes are ragged against the
32 x 4 x 2 output tiles.  The two-stage preconditioner and a solve with it attached are
checked end to end.
"""
import numpy as np
import pytest

import helm6_inputs as inputs
import oracle as O
from oracle import cnn

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


def _theta(seed, bias=0.1):
    th = cnn.init_params(inputs.standard_normal(seed, cnn.n_params()))
    o = 0
    for ci, co in zip(cnn.CHANNELS[:-1], cnn.CHANNELS[1:]):
        o += co * ci * 27
        th[o:o + co] = bias * inputs.standard_normal(seed + 1000 + o, co)
        o += co
    return th.astype(np.float32)


def _batch(seed, shape):
    return inputs.standard_normal(seed, int(np.prod(shape))).reshape(shape).astype(np.float32)


SHAPES = [(2, 5, 10, 40), (1, 3, 4, 32), (3, 4, 7, 9)]


@pytest.mark.parametrize("shape", SHAPES)
def test_forward_matches_oracle(H, shape):
    th = _theta(1)
    x = _batch(2, shape + (2,))
    with H.Trainer(*shape, th) as tr:
        y = tr.forward(torch.from_numpy(x).cuda()).cpu().numpy().astype(np.float64)
    ref = cnn.forward(th.astype(np.float64), x.astype(np.float64), bf16=True)
    assert rel2(y, ref) < 1e-3, rel2(y, ref)
    assert np.abs(y - ref).max() < 1e-2 * np.abs(ref).max()


@pytest.mark.parametrize("shape", SHAPES[:2])
def test_gradient_matches_oracle(H, shape):
    th = _theta(3)
    x = _batch(4, shape + (2,))
    t = _batch(5, shape + (2,))
    with H.Trainer(*shape, th) as tr:
        loss, g = tr.gradient(torch.from_numpy(x).cuda(), torch.from_numpy(t).cuda())
    g = g.cpu().numpy().astype(np.float64)
    lref, gref = cnn.loss_and_grad(th.astype(np.float64), x.astype(np.float64), t.astype(np.float64), bf16=True)
    assert abs(loss - lref) < 1e-5 * lref, (loss, lref)
    assert rel2(g, gref) < 1e-3, rel2(g, gref)
    o = 0
    for ci, co in zip(cnn.CHANNELS[:-1], cnn.CHANNELS[1:]):
        for size in (co * ci * 27, co):
            blk = slice(o, o + size)
            assert rel2(g[blk], gref[blk]) < 3e-3, (ci, co, size, rel2(g[blk], gref[blk]))
            o += size


def test_training_reduces_the_loss(H):
    shape = (2, 8, 8, 32)
    x = _batch(6, shape + (2,))
    # a target the network can represent: another network's output
    t = cnn.forward(_theta(7).astype(np.float64), x.astype(np.float64), bf16=True).astype(np.float32)
    xd, td = torch.from_numpy(x).cuda(), torch.from_numpy(t).cuda()
    with H.Trainer(*shape, _theta(8)) as tr:
        l0 = tr.step(xd, td, 0.0)  # lr 0: the loss of the initial parameters
        for _ in range(60):
            tr.step(xd, td, 3e-3, want_loss=False)
        l1 = tr.step(xd, td, 3e-3)
        th = tr.params()
    assert l1 < 0.5 * l0, (l0, l1)
    assert np.all(np.isfinite(th))


def _problem(n=14, k=9.0 + 0.2j, faces="DDNNSS"):
    return O.Problem(n, k, faces)


def test_stage2_matches_oracle(H):
    prob = _problem()
    th = _theta(9)
    c = 0.5
    u = inputs.complex_normal(10, prob.shape)
    with H.Solver(prob.n, prob.k, prob.faces, precision=H.MIXED, method=H.FGMRES) as s:
        s.set_cnn(th, c, H.CNN_ON)
        ud = torch.from_numpy(u).cuda()
        z = s.apply_stage2(ud).cpu().numpy()
        z1 = s.apply_Pinv(ud).cpu().numpy()
    pre = O.Preconditioner(prob)
    zr = cnn.stage2(th.astype(np.float64), c, u, pre, lambda v: O.apply_A(prob, v), bf16=True)
    zr1 = pre(u)
    # the direct part (BF16-split transforms: 1e-5) and the learned correction separately
    assert rel2(z1, zr1) < 1e-4
    assert rel2(z - z1, zr - zr1) < 3e-3, rel2(z - z1, zr - zr1)


@pytest.mark.parametrize("mode", ["CNN_ON", "CNN_AUTO"])
def test_solve_with_learned_stage_matches_oracle(H, mode):
    n, k, faces = 29, 10.0 + 0.1j, "DDNNSS"
    prob = O.Problem(n, k, faces)
    src = inputs.gaussian_sources(3, n, 2, margin_h=4)
    F = O.rhs(prob, O.sources.gaussians(src))
    Uref, _ = O.solve(prob, F, tol=1e-13)
    with H.Solver(n, k, faces, precision=H.MIXED, method=H.FGMRES, max_restart=10) as s:
        s.set_cnn(_theta(11), 0.05, getattr(H, mode))
        u, st = s.solve(torch.from_numpy(F).cuda(), tol=1e-8, restart=10, maxit=400)
    assert st["rc"] == 0 and st["relres"] <= 1e-8, st["status"]
    assert rel2(u.cpu().numpy(), Uref) < 1e-6
    if mode == "CNN_ON":
        assert st["cnn_cycles"] == st["outer"]
    else:
        assert st["cnn_cycles"] >= min(1, st["outer"] - 1)


@pytest.mark.parametrize("fault,mode", [("nan_weight", "CNN_ON"), ("overflow", "CNN_ON"),
                                        ("nan_weight", "CNN_AUTO")])
def test_failing_network_falls_back_to_the_direct_preconditioner(H, fault, mode):
    """Faults injected on the host into the network's parameters: one NaN weight (corrupt
    weights), or weights scaled by 1e30 so that the BF16/FP32 forward overflows (a failing
    network).  The learned-stage cycle's non-finite correction is discarded, the rest of the
    solve runs on A_p^-1 alone and still reaches the oracle's solution."""
    n, k, faces = 29, 10.0 + 0.1j, "DDNNSS"
    prob = O.Problem(n, k, faces)
    src = inputs.gaussian_sources(3, n, 2, margin_h=4)
    F = O.rhs(prob, O.sources.gaussians(src))
    Uref, _ = O.solve(prob, F, tol=1e-13)
    th = _theta(11)
    if fault == "nan_weight":
        th[5] = np.nan
    else:
        th = (th * np.float32(1e30)).astype(np.float32)
    with H.Solver(n, k, faces, precision=H.MIXED, method=H.FGMRES, max_restart=10) as s:
        _, st0 = s.solve(torch.from_numpy(F).cuda(), tol=1e-8, restart=10, maxit=400)
        s.set_cnn(th, 0.05, getattr(H, mode))
        u, st = s.solve(torch.from_numpy(F).cuda(), tol=1e-8, restart=10, maxit=400)
    assert st["rc"] == 0 and st["relres"] <= 1e-8, st["status"]
    assert st["cnn_fallbacks"] == 1 and st["cnn_cycles"] == 1, st
    assert np.isfinite(u.cpu().numpy()).all()
    assert rel2(u.cpu().numpy(), Uref) < 1e-6
    # the failed cycle's iterations are spent, the rest is the plain solve's work
    assert st["iters"] <= st0["iters"] + 10


def test_wavenumber_on_the_preconditioner_spectrum(H):
    """k^2 h^2 placed exactly on the spectrum of the 7-point operator (mode (1,1,1) of the
    Dirichlet cube): A_p is singular up to rounding, its z-line for that mode has a pivot at
    rounding level.  The solver must answer with a documented status, and a converged
    answer must satisfy the oracle's operator to the tolerance (A itself stays regular: its
    symbol differs from A_p's at O(h^2))."""
    n = 15
    h = 1.0 / (n + 1)
    k = float(np.sqrt(3 * 4 * np.sin(np.pi * h / 2) ** 2) / h)
    prob = O.Problem(n, k, "DDDDDD")
    F = O.rhs(prob, O.sources.gaussians(inputs.gaussian_sources(5, n, 1, margin_h=4)))
    for prec, meth in ((H.FP64, H.GMRES), (H.MIXED, H.FGMRES)):
        with H.Solver(n, k, "DDDDDD", precision=prec, method=meth, max_restart=20) as s:
            u, st = s.solve(torch.from_numpy(F).cuda(), tol=1e-8, restart=20, maxit=300)
        assert st["status"] in ("OK", "NOT_CONVERGED", "BREAKDOWN", "NONFINITE"), st["status"]
        if st["rc"] == 0:
            U = u.cpu().numpy()
            res = np.linalg.norm(F - O.apply_A(prob, U)) / np.linalg.norm(F)
            assert res <= 1.05e-8, (prec, res)


def test_learned_stage_argument_errors(H):
    th = _theta(12)
    with H.Solver(10, 5.0, "DDNNSS", precision=H.FP64, method=H.GMRES) as s:
        with pytest.raises(H.Helm6Error):
            s.set_cnn(th, 1.0)
    with H.Solver(10, 5.0, "DDNNSS", precision=H.MIXED, method=H.FGMRES) as s:
        x = s.empty()
        with pytest.raises(H.Helm6Error):
            s.apply_stage2(x)  # no network attached
        with pytest.raises(H.Helm6Error):
            s.set_cnn(th, float("nan"))
        s.set_cnn(th, 1.0)
        s.set_cnn(th, 1.0, H.CNN_OFF)
        with pytest.raises(H.Helm6Error):
            s.apply_stage2(x)


@pytest.mark.parametrize("shape", SHAPES[:2])
def test_residual_loss_gradient_matches_oracle(H, shape):
    k, h = 40.0 + 0.4j, 1.0 / 129
    th = _theta(13)
    x = _batch(14, shape + (2,))
    with H.Trainer(*shape, th) as tr:
        tr.set_residual_loss(k, h)
        xd = torch.from_numpy(x).cuda()
        loss, g = tr.gradient(xd, xd)
    g = g.cpu().numpy().astype(np.float64)
    lref, gref = cnn.residual_loss_and_grad(th.astype(np.float64), x.astype(np.float64),
                                            cnn.stencil_weights(k, h), bf16=True)
    assert abs(loss - lref) < 1e-5 * lref, (loss, lref)
    assert rel2(g, gref) < 1e-3, rel2(g, gref)


def _weights():
    import os
    from paper_1212_1397_gb300 import weights_path
    p = weights_path("stage2_kh031.npz")
    if not os.path.exists(p):
        pytest.skip("trained weights not present")
    return np.load(p)


def test_trained_network_gain(H, capsys):
    """What the trained network (weights trained on the GPU by the library's own kernels on
    kh = 0.31 workloads) gains over the direct preconditioner alone, at n = 48, k = 15 (kh =
    0.31), mixed faces: (1) the one-step residual u - A z of the preconditioner applied to a
    field u, z = A_p^-1 u alone versus the two-stage z, for u the residual of an iterate
    (the training distribution; the stage must cut it) and for u the source itself
    (reported); (2) iterations of mixed
    FGMRES(30) to 1e-8 without the stage, with it on every cycle, and in AUTO mode.  All
    three solutions must match the oracle's; the learned stage must cut the one-step
    residual; AUTO may cost at most its two probe columns over the plain solve."""
    w = _weights()
    theta, c = w["theta"], float(w["out_scale"])
    assert w["val"][-1] < 0.35  # held-out patches: residual energy left, relative to N = 0
    n, k, faces = 48, 15.0, "DDNNSS"
    prob = O.Problem(n, k, faces)
    src = inputs.gaussian_sources(1000, n, 1, margin_h=8)
    F = O.rhs(prob, O.sources.gaussians(src)) + 1e-3 * (prob.h ** 2) * inputs.complex_normal(8919, prob.shape)
    Uref, _ = O.solve(prob, F, tol=1e-12)
    Fd = torch.from_numpy(F).cuda()
    out = {}
    with H.Solver(n, k, faces, precision=H.MIXED, method=H.FGMRES, max_restart=30) as s, \
            H.Solver(n, k, faces, precision=H.FP64, method=H.GMRES, max_restart=1) as s64:
        # fields the stage was trained on: the residual of an iterate (one plain cycle)
        U1, _ = s.solve(Fd, tol=1e-12, restart=30, maxit=30)
        s.set_cnn(theta, c, H.CNN_ON)
        for name, v in (("iterate_residual", Fd - s64.apply_A(U1)), ("source", Fd)):
            u = v / v.norm()
            r1 = (u - s64.apply_A(s.apply_Pinv(u))).norm().item()
            r2 = (u - s64.apply_A(s.apply_stage2(u))).norm().item()
            out[name] = dict(direct=r1, two_stage=r2, ratio=r2 / r1)
        for mode in ("CNN_OFF", "CNN_ON", "CNN_AUTO"):
            s.set_cnn(theta, c, getattr(H, mode))
            U, st = s.solve(Fd, tol=1e-8, restart=30, maxit=600)
            assert st["rc"] == 0 and st["relres"] <= 1e-8, (mode, st["status"])
            assert rel2(U.cpu().numpy(), Uref) < 1e-6, mode
            out[mode] = dict(iters=st["iters"], cnn_cycles=st["cnn_cycles"], ms=st["t_total_ms"])
    with capsys.disabled():
        print("\nlearned stage gain:", out)
    assert out["iterate_residual"]["ratio"] < 0.8
    # AUTO's probe is 2 learned-stage columns: it may not cost more than a few iterations
    # over the direct preconditioner alone (time-to-solution is printed above)
    assert out["CNN_AUTO"]["iters"] <= out["CNN_OFF"]["iters"] + 4


def test_auto_fallback_finishes_as_one_graph(H):
    """AUTO mode in a context that runs its solves as one device-driven graph: once the probe
    (cycles 1 and 2) has decided against the learned stage, the rest of the solve is handed to
    the graph.  Iterations, cycles and the solution equal those of the host-driven AUTO solve,
    and the solution meets the oracle's."""
    w = _weights()
    theta, c = w["theta"], float(w["out_scale"])
    n, k, faces = 48, 15.0, "DDNNSS"
    prob = O.Problem(n, k, faces)
    src = inputs.gaussian_sources(1000, n, 1, margin_h=8)
    F = O.rhs(prob, O.sources.gaussians(src)) + 1e-3 * (prob.h ** 2) * inputs.complex_normal(8919, prob.shape)
    Uref, _ = O.solve(prob, F, tol=1e-12)
    Fd = torch.from_numpy(F).cuda()
    res = {}
    for ug in (False, 2):
        with H.Solver(n, k, faces, precision=H.MIXED, method=H.FGMRES, max_restart=3, use_graphs=ug) as s:
            s.set_cnn(theta, c, H.CNN_AUTO)
            U, st = s.solve(Fd, tol=1e-8, restart=3, maxit=600)
        assert st["rc"] == 0 and st["relres"] <= 1e-8, (ug, st["status"])
        assert rel2(U.cpu().numpy(), Uref) < 1e-6, ug
        res[ug] = (U.cpu().numpy(), st)
    (Uh, sh), (Ug, sg) = res[False], res[2]
    assert sh["outer"] >= 4  # the probe cycles and at least one cycle after them
    for key in ("iters", "outer", "cnn_cycles", "cnn_fallbacks"):
        assert sh[key] == sg[key], (key, sh[key], sg[key])
    assert rel2(Ug, Uh) < 1e-12

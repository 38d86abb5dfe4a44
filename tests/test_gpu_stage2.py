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
    assert st["cnn_cycles"] == st["outer"] if mode == "CNN_ON" else st["cnn_cycles"] >= min(2, st["outer"])


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

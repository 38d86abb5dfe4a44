"""Pins of the learned-stage oracle (oracle/cnn.py) against facts outside it.

* the convolution against scipy.ndimage.correlate (zero padding) channel pair by pair;
* GELU at x = +-1 against the standard normal distribution function's tabulated
  values, and its derivative against central differences;
* BF16 rounding against torch's float32 -> bfloat16 conversion and hand-picked ties;
* the two adjoint identities <conv(x), g> = <x, input_grad(g)> = <W, weight_grad(x, g)>;
* the full loss gradient against central finite differences (FP64, no rounding);
* the parameter count of the 2-16-16-16-2 network;
* the two-stage preconditioner reducing to M^-1 when every parameter is zero;
* the patch operator against the oracle's full 27-point operator on a Dirichlet cube
  (whose ghost values are zero too), its adjoint identity, and the residual-form loss
  gradient against central finite differences.
"""
import numpy as np
import pytest
import scipy.ndimage as ndi

import helm6_inputs as inputs
from oracle import cnn


def _rand(seed, shape):
    return inputs.standard_normal(seed, int(np.prod(shape))).reshape(shape)


def test_conv3d_matches_scipy_correlate():
    x = _rand(1, (2, 5, 6, 7, 3))
    W = _rand(2, (4, 3, 3, 3, 3))
    b = _rand(3, (4,))
    y = cnn.conv3d(x, W, b)
    for bi in range(2):
        for o in range(4):
            ref = b[o] + sum(ndi.correlate(x[bi, ..., c], W[o, c], mode="constant", cval=0.0) for c in range(3))
            assert np.allclose(y[bi, ..., o], ref, rtol=1e-13, atol=1e-12)


def test_gelu_values_and_derivative():
    # Phi(1) = 0.8413447460685429, Phi(-1) = 0.15865525393145707 (standard normal table)
    assert abs(cnn.gelu(np.array(1.0)) - 0.8413447460685429) < 1e-15
    assert abs(cnn.gelu(np.array(-1.0)) + 0.15865525393145707) < 1e-15
    assert cnn.gelu(np.array(0.0)) == 0.0
    assert abs(cnn.gelu(np.array(8.0)) - 8.0) < 1e-12
    xs = np.linspace(-4, 4, 33)
    e = 1e-5
    fd = (cnn.gelu(xs + e) - cnn.gelu(xs - e)) / (2 * e)
    assert np.max(np.abs(fd - cnn.gelu_grad(xs))) < 1e-9
    assert abs(cnn.gelu_grad(np.array(0.0)) - 0.5) < 1e-15


def test_bf16_rounding():
    torch = pytest.importorskip("torch")
    one = 1.0
    assert cnn.bf16_round(np.array([one + 2.0 ** -8]))[0] == 1.0          # tie -> even
    assert cnn.bf16_round(np.array([one + 3 * 2.0 ** -8]))[0] == 1.015625  # tie -> even (up)
    assert cnn.bf16_round(np.array([np.pi]))[0] == 3.140625
    assert cnn.bf16_round(np.array([-np.pi]))[0] == -3.140625
    v = _rand(7, (4096,)) * np.exp(_rand(8, (4096,)) * 5)
    ref = torch.from_numpy(v.astype(np.float32)).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(cnn.bf16_round(v), ref)


def test_conv_adjoints():
    x = _rand(11, (2, 4, 5, 6, 3))
    W = _rand(12, (2, 3, 3, 3, 3))
    g = _rand(13, (2, 4, 5, 6, 2))
    y = cnn.conv3d(x, W, np.zeros(2))
    lhs = float(np.sum(y * g))
    assert abs(lhs - float(np.sum(x * cnn.conv3d_input_grad(g, W)))) < 1e-10 * abs(lhs) + 1e-10
    assert abs(lhs - float(np.sum(W * cnn.conv3d_weight_grad(x, g)))) < 1e-10 * abs(lhs) + 1e-10


def test_loss_gradient_against_finite_differences():
    ch = (2, 3, 3, 2)
    theta = _rand(21, (cnn.n_params(ch),)) * 0.4
    x = _rand(22, (2, 3, 4, 5, 2))
    t = _rand(23, (2, 3, 4, 5, 2))
    loss, grad = cnn.loss_and_grad(theta, x, t, bf16=False, channels=ch)
    e = 1e-6
    fd = np.empty_like(theta)
    for i in range(theta.size):
        tp, tm = theta.copy(), theta.copy()
        tp[i] += e
        tm[i] -= e
        yp = cnn.forward(tp, x, False, ch)
        ym = cnn.forward(tm, x, False, ch)
        fd[i] = (np.mean((yp - t) ** 2) - np.mean((ym - t) ** 2)) / (2 * e)
    assert np.max(np.abs(fd - grad)) < 1e-7 * max(1.0, np.max(np.abs(grad)))
    assert loss > 0


def test_parameter_count():
    assert cnn.n_params() == 15602
    theta = np.arange(cnn.n_params(), dtype=np.float64)
    assert np.array_equal(cnn.pack(cnn.unpack(theta)), theta)


def test_stage2_with_zero_network_is_the_direct_preconditioner():
    from oracle import helm6_oracle as orc
    P = orc.Problem(6, 9.0 + 0.2j, "DDNNSS")
    pre = orc.Preconditioner(P)
    u = inputs.complex_normal(31, P.shape)
    z = cnn.stage2(np.zeros(cnn.n_params()), 3.0, u, pre, lambda v: orc.apply_A(P, v))
    assert np.allclose(z, pre(u), rtol=0, atol=1e-14 * np.abs(z).max())


def test_patch_operator_is_the_dirichlet_operator():
    from oracle import helm6_oracle as orc
    P = orc.Problem(7, 6.0 + 0.5j, "DDDDDD")
    U = inputs.complex_normal(41, P.shape)
    ref = orc.apply_A(P, U)
    out = cnn.patch_operator(U[None], cnn.stencil_weights(P.k, P.h))[0]
    assert np.allclose(out, ref, rtol=1e-13, atol=1e-13 * np.abs(ref).max())


def test_patch_operator_adjoint():
    w = (-5.1 + 0.2j, 0.6 - 0.1j, 0.09 + 0.03j, 0.033 - 0.01j)
    a = inputs.complex_normal(42, (2, 4, 5, 6))
    b = inputs.complex_normal(43, (2, 4, 5, 6))
    lhs = np.vdot(b, cnn.patch_operator(a, w))
    rhs = np.vdot(cnn.patch_operator(b, w, conj=True), a)
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)


def test_residual_loss_gradient_against_finite_differences():
    ch = (2, 3, 3, 2)
    w = (-5.1 + 0.2j, 0.6 - 0.1j, 0.09 + 0.03j, 0.033 - 0.01j)
    theta = _rand(51, (cnn.n_params(ch),)) * 0.4
    x = _rand(52, (2, 4, 4, 5, 2))
    loss, grad = cnn.residual_loss_and_grad(theta, x, w, bf16=False, channels=ch)

    def L(th):
        y = cnn.forward(th, x, False, ch)
        R = cnn.patch_operator(y[..., 0] + 1j * y[..., 1], w) - (x[..., 0] + 1j * x[..., 1])
        m = cnn.interior_mask(R.shape)
        return np.sum(np.abs(R[m]) ** 2) / (2 * m.sum())

    assert abs(L(theta) - loss) < 1e-14 * loss
    e = 1e-6
    fd = np.array([(L(theta + e * np.eye(theta.size)[i]) - L(theta - e * np.eye(theta.size)[i])) / (2 * e)
                   for i in range(theta.size)])
    assert np.max(np.abs(fd - grad)) < 1e-7 * max(1.0, np.max(np.abs(grad)))

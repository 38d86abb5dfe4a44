"""Plain FP64 CPU statement of the learned second preconditioner stage (test infrastructure).

TEST INFRASTRUCTURE ONLY: imported by tests/ and bench.py's CPU legs, never by the product
library, and sharing no code with the CUDA kernels.

The stage applies, after the direct second-order preconditioner M (Eq. 3DAP), a small 3D
convolutional network N to what that preconditioner leaves behind:

    z = M^-1 u + c * s * N((u - A M^-1 u) / s),   s = sqrt(mean |u - A M^-1 u|^2),

with A the sixth-order operator (Eq. scheme) and c a fixed output scale stored with the
weights.  The paper has no such stage; it is one of the three reshapings of the method
(precision, learned correction, batching) this project adds, and it lives inside flexible
GMRES, whose columns may come from any map.

Network (all arrays channel-last, [batch, z, y, x, channel], x fastest):
  * 4 layers of 3x3x3 cross-correlation with zero padding ("same" size), channels
    2 -> 16 -> 16 -> 16 -> 2, bias per output channel;
  * GELU x * Phi(x) (Phi the standard normal CDF, exact erf form) after layers 1-3;
  * channel 0 is the real part, channel 1 the imaginary part of a complex field.
Weights W[l] have shape [c_out, c_in, 3, 3, 3] (tap order dz, dy, dx); the flat parameter
vector packs, per layer in order, W (C order) then b.

Training losses.  `loss_and_grad`: mean squared error against a target (the error e~ the
stage should add).  `residual_loss_and_grad`: the residual form that makes N a local
approximate inverse of A: with X = x_0 + i x_1 the input, Y = y_0 + i y_1 the output and
A_h the interior 27-point operator of Eq. scheme on the patch with zero values outside it,

    L = sum over interior points p of |(A_h Y - X)_p|^2 / (2 * number of interior points),

interior meaning at least one point away from every face of the patch (there A_h needs no
value outside it).  Then A (c s N(t/s)) ~ t for c = 1, so z = A_p^-1 u + s N(t/s) removes
what the direct preconditioner left.

Precision model of the GPU kernels (`bf16=True`): the network input, the weights and the
activations after each GELU are rounded to BF16 (round to nearest, ties to even); sums
are exact here (FP64) and FP32 on the GPU; the last layer's output and all biases stay
in full precision.  The backward pass treats each rounding as the identity
(straight-through), uses the rounded weights and activations that the forward pass used,
and differentiates the GELU at the unrounded pre-activation.
"""
from __future__ import annotations

import numpy as np
from scipy.special import erf

CHANNELS = (2, 16, 16, 16, 2)


def n_params(channels=CHANNELS) -> int:
    """Number of scalars in the flat parameter vector (weights and biases of every layer)."""
    return sum(co * ci * 27 + co for ci, co in zip(channels[:-1], channels[1:]))


def unpack(theta: np.ndarray, channels=CHANNELS):
    """Flat vector -> [(W, b), ...] per layer (W [co, ci, 3, 3, 3], b [co])."""
    theta = np.asarray(theta, dtype=np.float64)
    out, o = [], 0
    for ci, co in zip(channels[:-1], channels[1:]):
        W = theta[o:o + co * ci * 27].reshape(co, ci, 3, 3, 3)
        o += co * ci * 27
        b = theta[o:o + co]
        o += co
        out.append((W, b))
    assert o == theta.size, (o, theta.size)
    return out


def pack(layers) -> np.ndarray:
    return np.concatenate([np.concatenate([W.ravel(), b.ravel()]) for W, b in layers])


def bf16_round(x: np.ndarray) -> np.ndarray:
    """Nearest BF16 value (8-bit significand), ties to even, of each element.

    BF16 keeps the top 16 bits of an IEEE binary32 pattern, so rounding a binary32 value
    to it is integer rounding of the pattern at bit 16.  The FP64 input is first taken to
    binary32 (the GPU rounds its FP32 results)."""
    f = np.asarray(x, dtype=np.float32)
    bits = f.view(np.uint32).astype(np.uint64)
    lower = bits & 0xFFFF
    upper = bits >> 16
    round_up = (lower > 0x8000) | ((lower == 0x8000) & ((upper & 1) == 1))
    upper = (upper + round_up.astype(np.uint64)) & 0xFFFF
    out = (upper << 16).astype(np.uint32).view(np.float32)
    # NaN and infinity keep their class (not produced by the network's finite inputs)
    out = np.where(np.isfinite(f), out, f)
    return out.astype(np.float64)


def gelu(x):
    """x Phi(x), Phi the standard normal distribution function."""
    return 0.5 * x * (1.0 + erf(x / np.sqrt(2.0)))


def gelu_grad(x):
    """d/dx x Phi(x) = Phi(x) + x phi(x)."""
    return 0.5 * (1.0 + erf(x / np.sqrt(2.0))) + x * np.exp(-0.5 * x * x) / np.sqrt(2.0 * np.pi)


def conv3d(x: np.ndarray, W: np.ndarray, b: np.ndarray) -> np.ndarray:
    """Zero-padded 3x3x3 cross-correlation: y[p, o] = b[o] + sum_{c, d} W[o, c, d] x[p + d - 1, c].

    x: [B, Z, Y, X, C_in]; W: [C_out, C_in, 3, 3, 3]; returns [B, Z, Y, X, C_out]."""
    B, Z, Y, X, _ = x.shape
    xp = np.zeros((B, Z + 2, Y + 2, X + 2, x.shape[4]))
    xp[:, 1:-1, 1:-1, 1:-1, :] = x
    y = np.broadcast_to(b, (B, Z, Y, X, W.shape[0])).copy()
    for dz in range(3):
        for dy in range(3):
            for dx in range(3):
                y += xp[:, dz:dz + Z, dy:dy + Y, dx:dx + X, :] @ W[:, :, dz, dy, dx].T
    return y


def conv3d_weight_grad(x: np.ndarray, g: np.ndarray) -> np.ndarray:
    """d(sum g * conv3d(x, W, b)) / dW: [C_out, C_in, 3, 3, 3]."""
    B, Z, Y, X, ci = x.shape
    xp = np.zeros((B, Z + 2, Y + 2, X + 2, ci))
    xp[:, 1:-1, 1:-1, 1:-1, :] = x
    gw = np.zeros((g.shape[4], ci, 3, 3, 3))
    gf = g.reshape(-1, g.shape[4])
    for dz in range(3):
        for dy in range(3):
            for dx in range(3):
                gw[:, :, dz, dy, dx] = gf.T @ xp[:, dz:dz + Z, dy:dy + Y, dx:dx + X, :].reshape(-1, ci)
    return gw


def conv3d_input_grad(g: np.ndarray, W: np.ndarray) -> np.ndarray:
    """d(sum g * conv3d(x, W, b)) / dx: each output point p sends W[o, c, d] g[p, o] to x[p + d - 1]."""
    B, Z, Y, X, _ = g.shape
    gx = np.zeros((B, Z + 2, Y + 2, X + 2, W.shape[1]))
    for dz in range(3):
        for dy in range(3):
            for dx in range(3):
                gx[:, dz:dz + Z, dy:dy + Y, dx:dx + X, :] += g @ W[:, :, dz, dy, dx]
    return gx[:, 1:-1, 1:-1, 1:-1, :]


def forward(theta, x, bf16=True, channels=CHANNELS, keep=False):
    """Network output for input x [B, Z, Y, X, 2]; with keep=True also the saved tensors."""
    q = bf16_round if bf16 else (lambda v: v)
    layers = unpack(theta, channels)
    a = q(x)
    acts, pre = [a], []
    for li, (W, b) in enumerate(layers):
        zl = conv3d(a, q(W), b)
        pre.append(zl)
        if li < len(layers) - 1:
            a = q(gelu(zl))
            acts.append(a)
        else:
            a = zl
    return (a, acts, pre) if keep else a


def loss_and_grad(theta, x, target, bf16=True, channels=CHANNELS):
    """Mean squared error over every element of the output, and its gradient with respect
    to the flat parameter vector (straight-through for the BF16 roundings)."""
    q = bf16_round if bf16 else (lambda v: v)
    layers = unpack(theta, channels)
    y, acts, pre = forward(theta, x, bf16, channels, keep=True)
    diff = y - target
    loss = float(np.mean(diff * diff))
    g = 2.0 * diff / diff.size
    grads = [None] * len(layers)
    for li in range(len(layers) - 1, -1, -1):
        W, _ = layers[li]
        grads[li] = (conv3d_weight_grad(acts[li], g), g.sum(axis=(0, 1, 2, 3)))
        if li > 0:
            g = conv3d_input_grad(g, q(W)) * gelu_grad(pre[li - 1])
    return loss, pack(grads)


def init_params(seed_normal: np.ndarray, channels=CHANNELS) -> np.ndarray:
    """Parameters from a vector of standard normal draws (one per parameter): weights
    scaled by 1/sqrt(27 c_in) (variance-preserving for unit inputs), biases zero."""
    theta = np.zeros(n_params(channels))
    o = 0
    for ci, co in zip(channels[:-1], channels[1:]):
        nw = co * ci * 27
        theta[o:o + nw] = seed_normal[o:o + nw] / np.sqrt(27.0 * ci)
        o += nw + co
    return theta


def stage2(theta, out_scale, u, precond, apply_A, bf16=True):
    """Two-stage preconditioner applied to a complex field u [Z, Y, X]:
    z1 = M^-1 u, t = u - A z1, s = rms(t), z = z1 + c s N(t / s)."""
    z1 = precond(u)
    t = u - apply_A(z1)
    s = float(np.sqrt(np.mean(np.abs(t) ** 2)))
    if s == 0.0:
        return z1
    xin = np.stack([t.real / s, t.imag / s], axis=-1)[None]
    y = forward(theta, xin, bf16)[0]
    return z1 + out_scale * s * (y[..., 0] + 1j * y[..., 1])


def stencil_weights(k: complex, h: float):
    """Class weights (centre, face, edge, corner) of the interior 27-point operator of
    Eq. scheme written as D_x+D_y+D_z + a(D_xD_y+D_xD_z+D_yD_z) + b D_xD_yD_z + kappa with
    D = [1, -2, 1]: the centre collects -6, 12a, -8b and kappa; a face neighbour 1, -4a
    (two products) and 4b; an edge neighbour a (one product) and -2b; a corner b."""
    from .helm6_oracle import scheme_coefficients
    s = scheme_coefficients(complex(k), h)
    a, b, kap = s["a"], s["b"], s["kappa"]
    return (-6 + 12 * a - 8 * b + kap, 1 - 4 * a + 4 * b, a - 2 * b, b + 0j)


def patch_operator(Y: np.ndarray, w, conj: bool = False) -> np.ndarray:
    """Interior 27-point operator (weights w = (c0 centre, c1 faces, c2 edges, c3 corners),
    complex) on complex arrays [B, Z, Y, X] with zero values outside the array; conj=True
    applies the conjugated weights (the adjoint: the stencil is symmetric)."""
    c = [complex(v).conjugate() if conj else complex(v) for v in w]
    B, Z, Yn, X = Y.shape
    P = np.zeros((B, Z + 2, Yn + 2, X + 2), dtype=complex)
    P[:, 1:-1, 1:-1, 1:-1] = Y
    out = np.zeros_like(Y, dtype=complex)
    for dz in (-1, 0, 1):
        for dy in (-1, 0, 1):
            for dx in (-1, 0, 1):
                m = abs(dz) + abs(dy) + abs(dx)
                out += c[m] * P[:, 1 + dz:1 + dz + Z, 1 + dy:1 + dy + Yn, 1 + dx:1 + dx + X]
    return out


def interior_mask(shape) -> np.ndarray:
    """True at the points of [B, Z, Y, X] at least one point away from every face."""
    m = np.zeros(shape, dtype=bool)
    m[:, 1:-1, 1:-1, 1:-1] = True
    return m


def residual_loss_and_grad(theta, x, w, bf16=True, channels=CHANNELS):
    """The residual-form loss above and its gradient with respect to the parameters."""
    q = bf16_round if bf16 else (lambda v: v)
    layers = unpack(theta, channels)
    y, acts, pre = forward(theta, x, bf16, channels, keep=True)
    X = x[..., 0] + 1j * x[..., 1]
    Yc = y[..., 0] + 1j * y[..., 1]
    mask = interior_mask(X.shape)
    M = int(mask.sum())
    R = np.where(mask, patch_operator(Yc, w) - X, 0.0)
    loss = float(np.sum(np.abs(R) ** 2) / (2 * M))
    # dL/dy_0 = Re(A^H R)/M, dL/dy_1 = Im(A^H R)/M
    AR = patch_operator(R, w, conj=True) / M
    g = np.stack([AR.real, AR.imag], axis=-1)
    grads = [None] * len(layers)
    for li in range(len(layers) - 1, -1, -1):
        W, _ = layers[li]
        grads[li] = (conv3d_weight_grad(acts[li], g), g.sum(axis=(0, 1, 2, 3)))
        if li > 0:
            g = conv3d_input_grad(g, q(W)) * gelu_grad(pre[li - 1])
    return loss, pack(grads)

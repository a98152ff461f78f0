"""FP64 CPU oracle of the small 3D CNN that supplies a learned initial guess.

TEST INFRASTRUCTURE ONLY (see the package docstring).  The network is not part
of the paper; it is the workload's learned-x0 form: four 3x3x3 convolutions
2 -> 16 -> 16 -> 16 -> 1 with "same" zero padding and bias, the erf form of
GELU after the first three, mapping the normalised input channels
(r0, x^(i)), r0 = b^(i+1) - A x^(i), to the normalised x^(i+1) - x^(i).
Training minimises the mean squared error with Adam.

Arrays are channels-first, (C, Z, Y, X) for one volume and (B, C, Z, Y, X)
for a batch; x is the fastest axis, as in the solver's vectors.  Weights are
(C_out, C_in, 3, 3, 3) with tap (dz, dy, dx) + 1 applied to the input voxel at
offset (dz, dy, dx) (cross-correlation).

Precision model of the CUDA path, which the oracle reproduces in FP64 on the
same rounded operands: weights and every operand of a convolution (input
volumes, hidden activations, gradients fed to the next contraction) are
rounded to bfloat16 (round to nearest even), accumulation and everything else
is wider.  ``bf16`` below performs that rounding.
"""

from __future__ import annotations

import math

import numpy as np

LAYERS = [(2, 16), (16, 16), (16, 16), (16, 1)]   # (C_in, C_out)
SQRT1_2 = 1.0 / math.sqrt(2.0)


def bf16(a: np.ndarray) -> np.ndarray:
    """Round to bfloat16 (8 significand bits, round to nearest even), as FP64.

    Goes through float32 first (as the device does with its FP32 values); the
    oracle's FP64 values are first rounded to the nearest float32."""
    f = np.asarray(a, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) >> 16) << 16
    out = r.astype(np.uint32).view(np.float32).astype(np.float64)
    nan = np.isnan(f)
    if nan.any():
        out[nan] = np.nan
    return out


def n_params() -> int:
    return sum(co * ci * 27 + co for ci, co in LAYERS)


def unpack(theta: np.ndarray):
    """Split the flat parameter vector into [(W, b)] per layer (W first)."""
    out, o = [], 0
    for ci, co in LAYERS:
        W = theta[o:o + co * ci * 27].reshape(co, ci, 3, 3, 3)
        o += co * ci * 27
        b = theta[o:o + co]
        o += co
        out.append((W, b))
    return out


def conv3d(x: np.ndarray, W: np.ndarray, b: np.ndarray) -> np.ndarray:
    """y[o, p] = b[o] + sum_{c, d} W[o, c, d + 1] x[c, p + d], zero outside."""
    C, Z, Y, X = x.shape
    xp = np.pad(x, ((0, 0), (1, 1), (1, 1), (1, 1)))
    y = np.zeros((W.shape[0], Z, Y, X)) + b[:, None, None, None]
    for dz in range(3):
        for dy in range(3):
            for dx in range(3):
                patch = xp[:, dz:dz + Z, dy:dy + Y, dx:dx + X]
                y += np.einsum("oc,czyx->ozyx", W[:, :, dz, dy, dx], patch)
    return y


def conv3d_backward(x: np.ndarray, W: np.ndarray, dy: np.ndarray):
    """Gradients of conv3d: (dx, dW, db) for upstream gradient dy."""
    C, Z, Y, X = x.shape
    xp = np.pad(x, ((0, 0), (1, 1), (1, 1), (1, 1)))
    dxp = np.zeros_like(xp)
    dW = np.zeros_like(W)
    for dz in range(3):
        for dy_ in range(3):
            for dx in range(3):
                patch = xp[:, dz:dz + Z, dy_:dy_ + Y, dx:dx + X]
                dW[:, :, dz, dy_, dx] = np.einsum("ozyx,czyx->oc", dy, patch)
                dxp[:, dz:dz + Z, dy_:dy_ + Y, dx:dx + X] += np.einsum("oc,ozyx->czyx", W[:, :, dz, dy_, dx], dy)
    return dxp[:, 1:-1, 1:-1, 1:-1], dW, dy.sum(axis=(1, 2, 3))


def _erf(a):
    from scipy.special import erf
    return erf(a)


def gelu(a: np.ndarray) -> np.ndarray:
    """GELU, erf form: a * Phi(a)."""
    return 0.5 * a * (1.0 + _erf(a * SQRT1_2))


def gelu_grad(a: np.ndarray) -> np.ndarray:
    """d GELU / d a = Phi(a) + a phi(a)."""
    return 0.5 * (1.0 + _erf(a * SQRT1_2)) + a * np.exp(-0.5 * a * a) / math.sqrt(2.0 * math.pi)


def _identity(a):
    return np.asarray(a, dtype=np.float64)


def forward(theta: np.ndarray, x: np.ndarray, keep: bool = False, rounding: bool = True):
    """Network output (1, Z, Y, X) for input x (2, Z, Y, X), with the rounding
    of the CUDA path (rounding=False: exact FP64, for derivative checks).
    With keep, also the per-layer (input, pre-activation)."""
    q = bf16 if rounding else _identity
    params = unpack(q(theta))
    h = q(x)
    cache = []
    for li, (W, b) in enumerate(params):
        z = conv3d(h, W, b)
        cache.append((h, z))
        if li < len(params) - 1:
            h = q(gelu(z))
        else:
            h = z
    return (h, cache) if keep else h


def loss_and_grad(theta: np.ndarray, xb: np.ndarray, tb: np.ndarray, rounding: bool = True,
                  stencil: np.ndarray = None):
    """Mean squared error over a batch (B, 2, ...) -> (B, 1, ...) and its
    gradient with respect to the (FP32 master) parameters; the convolutions
    use bfloat16-rounded weights, inputs and upstream gradients.

    With ``stencil`` (3, 3, 3), the error e = out - t is weighted by the
    operator first: the loss is the mean of (K * e)^2, K * e the
    cross-correlation with zero padding (for K taken from a row of A, the
    residual A e of the guess on the crop's interior).  The stencil step is
    exact here; the CUDA path does it in FP32."""
    q = bf16 if rounding else _identity
    params = unpack(q(theta))
    grads = [(np.zeros_like(W), np.zeros_like(b)) for W, b in params]
    total = 0.0
    count = tb.size
    K = None if stencil is None else np.asarray(stencil, dtype=np.float64).reshape(1, 1, 3, 3, 3)
    for x, t in zip(xb, tb):
        out, cache = forward(theta, x, keep=True, rounding=rounding)
        diff = out - t
        if K is None:
            total += float((diff * diff).sum())
            g = 2.0 * diff / count
        else:
            s = conv3d(diff, K, np.zeros(1))
            total += float((s * s).sum())
            g = conv3d_backward(diff, K, 2.0 * s / count)[0]
        for li in range(len(params) - 1, -1, -1):
            h, z = cache[li]
            W, _ = params[li]
            if li < len(params) - 1:
                g = g * gelu_grad(z)
            gq = q(g)
            dx, dW, db = conv3d_backward(h, W, gq)
            grads[li][0][...] += dW
            grads[li][1][...] += db
            g = dx
    flat = np.concatenate([np.concatenate([dW.ravel(), db]) for dW, db in grads])
    return total / count, flat


def adam_step(theta, m, v, grad, t, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (bias-corrected), returning (theta, m, v)."""
    m = beta1 * m + (1.0 - beta1) * grad
    v = beta2 * v + (1.0 - beta2) * grad * grad
    mh = m / (1.0 - beta1 ** t)
    vh = v / (1.0 - beta2 ** t)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v


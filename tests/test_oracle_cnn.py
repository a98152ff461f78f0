"""Pins of the CNN oracle: scipy's correlate for one channel, central finite
differences for every gradient, tabulated normal-CDF values for GELU, the
closed form of the first Adam step, and bfloat16 rounding cases."""

import numpy as np
import pytest

from oracle import cnn as C
from paper_1604_06043_gb300 import problems as pb


def test_conv3d_single_channel_is_scipy_correlate():
    from scipy.ndimage import correlate
    rng = np.random.default_rng(0)
    x = rng.standard_normal((1, 5, 6, 7))
    W = rng.standard_normal((1, 1, 3, 3, 3))
    y = C.conv3d(x, W, np.array([0.25]))
    ref = correlate(x[0], W[0, 0], mode="constant", cval=0.0) + 0.25
    np.testing.assert_allclose(y[0], ref, rtol=1e-12, atol=1e-12)


def test_conv3d_multichannel_is_sum_of_correlations():
    from scipy.ndimage import correlate
    rng = np.random.default_rng(1)
    x = rng.standard_normal((3, 4, 5, 4))
    W = rng.standard_normal((2, 3, 3, 3, 3))
    b = rng.standard_normal(2)
    y = C.conv3d(x, W, b)
    for o in range(2):
        ref = sum(correlate(x[c], W[o, c], mode="constant", cval=0.0) for c in range(3)) + b[o]
        np.testing.assert_allclose(y[o], ref, rtol=1e-12, atol=1e-12)


def test_conv3d_backward_finite_differences():
    rng = np.random.default_rng(2)
    x = rng.standard_normal((2, 3, 4, 3))
    W = rng.standard_normal((3, 2, 3, 3, 3))
    b = rng.standard_normal(3)
    g = rng.standard_normal((3, 3, 4, 3))
    f = lambda x_, W_, b_: float((g * C.conv3d(x_, W_, b_)).sum())
    dx, dW, db = C.conv3d_backward(x, W, g)
    eps = 1e-6
    for arr, grad in ((x, dx), (W, dW), (b, db)):
        idx = [tuple(rng.integers(0, s) for s in arr.shape) for _ in range(6)]
        for i in idx:
            old = arr[i]
            arr[i] = old + eps
            fp = f(x, W, b)
            arr[i] = old - eps
            fm = f(x, W, b)
            arr[i] = old
            assert abs((fp - fm) / (2 * eps) - grad[i]) <= 1e-6 * (1 + abs(grad[i]))


def test_gelu_tabulated_values():
    # Phi(x) from standard normal tables
    phi = {-1.0: 0.15865525393145707, 0.5: 0.6914624612740131, 1.0: 0.8413447460685429,
           2.0: 0.9772498680518208}
    for a, p in phi.items():
        assert abs(C.gelu(np.array(a)) - a * p) < 1e-15
    a = np.linspace(-4, 4, 41)
    fd = (C.gelu(a + 1e-6) - C.gelu(a - 1e-6)) / 2e-6
    np.testing.assert_allclose(C.gelu_grad(a), fd, rtol=1e-7, atol=1e-9)


def test_first_adam_step_is_signed_lr():
    g = np.array([0.3, -2.0, 1e-3])
    th, m, v = C.adam_step(np.zeros(3), np.zeros(3), np.zeros(3), g, t=1, lr=0.01)
    np.testing.assert_allclose(th, -0.01 * g / (np.abs(g) + 1e-8), rtol=1e-12)
    np.testing.assert_allclose(m, 0.1 * g)
    np.testing.assert_allclose(v, 0.001 * g * g)


def test_bf16_rounding_cases():
    cases = {1.0: 1.0, 1 + 2**-8: 1.0, 1 + 3 * 2**-8: 1 + 2**-6, 1 + 2**-7: 1 + 2**-7,
             -3.0: -3.0, 1 + 2**-8 + 2**-20: 1 + 2**-7}
    for a, r in cases.items():
        assert C.bf16(np.array([a]))[0] == r
    torch = pytest.importorskip("torch")
    v = np.random.default_rng(3).standard_normal(2000) * 10.0 ** np.random.default_rng(4).integers(-8, 8, 2000)
    ref = torch.tensor(v, dtype=torch.float32).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(C.bf16(v), ref)


def test_network_gradient_finite_differences():
    rng = np.random.default_rng(5)
    theta = pb.cnn_init_params(5) + 0.01 * rng.standard_normal(C.n_params())
    xb = rng.standard_normal((2, 2, 4, 4, 4))
    tb = rng.standard_normal((2, 1, 4, 4, 4))
    loss, grad = C.loss_and_grad(theta, xb, tb, rounding=False)
    eps = 1e-6
    idx = rng.choice(C.n_params(), size=12, replace=False)
    for i in idx:
        th = theta.copy()
        th[i] += eps
        lp, _ = C.loss_and_grad(th, xb, tb, rounding=False)
        th[i] -= 2 * eps
        lm, _ = C.loss_and_grad(th, xb, tb, rounding=False)
        assert abs((lp - lm) / (2 * eps) - grad[i]) <= 1e-5 * (1e-3 + abs(grad[i]))


def test_stencil_loss_is_operator_residual_and_gradient_checks():
    # with K the 7-point row of A, the loss is mean((A e)^2) on the crop
    # interior (zero padding outside), and its gradient passes finite differences
    rng = np.random.default_rng(6)
    A = pb.convdiff((6, 6, 6), (20.0, 10.0, 5.0), tau=0.005)
    K = pb.row_stencil(A, (6, 6, 6), (3, 3, 3))
    assert np.count_nonzero(K) == 7 and K[1, 1, 1] == A.to_dense()[3 * 36 + 3 * 6 + 3, 3 * 36 + 3 * 6 + 3]
    e = rng.standard_normal((1, 6, 6, 6))
    s = C.conv3d(e, K.reshape(1, 1, 3, 3, 3), np.zeros(1))
    Ae = (A.to_dense() @ e.reshape(-1)).reshape(6, 6, 6)
    # equal at every point: Dirichlet rows lack the outside neighbours, as the padding does
    np.testing.assert_allclose(s[0], Ae, rtol=1e-12, atol=1e-9 * np.abs(Ae).max())
    theta = pb.cnn_init_params(5) + 0.01 * rng.standard_normal(C.n_params())
    xb = rng.standard_normal((2, 2, 4, 4, 4))
    tb = rng.standard_normal((2, 1, 4, 4, 4))
    Kn = K / np.abs(K).max()
    loss, grad = C.loss_and_grad(theta, xb, tb, rounding=False, stencil=Kn)
    out = np.stack([C.forward(theta, x, rounding=False) for x in xb])
    s = np.stack([C.conv3d(o - tt, Kn.reshape(1, 1, 3, 3, 3), np.zeros(1)) for o, tt in zip(out, tb)])
    assert loss == pytest.approx(float((s * s).sum()) / tb.size, rel=1e-12)
    eps = 1e-6
    for i in rng.choice(C.n_params(), size=12, replace=False):
        th = theta.copy()
        th[i] += eps
        lp, _ = C.loss_and_grad(th, xb, tb, rounding=False, stencil=Kn)
        th[i] -= 2 * eps
        lm, _ = C.loss_and_grad(th, xb, tb, rounding=False, stencil=Kn)
        assert abs((lp - lm) / (2 * eps) - grad[i]) <= 1e-5 * (1e-3 + abs(grad[i]))


def test_param_count_and_layout():
    assert C.n_params() == 2 * 16 * 27 + 16 + 2 * (16 * 16 * 27 + 16) + 16 * 27 + 1
    theta = pb.cnn_init_params(5)
    assert theta.shape == (C.n_params(),)
    (W0, b0), *_ = C.unpack(theta)
    assert W0.shape == (16, 2, 3, 3, 3) and not b0.any()
    assert np.abs(W0).max() <= (6.0 / 54) ** 0.5


def test_training_reduces_loss():
    # the target is a fixed linear stencil of the inputs: learnable exactly
    rng = np.random.default_rng(6)
    xb = rng.standard_normal((4, 2, 6, 6, 6))
    K = np.zeros((1, 2, 3, 3, 3))
    K[0, 0, 1, 1, 1], K[0, 1, 1, 1, 2] = 0.5, -0.3
    tb = np.stack([C.conv3d(x, K, np.zeros(1)) for x in xb])
    theta = pb.cnn_init_params(5)
    m = np.zeros_like(theta)
    v = np.zeros_like(theta)
    l0, _ = C.loss_and_grad(theta, xb, tb, rounding=False)
    for t in range(1, 31):
        l, g = C.loss_and_grad(theta, xb, tb, rounding=False)
        theta, m, v = C.adam_step(theta, m, v, g, t, lr=3e-3)
    l1, _ = C.loss_and_grad(theta, xb, tb, rounding=False)
    assert l1 < 0.5 * l0

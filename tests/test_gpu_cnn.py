"""The learned-initial-guess CNN on the GPU against its FP64 oracle.

Both sides round the same operands to bfloat16 (weights, biases, inputs,
hidden activations, upstream gradients) and accumulate wider (FP32 on the GPU,
FP64 in the oracle).  A bfloat16 rounding can land on either side of a
rounding boundary when the FP32 and FP64 pre-rounding values straddle it (they
differ by ~1e-7 relative; the bfloat16 unit roundoff is U = 2^-8), and such a
flip moves every later value that reads it.  So every element is compared
against one bfloat16 unit roundoff of the sum of the absolute values of its
terms: an output o = b + sum W h within U (|b| + sum |W| |h|), a gradient
entry dW = sum g h within U sum |g| |h| (the terms of the oracle's own last
contraction).  Measured: at most 0.06 U (outputs) and 0.14 U (gradients) of
that scale.  The share of outputs that moved beyond FP32 accumulation slack
(1e-6 of the scale) -- the footprint of the flips -- is reported and bounded,
and the norm bounds stay as a second check.
"""

import numpy as np
import pytest

from oracle import cnn as C
from paper_1604_06043_gb300 import problems as pb

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
DEV = "cuda:0"


@pytest.fixture(scope="module")
def M():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1604_06043_gb300 import build, msstab
    build.build()
    return msstab


def _params(seed=5):
    rng = np.random.default_rng(seed)
    th = pb.cnn_init_params(seed)
    th += 0.05 * rng.standard_normal(th.size)      # non-zero biases, generic weights
    return th.astype(np.float32).astype(np.float64)


def _t(a, dt=torch.float32):
    return torch.tensor(np.ascontiguousarray(a), dtype=dt, device=DEV)


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


U_BF16 = 2.0 ** -8


def _output_terms(th, x):
    """|b| + sum |W| |h| of the last layer's outputs (the oracle's operands)."""
    _, cache = C.forward(th, x, keep=True)
    W, b = C.unpack(C.bf16(th))[-1]
    return C.conv3d(np.abs(cache[-1][0]), np.abs(W), np.abs(b))


def _gradient_terms(th, xb, tb, stencil=None):
    """sum |upstream| |input| of every gradient entry (flat, like the
    parameters), from the oracle's own backward pass."""
    params = C.unpack(C.bf16(th))
    acc = [(np.zeros_like(W), np.zeros_like(b)) for W, b in params]
    count = tb.size
    K = None if stencil is None else np.asarray(stencil, dtype=np.float64).reshape(1, 1, 3, 3, 3)
    for x, t_ in zip(xb, tb):
        out, cache = C.forward(th, x, keep=True)
        diff = out - t_
        if K is None:
            g = 2.0 * diff / count
        else:
            s_ = C.conv3d(diff, K, np.zeros(1))
            g = C.conv3d_backward(diff, K, 2.0 * s_ / count)[0]
        for li in range(len(params) - 1, -1, -1):
            h, z = cache[li]
            W, _ = params[li]
            if li < len(params) - 1:
                g = g * C.gelu_grad(z)
            gq = C.bf16(g)
            _, dWa, dba = C.conv3d_backward(np.abs(h), np.abs(W), np.abs(gq))
            acc[li][0][...] += dWa
            acc[li][1][...] += dba
            g = C.conv3d_backward(h, W, gq)[0]
    return np.concatenate([np.concatenate([a.ravel(), b]) for a, b in acc])


def _check_elementwise(got, ref, terms, moved_max):
    """Every element within U_BF16 of its terms; the share beyond FP32 slack
    (elements that a bfloat16 flip upstream moved) at most moved_max."""
    d = np.abs(got - ref)
    assert np.all(d <= U_BF16 * terms), float(np.max(d / (U_BF16 * terms)))
    moved = float(np.mean(d > 1e-6 * terms))
    assert moved <= moved_max, moved
    return moved


def test_forward_matches_oracle(M):
    B, D = 2, 12
    th = _params()
    rng = np.random.default_rng(1)
    x = rng.standard_normal((B, 2, D, D, D)).astype(np.float32)
    net = M.CNN((D, D, D), th, max_batch=B, crop=D, device=DEV)
    out = net.forward(_t(x), B, D).cpu().numpy().reshape(B, 1, D, D, D)
    ref = np.stack([C.forward(th, xb.astype(np.float64)) for xb in x])
    terms = np.stack([_output_terms(th, xb.astype(np.float64)) for xb in x])
    moved = _check_elementwise(out, ref, terms, 0.5)
    print("forward: %.1f %% of the outputs moved by a bfloat16 flip upstream" % (100 * moved))
    assert _rel(out, ref) <= 2e-3


def test_gradient_matches_oracle(M):
    B, D = 2, 10
    th = _params(6)
    rng = np.random.default_rng(2)
    x = rng.standard_normal((B, 2, D, D, D)).astype(np.float32)
    t = rng.standard_normal((B, 1, D, D, D)).astype(np.float32)
    net = M.CNN((D, D, D), th, max_batch=B, crop=D, device=DEV)
    g, loss = net.grad(_t(x), _t(t), B, D)
    ref_loss, ref_g = C.loss_and_grad(th, x.astype(np.float64), t.astype(np.float64))
    assert abs(loss - ref_loss) <= 1e-4 * ref_loss
    g = g.cpu().numpy()
    terms = _gradient_terms(th, x.astype(np.float64), t.astype(np.float64))
    # every gradient entry sums over all voxels, so nearly every entry sees a
    # flip somewhere: the share is reported, the element-wise bound is the test
    moved = _check_elementwise(g, ref_g, terms, 1.0)
    print("gradient: %.1f %% of the entries moved by a bfloat16 flip upstream" % (100 * moved))
    o = 0
    for ci, co in C.LAYERS:
        n = co * ci * 27 + co
        assert _rel(g[o:o + n], ref_g[o:o + n]) <= 5e-3, (ci, co)
        o += n


def test_gradient_matches_oracle_several_tiles_per_block(M):
    # 5 crops of 32^3 = 1280 tiles of 8 x 16 voxels: more than the persistent
    # grids of the convolutions (608 and 1064 blocks) and of the weight
    # gradient (304), so blocks take two or more tiles (the two-stage pipelines,
    # the accumulation over tiles in tensor memory, the mbarrier phases)
    B, D = 5, 32
    th = _params(8)
    rng = np.random.default_rng(12)
    x = rng.standard_normal((B, 2, D, D, D)).astype(np.float32)
    t = rng.standard_normal((B, 1, D, D, D)).astype(np.float32)
    net = M.CNN((D, D, D), th, max_batch=B, crop=D, device=DEV)
    g, loss = net.grad(_t(x), _t(t), B, D)
    ref_loss, ref_g = C.loss_and_grad(th, x.astype(np.float64), t.astype(np.float64))
    assert abs(loss - ref_loss) <= 1e-4 * ref_loss
    g = g.cpu().numpy()
    _check_elementwise(g, ref_g, _gradient_terms(th, x.astype(np.float64), t.astype(np.float64)), 1.0)
    o = 0
    for ci, co in C.LAYERS:
        n = co * ci * 27 + co
        assert _rel(g[o:o + n], ref_g[o:o + n]) <= 5e-3, (ci, co)
        o += n


def test_operator_weighted_gradient_matches_oracle(M):
    B, D = 2, 10
    th = _params(9)
    rng = np.random.default_rng(7)
    x = rng.standard_normal((B, 2, D, D, D)).astype(np.float32)
    t = rng.standard_normal((B, 1, D, D, D)).astype(np.float32)
    A = pb.convdiff((12, 12, 12), (20.0, 10.0, 5.0), tau=0.005)
    K = pb.row_stencil(A, (12, 12, 12), (6, 6, 6))
    K = K / np.abs(K).max()
    net = M.CNN((D, D, D), th, max_batch=B, crop=D, device=DEV)
    net.set_loss_stencil(K)
    g, loss = net.grad(_t(x), _t(t), B, D)
    ref_loss, ref_g = C.loss_and_grad(th, x.astype(np.float64), t.astype(np.float64), stencil=K)
    assert abs(loss - ref_loss) <= 1e-4 * ref_loss
    g = g.cpu().numpy()
    _check_elementwise(g, ref_g, _gradient_terms(th, x.astype(np.float64), t.astype(np.float64), K), 1.0)
    o = 0
    for ci, co in C.LAYERS:
        n = co * ci * 27 + co
        assert _rel(g[o:o + n], ref_g[o:o + n]) <= 5e-3, (ci, co)
        o += n
    net.set_loss_stencil(None)          # back to the mean squared error
    g2, loss2 = net.grad(_t(x), _t(t), B, D)
    assert abs(loss2 - C.loss_and_grad(th, x.astype(np.float64), t.astype(np.float64))[0]) <= 1e-4 * loss2


def test_adam_step_matches_oracle(M):
    th = _params(7)
    g = np.random.default_rng(3).standard_normal(th.size).astype(np.float32).astype(np.float64)
    net = M.CNN((8, 8, 8), th, max_batch=1, crop=8, device=DEV)
    net.adam_step(_t(g), 1e-3)
    net.adam_step(_t(0.5 * g), 1e-3)
    p = net.params().cpu().numpy()
    r, m, v = C.adam_step(th, np.zeros_like(th), np.zeros_like(th), g, 1, lr=1e-3)
    r, m, v = C.adam_step(r, m, v, 0.5 * g, 2, lr=1e-3)
    assert np.max(np.abs(p - r)) <= 1e-6 * (np.max(np.abs(th)) + 1e-3)


def test_training_reduces_loss_on_a_learnable_map(M):
    # x_next - x_prev is a fixed stencil of (r0, x_prev): exactly representable
    n = 16
    K = np.zeros((1, 2, 3, 3, 3))
    K[0, 0, 1, 1, 1], K[0, 1, 1, 1, 2], K[0, 1, 0, 1, 1] = 0.5, -0.3, 0.2
    rng = np.random.default_rng(4)
    net = M.CNN((n, n, n), pb.cnn_init_params(5), max_pairs=4, max_batch=4, crop=8, device=DEV)
    for k in range(4):
        r0 = rng.standard_normal(n ** 3)
        xp = rng.standard_normal(n ** 3)
        inp = np.stack([r0, xp]).reshape(2, n, n, n)
        xn = xp + C.conv3d(inp, K, np.zeros(1)).reshape(-1)
        net.add_pair(_t(r0, torch.float64), _t(xp, torch.float64), _t(xn, torch.float64))
    net.fit_scales()
    s = net.scales()
    assert all(v > 0 for v in s)
    origins = []
    for it in range(60):
        for bb in range(4):
            origins.append([rng.integers(0, 4), rng.integers(0, n - 8 + 1), rng.integers(0, n - 8 + 1),
                            rng.integers(0, n - 8 + 1)])
    hist = net.train(np.array(origins), 4, 8, 3e-3)
    assert np.isfinite(hist).all()
    assert hist[-10:].mean() < 0.3 * hist[:3].mean()


def test_infer_matches_oracle(M):
    n = 12
    th = _params(8)
    rng = np.random.default_rng(5)
    r0 = rng.standard_normal(n ** 3) * 50
    xp = rng.standard_normal(n ** 3)
    net = M.CNN((n, n, n), th, device=DEV, crop=8)
    net.set_scales(2.0, 4.0)
    delta = torch.empty(n ** 3, dtype=torch.float64, device=DEV)
    net.infer(_t(r0, torch.float64), _t(xp, torch.float64), delta)
    torch.cuda.synchronize()
    # per-instance residual scale s_r = 1/RMS(r0); global s_x = 2, c = 4
    s_r = np.float32(1.0 / np.sqrt(np.mean(r0 * r0)))
    s_x, c = np.float32(2.0), np.float32(4.0)
    inp = np.stack([(s_r * r0.astype(np.float32)), (s_x * xp.astype(np.float32))]).reshape(2, n, n, n)
    ref = C.forward(th, inp.astype(np.float64)).reshape(-1) / (float(c) * float(s_r))
    terms = _output_terms(th, inp.astype(np.float64)).reshape(-1) / (float(c) * float(s_r))
    _check_elementwise(delta.cpu().numpy(), ref, terms, 0.5)
    assert _rel(delta.cpu().numpy(), ref) <= 2e-3


def test_select_guess_keeps_only_a_better_start(M):
    w = pb.WORKLOADS["convdiff3d_24"]
    A = w.matrix()
    S = M.Solver(A, w.s, w.ell, w.p_raw(), device=DEV)
    xp = w.x0()
    b = xp / w.tau + w.f()
    import scipy.sparse.linalg as spla
    exact = spla.spsolve(A.to_scipy().tocsc(), b)
    bt, xpt = _t(b, torch.float64), _t(xp, torch.float64)
    x = torch.empty_like(xpt)
    good = _t(exact - xp, torch.float64)
    assert S.select_guess(bt, xpt, good, x)
    np.testing.assert_allclose(x.cpu().numpy(), xp + (exact - xp), rtol=0, atol=1e-12 * np.abs(exact).max())
    bad = _t(1e3 * np.random.default_rng(0).standard_normal(A.n), torch.float64)
    assert not S.select_guess(bt, xpt, bad, x)
    np.testing.assert_array_equal(x.cpu().numpy(), xp)
    # scaled: x_prev + alpha delta with the residual-minimising alpha (1 for the exact correction)
    used, alpha, red = S.select_guess_scaled(bt, xpt, good, x)
    assert used and abs(alpha - 1.0) < 1e-8 and red < 1e-6   # sqrt(1 - cos^2): floor near sqrt(eps)
    half = _t(0.5 * (exact - xp), torch.float64)
    used, alpha, red = S.select_guess_scaled(bt, xpt, half, x)
    assert used and abs(alpha - 2.0) < 1e-8
    used, alpha, red = S.select_guess_scaled(bt, xpt, bad, x)
    assert used and 0.0 < red <= 1.0
    r = b - A.to_scipy() @ x.cpu().numpy()
    r0 = b - A.to_scipy() @ xp
    assert abs(np.linalg.norm(r) / np.linalg.norm(r0) - red) < 1e-6

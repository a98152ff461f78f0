"""Kernel-level parity: every CUDA kernel of the solver against the FP64
oracle's definition of the same step, on the same seeded inputs.

Tolerance (FP64): 1e-12 relative to the sum of the absolute values of the
terms (|A||x| per row for products with A, sum |a_i b_i| for dot products,
the sum of |coefficient x operand| for block updates), so that cancellation
cannot make a correct result fail.  FP32 kernels: 1e-6 of the same scale
(a handful of FP32 roundings, unit roundoff 6e-8).
"""

import numpy as np
import pytest

from oracle import idrstab as O
from paper_1604_06043_gb300 import problems as pb

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DEV = "cuda:0"
TOL64 = 1e-12
TOL32 = 1e-6


@pytest.fixture(scope="module")
def msstab():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1604_06043_gb300 import build, msstab as M
    build.build()
    return M


@pytest.fixture(scope="module")
def case(msstab):
    w = pb.WORKLOADS["convdiff3d_33"]     # N = 35937: many blocks and a ragged tail
    A = w.matrix()
    return w, A


def _solver(msstab, A, s, ell, **opt):
    return msstab.Solver(A, s, ell, pb.randn_cols(A.n, s, pb.SEED_P), device=DEV, **opt)


def _t(x, dtype=torch.float64):
    return torch.tensor(np.ascontiguousarray(x), dtype=dtype, device=DEV)


def _abs_spmv(A, x):
    return abs(A.to_scipy()) @ np.abs(x)


def _random_csr(n, seed):
    rng = np.random.default_rng(seed)
    rows, cols, vals = [], [], []
    for i in range(n):
        k = int(rng.integers(0, 12))
        c = np.unique(rng.integers(0, n, size=k))
        rows += [i] * len(c)
        cols += list(c)
        vals += list(rng.standard_normal(len(c)))
    import scipy.sparse as sp
    M = sp.csr_matrix((vals, (rows, cols)), shape=(n, n))
    M.sort_indices()
    return pb.CSR(n, M.indptr.astype(np.int32), M.indices.astype(np.int32), M.data.astype(np.float64))


# ---------------------------------------------------------------------------
# products with A
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("fmt,sigma", [(0, 1), (1, 1), (0, 64)])
def test_spmv_fp64(msstab, case, fmt, sigma):
    w, A = case
    S = _solver(msstab, A, 4, 2, spmv_format=fmt, sell_sigma=sigma)
    x = pb.uniform(A.n, 11) - 0.5
    y = torch.empty(A.n, dtype=torch.float64, device=DEV)
    S.op_spmv(_t(x), y)
    ref = A.to_scipy() @ x
    err = np.abs(y.cpu().numpy() - ref)
    assert np.all(err <= TOL64 * _abs_spmv(A, x))


@pytest.mark.parametrize("fmt,sigma", [(0, 1), (1, 1), (0, 32), (0, 128)])
def test_spmv_irregular_rows(msstab, fmt, sigma):
    A = _random_csr(3001, 5)            # empty rows, ragged lengths, unsorted lengths
    S = _solver(msstab, A, 2, 1, spmv_format=fmt, sell_sigma=sigma)
    x = pb.uniform(A.n, 12) - 0.5
    y = torch.full((A.n,), np.nan, dtype=torch.float64, device=DEV)
    S.op_spmv(_t(x), y)
    ref = A.to_scipy() @ x
    err = np.abs(y.cpu().numpy() - ref)
    assert np.all(err <= TOL64 * _abs_spmv(A, x) + 1e-300)


@pytest.mark.parametrize("fmt", [0, 1])
def test_spmv_fp32_scaled_copy(msstab, case, fmt):
    w, A = case
    S = _solver(msstab, A, 4, 2, spmv_format=fmt)
    x32 = (pb.uniform(A.n, 13) - 0.5).astype(np.float32)
    y = torch.empty(A.n, dtype=torch.float32, device=DEV)
    S.op_spmv(_t(x32, torch.float32), y, prec=1)
    rho = np.max(np.abs(A.to_scipy().diagonal()))
    As = A.to_scipy() / rho
    ref = As @ x32.astype(np.float64)
    err = np.abs(y.cpu().numpy().astype(np.float64) - ref)
    assert np.all(err <= TOL32 * (abs(As) @ np.abs(x32.astype(np.float64))))


def test_residual_and_norms(msstab, case):
    w, A = case
    S = _solver(msstab, A, 4, 2)
    b = w.x0() / w.tau + w.f()
    x = pb.uniform(A.n, 14)
    r = torch.empty(A.n, dtype=torch.float64, device=DEV)
    out = torch.zeros(2, dtype=torch.float64, device=DEV)
    S.op_residual(_t(b), _t(x), r, out)
    ref = b - A.to_scipy() @ x
    scale = np.abs(b) + _abs_spmv(A, x)
    assert np.all(np.abs(r.cpu().numpy() - ref) <= TOL64 * scale)
    o = out.cpu().numpy()
    rg = r.cpu().numpy()
    # ||r||^2 is the dot of the kernel's own r (compared element-wise above)
    assert abs(o[0] - rg @ rg) <= TOL64 * (rg @ rg)
    assert abs(o[1] - b @ b) <= TOL64 * (b @ b)


# ---------------------------------------------------------------------------
# cut space and projections
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("s", [1, 3, 8, 16])
def test_cut_space_matches_oracle(msstab, case, s):
    w, A = case
    S = _solver(msstab, A, s, 2)
    P = torch.empty((s, A.n), dtype=torch.float64, device=DEV)
    S.op_get_p(P)
    ref = O.orthonormalize_mgs2(pb.randn_cols(A.n, s, pb.SEED_P))
    assert np.max(np.abs(P.cpu().numpy() - ref)) <= 1e-12


@pytest.mark.parametrize("fmt", [0, 1])
@pytest.mark.parametrize("s", [4, 8, 16])
def test_spmv_dot(msstab, case, fmt, s):
    w, A = case
    S = _solver(msstab, A, s, 2, spmv_format=fmt)
    x = pb.uniform(A.n, 15) - 0.5
    y = torch.empty(A.n, dtype=torch.float64, device=DEV)
    d = torch.zeros(s + 1, dtype=torch.float64, device=DEV)
    S.op_spmv_dot(_t(x), y, d)
    P = O.orthonormalize_mgs2(pb.randn_cols(A.n, s, pb.SEED_P))
    yr = A.to_scipy() @ x
    yabs = _abs_spmv(A, x)
    assert np.all(np.abs(y.cpu().numpy() - yr) <= TOL64 * yabs)
    dd = d.cpu().numpy()
    for c in range(s):
        assert abs(dd[c] - O.proj(P, yr)[c]) <= TOL64 * (np.abs(P[c]) @ yabs) * 4
    assert abs(dd[s] - yr @ yr) <= TOL64 * (yabs @ yabs) * 4


def test_spmv_dot_fp32(msstab, case):
    w, A = case
    s = 8
    S = _solver(msstab, A, s, 2)
    x = (pb.uniform(A.n, 16) - 0.5).astype(np.float32)
    y = torch.empty(A.n, dtype=torch.float32, device=DEV)
    d = torch.zeros(s + 1, dtype=torch.float64, device=DEV)
    S.op_spmv_dot(_t(x, torch.float32), y, d, prec=1)
    P32 = torch.empty((s, A.n), dtype=torch.float32, device=DEV)
    S.op_get_p(P32, prec=1)
    yv = y.cpu().numpy().astype(np.float64)
    P = P32.cpu().numpy().astype(np.float64)
    dd = d.cpu().numpy()
    # per-thread FP32 partials of the stored FP32 values, FP64 across threads
    ref = P @ yv
    assert np.all(np.abs(dd[:s] - ref) <= TOL32 * (np.abs(P) @ np.abs(yv)))


@pytest.mark.parametrize("nx,ny", [(1, 1), (2, 4), (5, 5), (16, 16), (3, 9)])
def test_multidot(msstab, case, nx, ny):
    w, A = case
    S = _solver(msstab, A, 4, 2)
    rng = np.random.default_rng(nx * 100 + ny)
    X = rng.standard_normal((nx, A.n))
    Y = rng.standard_normal((ny, A.n))
    out = torch.zeros(nx * ny, dtype=torch.float64, device=DEV)
    S.op_multidot(_t(X), _t(Y), out)
    ref = X @ Y.T
    scale = np.abs(X) @ np.abs(Y).T
    assert np.all(np.abs(out.cpu().numpy().reshape(nx, ny) - ref) <= TOL64 * scale)


@pytest.mark.parametrize("nx,ny", [(2, 2), (1, 4), (4, 8), (3, 16)])
def test_multidot_fp32(msstab, case, nx, ny):
    """FP32 multi-dot (the Gram of the FP32 inner form's degree-1 step and the
    Arnoldi and Cholesky QR projections): FP32 partials per thread and warp,
    FP64 across warps and blocks, against FP64 dots of the same FP32 values."""
    w, A = case
    S = _solver(msstab, A, 4, 2)
    rng = np.random.default_rng(nx * 1000 + ny)
    X = rng.standard_normal((nx, A.n)).astype(np.float32)
    Y = rng.standard_normal((ny, A.n)).astype(np.float32)
    out = torch.zeros(nx * ny, dtype=torch.float64, device=DEV)
    S.op_multidot(_t(X, torch.float32), _t(Y, torch.float32), out, prec=1)
    Xd, Yd = X.astype(np.float64), Y.astype(np.float64)
    ref = Xd @ Yd.T
    scale = np.abs(Xd) @ np.abs(Yd).T
    assert np.all(np.abs(out.cpu().numpy().reshape(nx, ny) - ref) <= TOL32 * scale)


# ---------------------------------------------------------------------------
# block updates of Algorithm 1
# ---------------------------------------------------------------------------

def _levels(n, s, ell, seed):
    rng = np.random.default_rng(seed)
    R = [rng.standard_normal(n) for _ in range(ell + 1)]
    Vl = [rng.standard_normal((s, n)) for _ in range(ell + 2)]
    return R, Vl


def _pack(R, Vl):
    return np.stack(R), np.concatenate(Vl, axis=0)


def _unpack(Rg, Vg, s, ell):
    R = [Rg[i] for i in range(ell + 1)]
    Vl = [Vg[(i + 1) * s:(i + 2) * s] for i in range(-1, ell + 1)]
    return R, Vl


@pytest.mark.parametrize("s,ell,k", [(8, 4, 0), (8, 4, 3), (4, 2, 1), (16, 4, 2), (1, 1, 0)])
def test_gamma_update(msstab, case, s, ell, k):
    w, A = case
    S = _solver(msstab, A, s, ell)
    R, Vl = _levels(A.n, s, ell, 20 + k)
    gamma = np.random.default_rng(7).standard_normal(s)
    Rg, Vg = _pack(R, Vl)
    Rt, Vt = _t(Rg), _t(Vg)
    S.op_gamma_update(Rt, Vt, k, _t(gamma))
    R2 = [r.copy() for r in R]
    R2[k] = R[k] - gamma @ Vl[k + 1]
    scale = np.abs(R[k]) + np.abs(gamma) @ np.abs(Vl[k + 1])
    got = Rt.cpu().numpy()
    assert np.all(np.abs(got[k] - R2[k]) <= TOL64 * scale)
    for i in range(ell + 1):
        if i != k:
            np.testing.assert_array_equal(got[i], R[i])


@pytest.mark.parametrize("s,ell,k,q", [(8, 4, 0, 0), (8, 4, 2, 5), (8, 4, 3, 7), (16, 4, 1, 9), (1, 1, 0, 0)])
def test_eta_update_top_level(msstab, case, s, ell, k, q):
    w, A = case
    S = _solver(msstab, A, s, ell)
    R, Vl = _levels(A.n, s, ell, 40 + q)
    eta = np.random.default_rng(8).standard_normal(s)
    Rg, Vg = _pack(R, Vl)
    Rt, Vt = _t(Rg), _t(Vg)
    S.op_eta_update(Rt, Vt, k, q, _t(eta))
    Wk = O.w_block(Vl, k, q)
    ref = R[k + 1] - eta @ Wk
    scale = np.abs(R[k + 1]) + np.abs(eta) @ np.abs(Wk)
    _, V2 = _unpack(Rt.cpu().numpy(), Vt.cpu().numpy(), s, ell)
    assert np.all(np.abs(V2[k + 1][q] - ref) <= TOL64 * scale)


@pytest.mark.parametrize("s,ell,k", [(8, 4, 0), (8, 4, 1), (8, 4, 3), (4, 2, 1), (3, 3, 2), (16, 4, 3), (1, 1, 0)])
def test_level_step_equals_algorithm1(msstab, case, s, ell, k):
    """One level step k as Algorithm 1 writes it (gamma update of all levels,
    then for each q the eta update of all levels and the product with A)
    against the CUDA path's split: top-level gamma and eta updates plus the
    products, then the lazy update of the levels below k."""
    w, A = case
    S = _solver(msstab, A, s, ell)
    R, Vl = _levels(A.n, s, ell, 60 + k)
    x0 = np.random.default_rng(9).standard_normal(A.n)
    rng = np.random.default_rng(10)
    gamma = rng.standard_normal(s)
    etas = rng.standard_normal((s, s)) * 0.5
    # oracle, in the order of Algorithm 1
    Ro = [r.copy() for r in R]
    Vo = [v.copy() for v in Vl]
    xo = x0.copy()
    O.gamma_update(Ro, Vo, xo, gamma, k)
    Ro[k + 1] = A.to_scipy() @ Ro[k]
    for q in range(s):
        O.eta_update(Ro, Vo, k, q, etas[q])
        Vo[k + 2][q] = A.to_scipy() @ Vo[k + 1][q]
    # CUDA path
    Rg, Vg = _pack(R, Vl)
    Rt, Vt, xt = _t(Rg), _t(Vg), _t(x0)
    ld = A.n
    S.op_gamma_update(Rt, Vt, k, _t(gamma))
    S.op_spmv(Rt[k], Rt[k + 1])
    for q in range(s):
        S.op_eta_update(Rt, Vt, k, q, _t(etas[q]))
        S.op_spmv(Vt[(k + 1) * s + q], Vt[(k + 2) * s + q])
    gram = torch.zeros((ell + 1) ** 2, dtype=torch.float64, device=DEV)
    S.op_lazy_update(Rt, Vt, xt, k, _t(gamma), _t(etas), gram)
    Rc, Vc = _unpack(Rt.cpu().numpy(), Vt.cpu().numpy(), s, ell)
    # element-wise against the oracle, each entry within 1e-12 of its
    # propagated scale: the scale of a combination b - sum_j c_j w_j is
    # |b| + sum_j |c_j| scale(w_j), of a product A v it is |A| scale(v) --
    # the bound that the rounding errors of both sides obey (a few dozen
    # chained operations of at most s + 1 terms: far below 1e-12 / 2^-53)
    Sr, Sv, sx = _level_step_scales(A, R, Vl, x0, gamma, etas, k)
    for i in range(ell + 1):
        assert np.all(np.abs(Rc[i] - Ro[i]) <= TOL64 * Sr[i]), ("r", i)
    for i in range(ell + 2):
        assert np.all(np.abs(Vc[i] - Vo[i]) <= TOL64 * Sv[i]), ("V", i - 1)
    assert np.all(np.abs(xt.cpu().numpy() - xo) <= TOL64 * sx)
    # the Gram matrix the lazy kernel returns: the dots of its own output
    # vectors, within 1e-12 of sum |a_i b_i|
    G = np.array([[Rc[a] @ Rc[c] for c in range(ell + 1)] for a in range(ell + 1)])
    Gs = np.array([[np.abs(Rc[a]) @ np.abs(Rc[c]) for c in range(ell + 1)] for a in range(ell + 1)])
    assert np.all(np.abs(gram.cpu().numpy().reshape(ell + 1, ell + 1) - G) <= TOL64 * Gs)


@pytest.mark.parametrize("s", [8, 5, 4])
def test_tau_step_with_fused_lower_level_updates(msstab, s):
    """The FP32 degree-1 step that first applies the level -1 updates of level
    step 0 (x += V^(-1) gamma_0, v_q^(-1) = r^(0) - [V^(0)_{0:q-1}, V^(-1)_{q:s-1}]
    eta_q) in the same pass equals the lower-level update followed by the
    degree-1 step bit for bit (vectors and projections), and both equal the
    oracle's Algorithm-1 order within the FP32 bound."""
    w = pb.WORKLOADS["convdiff3d_24"]      # n = 13824: a multiple of 4
    A = w.matrix()
    ell = 1
    S = _solver(msstab, A, s, ell)
    R, Vl = _levels(A.n, s, ell, 120 + s)
    R = [r_.astype(np.float32).astype(np.float64) for r_ in R]
    Vl = [v_.astype(np.float32).astype(np.float64) for v_ in Vl]
    x0 = np.random.default_rng(17).standard_normal(A.n).astype(np.float32).astype(np.float64)
    rng = np.random.default_rng(18)
    gamma = rng.standard_normal(s)
    etas = rng.standard_normal((s, s)) * 0.5
    tau = rng.standard_normal(ell)
    Rg, Vg = _pack(R, Vl)
    n = A.n
    res = []
    for fused in (False, True):
        Rt, Vt, xt = _padded(Rg, torch.float32), _padded(Vg, torch.float32), _padded(x0[None, :], torch.float32)[0]
        out = torch.zeros(s * s + s + 1, dtype=torch.float64, device=DEV)
        if fused:
            S.op_tau_step(Rt, Vt, xt, _t(tau), out, prec=1, lazy_gamma=_t(gamma), lazy_eta=_t(etas))
        else:
            S.op_lazy_update(Rt, Vt, xt, 0, _t(gamma), _t(etas), prec=1)
            S.op_tau_step(Rt, Vt, xt, _t(tau), out, prec=1)
        res.append((Rt[:, :n].clone(), Vt[:, :n].clone(), xt[:n].clone(), out.clone()))
    (Ra, Va, xa, oa), (Rb, Vb, xb, ob) = res
    assert torch.equal(Ra, Rb) and torch.equal(Va, Vb) and torch.equal(xa, xb) and torch.equal(oa, ob)
    # the oracle: the level -1 part of the gamma and eta updates of level step 0, then the degree-1 step
    Ro, Vo, xo = [r.copy() for r in R], [v.copy() for v in Vl], x0.copy()
    xo = xo + gamma @ Vo[0]
    newV = [Ro[0] - etas[q] @ np.concatenate([Vo[1][:q], Vo[0][q:]], axis=0) for q in range(s)]
    Vo[0] = np.array(newV)
    r, x, U, V = O.tau_update(Ro, Vo, xo, tau)
    Rc, Vc = _unpack(Ra.cpu().numpy().astype(np.float64), Va.cpu().numpy().astype(np.float64), s, ell)
    sc_u = [np.abs(R[0]) + np.abs(etas[q]) @ np.abs(np.concatenate([Vl[1][:q], Vl[0][q:]], axis=0))
            for q in range(s)]
    for q in range(s):
        assert np.all(np.abs(Vc[0][q] - U[q]) <= TOL32 * (sc_u[q] + abs(tau[0]) * np.abs(Vl[1][q]))), q
        assert np.all(np.abs(Vc[1][q] - V[q]) <= TOL32 * (np.abs(Vl[1][q]) + abs(tau[0]) * np.abs(Vl[2][q]))), q
    sx = np.abs(x0) + np.abs(gamma) @ np.abs(Vl[0]) + abs(tau[0]) * np.abs(R[0])
    assert np.all(np.abs(xa.cpu().numpy().astype(np.float64) - x) <= TOL32 * sx)
    assert np.all(np.abs(Rc[0] - r) <= TOL32 * (np.abs(R[0]) + abs(tau[0]) * np.abs(R[1])))


@pytest.mark.parametrize("k", [0, 1, 3])
def test_level_updates_fp32_four_rows(msstab, case, k):
    """The FP32 inner form's gamma, eta and lower-level updates of level step k
    (products with A left out: they only touch levels above k) with the
    solver's vector layout, so that every kernel takes four rows per thread,
    against Algorithm 1's order on the same FP32 values; and bit for bit
    against the row-by-row kernels, which run when the columns are not
    16-byte aligned (leading dimension n = 35937)."""
    w, A = case
    s, ell = 8, 4
    S = _solver(msstab, A, s, ell)
    R, Vl = _levels(A.n, s, ell, 70 + k)
    R = [r_.astype(np.float32).astype(np.float64) for r_ in R]
    Vl = [v_.astype(np.float32).astype(np.float64) for v_ in Vl]
    x0 = np.random.default_rng(15).standard_normal(A.n).astype(np.float32).astype(np.float64)
    rng = np.random.default_rng(16)
    gamma = rng.standard_normal(s)
    etas = rng.standard_normal((s, s)) * 0.5
    Ro, Vo, xo = [r.copy() for r in R], [v.copy() for v in Vl], x0.copy()
    O.gamma_update(Ro, Vo, xo, gamma, k)
    for q in range(s):
        O.eta_update(Ro, Vo, k, q, etas[q])
    Rg, Vg = _pack(R, Vl)
    n = A.n
    runs = []
    for pad in (True, False):
        if pad:
            Rt, Vt, xt = _padded(Rg, torch.float32), _padded(Vg, torch.float32), _padded(x0[None, :], torch.float32)[0]
        else:
            Rt, Vt, xt = _t(Rg, torch.float32), _t(Vg, torch.float32), _t(x0, torch.float32)
        S.op_gamma_update(Rt, Vt, k, _t(gamma), prec=1)
        for q in range(s):
            S.op_eta_update(Rt, Vt, k, q, _t(etas[q]), prec=1)
        S.op_lazy_update(Rt, Vt, xt, k, _t(gamma), _t(etas), prec=1)
        runs.append((Rt[:, :n].clone(), Vt[:, :n].clone(), xt[:n].clone()))
    (Ra, Va, xa), (Rb, Vb, xb) = runs
    assert torch.equal(Ra, Rb) and torch.equal(Va, Vb) and torch.equal(xa, xb)
    Rc, Vc = _unpack(Ra.cpu().numpy().astype(np.float64), Va.cpu().numpy().astype(np.float64), s, ell)
    # the propagated scales of the same operations on absolute values
    Sr = [np.abs(r) for r in R]
    Sv = [np.abs(v) for v in Vl]
    g = np.abs(gamma)
    for i in range(k + 1):
        Sr[i] = Sr[i] + g @ Sv[i + 1]
    sx = np.abs(x0) + g @ Sv[0]
    for q in range(s):
        e = np.abs(etas[q])
        new = [Sr[i + 1] + e @ np.concatenate([Sv[i + 2][:q], Sv[i + 1][q:]], axis=0) for i in range(-1, k + 1)]
        for i, v in zip(range(-1, k + 1), new):
            Sv[i + 1][q] = v
    for i in range(k + 1):
        assert np.all(np.abs(Rc[i] - Ro[i]) <= TOL32 * Sr[i]), ("r", i)
    for i in range(k + 2):
        assert np.all(np.abs(Vc[i] - Vo[i]) <= TOL32 * Sv[i]), ("V", i - 1)
    assert np.all(np.abs(xa.cpu().numpy().astype(np.float64) - xo) <= TOL32 * sx)


def _level_step_scales(A, R, Vl, x0, gamma, etas, k):
    """The propagated magnitudes of one level step of Algorithm 1 (the same
    sequence of operations as the oracle, on absolute values)."""
    Aa = abs(A.to_scipy())
    Sr = [np.abs(r) for r in R]
    Sv = [np.abs(v) for v in Vl]
    g = np.abs(gamma)
    for i in range(k + 1):
        Sr[i] = Sr[i] + g @ Sv[i + 1]
    sx = np.abs(x0) + g @ Sv[0]
    Sr[k + 1] = Aa @ Sr[k]
    for q in range(etas.shape[0]):
        e = np.abs(etas[q])
        new = [Sr[i + 1] + e @ np.concatenate([Sv[i + 2][:q], Sv[i + 1][q:]], axis=0) for i in range(-1, k + 1)]
        for i, v in zip(range(-1, k + 1), new):
            Sv[i + 1][q] = v
        Sv[k + 2][q] = Aa @ Sv[k + 1][q]
    return Sr, Sv, sx


@pytest.mark.parametrize("s,ell", [(8, 4), (4, 2), (1, 1), (16, 4), (5, 3)])
def test_tau_update(msstab, case, s, ell):
    w, A = case
    S = _solver(msstab, A, s, ell)
    R, Vl = _levels(A.n, s, ell, 80 + s)
    x0 = np.random.default_rng(11).standard_normal(A.n)
    tau = np.random.default_rng(12).standard_normal(ell)
    r, x, U, V = O.tau_update(R, Vl, x0, tau)
    Rg, Vg = _pack(R, Vl)
    Rt, Vt, xt = _t(Rg), _t(Vg), _t(x0)
    S.op_tau_update(Rt, Vt, xt, _t(tau))
    Rc, Vc = _unpack(Rt.cpu().numpy(), Vt.cpu().numpy(), s, ell)
    sc = lambda a, terms: np.abs(a) + sum(abs(t_) * np.abs(v_) for t_, v_ in terms)
    assert np.all(np.abs(Rc[0] - r) <= TOL64 * sc(R[0], [(tau[i - 1], R[i]) for i in range(1, ell + 1)]))
    assert np.all(np.abs(xt.cpu().numpy() - x) <= TOL64 * sc(x0, [(tau[i - 1], R[i - 1]) for i in range(1, ell + 1)]))
    for q in range(s):
        assert np.all(np.abs(Vc[1][q] - V[q]) <= TOL64 * sc(Vl[1][q], [(tau[i - 1], Vl[i + 1][q]) for i in range(1, ell + 1)]))
        assert np.all(np.abs(Vc[0][q] - U[q]) <= TOL64 * sc(Vl[0][q], [(tau[i - 1], Vl[i][q]) for i in range(1, ell + 1)]))


def _padded(a, dtype):
    """a (rows x n) in a device array whose leading dimension is n rounded up
    to 64 elements, as the solver's workspace lays its vectors out."""
    rows, n = a.shape
    ld = (n + 63) // 64 * 64
    out = torch.zeros((rows, ld), dtype=dtype, device=DEV)
    out[:, :n] = _t(a, dtype)
    return out


@pytest.mark.parametrize("prec,s,ell,upd,pad", [(0, 8, 4, True, False), (0, 4, 1, True, False),
                                                  (1, 8, 1, True, True), (1, 5, 1, True, True),
                                                  (1, 4, 1, True, True), (1, 8, 1, False, True),
                                                  (1, 8, 1, True, False), (1, 16, 1, True, True),
                                                  (1, 8, 2, True, True)])
def test_tau_step_projections(msstab, case, prec, s, ell, upd, pad):
    """The degree-l step with the fused projections of the next cycle's first
    gamma solve (P^T V^(0), P^T r, r.r), in FP64 and in the FP32 inner form
    (l = 1, s <= 8 and 16-byte aligned columns: four rows per thread, warps
    over chunks of vector groups; otherwise the per-group kernel), against the
    oracle's update and plain FP64 dots of the oracle's vectors.  The padded
    cases lay the vectors out as the solver does (leading dimension a multiple
    of 64), the others with leading dimension n (35937: not 16-byte aligned)."""
    w, A = case
    S = _solver(msstab, A, s, ell)
    R, Vl = _levels(A.n, s, ell, 90 + s + ell)
    x0 = np.random.default_rng(13).standard_normal(A.n)
    tau = np.random.default_rng(14).standard_normal(ell)
    P = O.orthonormalize_mgs2(pb.randn_cols(A.n, s, pb.SEED_P))
    if prec == 1:
        # the FP32 form works on FP32 copies; the oracle takes the same values
        R = [r_.astype(np.float32).astype(np.float64) for r_ in R]
        Vl = [v_.astype(np.float32).astype(np.float64) for v_ in Vl]
        x0 = x0.astype(np.float32).astype(np.float64)
        P = P.astype(np.float32).astype(np.float64)
    dt, tol = (torch.float64, TOL64) if prec == 0 else (torch.float32, TOL32)
    t_ = tau if upd else np.zeros(ell)
    r, x, U, V = O.tau_update(R, Vl, x0, t_)
    Rg, Vg = _pack(R, Vl)
    if pad:
        Rt, Vt, xt = _padded(Rg, dt), _padded(Vg, dt), _padded(x0[None, :], dt)[0]
    else:
        Rt, Vt, xt = _t(Rg, dt), _t(Vg, dt), _t(x0, dt)
    out = torch.zeros(s * s + s + 1, dtype=torch.float64, device=DEV)
    S.op_tau_step(Rt, Vt, xt, _t(tau), out, do_update=upd, prec=prec)
    n = A.n
    Rc, Vc = _unpack(Rt[:, :n].cpu().numpy().astype(np.float64), Vt[:, :n].cpu().numpy().astype(np.float64), s, ell)
    xt = xt[:n]
    sc = lambda a, terms: np.abs(a) + sum(abs(c_) * np.abs(v_) for c_, v_ in terms)
    sr = sc(R[0], [(t_[i - 1], R[i]) for i in range(1, ell + 1)])
    assert np.all(np.abs(Rc[0] - r) <= tol * sr)
    assert np.all(np.abs(xt.cpu().numpy().astype(np.float64) - x)
                  <= tol * sc(x0, [(t_[i - 1], R[i - 1]) for i in range(1, ell + 1)]))
    sv = []
    for q in range(s):
        sv.append(sc(Vl[1][q], [(t_[i - 1], Vl[i + 1][q]) for i in range(1, ell + 1)]))
        assert np.all(np.abs(Vc[1][q] - V[q]) <= tol * sv[q])
        assert np.all(np.abs(Vc[0][q] - U[q]) <= tol * sc(Vl[0][q], [(t_[i - 1], Vl[i][q]) for i in range(1, ell + 1)]))
    o = out.cpu().numpy()
    pv = o[:s * s].reshape(s, s)
    for q in range(s):
        # rounding of the update (scale sv) and of the sums (scale |P||v|)
        bound = tol * (np.abs(P) @ sv[q]) * 4
        assert np.all(np.abs(pv[q] - P @ V[q]) <= bound), (q, np.max(np.abs(pv[q] - P @ V[q]) / bound))
    assert np.all(np.abs(o[s * s:s * s + s] - P @ r) <= tol * (np.abs(P) @ sr) * 4)
    assert abs(o[s * s + s] - r @ r) <= tol * (sr @ sr) * 4


@pytest.mark.parametrize("n", [1, 2, 4, 8, 16])
def test_small_solve(msstab, case, n):
    w, A = case
    S = _solver(msstab, A, 2, 1)
    rng = np.random.default_rng(n)
    for trial in range(5):
        M = rng.standard_normal((n, n))
        z = rng.standard_normal(n)
        out = torch.zeros(n, dtype=torch.float64, device=DEV)
        flag = torch.full((1,), 7, dtype=torch.int32, device=DEV)
        S.op_small_solve(_t(M), _t(z), out, flag)
        assert int(flag.item()) == 0
        ref = O.lu_solve_pp(M, z)
        # componentwise (Skeel) scale |M^-1| |M| |z|: the forward error bound
        # of Gaussian elimination with partial pivoting (the GPU's Gauss-Jordan
        # makes the same eliminations, and its back substitution column-wise)
        scale = np.abs(np.linalg.inv(M)) @ (np.abs(M) @ np.abs(ref))
        assert np.all(np.abs(out.cpu().numpy() - ref) <= TOL64 * scale)


def test_small_solve_breakdown(msstab, case):
    w, A = case
    S = _solver(msstab, A, 2, 1)
    M = np.array([[1.0, 2.0, 3.0], [2.0, 4.0, 6.0], [0.0, 1.0, 1.0]])
    out = torch.zeros(3, dtype=torch.float64, device=DEV)
    flag = torch.zeros(1, dtype=torch.int32, device=DEV)
    S.op_small_solve(_t(M), _t(np.ones(3)), out, flag)
    with pytest.raises(O.Breakdown):
        O.lu_solve_pp(M, np.ones(3))
    assert int(flag.item()) == 1 and not out.cpu().numpy().any()


@pytest.mark.parametrize("ell", [1, 2, 4, 8])
def test_tau_solve(msstab, case, ell):
    w, A = case
    S = _solver(msstab, A, 2, 1)
    rng = np.random.default_rng(ell)
    R = [rng.standard_normal(200) * 10.0 ** rng.integers(-4, 4) for _ in range(ell + 1)]
    G = np.array([[R[a] @ R[c] for c in range(ell + 1)] for a in range(ell + 1)])
    tau = torch.zeros(ell, dtype=torch.float64, device=DEV)
    S.op_tau_solve(_t(G), tau)
    ref = O.tau_from_gram(G)
    # the scaled normal equations Ms y = rs (Ms = D G11 D, rs = D g, tau = D y)
    # in the componentwise scale |Ms^-1| (|Ms| |y| + |rs|), mapped back by D
    d = 1.0 / np.sqrt(np.diag(G)[1:])
    Ms = d[:, None] * G[1:, 1:] * d[None, :]
    rs = d * G[1:, 0]
    y = ref / d
    scale = d * (np.abs(np.linalg.inv(Ms)) @ (np.abs(Ms) @ np.abs(y) + np.abs(rs)))
    assert np.all(np.abs(tau.cpu().numpy() - ref) <= TOL64 * scale)

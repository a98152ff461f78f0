"""ILU(0) split preconditioning (Section 5.1) on the GPU against the oracle.

* The factor is bit-exact: both sides run the IKJ elimination in the same
  order with rounded products and differences (no fused multiply-add).
* The level of every row is an integer fixed by the dependency graph (the
  longest chain below it), checked exactly against its definition.
* Triangular solves (the barrier-free packed sweep for rows with at most 8
  dependencies, the level-by-level sweep otherwise):
  |y_gpu - y_oracle| <= 1e-12 * M(T)^-1 |T| |y|
  componentwise (M(T) the comparison matrix), the bound of the componentwise
  backward error of a triangular solve with c*u = 1e-12 (c17 of the readings:
  1e-12 of the scale of the terms).  U x: 1e-12 of |U| |x| per row.
* The preconditioned operator L^-1 A U^-1: normwise 1e-11 (three stages, each
  within its componentwise bound; the factors of these diagonally dominant
  matrices are well conditioned).
* Solves: the decision-based MV rule of the other solve tests, the true
  preconditioned residual <= tol, the solution against the oracle's.
* At 128^3 (the size the oracle cannot factor in Python in reasonable time)
  the 7-point stencil's factor is checked in closed form on every row: U keeps
  A's strict upper part, l_ik = a_ik / u_kk, and u_ii = a_ii - sum_k l_ik a_ki
  with the same rounded operations, bit for bit.
"""

import numpy as np
import pytest

from oracle import idrstab as O
from oracle import ilu as I
from paper_1604_06043_gb300 import problems as pb
from parity_rules import mvs_match

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


def _t(x, dt=torch.float64):
    return torch.tensor(np.ascontiguousarray(x), dtype=dt, device=DEV)


def _solver(M, A, s=4, ell=2, seed=3, **opt):
    return M.Solver(A, s, ell, pb.randn_cols(A.n, s, seed), device=DEV, precond=M.PRECOND_ILU0, **opt)


def _levels(A, upper):
    """Level of each row from its definition (the longest dependency chain below it)."""
    rp, col = A.row_ptr, A.col
    lev = np.zeros(A.n, dtype=np.int64)
    order = range(A.n - 1, -1, -1) if upper else range(A.n)
    for i in order:
        c = col[rp[i]:rp[i + 1]]
        dep = c[c > i] if upper else c[c < i]
        lev[i] = 1 + lev[dep].max() if dep.size else 0
    return lev


def _stencil_closed_form(A, lu):
    """For a 5/7-point stencil in natural order ILU(0) modifies only the
    diagonal: U's strict upper part is A's, l_ik = a_ik / u_kk, and
    u_ii = a_ii - l_ik1 a_k1i - l_ik2 a_k2i - ... in column order, each product
    and difference rounded (the IKJ elimination's own operations)."""
    rp, col, val = A.row_ptr.astype(np.int64), A.col.astype(np.int64), A.val
    rows = np.repeat(np.arange(A.n), np.diff(rp))
    up, low = col > rows, col < rows
    diag = np.nonzero(col == rows)[0]
    if diag.size != A.n or not np.array_equal(lu[up], val[up]):
        return False
    u = lu[diag]
    if not np.array_equal(lu[low], val[low] / u[col[low]]):
        return False
    key = rows * A.n + col                   # increasing: rows ascending, columns sorted
    exp = val[diag].copy()
    lower_idx = np.nonzero(low)[0]
    first = np.searchsorted(lower_idx, rp[:-1])
    cnt = np.bincount(rows[low], minlength=A.n)
    for j in range(int(cnt.max())):
        has = cnt > j
        p = lower_idx[first[has] + j]
        i_rows = np.nonzero(has)[0]
        q = np.searchsorted(key, col[p] * A.n + i_rows)     # a_ki, row k's entry in column i
        if not np.array_equal(key[q], col[p] * A.n + i_rows):
            return False
        exp[has] = exp[has] - lu[p] * val[q]
    return bool(np.array_equal(u, exp))


MATRICES = {
    "convdiff3d_24": lambda: pb.WORKLOADS["convdiff3d_24"].matrix(),
    "convdiff2d_32": lambda: pb.WORKLOADS["convdiff2d_32"].matrix(),
    "random_3000": lambda: pb.random_sparse(3000, 6, seed=21),
    "random_band_5000": lambda: pb.random_sparse(5000, 5, seed=22, band=40),
    "tridiag_40": lambda: pb.tridiag(40, 2.0, 3.0, 1.0),
    "random_wide_2000": lambda: pb.random_sparse(2000, 24, seed=23),   # > 8 per side: level-by-level sweeps
}


@pytest.mark.parametrize("name", list(MATRICES))
def test_factor_bit_exact_and_levels(M, name):
    A = MATRICES[name]()
    S = _solver(M, A, s=2)
    lu = torch.empty(A.nnz, dtype=torch.float64, device=DEV)
    S.op_ilu_factor(lu)
    assert np.array_equal(lu.cpu().numpy(), I.ilu0(A))
    ll = torch.empty(A.n, dtype=torch.int32, device=DEV)
    lup = torch.empty(A.n, dtype=torch.int32, device=DEV)
    info = S.op_ilu_levels(ll, lup)
    el, eu = _levels(A, False), _levels(A, True)
    assert np.array_equal(ll.cpu().numpy(), el) and np.array_equal(lup.cpu().numpy(), eu)
    assert info[0] == el.max() + 1 and info[1] == eu.max() + 1
    assert info[2] == np.bincount(el).max() and info[3] == np.bincount(eu).max()
    if name == "convdiff3d_24":
        assert info[0] == info[1] == 3 * 24 - 2      # the planes x + y + z = const
    S.close()


@pytest.mark.parametrize("name", ["convdiff3d_24", "random_3000", "random_band_5000", "random_wide_2000",
                                  "tridiag_40"])
def test_triangular_solves_and_operator(M, name):
    A = MATRICES[name]()
    F = I.Factors.from_values(A, I.ilu0(A))
    S = _solver(M, A, s=2)
    rng = np.random.default_rng(5)
    z = rng.standard_normal(A.n)
    zt = _t(z)
    y = torch.empty_like(zt)
    for which, low in ((0, True), (1, False)):
        S.op_ilu_apply(which, zt, y)
        ref = F.lower_solve(z) if low else F.upper_solve(z)
        sc = I.comparison_scale(F, ref, lower=low)
        err = np.abs(y.cpu().numpy() - ref)
        assert np.all(err <= 1e-12 * sc), (which, float((err / sc).max()))
        # in place
        w_ = zt.clone()
        S.op_ilu_apply(which, w_, w_)
        assert torch.equal(w_, y)
    S.op_ilu_apply(2, zt, y)
    absU = abs(F.U)
    ref = F.upper_mul(z)
    assert np.all(np.abs(y.cpu().numpy() - ref) <= 1e-12 * (absU @ np.abs(z)))
    S.op_ilu_apply(3, zt, y)
    ref = I.SplitOperator(A, F) @ z
    assert np.linalg.norm(y.cpu().numpy() - ref) <= 1e-11 * np.linalg.norm(ref)
    S.close()


def test_large_level_groups_in_a_chunk(M):
    """Runs of 1400 independent rows coupled to the runs beside them: with one
    row chunk per SM (about 3000 rows) a chunk's level holds more rows than the
    1024 values the sweep keeps in shared memory and than the 512 threads of a
    block, so that dependencies beyond the buffer come from the global vector
    and threads take several positions of one level; chunk borders fall inside
    levels."""
    A = pb.offset_coupled(152 * 3000, 1400, -1.0, 4.0, -1.5)
    F = I.Factors.from_values(A, I.ilu0(A))
    S = _solver(M, A, s=2)
    lev = S.op_ilu_levels()
    assert lev[0] == lev[1] == -(-A.n // 1400) and lev[2] == lev[3] == 1400   # the runs are the levels
    z = np.random.default_rng(8).standard_normal(A.n)
    zt = _t(z)
    y = torch.empty_like(zt)
    for which, low in ((0, True), (1, False)):
        S.op_ilu_apply(which, zt, y)
        ref = F.lower_solve(z) if low else F.upper_solve(z)
        sc = I.comparison_scale(F, ref, lower=low)
        err = np.abs(y.cpu().numpy() - ref)
        assert np.all(err <= 1e-12 * sc), (which, float((err / sc).max()))
    S.close()


def test_exact_factor_gives_the_identity(M):
    A = MATRICES["tridiag_40"]()
    S = _solver(M, A, s=2)
    v = _t(np.random.default_rng(6).standard_normal(A.n))
    y = torch.empty_like(v)
    S.op_ilu_apply(3, v, y)
    assert torch.max(torch.abs(y - v)).item() <= 1e-13 * torch.max(torch.abs(v)).item()
    S.close()


def test_preconditioned_solve_matches_oracle(M):
    w = pb.WORKLOADS["convdiff3d_24"]
    A = w.matrix()
    b = w.x0() / w.tau + w.f()
    F = I.Factors.from_values(A, I.ilu0(A))
    P = O.orthonormalize_mgs2(w.p_raw())
    ref, xo, rel = I.precond_solve(A, F, b, w.x0(), w.s, w.ell, P, tol=w.tol)
    S = M.Solver(A, w.s, w.ell, w.p_raw(), device=DEV, precond=M.PRECOND_ILU0, replace_every=1,
                 fetch_policy=M.FETCH_NEVER, kernel_timing=1)
    x = _t(w.x0())
    st = S.solve(_t(b), x, w.tol)
    hist, _ = S.history()
    assert st.status == 0 and st.relres_true <= w.tol
    assert mvs_match(st.mvs, ref.mvs, hist, ref.history, w.tol), (st.mvs, ref.mvs, hist, ref.history)
    xn = x.cpu().numpy()
    assert np.linalg.norm(xn - xo) <= 1e-6 * np.linalg.norm(xo)
    r = b - A.to_scipy() @ xn
    assert abs(st.relres_orig - np.linalg.norm(r) / np.linalg.norm(b)) <= 1e-3 * st.relres_orig
    assert st.n_launch[8] > 0          # the ILU(0) sweeps ran
    S.close()


def test_preconditioned_sequence_matches_oracle(M):
    w = pb.WORKLOADS["convdiff3d_33"]
    A = w.matrix()
    steps = 3
    o = I.precond_sequence(A, w.f(), w.x0(), w.tau, steps, w.s, w.ell, w.p_raw(), tol=w.tol)
    S = M.Solver(A, w.s, w.ell, w.p_raw(), device=DEV, precond=M.PRECOND_ILU0, replace_every=1)
    f = _t(w.f())
    x = _t(w.x0())
    b = torch.empty_like(x)
    As = A.to_scipy()
    xprev = w.x0()
    for i, r in enumerate(o.solves):
        S.op_axpby(1.0 / w.tau, x, 1.0, f, b)
        st = S.solve(b, x, w.tol)
        hist, _ = S.history()
        assert st.status == 0 and st.relres_true <= w.tol, i
        assert mvs_match(st.mvs, r.mvs, hist, r.history, w.tol), (i, st.mvs, r.mvs, hist, r.history)
        xn = x.cpu().numpy()
        bn = xprev / w.tau + w.f()
        assert abs(st.relres_orig - np.linalg.norm(bn - As @ xn) / np.linalg.norm(bn)) <= 1e-3 * st.relres_orig
        if i == 0:
            assert st.fetched == 1
        else:
            assert st.used_recycle == 1
        xprev = xn
    assert np.linalg.norm(xprev - o.x) <= 1e-6 * np.linalg.norm(o.x)
    S.close()


def test_invalid_inputs_are_rejected(M):
    A = pb.WORKLOADS["convdiff3d_24"].matrix()
    with pytest.raises(M.MsstabError) as e:
        M.Solver(A, 2, 2, pb.randn_cols(A.n, 2, 3), device=DEV, precond=M.PRECOND_ILU0,
                 precision=M.PREC_FP32_INNER)
    assert e.value.status == M.ERR_INVALID_ARG
    with pytest.raises(M.MsstabError) as e:
        M.Solver(A, 2, 2, pb.randn_cols(A.n, 2, 3), device=DEV, precond=7)
    assert e.value.status == M.ERR_INVALID_ARG
    # no diagonal in row 1; unsorted columns; a zero pivot
    nodiag = pb.CSR(2, np.array([0, 1, 2], dtype=np.int32), np.array([0, 0], dtype=np.int32), np.array([1.0, 1.0]))
    unsorted = pb.CSR(2, np.array([0, 2, 3], dtype=np.int32), np.array([1, 0, 1], dtype=np.int32),
                      np.array([1.0, 2.0, 1.0]))
    zero = pb.CSR(2, np.array([0, 2, 4], dtype=np.int32), np.array([0, 1, 0, 1], dtype=np.int32),
                  np.array([0.0, 1.0, 1.0, 0.0]))
    for B, code in ((nodiag, M.ERR_INVALID_ARG), (unsorted, M.ERR_INVALID_ARG), (zero, M.ERR_BREAKDOWN)):
        with pytest.raises(M.MsstabError) as e:
            M.Solver(B, 1, 1, pb.randn_cols(2, 1, 3), device=DEV, precond=M.PRECOND_ILU0)
        assert e.value.status == code
    S = M.Solver(A, 2, 2, pb.randn_cols(A.n, 2, 3), device=DEV)
    with pytest.raises(M.MsstabError):
        S.op_ilu_factor(torch.empty(A.nnz, dtype=torch.float64, device=DEV))
    S.close()


def test_128_factor_closed_form_every_row(M):
    w = pb.WORKLOADS["convdiff3d_128"]
    A = w.matrix()
    S = M.Solver(A, w.s, w.ell, w.p_raw(), device=DEV, precond=M.PRECOND_ILU0, replace_every=1)
    lu_t = torch.empty(A.nnz, dtype=torch.float64, device=DEV)
    S.op_ilu_factor(lu_t)
    lu = lu_t.cpu().numpy()
    info = S.op_ilu_levels()
    assert info[0] == info[1] == 3 * 128 - 2
    assert _stencil_closed_form(A, lu)
    # one preconditioned solve of the sequence's first system
    b = w.x0() / w.tau + w.f()
    x = _t(w.x0())
    st = S.solve(_t(b), x, w.tol)
    assert st.status == 0 and st.relres_true <= w.tol
    r = b - A.to_scipy() @ x.cpu().numpy()
    assert abs(np.linalg.norm(r) / np.linalg.norm(b) - st.relres_orig) <= 1e-3 * st.relres_orig
    print("128^3 ILU(0): first system %d MVs, %d cycles, %.1f ms, preconditioned relres %.2e, original %.2e"
          % (st.mvs, st.cycles, st.ms, st.relres_true, st.relres_orig))
    S.close()


def test_csr_format_and_zero_rhs(M):
    # the operator with the CSR product (the factor and sweeps are format-independent)
    w = pb.WORKLOADS["convdiff3d_24"]
    A = w.matrix()
    b = w.x0() / w.tau + w.f()
    F = I.Factors.from_values(A, I.ilu0(A))
    ref, xo, _ = I.precond_solve(A, F, b, w.x0(), w.s, w.ell, O.orthonormalize_mgs2(w.p_raw()), tol=w.tol)
    S = M.Solver(A, w.s, w.ell, w.p_raw(), device=DEV, precond=M.PRECOND_ILU0, replace_every=1,
                 fetch_policy=M.FETCH_NEVER, spmv_format=M.FORMAT_CSR)
    x = _t(w.x0())
    st = S.solve(_t(b), x, w.tol)
    hist, _ = S.history()
    assert st.status == 0 and mvs_match(st.mvs, ref.mvs, hist, ref.history, w.tol)
    assert np.linalg.norm(x.cpu().numpy() - xo) <= 1e-6 * np.linalg.norm(xo)
    # b = 0: x = 0 without a product
    x = _t(w.x0())
    st = S.solve(torch.zeros(A.n, dtype=torch.float64, device=DEV), x, w.tol)
    assert st.status == 0 and st.mvs == 0 and not x.cpu().numpy().any()
    # entry-point argument checks
    y = torch.empty_like(x)
    with pytest.raises(M.MsstabError) as e:
        S.op_ilu_apply(4, x, y)
    assert e.value.status == M.ERR_INVALID_ARG
    with pytest.raises(M.MsstabError) as e:
        S.op_ilu_apply(2, x, x)
    assert e.value.status == M.ERR_INVALID_ARG
    S.close()

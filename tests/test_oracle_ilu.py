"""Pins of the ILU(0) oracle (split preconditioning of Section 5.1).

ILU(0) is fixed by its definition: L unit lower and U upper triangular, the
pattern of L + U that of A, and (L U)_ij = a_ij on that pattern.  These
equations have one solution when the pivots are non-zero, so checking them by
a dense product pins the factor completely.  Further pins: a tridiagonal
matrix has no fill, so ILU(0) is its exact LU (scipy's LU, with no row swaps
for these matrices); for the 5-point stencil in natural ordering L U - A is
non-zero exactly on the two fill diagonals at offsets +-(n - 1); for the
5- and 7-point stencils U keeps A's strict upper part (only the diagonal is
modified); triangular solves against dense solves; on an exactly factorised
matrix the preconditioned operator is the identity; and the preconditioned
solver's residual replacement, MV count and solution.
"""

import numpy as np
import pytest
import scipy.linalg as sla

from oracle import ilu as I
from oracle import idrstab as O
from paper_1604_06043_gb300 import problems as pb


def _dense_factors(A, lu):
    F = I.Factors.from_values(A, lu)
    return F, F.L.toarray(), F.U.toarray()


def _check_definition(A, lu, rtol=1e-13):
    F, L, U = _dense_factors(A, lu)
    D = A.to_dense()
    mask = D != 0
    assert np.array_equal(np.diag(L), np.ones(A.n))
    assert np.all(np.triu(L, 1) == 0) and np.all(np.tril(U, -1) == 0)
    assert not np.any((L - np.eye(A.n) != 0) & ~mask) and not np.any((U != 0) & ~mask)
    LU = L @ U
    scale = np.abs(L) @ np.abs(U)
    err = np.abs(LU - D)[mask]
    return bool(np.all(err <= rtol * scale[mask])), LU, D


@pytest.mark.parametrize("A", [pb.convdiff((6, 6, 6), (20.0, 10.0, 5.0), tau=0.005),
                               pb.convdiff((9, 9), (10.0, 10.0), tau=0.01),
                               pb.random_sparse(80, 5, seed=11),
                               pb.random_sparse(120, 4, seed=12, band=9)])
def test_factor_satisfies_the_definition(A):
    ok, _, _ = _check_definition(A, I.ilu0(A))
    assert ok


def test_definition_check_rejects_planted_mistakes():
    A = pb.random_sparse(60, 5, seed=13)
    lu = I.ilu0(A)
    dg = I.diag_positions(A)
    rows = np.repeat(np.arange(A.n), np.diff(A.row_ptr))
    low = np.nonzero(A.col < rows)[0]
    # an L entry left undivided by its pivot
    bad = lu.copy()
    p = low[len(low) // 2]
    bad[p] = A.val[p]
    assert not _check_definition(A, bad)[0]
    # an update with the wrong sign on one diagonal
    i = int(np.nonzero(lu[dg] != A.val[dg])[0][-1])     # a row whose diagonal was updated
    bad = lu.copy()
    bad[dg[i]] = 2 * A.val[dg[i]] - lu[dg[i]]
    assert not _check_definition(A, bad)[0]
    # the factor of the transpose
    At = pb.CSR(A.n, *(lambda m: (m.indptr.astype(np.int32), m.indices.astype(np.int32), m.data))(
        A.to_scipy().T.tocsr().sorted_indices()))
    assert not np.allclose(I.ilu0(At), lu)


def test_tridiagonal_factor_is_the_exact_lu():
    # tridiag(2, 3, 1) of the termination experiments: no fill, so ILU(0) = LU;
    # |u_ii| > 2 keeps partial pivoting from swapping rows
    A = pb.tridiag(40, 2.0, 3.0, 1.0)
    _, L, U = _dense_factors(A, I.ilu0(A))
    Pm, Ls, Us = sla.lu(A.to_dense())
    assert np.array_equal(Pm, np.eye(A.n))
    np.testing.assert_allclose(L, Ls, rtol=0, atol=1e-15)
    np.testing.assert_allclose(U, Us, rtol=0, atol=1e-14)


def test_five_point_fill_lies_on_the_two_dropped_diagonals():
    nx, ny = 7, 7
    A = pb.convdiff((nx, ny), (10.0, 5.0), tau=0.01)
    ok, LU, D = _check_definition(A, I.ilu0(A))
    assert ok
    R = LU - D
    i, j = np.nonzero(np.abs(R) > 1e-12 * np.abs(D).max())
    assert set((j - i).tolist()) == {nx - 1, -(nx - 1)}


@pytest.mark.parametrize("shape", [(7, 7), (5, 5, 5)])
def test_stencil_factor_keeps_the_strict_upper_part(shape):
    A = pb.convdiff(shape, (20.0, 10.0, 5.0)[:len(shape)], tau=0.005)
    lu = I.ilu0(A)
    rows = np.repeat(np.arange(A.n), np.diff(A.row_ptr))
    up = A.col > rows
    assert np.array_equal(lu[up], A.val[up])


def test_triangular_solves_match_dense_solves():
    A = pb.convdiff((8, 8, 8), (20.0, 10.0, 5.0), tau=0.005)
    F, L, U = _dense_factors(A, I.ilu0(A))
    z = np.random.default_rng(1).standard_normal(A.n)
    np.testing.assert_allclose(F.lower_solve(z), np.linalg.solve(L, z), rtol=1e-12, atol=1e-12 * np.abs(z).max())
    y = F.upper_solve(z)
    np.testing.assert_allclose(y, np.linalg.solve(U, z), rtol=1e-12, atol=1e-12 * np.abs(y).max())
    np.testing.assert_allclose(F.upper_mul(z), U @ z, rtol=1e-14, atol=1e-14 * np.abs(U @ z).max())
    # the comparison-matrix scale bounds |y| componentwise (|y| = |T^-1 T y|)
    for low, yy in ((True, F.lower_solve(z)), (False, y)):
        sc = I.comparison_scale(F, yy, lower=low)
        assert np.all(sc >= np.abs(yy) * (1 - 1e-12))


def test_exact_factor_gives_the_identity_operator():
    # (the preconditioned method itself has nothing to do then: its Krylov
    # spaces are one-dimensional and the s x s projections degenerate)
    A = pb.tridiag(64, 2.0, 3.0, 1.0)
    F = I.Factors.from_values(A, I.ilu0(A))
    v = np.random.default_rng(2).standard_normal(A.n)
    np.testing.assert_allclose(I.SplitOperator(A, F) @ v, v, rtol=0, atol=1e-12 * np.abs(v).max())
    b = np.random.default_rng(3).random(A.n)
    np.testing.assert_allclose(F.upper_solve(F.lower_solve(b)), np.linalg.solve(A.to_dense(), b), rtol=1e-12)


def test_preconditioned_solve_counts_and_residuals():
    w = pb.WORKLOADS["convdiff3d_24"]
    A = w.matrix()
    s, ell = w.s, w.ell
    P = O.orthonormalize_mgs2(w.p_raw())
    b = w.x0() / w.tau + w.f()
    F = I.Factors.from_values(A, I.ilu0(A))
    res, x, rel = I.precond_solve(A, F, b, w.x0(), s, ell, P, tol=1e-8)
    assert res.status == O.OK
    # replacement after every cycle: the final recursive residual is the true preconditioned one
    bt = F.lower_solve(b)
    rt = bt - I.SplitOperator(A, F) @ F.upper_mul(x)
    assert np.linalg.norm(rt) <= 1e-8 * np.linalg.norm(bt) * 1.0001
    assert res.mvs == 1 + s + res.cycles * (ell * (s + 1) + 1)
    assert rel < 1e-6
    plain = O.idrstab(A, b, w.x0(), s, ell, P, tol=1e-8, replace_every=1)
    assert res.mvs < plain.mvs


def test_zero_pivot_is_reported():
    # [[0, 1], [1, 0]] has a structural diagonal but ILU(0) = LU needs u_11 != 0
    A = pb.CSR(2, np.array([0, 2, 4], dtype=np.int32), np.array([0, 1, 0, 1], dtype=np.int32),
               np.array([0.0, 1.0, 1.0, 0.0]))
    with pytest.raises(I.ZeroPivot):
        I.ilu0(A)
    B = pb.CSR(2, np.array([0, 1, 2], dtype=np.int32), np.array([1, 0], dtype=np.int32), np.array([1.0, 1.0]))
    with pytest.raises(ValueError):
        I.ilu0(B)


def test_preconditioned_sequence_recycles_in_the_preconditioned_space():
    w = pb.WORKLOADS["convdiff3d_24"]
    A = w.matrix()
    seq = I.precond_sequence(A, w.f(), w.x0(), w.tau, 3, w.s, w.ell, w.p_raw(), tol=1e-8)
    s, ell = w.s, w.ell
    first, later = seq.solves[0], seq.solves[1:]
    assert all(r.status == O.OK for r in seq.solves) and len(seq.solves) == 3
    # system 1: Arnoldi start, fetch with V := A~ U (s products); later: recycled start
    assert first.mvs == 1 + s + first.cycles * (ell * (s + 1) + 1) + s
    for r in later:
        assert r.mvs == 1 + r.cycles * (ell * (s + 1) + 1)
    assert max(seq.relres_orig) < 1e-6

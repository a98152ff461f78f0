"""The seeded input generators: stencils against an explicit loop assembly,
sizes of the measured workloads, and properties of the coefficient field."""

import numpy as np
import pytest

from paper_1604_06043_gb300 import problems as pb


def _dense_2d(n, beta, tau):
    h = 1.0 / (n + 1)
    N = n * n
    A = np.zeros((N, N))
    for j in range(n):
        for i in range(n):
            p = i + n * j
            A[p, p] = 1.0 / tau + 4.0 / h**2
            for di, dj, b in ((1, 0, beta[0]), (-1, 0, -beta[0]), (0, 1, beta[1]), (0, -1, -beta[1])):
                ii, jj = i + di, j + dj
                if 0 <= ii < n and 0 <= jj < n:
                    A[p, ii + n * jj] = -1.0 / h**2 + b / (2.0 * h)
    return A


def test_convdiff_2d_matches_loop_assembly():
    A = pb.convdiff((6, 6), (10.0, -3.0), tau=0.01)
    np.testing.assert_allclose(A.to_dense(), _dense_2d(6, (10.0, -3.0), 0.01), rtol=1e-15)
    # columns ascending within each row
    for i in range(A.n):
        c = A.col[A.row_ptr[i]:A.row_ptr[i + 1]]
        assert np.all(np.diff(c) > 0)


def test_convdiff_3d_constant_kappa_is_kronecker_sum():
    n, beta, tau = 5, (20.0, 10.0, 5.0), 0.005
    h = 1.0 / (n + 1)
    I = np.eye(n)

    def d1(b):
        return (np.diag(np.full(n, 2.0)) - np.eye(n, k=1) - np.eye(n, k=-1)) / h**2 + \
            b * (np.eye(n, k=1) - np.eye(n, k=-1)) / (2 * h)

    # x fastest: index = i + n j + n^2 k  ->  kron(z, y, x)
    L = np.kron(np.kron(I, I), d1(beta[0])) + np.kron(np.kron(I, d1(beta[1])), I) + \
        np.kron(np.kron(d1(beta[2]), I), I)
    ref = L + np.eye(n**3) / tau
    np.testing.assert_allclose(pb.convdiff((n, n, n), beta, tau=tau).to_dense(), ref, rtol=1e-14, atol=1e-9)


def test_variable_kappa_symmetric_without_convection():
    kap = pb.lognormal_kappa((6, 6, 6), corr=2.0)
    A = pb.convdiff((6, 6, 6), (0.0, 0.0, 0.0), kappa=kap).to_dense()
    np.testing.assert_allclose(A, A.T, rtol=1e-14)
    # weakly diagonally dominant, strictly on rows touching the boundary
    off = np.abs(A).sum(1) - np.abs(np.diag(A))
    assert np.all(np.diag(A) >= off * (1 - 1e-12))


def test_lognormal_field_statistics():
    kap = pb.lognormal_kappa((32, 32, 32), sigma=1.0, corr=4.0)
    g = np.log(kap)
    assert abs(g.mean()) < 1e-12 and abs(g.std() - 1.0) < 1e-12
    # correlated: neighbours along x are much more alike than independent draws
    g3 = g.reshape(32, 32, 32)
    c = np.corrcoef(g3[:, :, :-1].ravel(), g3[:, :, 1:].ravel())[0, 1]
    assert c > 0.9


@pytest.mark.parametrize("name,n,nnz", [("convdiff2d_32", 1024, 4992)])
def test_workload_sizes_small(name, n, nnz):
    A = pb.WORKLOADS[name].matrix()
    assert A.n == n and A.nnz == nnz


def test_workload_size_formulas():
    # 7-point stencil: 7 N - 6 n^2 entries (one missing neighbour per boundary face)
    for n in (128, 256):
        assert 7 * n**3 - 6 * n**2 == {128: 14581760, 256: 117047296}[n]
    A = pb.convdiff((12, 12, 12), (1.0, 1.0, 1.0), tau=1.0)
    assert A.nnz == 7 * 12**3 - 6 * 12**2


def test_seeds_are_reproducible():
    w = pb.WORKLOADS["convdiff2d_32"]
    np.testing.assert_array_equal(w.f(), pb.uniform(1024, 1))
    assert not np.array_equal(w.f(), w.x0())
    assert w.p_raw().shape == (4, 1024)


def test_tridiag_orientation():
    T = pb.tridiag(5, 2.0, 3.0, 1.0).to_dense()
    assert T[1, 0] == 2.0 and T[1, 1] == 3.0 and T[1, 2] == 1.0


def test_random_sparse_pattern():
    for band in (None, 7):
        A = pb.random_sparse(300, 6, seed=9, band=band)
        rp, col, val = A.row_ptr, A.col, A.val
        assert rp[0] == 0 and rp[-1] == col.size == val.size
        for i in range(A.n):
            c = col[rp[i]:rp[i + 1]]
            v = val[rp[i]:rp[i + 1]]
            assert np.all(np.diff(c) > 0) and i in c                 # sorted, unique, diagonal present
            if band is not None:
                assert np.all(np.abs(c - i) <= band)
            d = v[c == i][0]
            assert d > np.abs(v[c != i]).sum()                        # strict diagonal dominance
    B = pb.random_sparse(300, 6, seed=9)
    C = pb.random_sparse(300, 6, seed=9)
    assert np.array_equal(B.col, C.col) and np.array_equal(B.val, C.val)


def test_offset_coupled_pattern():
    A = pb.offset_coupled(50, 7, -1.0, 4.0, -1.5)
    D = A.to_scipy().toarray()
    i = np.arange(50)
    ref = 4.0 * np.eye(50) - np.eye(50, k=-7) - 1.5 * np.eye(50, k=7)
    assert np.array_equal(D, ref)
    for r in range(A.n):
        c = A.col[A.row_ptr[r]:A.row_ptr[r + 1]]
        assert np.all(np.diff(c) > 0) and r in c
    assert A.nnz == 50 + 2 * (50 - 7) and i.size == 50

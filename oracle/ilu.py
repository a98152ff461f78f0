"""FP64 CPU oracle: ILU(0) split preconditioning of the systems of a sequence.

TEST INFRASTRUCTURE ONLY (see the package docstring): the product path never
imports this module.

Section 5.1 solves its ocean sequence with a split preconditioner from an
incomplete LU factorisation with zero fill-in: the systems become
L^-1 A R^-1 x~ = L^-1 b, the solution is x = R^-1 x~, and after each cycle the
recursive residual is replaced by L^-1 (b - A R^-1 x~).  Here L is unit lower
triangular and R (called U below, as in most texts) upper triangular, both on
the sparsity pattern of A.

ILU(0) is the plain definition: the factors L (unit lower) and U (upper) whose
combined pattern is the pattern of A and whose product agrees with A on that
pattern, computed row by row by Gaussian elimination in which every update that
would land outside the pattern is dropped (the IKJ ordering of the
elimination: row i is reduced by the already finished rows k < i of its strict
lower part, in increasing k).  The factor values are stored on A's own CSR
pattern: entries left of the diagonal hold L (its unit diagonal is implicit),
the rest hold U.

Python floats are IEEE doubles, and every update here is one multiplication
and one subtraction, each rounded (no fused multiply-add), so a device
implementation that performs the same operations in the same order without
contraction reproduces these values bit for bit.

The triangular solves use scipy's sparse triangular solver as a library step.
"""

from __future__ import annotations

import dataclasses
import math
from typing import Optional

import numpy as np

from .idrstab import MatVec, OK, idrstab, orthonormalize_mgs2, cholqr2


class ZeroPivot(ArithmeticError):
    """A diagonal entry of U is zero: ILU(0) does not exist for this ordering."""


def diag_positions(A) -> np.ndarray:
    """Index of the diagonal entry in each row (columns must be strictly increasing)."""
    rp, col = A.row_ptr, A.col
    dg = np.empty(A.n, dtype=np.int64)
    for i in range(A.n):
        row = col[rp[i]:rp[i + 1]]
        if np.any(np.diff(row) <= 0):
            raise ValueError("columns of row %d are not strictly increasing" % i)
        hit = np.nonzero(row == i)[0]
        if hit.size != 1:
            raise ValueError("row %d has no diagonal entry" % i)
        dg[i] = rp[i] + hit[0]
    return dg


def ilu0(A) -> np.ndarray:
    """The ILU(0) factor values on A's pattern (IKJ elimination, Python loops)."""
    rp = [int(v) for v in A.row_ptr]
    col = [int(v) for v in A.col]
    lu = [float(v) for v in A.val]
    dg = [int(v) for v in diag_positions(A)]
    for i in range(A.n):
        end_i = rp[i + 1]
        for p in range(rp[i], dg[i]):
            k = col[p]
            piv = lu[dg[k]]
            if piv == 0.0:
                raise ZeroPivot(k)
            lik = lu[p] / piv
            lu[p] = lik
            # row i minus l_ik times the upper part of row k, on row i's pattern
            q, t, end_k = dg[k] + 1, p + 1, rp[k + 1]
            while q < end_k and t < end_i:
                if col[q] == col[t]:
                    lu[t] = lu[t] - lik * lu[q]
                    q += 1
                    t += 1
                elif col[q] < col[t]:
                    q += 1
                else:
                    t += 1
        if lu[dg[i]] == 0.0:
            raise ZeroPivot(i)
    return np.array(lu, dtype=np.float64)


@dataclasses.dataclass
class Factors:
    """L (unit lower, strict part stored) and U (upper with diagonal) as scipy CSR."""

    L: object
    U: object

    @staticmethod
    def from_values(A, lu: np.ndarray) -> "Factors":
        import scipy.sparse as sp
        rows = np.repeat(np.arange(A.n), np.diff(A.row_ptr))
        col = A.col.astype(np.int64)
        lower = col < rows
        Ls = sp.csr_matrix((lu[lower], (rows[lower], col[lower])), shape=(A.n, A.n))
        Ls = Ls + sp.identity(A.n, format="csr")
        Us = sp.csr_matrix((lu[~lower], (rows[~lower], col[~lower])), shape=(A.n, A.n))
        Ls.sort_indices()
        Us.sort_indices()
        return Factors(Ls, Us)

    def lower_solve(self, z: np.ndarray) -> np.ndarray:
        """L^-1 z."""
        from scipy.sparse.linalg import spsolve_triangular
        return spsolve_triangular(self.L, z, lower=True, unit_diagonal=True)

    def upper_solve(self, v: np.ndarray) -> np.ndarray:
        """U^-1 v."""
        from scipy.sparse.linalg import spsolve_triangular
        return spsolve_triangular(self.U, v, lower=False)

    def upper_mul(self, x: np.ndarray) -> np.ndarray:
        """U x."""
        return self.U @ x


class SplitOperator:
    """v -> L^-1 A U^-1 v, the operator of the split-preconditioned system."""

    def __init__(self, A, F: Factors):
        self.A = A.to_scipy()
        self.F = F
        self.shape = self.A.shape

    def __matmul__(self, v: np.ndarray) -> np.ndarray:
        return self.F.lower_solve(self.A @ self.F.upper_solve(v))


def comparison_scale(F: Factors, y: np.ndarray, lower: bool) -> np.ndarray:
    """Componentwise scale of the rounding error of a triangular solve T y = z.

    The computed solution satisfies (T + dT) y^ = z with |dT| <= c u |T|, so
    |y^ - y| <= c u |T^-1| |T| |y^|; and |T^-1| <= M(T)^-1 for the comparison
    matrix M(T) (diagonal |t_ii|, off-diagonals -|t_ij|) of a triangular T.
    Returns M(T)^-1 (|T| |y|), computed without cancellation (all terms >= 0)."""
    from scipy.sparse.linalg import spsolve_triangular
    T = (F.L if lower else F.U).tocsr(copy=True)
    T.data = np.abs(T.data)
    rhs = T @ np.abs(y)
    d = T.diagonal()
    M = -T
    M.setdiag(d)
    M.sort_indices()
    return spsolve_triangular(M.tocsr(), rhs, lower=lower)


def precond_solve(A, F: Factors, b, x, s, ell, P, U=None, V=None, tol=1e-8, *, mv: Optional[MatVec] = None,
                  **kw):
    """One split-preconditioned solve: b~ = L^-1 b, x~ = U x, IDR(s)stab(l) on
    L^-1 A U^-1 with the true residual L^-1 (b - A U^-1 x~) replacing the
    recursive one after every cycle (Section 5.1), then x = U^-1 x~.

    Returns (result of the preconditioned solve, x, ||b - A x|| / ||b||)."""
    mv = mv or MatVec(SplitOperator(A, F))
    bt = F.lower_solve(np.asarray(b, dtype=np.float64))
    xt = F.upper_mul(np.asarray(x, dtype=np.float64))
    kw.setdefault("replace_every", 1)
    res = idrstab(mv.A, bt, xt, s, ell, P, U, V, tol, mv=mv, **kw)
    xo = F.upper_solve(res.x)
    nb = float(np.linalg.norm(b))
    rel = float(np.linalg.norm(b - A.to_scipy() @ xo)) / nb if nb > 0 else 0.0
    return res, xo, rel


@dataclasses.dataclass
class PrecondSequenceResult:
    x: np.ndarray
    solves: list
    relres_orig: list


def precond_sequence(A, f, x0, tau_t, steps, s, ell, P_raw, tol=1e-8, *, policy="once", lu=None,
                     fetch_threshold=None, max_mvs=None, on_solve=None) -> PrecondSequenceResult:
    """The implicit-Euler sequence of the M(s)stab driver, each system solved
    with the ILU(0) split preconditioner; the recycled U, V live in the
    preconditioned space (V = L^-1 A U^-1 U), which is fixed because A is.
    Policies "once" and "never" as in the unpreconditioned driver; the basis is
    conditioned at the fetch (V := A~ U, s counted products, Cholesky QR twice)."""
    if lu is None:
        lu = ilu0(A)
    F = Factors.from_values(A, lu)
    mv = MatVec(SplitOperator(A, F))
    P = orthonormalize_mgs2(P_raw)
    thr = math.sqrt(tol) if fetch_threshold is None else fetch_threshold
    x = np.array(x0, dtype=np.float64, copy=True)
    rec = None
    solves, rel = [], []
    for _ in range(steps):
        b = x / tau_t + f
        U = V = None
        if policy == "once" and rec is not None:
            U, V = rec
        want_fetch = policy == "once" and rec is None
        res, x, r = precond_solve(A, F, b, x, s, ell, P, U, V, tol, mv=mv, max_mvs=max_mvs,
                                  fetch_threshold=thr if want_fetch else None, fetch_refresh=True)
        if want_fetch and res.fetched is not None:
            try:
                rec = cholqr2(*res.fetched)
            except ValueError:
                rec = None
        solves.append(res)
        rel.append(r)
        if on_solve is not None:
            on_solve(res)
        if res.status != OK:
            break
    return PrecondSequenceResult(x, solves, rel)

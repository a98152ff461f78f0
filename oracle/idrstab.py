"""FP64 CPU oracle: IDR(s)stab(l) (Algorithm 1) and M(s)stab(l) (Section 4.2).

TEST INFRASTRUCTURE ONLY (see the package docstring): the product path never
imports this module.

Everything is plain numpy in float64, real arithmetic (the paper's Hermitian
transposes become transposes).  A library routine serves only as a single step
(a sparse matrix-vector product, a dot product, a triangular solve); nothing is
fused, blocked or tracked algebraically: every projection P^T w is recomputed
from the vectors as they stand, in the order of Algorithm 1.

Storage: a block of s columns of length N (P, U, V, the level arrays V^(i)) is
an (s, N) array whose row q is column q.  The level arrays of one cycle are
kept as lists with an offset: R[i] = r^(i) for i = 0..l and Vl[i + 1] = V^(i)
for i = -1..l (V^(-1) = U, the pre-images).

Readings of points the paper leaves open (the same on the CUDA side):
  * stopping test: the recursive residual at a cycle end against tol*||b||,
    then one extra MV for the true residual b - Ax; if that fails, r is
    replaced by it and the cycles continue (residual replacement as used in
    the ocean experiment of Section 5.1);
  * MV count: every product with A (r0, the s products of the Arnoldi start,
    l(s+1) per cycle, one per true-residual check);
  * the garbled recapture of the solution after the residual minimisation is
    read as x = x^(0) + sum_{i=1..l} tau_i r^(i-1);
  * s x s solves: Gaussian elimination with partial pivoting; a pivot below
    1e-14 * (largest magnitude in its column of the projected matrix) is a
    breakdown (a per-column test: the columns differ in scale by orders);
  * tau = Z^+ r^(0) through the normal equations of the Gram matrix of
    [r^(0..l)], diagonally scaled, by Cholesky with LU as the fallback;
  * fetching point: the first cycle end whose recursive relative residual is
    at most sqrt(tol) ("half the tolerance" on a log scale), or a fixed cycle
    number;
  * recycled-basis orthonormalisation (optional): V <- V R^-1, U <- U R^-1
    with R the Cholesky factor of V^T V, applied twice.
"""

from __future__ import annotations

import dataclasses
import math
from typing import Callable, List, Optional

import numpy as np

PIVOT_REL_TOL = 1e-14

OK, BREAKDOWN, MAXIT, NAN = "ok", "breakdown", "maxit", "nan"


class Breakdown(Exception):
    """A small projected system was numerically singular (the paper assumes the
    canonical case, in which this does not happen)."""


# ----------------------------------------------------------------------------
# small dense solves
# ----------------------------------------------------------------------------

def lu_solve_pp(M: np.ndarray, rhs: np.ndarray) -> np.ndarray:
    """Solve M z = rhs by Gaussian elimination with row (partial) pivoting.

    Raises Breakdown if the pivot of column k falls below 1e-14 times the
    largest magnitude in column k of M (a zero column included).  The test is
    per column because the columns of a projected matrix P^T W can differ in
    scale by many orders (P^T of an orthonormal column is O(sqrt(s/N)), P^T of
    a product with A is O(||A||)); scaling a column changes neither
    solvability nor the pivot rows that partial pivoting picks."""
    a = np.array(M, dtype=np.float64, copy=True)
    z = np.array(rhs, dtype=np.float64, copy=True)
    n = z.shape[0]
    colmax = np.max(np.abs(a), axis=0) if n else np.zeros(0)
    if not (np.all(colmax > 0.0) and np.all(np.isfinite(colmax))):
        raise Breakdown("projected matrix has a zero or non-finite column")
    for k in range(n):
        p = k + int(np.argmax(np.abs(a[k:, k])))
        if abs(a[p, k]) < PIVOT_REL_TOL * colmax[k]:
            raise Breakdown(f"pivot {a[p, k]:.3e} at step {k}")
        if p != k:
            a[[k, p], :] = a[[p, k], :]
            z[[k, p]] = z[[p, k]]
        for i in range(k + 1, n):
            l = a[i, k] / a[k, k]
            a[i, k:] -= l * a[k, k:]
            z[i] -= l * z[k]
    for k in range(n - 1, -1, -1):
        z[k] = (z[k] - a[k, k + 1:] @ z[k + 1:]) / a[k, k]
    return z


CHOLQR_REL_TOL = 1e-14


def cholesky_upper(G: np.ndarray, rel_tol: float = 0.0) -> np.ndarray:
    """Upper triangular R with R^T R = G, written out; raises ValueError when a
    pivot is not above rel_tol * G_jj (rel_tol = 0: not positive)."""
    n = G.shape[0]
    R = np.zeros_like(G, dtype=np.float64)
    for j in range(n):
        d = G[j, j] - R[:j, j] @ R[:j, j]
        if not d > rel_tol * G[j, j]:
            raise ValueError("matrix not positive definite")
        R[j, j] = math.sqrt(d)
        for k in range(j + 1, n):
            R[j, k] = (G[j, k] - R[:j, j] @ R[:j, k]) / R[j, j]
    return R


def tau_from_gram(G: np.ndarray) -> np.ndarray:
    """tau = Z^+ r^(0) for Z = [r^(1..l)], from the Gram matrix G of [r^(0..l)]
    (Algorithm 1, degree-l residual minimisation).

    Normal equations (Z^T Z) tau = Z^T r^(0), scaled by D = diag(Z^T Z)^-1/2,
    solved by Cholesky, with LU (partial pivoting) when Cholesky fails.  If a
    level vector is exactly zero the minimisation is skipped (tau = 0)."""
    M = G[1:, 1:]
    rhs = G[1:, 0]
    dg = np.diag(M).copy()
    if not np.all(dg > 0.0):
        return np.zeros(M.shape[0])
    d = 1.0 / np.sqrt(dg)
    Ms = d[:, None] * M * d[None, :]
    rs = d * rhs
    try:
        R = cholesky_upper(Ms)
        y = np.zeros_like(rs)
        for i in range(len(rs)):                      # R^T y = rs
            y[i] = (rs[i] - R[:i, i] @ y[:i]) / R[i, i]
        z = np.zeros_like(rs)
        for i in range(len(rs) - 1, -1, -1):          # R z = y
            z[i] = (y[i] - R[i, i + 1:] @ z[i + 1:]) / R[i, i]
    except ValueError:
        z = lu_solve_pp(Ms, rs)
    return d * z


# ----------------------------------------------------------------------------
# bases: the cut space P, the Arnoldi start, the recycled basis
# ----------------------------------------------------------------------------

def orthonormalize_mgs2(X: np.ndarray) -> np.ndarray:
    """Orthonormal basis of the columns of X ((s, N) layout), by modified
    Gram-Schmidt applied twice; used for the random cut space P (Section 2.4:
    the basis vectors of P may be chosen randomly)."""
    Q = np.array(X, dtype=np.float64, copy=True)
    s = Q.shape[0]
    for j in range(s):
        for _ in range(2):
            for i in range(j):
                Q[j] -= (Q[i] @ Q[j]) * Q[i]
        Q[j] /= np.linalg.norm(Q[j])
    return Q


def cholqr2(U: np.ndarray, V: np.ndarray):
    """Orthonormalise the recycled V and carry U along: V <- V R^-1, U <- U R^-1
    with R^T R = V^T V, twice.  Keeps V = A U and range(V) (only the basis of
    the recycled space changes).  Raises ValueError if V is numerically rank
    deficient (a Cholesky pivot below 1e-14 of its diagonal entry)."""
    U = np.array(U, dtype=np.float64, copy=True)
    V = np.array(V, dtype=np.float64, copy=True)
    s = V.shape[0]
    for _ in range(2):
        G = V @ V.T
        R = cholesky_upper(G, CHOLQR_REL_TOL)
        # columns: V_new[:, j] = (V[:, j] - sum_{i<j} V_new[:, i] R[i, j]) / R[j, j]
        for j in range(s):
            for i in range(j):
                V[j] -= R[i, j] * V[i]
                U[j] -= R[i, j] * U[i]
            V[j] /= R[j, j]
            U[j] /= R[j, j]
    return U, V


class MatVec:
    """y = A v with a counter of matrix-vector products (MVs)."""

    def __init__(self, A):
        self.A = A.to_scipy() if hasattr(A, "to_scipy") else A
        self.count = 0

    def __call__(self, v: np.ndarray) -> np.ndarray:
        self.count += 1
        return self.A @ v

    def uncounted(self, v: np.ndarray) -> np.ndarray:
        return self.A @ v


def arnoldi_start(mv: MatVec, r0: np.ndarray, s: int, Pq: np.ndarray):
    """U, V for the first system: U = the first s Arnoldi vectors of K(A; r0)
    (modified Gram-Schmidt, applied twice), V = A U (s MVs), following the
    "Arnoldi scheme of level s" of Section 5.

    Should the Krylov space end before s vectors (happy breakdown), the next
    column of the orthonormal cut-space basis Pq, orthogonalised against the
    vectors so far, continues the basis."""
    N = r0.shape[0]
    U = np.zeros((s, N))
    V = np.zeros((s, N))
    q = r0 / np.linalg.norm(r0)
    for j in range(s):
        U[j] = q
        V[j] = mv(q)
        if j == s - 1:
            break
        w = V[j].copy()
        for _ in range(2):
            for i in range(j + 1):
                w -= (U[i] @ w) * U[i]
        nw = np.linalg.norm(w)
        if not nw > 1e-12 * np.linalg.norm(V[j]):
            w = Pq[j + 1].copy()
            for _ in range(2):
                for i in range(j + 1):
                    w -= (U[i] @ w) * U[i]
            nw = np.linalg.norm(w)
        q = w / nw
    return U, V


# ----------------------------------------------------------------------------
# the steps of one cycle of Algorithm 1
# ----------------------------------------------------------------------------

def proj(P: np.ndarray, w: np.ndarray) -> np.ndarray:
    """P^T w: the s inner products of w with the cut-space basis vectors."""
    return P @ w


def w_block(Vl: List[np.ndarray], i: int, q: int) -> np.ndarray:
    """W^(i) = [V^(i+1)_{1:q-1}, V^(i)_{q:s}] for the 0-based column q
    (columns 0..q-1 from level i+1, q..s-1 from level i)."""
    return np.concatenate([Vl[i + 2][:q], Vl[i + 1][q:]], axis=0)


def gamma_step(P, R, Vl, k):
    """gamma with r^(k) - V^(k) gamma orthogonal to P: (P^T V^(k)) gamma = P^T r^(k)."""
    M = np.stack([proj(P, v) for v in Vl[k + 1]], axis=1)
    return lu_solve_pp(M, proj(P, R[k]))


def gamma_update(R, Vl, x0, gamma, k):
    """r^(i) -= V^(i) gamma for i = 0..k, and x^(0) += V^(-1) gamma (in place)."""
    for i in range(k + 1):
        R[i] = R[i] - gamma @ Vl[i + 1]
    x0 += gamma @ Vl[0]


def eta_step(P, R, Vl, k, q):
    """eta_q with r^(k+1) - W^(k) eta_q orthogonal to P."""
    W = w_block(Vl, k, q)
    M = np.stack([proj(P, w) for w in W], axis=1)
    return lu_solve_pp(M, proj(P, R[k + 1]))


def eta_update(R, Vl, k, q, eta):
    """v_q^(i) = r^(i+1) - W^(i) eta_q for i = -1..k; all new values are formed
    before any is stored."""
    new = [R[i + 1] - eta @ w_block(Vl, i, q) for i in range(-1, k + 1)]
    for i, v in zip(range(-1, k + 1), new):
        Vl[i + 1][q] = v


def tau_step(R):
    """tau = Z^+ r^(0) with Z = [r^(1), ..., r^(l)]."""
    L = len(R)
    G = np.array([[R[a] @ R[c] for c in range(L)] for a in range(L)])
    return tau_from_gram(G)


def tau_update(R, Vl, x0, tau):
    """Degree-l polynomial step of Algorithm 1:
        r   = r^(0)      - sum_{i=1..l} tau_i r^(i)
        x   = x^(0)      + sum_{i=1..l} tau_i r^(i-1)
        v_q = v_q^(0)    - sum_{i=1..l} tau_i v_q^(i)
        u_q = v_q^(-1)   - sum_{i=1..l} tau_i v_q^(i-1)."""
    ell = len(tau)
    r = R[0].copy()
    x = x0.copy()
    V = Vl[1].copy()
    U = Vl[0].copy()
    for i in range(1, ell + 1):
        r -= tau[i - 1] * R[i]
        x += tau[i - 1] * R[i - 1]
        V -= tau[i - 1] * Vl[i + 1]
        U -= tau[i - 1] * Vl[i]
    return r, x, U, V


# ----------------------------------------------------------------------------
# Algorithm 1
# ----------------------------------------------------------------------------

@dataclasses.dataclass
class SolveResult:
    x: np.ndarray
    r: np.ndarray
    U: Optional[np.ndarray]
    V: Optional[np.ndarray]
    J: int                      # level reached (j in Algorithm 1)
    cycles: int
    mvs: int
    status: str
    relres_rec: float
    relres_true: float
    history: List[float]        # relative recursive residual: start, then each cycle end
    mv_history: List[int]       # MV count at the same points
    fetched: Optional[tuple] = None   # (U, V) written out at the fetching point
    fetch_cycle: int = 0


def slope_fires(history: List[float], k: int) -> bool:
    """The online drop test at the end of cycle k (history[i]: relative
    residual at the start, i = 0, and after cycle i): the residual fell in
    cycle k by at least one decade and by at least twice the mean decrease (in
    log10) of cycles 1..k-1.  A reading of "shortly before the residual drops"
    (section on choosing the fetching point) as a test a solver can apply as it
    runs; needs k >= 2."""
    if k < 2:
        return False
    lg = [math.log10(max(h, 1e-300)) for h in history[:k + 1]]
    drop = lg[k - 1] - lg[k]
    mean = (lg[0] - lg[k - 1]) / (k - 1)
    return drop >= 1.0 and drop >= 2.0 * mean


def fetch_estimate(history: List[float]) -> Optional[int]:
    """The fetching point estimated from a complete residual history (the
    probe solve of the section on choosing the fetching point): the cycle end
    just before the steepest one-cycle decrease of log10 relres, at least 1;
    None if the solve ran no cycle."""
    K = len(history) - 1
    if K < 1:
        return None
    lg = [math.log10(max(h, 1e-300)) for h in history]
    drops = [lg[k - 1] - lg[k] for k in range(1, K + 1)]
    k_star = 1 + max(range(K), key=lambda i: (drops[i], -i))   # first of the steepest
    return max(1, k_star - 1)


def idrstab(A, b, x, s, ell, P, U=None, V=None, tol=1e-8, *, max_mvs=None,
            fetch_threshold=None, fetch_cycle=None, fetch_refresh=False, fetch_slope=False,
            fetch_at_end=False, replace_every=0, inspect: Optional[Callable] = None,
            mv: Optional[MatVec] = None) -> SolveResult:
    """IDR(s)stab(l), Algorithm 1, with inputs A, b, x, s, l, P, U, V.

    Precondition V = A U, dim P = s (P orthonormal, (s, N) layout).  With
    U = V = None the start basis is the Arnoldi basis of the initial residual
    (first system / IDRstab); with U, V from an earlier solve this is M(s)stab
    (Section 4.2: pass the earlier outputs P, U, V on unchanged).

    ``fetch_threshold`` / ``fetch_cycle`` write out (U, V) at the fetching point
    (Section 5): the first cycle end with relative recursive residual at most
    the threshold, or the end of cycle number ``fetch_cycle``.  With
    ``fetch_refresh`` the written V is recomputed as A U (s counted MVs): the
    recursions keep V = A U only up to a drift (about 1e-6 relative here), and
    Algorithm 1 requires V = A U of its inputs.
    ``fetch_slope`` fetches instead the basis of the cycle before the first
    cycle at whose end ``slope_fires``; ``fetch_at_end`` fetches the final
    basis of a converged solve that fetched nothing before.
    ``replace_every`` > 0 replaces the recursive residual by b - A x (one
    counted MV) at the end of every replace_every-th cycle, as the
    preconditioned experiment of Section 5.1 does after each cycle; the stopping
    test then needs no confirming product.
    ``inspect(stage, state)`` is called after the level loop ("levels") and at
    each cycle end ("cycle") for the invariant tests."""
    mv = mv or MatVec(A)
    b = np.asarray(b, dtype=np.float64)
    x = np.array(x, dtype=np.float64, copy=True)
    N = b.shape[0]
    if max_mvs is None:
        max_mvs = min(100000, int(20 * math.sqrt(N)) + 1 + s + 2 * ell * (s + 1))
    nb = float(np.linalg.norm(b))
    if nb == 0.0:
        x[:] = 0.0
        return SolveResult(x, np.zeros(N), U, V, 0, 0, 0, OK, 0.0, 0.0, [0.0], [0])

    m0 = mv.count
    r = b - mv(x)
    r_is_true = True
    j = 0
    cycles = 0
    history = [float(np.linalg.norm(r)) / nb]
    mv_history = [mv.count - m0]
    fetched = None
    fetch_at = 0
    prev_basis = None
    status = OK
    if U is not None:
        U = np.array(U, dtype=np.float64, copy=True)
        V = np.array(V, dtype=np.float64, copy=True)

    while True:
        nr = float(np.linalg.norm(r))
        if not math.isfinite(nr):
            status = NAN
            break
        if nr <= tol * nb:
            if r_is_true:
                break
            r_true = b - mv(x)
            if float(np.linalg.norm(r_true)) <= tol * nb:
                r = r_true
                break
            r = r_true                     # residual replacement
            r_is_true = True
            continue
        if U is None:
            if mv.count - m0 + s > max_mvs:
                status = MAXIT
                break
            U, V = arnoldi_start(mv, r, s, P)
        if mv.count - m0 + ell * (s + 1) > max_mvs:
            status = MAXIT
            break

        # one cycle: level iteration k = 0..l-1, then the degree-l minimisation
        R = [r.copy()] + [None] * ell
        Vl = [U.copy(), V.copy()] + [np.zeros((s, N)) for _ in range(ell)]
        x0 = x.copy()
        try:
            for k in range(ell):
                gamma = gamma_step(P, R, Vl, k)
                gamma_update(R, Vl, x0, gamma, k)
                R[k + 1] = mv(R[k])
                for q in range(s):
                    eta = eta_step(P, R, Vl, k, q)
                    eta_update(R, Vl, k, q, eta)
                    Vl[k + 2][q] = mv(Vl[k + 1][q])
            if inspect is not None:
                inspect("levels", dict(R=R, Vl=Vl, x0=x0, P=P, b=b, mv=mv))
            tau = tau_step(R)
        except Breakdown:
            status = BREAKDOWN
            break
        r, x, U, V = tau_update(R, Vl, x0, tau)
        r_is_true = False
        j += ell
        cycles += 1
        if replace_every and cycles % replace_every == 0:
            r = b - mv(x)
            r_is_true = True
        relres = float(np.linalg.norm(r)) / nb
        history.append(relres)
        mv_history.append(mv.count - m0)
        if inspect is not None:
            inspect("cycle", dict(r=r, x=x, U=U, V=V, R=R, tau=tau, P=P, b=b, mv=mv))
        if fetched is None:
            if fetch_slope:
                if prev_basis is not None and slope_fires(history, cycles):
                    Up, Vp = prev_basis
                    fetched = (Up, np.stack([mv(u) for u in Up]) if fetch_refresh else Vp)
                    fetch_at = cycles - 1
                prev_basis = (U.copy(), V.copy())
            elif (fetch_cycle is not None and cycles == fetch_cycle) or \
                    (fetch_cycle is None and fetch_threshold is not None and relres <= fetch_threshold):
                Vf = np.stack([mv(u) for u in U]) if fetch_refresh else V.copy()
                fetched = (U.copy(), Vf)
                fetch_at = cycles

    if fetch_at_end and fetched is None and status == OK and cycles > 0:
        fetched = (U.copy(), np.stack([mv(u) for u in U]) if fetch_refresh else V.copy())
        fetch_at = cycles
    relres_rec = float(np.linalg.norm(r)) / nb
    relres_true = float(np.linalg.norm(b - mv.uncounted(x))) / nb
    return SolveResult(x, r, U, V, j, cycles, mv.count - m0, status, relres_rec, relres_true,
                       history, mv_history, fetched, fetch_at)


# ----------------------------------------------------------------------------
# M(s)stab over a sequence of systems
# ----------------------------------------------------------------------------

def _orth_or_none(UV):
    """The orthonormalised recycled basis, or None (no fetch) if V is rank deficient."""
    try:
        return cholqr2(*UV)
    except ValueError:
        return None


@dataclasses.dataclass
class SequenceResult:
    x: np.ndarray
    solves: List[SolveResult]


def msstab_sequence(A, f, x0, tau_t, steps, s, ell, P_raw, tol=1e-8, *, policy="once",
                    fetch_threshold=None, fetch_cycle=None, orth_recycle=True, first_step=0,
                    max_mvs=None, replace_every=0, on_solve: Optional[Callable] = None) -> SequenceResult:
    """Solve the implicit-Euler sequence A x^(i+1) = x^(i)/tau_t + f, one system
    after the other, from x^(0).

    policy "once":  the first system is solved by IDRstab (Arnoldi start); U, V
                    are fetched at the fetching point of that solve and passed,
                    with P, to every later system (Section 5.1 fetches once and
                    reuses the data for all right-hand sides).
    policy "never": every system is solved by IDRstab with its own Arnoldi start
                    (the IDRstab baseline).
    policy "every": the final U, V of each solve are passed to the next
                    (Miltenberger's chaining, Section 3.1).
    policy "slope": as "once", with the fetching point of the first solve found
                    as it runs: the basis of the cycle before the residual
                    drops (``slope_fires``), else the final basis.
    policy "probe": the first system is a probe solved by IDRstab without a
                    fetch; its history gives the fetching point
                    (``fetch_estimate``), at which the second system, again
                    solved by IDRstab, writes U, V (the final basis if it
                    converges earlier); the later systems recycle them.
    With ``orth_recycle`` (default) the passed basis is conditioned: V := A U
    (s MVs, counted in the solve that wrote it), then Cholesky QR twice.
    ``fetch_cycle`` (policy "once") fetches at the end of that cycle of the
    first solve instead of at the threshold (the fixed fetching cycles of the
    finite-termination experiments of Section 5.2).
    ``first_step``/``steps`` select the slice of the sequence that is solved;
    x0 is then the solution of the step before the slice."""
    mv = MatVec(A)
    P = orthonormalize_mgs2(P_raw)
    thr = math.sqrt(tol) if fetch_threshold is None else fetch_threshold
    x = np.array(x0, dtype=np.float64, copy=True)
    rec = None
    solves = []
    probe_cycle = None
    for _ in range(first_step, first_step + steps):
        b = x / tau_t + f
        if policy == "never" or rec is None:
            U = V = None
        else:
            U, V = rec
        kw = {}
        want_fetch = rec is None and policy in ("once", "slope", "probe")
        if policy == "once" and want_fetch:
            kw = dict(fetch_cycle=fetch_cycle) if fetch_cycle else dict(fetch_threshold=thr)
        elif policy == "slope" and want_fetch:
            kw = dict(fetch_slope=True, fetch_at_end=True)
        elif policy == "probe" and want_fetch:
            if probe_cycle is None:
                want_fetch = False            # the probe itself writes nothing
            else:
                kw = dict(fetch_cycle=probe_cycle, fetch_at_end=True)
        res = idrstab(mv.A, b, x, s, ell, P, U, V, tol, max_mvs=max_mvs, fetch_refresh=orth_recycle,
                      replace_every=replace_every, mv=mv, **kw)
        if policy == "probe" and rec is None and probe_cycle is None and res.status == OK:
            probe_cycle = fetch_estimate(res.history)
        if want_fetch and res.fetched is not None:
            rec = _orth_or_none(res.fetched) if orth_recycle else res.fetched
        elif policy == "every" and res.U is not None and res.cycles > 0 and res.status == OK:
            if orth_recycle:
                Vf = np.stack([mv(u) for u in res.U])
                res.mvs += s
                rec = _orth_or_none((res.U, Vf))
            else:
                rec = (res.U, res.V)
        solves.append(res)
        if on_solve is not None:
            on_solve(res)
        x = res.x
    return SequenceResult(x, solves)


# ----------------------------------------------------------------------------
# textbook BiCGStab (the s = l = 1 special case, Section 2.3)
# ----------------------------------------------------------------------------

def bicgstab(A, b, x, p, tol=1e-8, max_iter=1000):
    """BiCGStab with fixed shadow vector p (van der Vorst's formulation).

    Returns (x, relative residual after each iteration, MVs)."""
    mv = MatVec(A)
    x = np.array(x, dtype=np.float64, copy=True)
    nb = np.linalg.norm(b)
    r = b - mv(x)
    rho_old = alpha = omega = 1.0
    v = np.zeros_like(b)
    d = np.zeros_like(b)
    hist = [np.linalg.norm(r) / nb]
    for _ in range(max_iter):
        rho = p @ r
        beta = (rho / rho_old) * (alpha / omega)
        d = r + beta * (d - omega * v)
        v = mv(d)
        alpha = rho / (p @ v)
        sv = r - alpha * v
        t = mv(sv)
        omega = (t @ sv) / (t @ t)
        x = x + alpha * d + omega * sv
        r = sv - omega * t
        rho_old = rho
        hist.append(np.linalg.norm(r) / nb)
        if hist[-1] <= tol:
            break
    return x, hist, mv.count

"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test ties the oracle to something other than itself: a library routine
for a special case, a closed form, an invariant of Algorithm 1, or the
finite-termination levels that Section 5.2 derives from the dimension bounds
of Sonneveld and M-spaces.  The mutation tests at the end plant plausible
mistakes into the oracle and check that these pins catch them.
"""

import json
import math
import os

import numpy as np
import pytest

from oracle import idrstab as O
from paper_1604_06043_gb300 import problems as pb

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


# ---------------------------------------------------------------------------
# small dense building blocks against library routines
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("n", [1, 2, 5, 8, 16])
def test_lu_solve_pp_matches_numpy(n):
    rng = np.random.default_rng(10 + n)
    for _ in range(20):
        M = rng.standard_normal((n, n))
        z = rng.standard_normal(n)
        np.testing.assert_allclose(O.lu_solve_pp(M, z), np.linalg.solve(M, z), rtol=1e-9, atol=1e-12)


def test_lu_solve_pp_needs_pivoting():
    M = np.array([[0.0, 1.0], [1.0, 1.0]])
    np.testing.assert_allclose(O.lu_solve_pp(M, np.array([1.0, 3.0])), [2.0, 1.0])


def test_lu_solve_pp_breakdown():
    M = np.array([[1.0, 2.0], [2.0, 4.0]])
    with pytest.raises(O.Breakdown):
        O.lu_solve_pp(M, np.array([1.0, 1.0]))
    with pytest.raises(O.Breakdown):
        O.lu_solve_pp(np.zeros((3, 3)), np.ones(3))


def test_cholesky_upper_matches_numpy():
    rng = np.random.default_rng(1)
    X = rng.standard_normal((6, 40))
    G = X @ X.T
    R = O.cholesky_upper(G)
    np.testing.assert_allclose(R, np.linalg.cholesky(G).T, rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("ell", [1, 2, 4])
def test_tau_is_least_squares_solution(ell):
    rng = np.random.default_rng(ell)
    R = [rng.standard_normal(50) * 10.0 ** rng.integers(-3, 3) for _ in range(ell + 1)]
    tau = O.tau_step(R)
    Z = np.stack(R[1:], axis=1)
    ref = np.linalg.lstsq(Z, R[0], rcond=None)[0]
    np.testing.assert_allclose(tau, ref, rtol=1e-9)
    # the residual r^(0) - Z tau is orthogonal to the columns of Z
    r = R[0] - Z @ tau
    assert np.max(np.abs(Z.T @ r)) <= 1e-11 * np.linalg.norm(Z) * np.linalg.norm(R[0])


def test_tau_zero_level_vector():
    R = [np.ones(4), np.zeros(4)]
    np.testing.assert_array_equal(O.tau_step(R), [0.0])


def test_orthonormalize_mgs2():
    X = pb.randn_cols(500, 8, 3)
    Q = O.orthonormalize_mgs2(X)
    np.testing.assert_allclose(Q @ Q.T, np.eye(8), atol=1e-14)
    # same span, same orientation as a Householder QR with positive diagonal
    q, r = np.linalg.qr(X.T)
    q = q * np.sign(np.diag(r))[None, :]
    np.testing.assert_allclose(Q, q.T, atol=1e-12)


def test_cholqr2_keeps_relation_and_span():
    rng = np.random.default_rng(7)
    A = pb.convdiff((8, 8), (10.0, 10.0), tau=0.01).to_scipy()
    U = rng.standard_normal((4, 64))
    V = np.stack([A @ u for u in U])
    U2, V2 = O.cholqr2(U, V)
    np.testing.assert_allclose(V2 @ V2.T, np.eye(4), atol=1e-13)
    np.testing.assert_allclose(np.stack([A @ u for u in U2]), V2, atol=1e-10)
    # span unchanged: projecting V onto span(V2) reproduces V
    np.testing.assert_allclose((V @ V2.T) @ V2, V, rtol=1e-10, atol=1e-10)


def test_arnoldi_start_is_krylov_basis():
    A = pb.convdiff((8, 8), (10.0, 10.0), tau=0.01)
    mv = O.MatVec(A)
    r0 = pb.uniform(64, 2)
    U, V = O.arnoldi_start(mv, r0, 5, O.orthonormalize_mgs2(pb.randn_cols(64, 5, 3)))
    assert mv.count == 5
    np.testing.assert_allclose(U @ U.T, np.eye(5), atol=1e-13)
    np.testing.assert_allclose(np.stack([mv.A @ u for u in U]), V, rtol=1e-13, atol=1e-10)
    K = [r0]
    for _ in range(4):
        K.append(mv.A @ K[-1])
    q, r = np.linalg.qr(np.stack(K, axis=1))
    q = q * np.sign(np.diag(r))[None, :]
    np.testing.assert_allclose(U, q.T, atol=1e-9)


# ---------------------------------------------------------------------------
# Section 5.2: finite termination on A = tridiag(2, 3, 1), N = 40; the paper's
# printed values are in tests/golden/paper_finite_termination.json
# ---------------------------------------------------------------------------

FT = json.load(open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden",
                                 "paper_finite_termination.json")))
_MT = FT["matrix"]
TRI = pb.tridiag(_MT["N"], _MT["sub"], _MT["diag"], _MT["sup"])
B1, B2 = pb.termination_rhs(_MT["N"])


def _P(s):
    return O.orthonormalize_mgs2(pb.randn_cols(40, s, pb.SEED_P))


def _first_cycle_below(hist, thr):
    for c, h in enumerate(hist):
        if h < thr:
            return c
    return None


def test_fixture_values_follow_the_printed_bounds():
    """The fixture's numbers are those of the paper's dimension bounds."""
    N = _MT["N"]
    for g in FT["idrstab"]:
        assert N - (g["last_nonzero_G"] + 1) * g["s"] <= 0 < N - g["last_nonzero_G"] * g["s"]
    for m in FT["msstab"]:
        s, G = m["s"], m["data"][0]["G"]
        assert all(d["G"] == G for d in m["data"])
        assert m["dim_G"] == N - G * s and m["dim_M"] == m["dim_G"] + G
        last = m["last_nonzero_M"]
        assert m["dim_M"] - (last - G) * s > 0 >= m["dim_M"] - (last + 1 - G) * s
    f = FT["fetch_after_mvs"]
    assert f["mvs"] == 1 + f["s"] + f["G"] * f["ell"] * (f["s"] + 1)     # r0 + Arnoldi + G cycles (c3)


def test_table1_reduced_dimensions_agree_with_the_m_space_bounds():
    """Table 1's count of reduced dimensions, j s + J (s - 1) after j level
    steps from data of G_J, reaches N at the level after the last non-zero
    M-space of Section 5.2 (two statements of the paper, one termination)."""
    N = _MT["N"]
    for m in FT["msstab"]:
        s, G = m["s"], m["data"][0]["G"]
        j = next(j for j in range(1, N + 1) if j * s + G * (s - 1) >= N)
        assert G + j == m["last_nonzero_M"] + 1


def test_termination_rhs_orthogonal():
    assert FT["rhs"]["orthogonal"] and abs(B1 @ B2) < 1e-12


@pytest.mark.parametrize("g", FT["idrstab"], ids=lambda g: f"s{g['s']}l{g['ell']}")
def test_idrstab_terminates_when_sonneveld_space_vanishes(g):
    # G_j = {0} from the level after the last non-zero one on
    s, ell, level = g["s"], g["ell"], g["last_nonzero_G"] + 1
    res = O.idrstab(TRI, B1, np.zeros(40), s, ell, _P(s), tol=1e-13, max_mvs=2000)
    c = _first_cycle_below(res.history, 1e-10)
    assert c is not None and c * ell <= level + ell      # one extra cycle for rounding
    assert res.history[(level // ell) - 1] > 1e-6         # not before the level


def test_fetch_after_60_mvs_is_level_19():
    # 1 (r0) + 2 (Arnoldi) + 19 cycles x 3 MVs = 60 MVs <=> range(V) in G_19
    f = FT["fetch_after_mvs"]
    res = O.idrstab(TRI, B1, np.zeros(40), f["s"], f["ell"], _P(f["s"]), tol=1e-14, max_mvs=2000,
                    fetch_cycle=f["G"] // f["ell"])
    assert res.fetch_cycle == f["G"]
    assert res.mv_history[f["G"]] == f["mvs"]


def _m_solve(s, ell_src, fetch_cycle, ell):
    P = _P(s)
    src = O.idrstab(TRI, B1, np.zeros(40), s, ell_src, P, tol=1e-15, max_mvs=2000,
                    fetch_cycle=fetch_cycle)
    U, V = src.fetched
    return O.idrstab(TRI, B2, np.zeros(40), s, ell, P, U, V, tol=1e-13, max_mvs=2000)


M_CASES = [(m, d, ell) for m in FT["msstab"] for d in m["data"] for ell in m["ell"]]


@pytest.mark.parametrize("m,d,ell", M_CASES,
                         ids=[f"s{m['s']}_G{d['G']}_src_l{d['ell']}_l{ell}" for m, d, ell in M_CASES])
def test_msstab_terminates_after_the_last_nonzero_m_space(m, d, ell):
    # the M-space levels continue from the fetch level G; the residual is zero
    # once a residual of the level after the last non-zero M-space is computed
    s, G, last = m["s"], d["G"], m["last_nonzero_M"]
    res = _m_solve(s, d["ell"], G // d["ell"], ell)
    cz = -(-(last + 1 - G) // ell)             # cycles to reach level last + 1
    c = _first_cycle_below(res.history, 1e-10)
    assert c is not None and cz <= c <= cz + 1  # one extra cycle for rounding
    assert res.history[cz - 1] > 1e-8           # not a cycle earlier


# ---------------------------------------------------------------------------
# special cases: dense LU on tiny systems, BiCGStab for s = l = 1
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("s,ell", [(1, 1), (2, 2), (4, 2), (4, 4)])
def test_tiny_systems_match_dense_lu(s, ell):
    A = pb.convdiff((8, 8), (10.0, 10.0), tau=0.01)
    b = pb.uniform(64, 1) / 0.01 + pb.uniform(64, 2)
    P = O.orthonormalize_mgs2(pb.randn_cols(64, s, 3))
    res = O.idrstab(A, b, np.zeros(64), s, ell, P, tol=1e-12, max_mvs=5000)
    assert res.status == O.OK
    ref = np.linalg.solve(A.to_dense(), b)
    assert np.linalg.norm(res.x - ref) <= 1e-8 * np.linalg.norm(ref)
    assert res.relres_true <= 1e-12 * 1.01


def test_tridiag_matches_dense_lu():
    P = _P(4)
    res = O.idrstab(TRI, B2, np.zeros(40), 4, 2, P, tol=1e-12, max_mvs=2000)
    ref = np.linalg.solve(TRI.to_dense(), B2)
    assert np.linalg.norm(res.x - ref) <= 1e-10 * np.linalg.norm(ref)


def test_s1_l1_reproduces_bicgstab():
    w = pb.WORKLOADS["convdiff2d_32"]
    A = w.matrix()
    b = w.x0() / w.tau + w.f()
    x0 = np.zeros(w.n)
    p = O.orthonormalize_mgs2(pb.randn_cols(w.n, 1, 3))
    res = O.idrstab(A, b, x0, 1, 1, p, tol=1e-10, max_mvs=5000)
    _, hist, mvs = O.bicgstab(A, b, x0, p[0], tol=1e-10)
    n = min(15, len(hist) - 1, len(res.history) - 1)
    assert n == 15
    np.testing.assert_allclose(res.history[: n + 1], hist[: n + 1], rtol=1e-8)
    # the same number of iterations to tolerance; IDR(1)stab(1) pays one MV for
    # its Arnoldi start and one for the true-residual check
    assert abs(res.mvs - (mvs + 2)) <= 2


# ---------------------------------------------------------------------------
# invariants of Algorithm 1 and the counts of Table 1
# ---------------------------------------------------------------------------

def _invariant_run(s, ell, U=None, V=None, b=None):
    w = pb.WORKLOADS["convdiff2d_32"]
    A = w.matrix()
    b = w.x0() / w.tau + w.f() if b is None else b
    P = O.orthonormalize_mgs2(pb.randn_cols(w.n, s, 3))
    seen = {"levels": [], "cycle": []}

    def inspect(stage, st):
        mv = st["mv"]
        if stage == "levels":
            R, Vl = st["R"], st["Vl"]
            lv = []
            for i in range(ell):
                lv.append(np.linalg.norm(mv.uncounted(R[i]) - R[i + 1]) / np.linalg.norm(R[i + 1]))
                for q in range(s):
                    lv.append(np.linalg.norm(mv.uncounted(Vl[i + 1][q]) - Vl[i + 2][q])
                              / np.linalg.norm(Vl[i + 2][q]))
            for q in range(s):   # pre-images: A v^(-1) = v^(0)
                lv.append(np.linalg.norm(mv.uncounted(Vl[0][q]) - Vl[1][q]) / np.linalg.norm(Vl[1][q]))
            orth = [np.linalg.norm(P @ R[i]) / np.linalg.norm(R[i]) for i in range(ell)]
            orth += [np.linalg.norm(P @ Vl[i + 1][q]) / np.linalg.norm(Vl[i + 1][q])
                     for i in range(ell) for q in range(s)]
            seen["levels"].append((max(lv), max(orth)))
        else:
            r, x, U_, V_, R = st["r"], st["x"], st["U"], st["V"], st["R"]
            AU = np.stack([mv.uncounted(u) for u in U_])
            zr = max(abs(R[i] @ r) / (np.linalg.norm(R[i]) * np.linalg.norm(R[0])) for i in range(1, ell + 1))
            gap = np.linalg.norm(st["b"] - mv.uncounted(x) - r) / np.linalg.norm(st["b"])
            seen["cycle"].append((np.linalg.norm(AU - V_) / np.linalg.norm(V_), zr, gap))

    res = O.idrstab(A, b, np.zeros(w.n), s, ell, P, U, V, tol=1e-10, max_mvs=20000, inspect=inspect)
    return res, seen


@pytest.mark.parametrize("s,ell", [(1, 1), (2, 3), (4, 2)])
def test_invariants_hold_every_cycle(s, ell):
    res, seen = _invariant_run(s, ell)
    assert res.status == O.OK and res.cycles >= 3
    for lv, orth in seen["levels"]:
        assert lv < 1e-9          # level vectors: A r^(i) = r^(i+1), A v^(i) = v^(i+1)
        assert orth < 1e-9        # r^(i), v_q^(i) orthogonal to P for i < l
    for vau, zr, gap in seen["cycle"]:
        assert vau < 1e-9         # V = A U (precondition of Algorithm 1, kept by each cycle)
        assert zr < 1e-10         # Z^T r = 0 after the minimisation
        assert gap < 1e-9         # recursive residual = b - A x


@pytest.mark.parametrize("s,ell", [(2, 1), (4, 2), (3, 3)])
def test_mv_counts_table1(s, ell):
    w = pb.WORKLOADS["convdiff2d_32"]
    A = w.matrix()
    b = w.x0() / w.tau + w.f()
    P = O.orthonormalize_mgs2(pb.randn_cols(w.n, s, 3))
    res = O.idrstab(A, b, np.zeros(w.n), s, ell, P, tol=1e-8, max_mvs=20000)
    checks = res.mvs - (1 + s + ell * (s + 1) * res.cycles)
    assert checks >= 1 and checks <= 3
    # M(s)stab: no Arnoldi start; #MVs = j (s+1) with j = l cycles' levels (Table 1)
    res2 = O.idrstab(A, b * 1.5 + 1.0, res.x, s, ell, P, res.U, res.V, tol=1e-8, max_mvs=20000)
    assert res2.mvs - 1 - (res2.J * (s + 1)) in (1, 2, 3)
    assert res2.J == ell * res2.cycles
    # Table 1, #Columns: r^(0..l), x^(0) and V^(-1..l)
    assert (ell + 1) + 1 + s * (ell + 2) == (s + 1) * (ell + 2)


def test_residual_replacement_every_cycle():
    """r := b - A x at each cycle end (the preconditioned experiment of Section 5.1
    replaces the residual this way): the iteration is unchanged in exact
    arithmetic, the recursive residual equals the true one at every cycle end,
    each cycle pays one product more and no confirmation product is needed."""
    A = pb.convdiff((48, 48, 48), (20.0, 10.0, 5.0), tau=0.005)
    As = A.to_scipy()
    b = pb.uniform(A.n, 2) / 0.005 + pb.uniform(A.n, 1)
    x0 = pb.uniform(A.n, 2)
    s, ell = 8, 4
    P = O.orthonormalize_mgs2(pb.randn_cols(A.n, s, 3))
    runs = {}
    for re in (0, 1):
        gaps = []

        def inspect(stage, st):
            if stage == "cycle":
                gaps.append(np.linalg.norm(st["b"] - As @ st["x"] - st["r"]) / np.linalg.norm(st["b"]))

        runs[re] = (O.idrstab(A, b, x0, s, ell, P, tol=1e-8, replace_every=re, inspect=inspect), gaps)
    plain, gp = runs[0]
    repl, gr = runs[1]
    assert plain.status == O.OK and repl.status == O.OK
    assert max(gr) == 0.0
    assert repl.mvs == 1 + s + repl.cycles * (ell * (s + 1) + 1)
    assert repl.relres_true <= 1e-8
    # the first cycle is the same iteration (it starts from the same true residual)
    assert plain.history[1] == pytest.approx(repl.history[1], rel=1e-7)
    # on this stiff problem the drift of V from A U opens a gap larger than tol
    # in the plain recursion (the level vectors grow like ||A||^k), so its
    # convergence check fails once and costs a cycle; the replaced run does not
    assert max(gp) > 1e-8 and plain.cycles > repl.cycles


def test_m_equals_idr_on_a_single_system():
    w = pb.WORKLOADS["convdiff2d_32"]
    A = w.matrix()
    seq = O.msstab_sequence(A, w.f(), w.x0(), w.tau, 1, w.s, w.ell, w.p_raw(), policy="once")
    P = O.orthonormalize_mgs2(w.p_raw())
    one = O.idrstab(A, w.x0() / w.tau + w.f(), w.x0(), w.s, w.ell, P, tol=1e-8)
    np.testing.assert_array_equal(seq.solves[0].x, one.x)
    # identical iterates; the M(s)stab run also pays the s products of V := A U at its fetch
    assert seq.solves[0].fetched is not None
    assert seq.solves[0].mvs == one.mvs + w.s


def test_msstab_sequence_converges_and_recycles():
    w = pb.WORKLOADS["convdiff2d_32"]
    A = w.matrix()
    m = O.msstab_sequence(A, w.f(), w.x0(), w.tau, w.steps, w.s, w.ell, w.p_raw(), policy="once")
    i = O.msstab_sequence(A, w.f(), w.x0(), w.tau, w.steps, w.s, w.ell, w.p_raw(), policy="never")
    for a, c in zip(m.solves, i.solves):
        assert a.status == O.OK and c.status == O.OK
        assert a.relres_true <= 1e-8 and c.relres_true <= 1e-8
    assert m.solves[0].fetched is not None
    # the recycled systems start without the s MVs of the Arnoldi start
    assert sum(s.mvs for s in m.solves[1:]) < sum(s.mvs for s in i.solves[1:])
    ref = np.linalg.solve(A.to_dense(), w.x0() / w.tau + w.f())
    np.testing.assert_allclose(m.solves[0].x, ref, rtol=1e-6, atol=1e-6 * np.abs(ref).max())


def test_zero_rhs_and_exact_start():
    A = pb.convdiff((8, 8), (10.0, 10.0), tau=0.01)
    P = O.orthonormalize_mgs2(pb.randn_cols(64, 2, 3))
    res = O.idrstab(A, np.zeros(64), np.ones(64), 2, 2, P)
    assert res.status == O.OK and res.mvs == 0 and not res.x.any()
    b = A.to_scipy() @ np.ones(64)
    res = O.idrstab(A, b, np.ones(64), 2, 2, P)
    assert res.status == O.OK and res.mvs == 1 and res.cycles == 0


def test_maxit_status():
    A = pb.convdiff((8, 8), (10.0, 10.0), tau=0.01)
    P = O.orthonormalize_mgs2(pb.randn_cols(64, 2, 3))
    res = O.idrstab(A, pb.uniform(64, 1), np.zeros(64), 2, 2, P, tol=1e-14, max_mvs=10)
    assert res.status == O.MAXIT and res.mvs <= 10


# ---------------------------------------------------------------------------
# planted mistakes: each must make one of the pins above fail
# ---------------------------------------------------------------------------

def _tau_update_wrong_x_index(R, Vl, x0, tau):
    r, x, U, V = ORIG["tau_update"](R, Vl, x0, tau)
    x = x0.copy()
    for i in range(1, len(tau) + 1):
        x += tau[i - 1] * R[i]                 # r^(i) instead of r^(i-1)
    return r, x, U, V


def _gamma_update_no_lower_levels(R, Vl, x0, gamma, k):
    R[k] = R[k] - gamma @ Vl[k + 1]            # only level k, not 0..k
    x0 += gamma @ Vl[0]


def _eta_update_wrong_block(R, Vl, k, q, eta):
    new = [R[i + 1] - eta @ Vl[i + 1] for i in range(-1, k + 1)]   # drops V^(i+1)_{1:q-1}
    for i, v in zip(range(-1, k + 1), new):
        Vl[i + 1][q] = v


def _tau_update_wrong_sign_u(R, Vl, x0, tau):
    r, x, U, V = ORIG["tau_update"](R, Vl, x0, tau)
    U = Vl[0].copy()
    for i in range(1, len(tau) + 1):
        U += tau[i - 1] * Vl[i]
    return r, x, U, V


ORIG = {"tau_update": O.tau_update}


@pytest.mark.parametrize("name,fn", [
    ("tau_update", _tau_update_wrong_x_index),
    ("gamma_update", _gamma_update_no_lower_levels),
    ("eta_update", _eta_update_wrong_block),
    ("tau_update", _tau_update_wrong_sign_u),
])
def test_planted_mistakes_are_caught(monkeypatch, name, fn):
    monkeypatch.setattr(O, name, fn)
    caught = False
    try:
        test_invariants_hold_every_cycle(2, 2)
    except AssertionError:
        caught = True
    m = next(m for m in FT["msstab"] if m["s"] == 4 and m["data"][0]["G"] == 9)   # M(4)stab(1), data from G_9
    try:
        test_msstab_terminates_after_the_last_nonzero_m_space(m, m["data"][0], 1)
    except AssertionError:
        caught = True
    assert caught

"""Pins of the guess-selection oracle (oracle/guess.py) by what the
mathematics fixes: an exact correction in the span is found with zero
residual; one direction has the closed-form coefficient (w . r0)/(w . w); the
optimal residual is orthogonal to A times every direction; a zero direction
gets no weight; the selection never raises the residual.  Also the identity
that makes the previous step's change a natural direction for implicit-Euler
sequences: with exact solutions, b^(i+1) - A x^(i) = (x^(i) - x^(i-1)) / tau."""

import numpy as np
import scipy.sparse.linalg as spla

from oracle import guess as G
from paper_1604_06043_gb300 import problems as pb


def _system():
    w = pb.WORKLOADS["convdiff3d_24"]
    A = w.matrix()
    xp = w.x0()
    b = xp / w.tau + w.f()
    exact = spla.spsolve(A.to_scipy().tocsc(), b)
    return w, A, xp, b, exact


def test_exact_correction_in_the_span_is_found():
    w, A, xp, b, exact = _system()
    rnd = np.random.default_rng(1).standard_normal(A.n)
    x, a, red, used = G.select_span(A, b, xp, np.stack([rnd, exact - xp]))
    assert used and red < 1e-10
    assert abs(a[0]) < 1e-8 and abs(a[1] - 1.0) < 1e-8
    assert np.linalg.norm(x - exact) <= 1e-8 * np.linalg.norm(exact)


def test_single_direction_closed_form_and_orthogonality():
    w, A, xp, b, exact = _system()
    As = A.to_scipy()
    rng = np.random.default_rng(2)
    d1 = (exact - xp) + 0.3 * rng.standard_normal(A.n) * np.abs(exact - xp).max()
    x, a, red, used = G.select_span(A, b, xp, d1[None, :])
    r0 = b - As @ xp
    wv = As @ d1
    assert used and abs(a[0] - (wv @ r0) / (wv @ wv)) <= 1e-12 * abs(a[0])
    r = b - As @ x
    assert abs(np.linalg.norm(r) / np.linalg.norm(r0) - red) <= 1e-12
    # two directions: the optimal residual is orthogonal to A dir_j
    d2 = rng.standard_normal(A.n)
    x, a, red, used = G.select_span(A, b, xp, np.stack([d1, d2]))
    r = b - As @ x
    for d in (d1, d2):
        wd = As @ d
        assert abs(wd @ r) <= 1e-10 * np.linalg.norm(wd) * np.linalg.norm(r0)


def test_zero_direction_and_no_increase():
    w, A, xp, b, exact = _system()
    rng = np.random.default_rng(3)
    d = rng.standard_normal(A.n)
    x1, a1, red1, _ = G.select_span(A, b, xp, d[None, :])
    x2, a2, red2, _ = G.select_span(A, b, xp, np.stack([np.zeros(A.n), d]))
    assert a2[0] == 0.0 and abs(a2[1] - a1[0]) <= 1e-12 * abs(a1[0])
    assert red1 <= 1.0 and abs(red1 - red2) <= 1e-12
    # a direction orthogonal (through A) to r0 changes nothing: not kept
    As = A.to_scipy()
    r0 = b - As @ xp
    wd = As @ d
    # d' = d - (component whose image is along r0): pick d' with (A d') . r0 = 0
    e = np.zeros(A.n)
    e[0] = 1.0
    we = As @ e
    dp = d - ((wd @ r0) / (we @ r0)) * e
    x3, a3, red3, used3 = G.select_span(A, b, xp, dp[None, :])
    assert not used3 and red3 == 1.0 and np.array_equal(x3, xp)


def test_implicit_euler_residual_is_the_last_change_over_tau():
    w = pb.WORKLOADS["convdiff3d_24"]
    A = w.matrix()
    As = A.to_scipy().tocsc()
    f = w.f()
    x0 = w.x0()
    x1 = spla.spsolve(As, x0 / w.tau + f)
    x2 = spla.spsolve(As, x1 / w.tau + f)
    r0 = (x2 / w.tau + f) - As @ x2
    d = x2 - x1
    assert np.linalg.norm(r0 - d / w.tau) <= 1e-9 * np.linalg.norm(r0)

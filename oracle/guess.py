"""FP64 CPU oracle of the initial-guess selection of the learned-x0 form.

TEST INFRASTRUCTURE ONLY (see the package docstring).  Not part of the paper:
the workload's learned initial guess seeds x0 of a solve, and the solver still
runs to tolerance.  Given the previous solution x_prev of a sequence and a few
directions (the network's predicted change, the previous step's change
x^(i) - x^(i-1)), the start vector is the residual-minimising point of the
affine span

    x = x_prev + sum_j a_j dir_j,   a = argmin || r0 - W a ||_2,
    r0 = b - A x_prev,  W = [A dir_1, ..., A dir_m],

written out by its definition: the products with A, then a least-squares
solve (numpy's lstsq as the one library step).  The selection keeps the
combination only when it lowers the residual.
"""

from __future__ import annotations

import numpy as np


def select_span(A, b: np.ndarray, x_prev: np.ndarray, dirs: np.ndarray):
    """Returns (x, a, reduction, used): the start vector, the coefficients, the
    ratio ||b - A x|| / ||b - A x_prev|| and whether the combination was kept
    (x = x_prev, a = 0, reduction = 1 otherwise).  dirs: (m, N)."""
    As = A.to_scipy() if hasattr(A, "to_scipy") else A
    dirs = np.atleast_2d(np.asarray(dirs, dtype=np.float64))
    r0 = b - As @ x_prev
    W = np.stack([As @ d for d in dirs], axis=1)          # N x m
    a, *_ = np.linalg.lstsq(W, r0, rcond=None)
    r = r0 - W @ a
    n0 = float(np.linalg.norm(r0))
    if n0 == 0.0 or not np.all(np.isfinite(a)):
        return x_prev.copy(), np.zeros(len(dirs)), 1.0, False
    red = float(np.linalg.norm(r)) / n0
    if not red < 1.0:
        return x_prev.copy(), np.zeros(len(dirs)), 1.0, False
    return x_prev + a @ dirs, a, red, True

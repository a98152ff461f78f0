"""Seeded synthetic inputs for sequences A x^(i) = b^(i) with a fixed sparse A.

This module generates inputs only. It holds none of the solver's arithmetic and
is the one module that both the CUDA path (through the tests and the benchmark)
and the CPU oracle draw their inputs from:

* finite-difference convection-diffusion matrices in CSR form (int32 indices,
  float64 values, columns sorted within each row);
* the implicit-Euler data of a time-stepping sequence: the source term f and
  the start vector x^(0), both i.i.d. uniform [0, 1);
* the raw random basis from which the s-dimensional cut space P is built
  (i.i.d. standard normal; each side orthonormalises it on its own);
* a lognormal coefficient field for the variable-coefficient problem;
* the tridiag(2, 3, 1) test matrix and right-hand sides of the paper's
  finite-termination experiments (Section 5.2).

Discretisation (one reading of the workloads, applied everywhere): unit square
or cube, n interior points per axis, h = 1/(n+1), homogeneous Dirichlet
boundary, -div(kappa grad u) by the standard 2d+1 point stencil with face
coefficients taken as the harmonic mean of the two adjacent cell values
(kappa = 1 for the constant-coefficient problems), beta . grad u by central
differences, lexicographic ordering with x fastest.  The implicit-Euler matrix
is A = I/tau + L_h, and step i+1 has b = x^(i)/tau + f.

Seeds (numpy PCG64 ``default_rng``): f = 1, x^(0) = 2, P = 3, kappa = 4,
CNN initialisation = 5.
"""

from __future__ import annotations

import dataclasses
from typing import Optional, Sequence

import numpy as np

SEED_F = 1
SEED_X0 = 2
SEED_P = 3
SEED_KAPPA = 4
SEED_CNN = 5


@dataclasses.dataclass
class CSR:
    """Compressed sparse rows: row i holds col[row_ptr[i]:row_ptr[i+1]]."""

    n: int
    row_ptr: np.ndarray  # int32, n + 1
    col: np.ndarray      # int32, nnz
    val: np.ndarray      # float64, nnz

    @property
    def nnz(self) -> int:
        return int(self.row_ptr[-1])

    def to_scipy(self):
        import scipy.sparse as sp
        return sp.csr_matrix((self.val, self.col, self.row_ptr), shape=(self.n, self.n))

    def to_dense(self) -> np.ndarray:
        d = np.zeros((self.n, self.n))
        for i in range(self.n):
            for p in range(self.row_ptr[i], self.row_ptr[i + 1]):
                d[i, self.col[p]] += self.val[p]
        return d


def _from_stencil(cols: np.ndarray, vals: np.ndarray, mask: np.ndarray) -> CSR:
    """Pack an (n, m) stencil table (columns already ascending per row) into CSR."""
    n = cols.shape[0]
    counts = mask.sum(axis=1)
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=row_ptr[1:])
    if row_ptr[-1] >= 2**31:
        raise ValueError("nnz does not fit int32 indices")
    return CSR(n=n, row_ptr=row_ptr.astype(np.int32), col=cols[mask].astype(np.int32),
               val=vals[mask].astype(np.float64))


def convdiff(shape: Sequence[int], beta: Sequence[float], tau: Optional[float] = None,
             kappa: Optional[np.ndarray] = None) -> CSR:
    """Matrix of I/tau + (-div(kappa grad) + beta . grad) on an n_1 x ... x n_d grid.

    ``shape`` lists the interior points per axis in order (x, y[, z]); the grid
    is uniform with h = 1/(n+1) (all axes must have the same n).  ``tau=None``
    omits the identity term.  ``kappa`` (same shape, x fastest: kappa[z, y, x]
    in C order reversed, i.e. a flat array of length N in row order) gives the
    cell coefficients; None means kappa = 1.
    """
    shape = tuple(int(v) for v in shape)
    d = len(shape)
    if d not in (2, 3) or len(set(shape)) != 1:
        raise ValueError("shape must be (n, n) or (n, n, n)")
    n = shape[0]
    h = 1.0 / (n + 1)
    N = n ** d
    idx = np.arange(N, dtype=np.int64)
    # coordinate along each axis; axis 0 (x) is the fastest
    coord = [(idx // n ** a) % n for a in range(d)]
    kap = np.ones(N) if kappa is None else np.asarray(kappa, dtype=np.float64).reshape(N)
    if np.any(kap <= 0):
        raise ValueError("kappa must be positive")

    m = 2 * d + 1
    cols = np.zeros((N, m), dtype=np.int64)
    vals = np.zeros((N, m))
    mask = np.zeros((N, m), dtype=bool)
    diag = np.zeros(N) if tau is None else np.full(N, 1.0 / tau)
    # stencil slots in ascending column order: -e_{d-1}, ..., -e_0, centre, +e_0, ..., +e_{d-1}
    centre = d
    for a in range(d):
        stride = n ** a
        for sign in (-1, +1):
            slot = centre + sign * (a + 1)
            inside = (coord[a] + sign >= 0) & (coord[a] + sign < n)
            nb = np.where(inside, idx + sign * stride, idx)
            kface = np.where(inside, 2.0 * kap * kap[nb] / (kap + kap[nb]), kap)
            diag += kface / h**2
            c = -kface / h**2 + sign * float(beta[a]) / (2.0 * h)
            cols[:, slot] = nb
            vals[:, slot] = np.where(inside, c, 0.0)
            mask[:, slot] = inside
    cols[:, centre] = idx
    vals[:, centre] = diag
    mask[:, centre] = True
    return _from_stencil(cols, vals, mask)


def tridiag(n: int, sub: float, diag: float, sup: float) -> CSR:
    """tridiag(sub, diag, sup): sub-diagonal, diagonal and super-diagonal values."""
    idx = np.arange(n, dtype=np.int64)
    cols = np.stack([idx - 1, idx, idx + 1], axis=1)
    vals = np.tile(np.array([sub, diag, sup], dtype=np.float64), (n, 1))
    mask = (cols >= 0) & (cols < n)
    cols = np.where(mask, cols, 0)
    return _from_stencil(cols, vals, mask)


def offset_coupled(n: int, offset: int, sub: float, diag: float, sup: float) -> CSR:
    """Row i: sub in column i - offset, diag on the diagonal, sup in column
    i + offset (where those exist).  The rows split into runs of `offset`
    mutually independent rows, each coupled only to the runs beside it."""
    idx = np.arange(n, dtype=np.int64)
    cols = np.stack([idx - offset, idx, idx + offset], axis=1)
    vals = np.tile(np.array([sub, diag, sup], dtype=np.float64), (n, 1))
    mask = (cols >= 0) & (cols < n)
    cols = np.where(mask, cols, 0)
    return _from_stencil(cols, vals, mask)


def random_sparse(n: int, per_row: int, seed: int, band: Optional[int] = None) -> CSR:
    """A random sparse matrix with a general (non-stencil) pattern: each row
    holds its diagonal and up to per_row distinct off-diagonal columns drawn
    uniformly (from |j - i| <= band if band is given), columns sorted; the
    off-diagonal values are uniform in [-1, 1) and the diagonal is one plus the
    row's sum of their magnitudes (strict diagonal dominance)."""
    rng = np.random.default_rng(seed)
    rp = [0]
    cols, vals = [], []
    for i in range(n):
        lo, hi = (0, n) if band is None else (max(0, i - band), min(n, i + band + 1))
        cand = rng.integers(lo, hi, size=per_row)
        off = np.unique(cand[cand != i])
        v = rng.uniform(-1.0, 1.0, size=off.size)
        c = np.concatenate([off, [i]])
        w = np.concatenate([v, [1.0 + np.abs(v).sum()]])
        o = np.argsort(c)
        cols.append(c[o])
        vals.append(w[o])
        rp.append(rp[-1] + c.size)
    return CSR(n, np.array(rp, dtype=np.int32), np.concatenate(cols).astype(np.int32),
               np.concatenate(vals).astype(np.float64))


def termination_rhs(n: int = 40):
    """The two right-hand sides of the finite-termination experiments (Section 5.2):
    b1 = (1, ..., 1) and b2_i = sin(2 pi i / n), i = 1..n."""
    b1 = np.ones(n)
    b2 = np.sin(2.0 * np.pi / n * np.arange(1, n + 1))
    return b1, b2


def uniform(n: int, seed: int) -> np.ndarray:
    """n i.i.d. uniform [0, 1) values (float64)."""
    return np.random.default_rng(seed).random(n)


def randn_cols(n: int, s: int, seed: int = SEED_P) -> np.ndarray:
    """Raw cut-space basis: s columns of n i.i.d. N(0, 1) values, returned as an
    (s, n) array so that column q is the contiguous row q."""
    return np.random.default_rng(seed).standard_normal((s, n))


def randn_block_partitioned(n: int, s: int, seed: int) -> np.ndarray:
    """(s, n) raw cut space whose row i has its only non-zero, N(0,1), in
    column (i // 32) mod s: 32-row blocks dealt round-robin to the s columns.
    A random P with disjoint column supports (the columns are orthogonal
    already); the CUDA path detects this form and needs one multiply-add per
    row for P^T y."""
    rng = np.random.default_rng(seed)
    P = np.zeros((s, n))
    rows = np.arange(n)
    P[(rows // 32) % s, rows] = rng.standard_normal(n)
    return P


def lognormal_kappa(shape: Sequence[int], sigma: float = 1.0, corr: float = 8.0,
                    seed: int = SEED_KAPPA) -> np.ndarray:
    """kappa = exp(sigma g): g is white noise smoothed by a separable Gaussian of
    standard deviation ``corr`` cells (periodic, by FFT) and normalised to mean 0
    and variance 1.  Returns a flat array in row order (x fastest)."""
    shape = tuple(int(v) for v in shape)
    rng = np.random.default_rng(seed)
    # numpy axes are (z, y, x) so that the flattened array has x fastest
    noise = rng.standard_normal(shape[::-1])
    spec = np.fft.rfftn(noise)
    for ax, length in enumerate(shape[::-1]):
        freq = np.fft.rfftfreq(length) if ax == len(shape) - 1 else np.fft.fftfreq(length)
        gain = np.exp(-2.0 * (np.pi * corr * freq) ** 2)
        view = [1] * len(shape)
        view[ax] = gain.size
        spec *= gain.reshape(view)
    g = np.fft.irfftn(spec, s=shape[::-1], axes=tuple(range(len(shape))))
    g = (g - g.mean()) / g.std()
    return np.exp(sigma * g).reshape(-1)


CNN_LAYERS = [(2, 16), (16, 16), (16, 16), (16, 1)]   # (C_in, C_out), 3x3x3 kernels


def cnn_init_params(seed: int = SEED_CNN) -> np.ndarray:
    """Initial parameters of the learned-guess CNN as one flat float64 vector:
    per layer, weights (C_out, C_in, 3, 3, 3) He-uniform with bound
    sqrt(6 / fan_in), then C_out zero biases."""
    rng = np.random.default_rng(seed)
    parts = []
    for ci, co in CNN_LAYERS:
        bound = (6.0 / (ci * 27)) ** 0.5
        parts.append(rng.uniform(-bound, bound, size=co * ci * 27))
        parts.append(np.zeros(co))
    return np.concatenate(parts)


def row_stencil(A: CSR, shape: tuple, point: tuple) -> np.ndarray:
    """The 3x3x3 stencil of row `point` (z, y, x) of a matrix on the grid
    `shape` (x fastest): K[dz+1, dy+1, dx+1] = a(point, point + (dz, dy, dx)).
    Entries reaching beyond one cell raise."""
    nz, ny, nx = shape if len(shape) == 3 else (1,) + tuple(shape)
    z, y, x = point
    row = (z * ny + y) * nx + x
    K = np.zeros((3, 3, 3))
    for p in range(A.row_ptr[row], A.row_ptr[row + 1]):
        c = int(A.col[p])
        cz, rem = divmod(c, ny * nx)
        cy, cx = divmod(rem, nx)
        dz, dy, dx = cz - z, cy - y, cx - x
        if max(abs(dz), abs(dy), abs(dx)) > 1:
            raise ValueError("row reaches beyond the 3x3x3 neighbourhood")
        K[dz + 1, dy + 1, dx + 1] = A.val[p]
    return K


def crop_origins(shape, crop: int, count: int, seed: int) -> np.ndarray:
    """count random crop origins (z, y, x) of a crop^3 box inside a grid of the
    given (x, y, z) shape, as an int32 array (count, 3)."""
    rng = np.random.default_rng(seed)
    nx, ny, nz = shape
    return np.stack([rng.integers(0, nz - crop + 1, count), rng.integers(0, ny - crop + 1, count),
                     rng.integers(0, nx - crop + 1, count)], axis=1).astype(np.int32)


def cnn_crop_batches(n_pairs: int, shape, crop: int, batch: int, iters: int, seed: int = SEED_CNN) -> np.ndarray:
    """Crop origins for training the learned-guess CNN: iters x batch rows of
    (pair index, z0, y0, x0), int32, uniform over the stored pairs and over
    the positions of a crop^3 box inside the (x, y, z) grid."""
    rng = np.random.default_rng(seed)
    nx, ny, nz = shape
    m = iters * batch
    return np.stack([rng.integers(0, n_pairs, m), rng.integers(0, nz - crop + 1, m),
                     rng.integers(0, ny - crop + 1, m), rng.integers(0, nx - crop + 1, m)], axis=1).astype(np.int32)


@dataclasses.dataclass
class Workload:
    """One implicit-Euler sequence: A = I/tau + L_h, b^(i+1) = x^(i)/tau + f."""

    name: str
    shape: tuple
    beta: tuple
    tau: float
    steps: int
    s: int
    ell: int
    tol: float = 1e-8
    variable_kappa: bool = False
    replace_every: int = 0      # r := b - A x after every this many cycles (0: only to confirm)

    @property
    def n(self) -> int:
        return int(np.prod(self.shape))

    def matrix(self) -> CSR:
        kap = lognormal_kappa(self.shape) if self.variable_kappa else None
        return convdiff(self.shape, self.beta, tau=self.tau, kappa=kap)

    def f(self) -> np.ndarray:
        return uniform(self.n, SEED_F)

    def x0(self) -> np.ndarray:
        return uniform(self.n, SEED_X0)

    def p_raw(self) -> np.ndarray:
        return randn_cols(self.n, self.s, SEED_P)


# The sequences the solver is measured and tested on, named by what they are.
WORKLOADS = {
    # 2D, 32 x 32 interior grid, beta = (10, 10), 10 steps of tau = 0.01, s = 4, l = 2
    "convdiff2d_32": Workload("convdiff2d_32", (32, 32), (10.0, 10.0), 0.01, 10, 4, 2),
    # 3D, 128^3 grid, beta = (20, 10, 5), 50 steps of tau = 0.005, s = 8, l = 4
    # (true residual at every cycle end: the level vectors grow like ||A||^k and
    # the drift of V from A U would otherwise open a gap above tol)
    "convdiff3d_128": Workload("convdiff3d_128", (128, 128, 128), (20.0, 10.0, 5.0), 0.005, 50, 8, 4,
                               replace_every=1),
    # the same 128^3 sequence extended to 100 steps (learned initial guess)
    "convdiff3d_128_long": Workload("convdiff3d_128_long", (128, 128, 128), (20.0, 10.0, 5.0),
                                    0.005, 100, 8, 4, replace_every=1),
    # 3D variable-coefficient (lognormal kappa), 256^3, 100 steps, s = 16, l = 4;
    # beta and tau are not given for it and are taken equal to the 128^3 sequence
    "kappa3d_256": Workload("kappa3d_256", (256, 256, 256), (20.0, 10.0, 5.0), 0.005, 100, 16, 4,
                            variable_kappa=True, replace_every=1),
    # small 3D cases with the 128^3 sequence's physics, for parity tests that
    # span many thread blocks and a ragged tail
    "convdiff3d_24": Workload("convdiff3d_24", (24, 24, 24), (20.0, 10.0, 5.0), 0.005, 4, 8, 4),
    "convdiff3d_33": Workload("convdiff3d_33", (33, 33, 33), (20.0, 10.0, 5.0), 0.005, 3, 8, 4),
}

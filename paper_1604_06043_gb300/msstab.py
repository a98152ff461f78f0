"""Thin ctypes binding to libmsstab (include/msstab.h).

Argument marshalling only: every step of the solver runs in the library's
CUDA kernels.  Device buffers are torch CUDA tensors (PyTorch provides device
memory and the stream); their data pointers are passed straight through.  If
the library is not built, every call raises -- there is no CPU fallback.
"""

from __future__ import annotations

import ctypes
import os
from typing import Optional

import numpy as np

from . import build as _build

# status codes (msstab_status)
OK, ERR_INVALID_ARG, ERR_CUDA, ERR_OOM, ERR_BREAKDOWN, ERR_MAXIT, ERR_NAN = range(7)
STATUS_NAMES = {0: "ok", 1: "invalid_arg", 2: "cuda", 3: "oom", 4: "breakdown", 5: "maxit", 6: "nan"}
PREC_FP64, PREC_FP32_INNER = 0, 1
FETCH_ONCE, FETCH_EVERY, FETCH_NEVER, FETCH_SLOPE, FETCH_PROBE = 0, 1, 2, 3, 4
FORMAT_SELL, FORMAT_CSR = 0, 1
PRECOND_NONE, PRECOND_ILU0 = 0, 1
KERNEL_FAMILIES = ["spmv", "spmv_dot", "gamma", "eta", "lazy", "tau", "other", "cnn", "precond", "level"]


class Options(ctypes.Structure):
    _fields_ = [
        ("precision", ctypes.c_int32),
        ("fetch_policy", ctypes.c_int32),
        ("fetch_threshold", ctypes.c_double),
        ("fetch_cycle", ctypes.c_int32),
        ("orth_recycle", ctypes.c_int32),
        ("max_mvs", ctypes.c_int64),
        ("inner_tol", ctypes.c_double),
        ("spmv_format", ctypes.c_int32),
        ("sell_sigma", ctypes.c_int32),
        ("kernel_timing", ctypes.c_int32),
        ("max_outer", ctypes.c_int32),
        ("inner_ell", ctypes.c_int32),
        ("replace_every", ctypes.c_int32),
        ("precond", ctypes.c_int32),
        ("persistent", ctypes.c_int32),
        ("stream", ctypes.c_void_p),
        ("spin_limit", ctypes.c_int64),
    ]


class Stats(ctypes.Structure):
    _fields_ = [
        ("mvs", ctypes.c_int64),
        ("mvs_fp32", ctypes.c_int64),
        ("cycles", ctypes.c_int64),
        ("outer", ctypes.c_int64),
        ("launches", ctypes.c_int64),
        ("relres_true", ctypes.c_double),
        ("relres_rec", ctypes.c_double),
        ("ms", ctypes.c_double),
        ("status", ctypes.c_int32),
        ("fetched", ctypes.c_int32),
        ("used_recycle", ctypes.c_int32),
        ("guess_used", ctypes.c_int32),
        ("fp64_finish", ctypes.c_int32),
        ("fetch_at", ctypes.c_int32),
        ("relres_orig", ctypes.c_double),
        ("t_ms", ctypes.c_double * 10),
        ("n_launch", ctypes.c_int64 * 10),
    ]

    def as_dict(self):
        d = {f: getattr(self, f) for f, _ in self._fields_ if f not in ("t_ms", "n_launch")}
        d["status_name"] = STATUS_NAMES.get(self.status, str(self.status))
        d["t_ms"] = dict(zip(KERNEL_FAMILIES, list(self.t_ms)))
        d["n_launch"] = dict(zip(KERNEL_FAMILIES, list(self.n_launch)))
        return d


class MsstabError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


_P = ctypes.c_void_p
_I32, _I64, _D = ctypes.c_int32, ctypes.c_int64, ctypes.c_double
_SIGS = {
    "msstab_default_options": (None, [ctypes.POINTER(Options)]),
    "msstab_create": (_I32, [_I64, _I64, _P, _P, _P, _I32, _I32, _P, ctypes.POINTER(Options), ctypes.POINTER(_P)]),
    "msstab_solve": (_I32, [_P, _P, _P, _D, ctypes.POINTER(Stats)]),
    "msstab_solve_host": (_I32, [_P, _P, _P, _D, ctypes.POINTER(Stats)]),
    "msstab_destroy": (_I32, [_P]),
    "msstab_last_error": (ctypes.c_char_p, [_P]),
    "msstab_history": (_I32, [_P, _P, _P, _I32, ctypes.POINTER(_I32)]),
    "msstab_reset_recycle": (_I32, [_P]),
    "msstab_set_spin_limit": (_I32, [_P, _I64]),
    "msstab_has_recycle": (_I32, [_P, ctypes.POINTER(_I32)]),
    "msstab_export_recycle": (_I32, [_P, _P, _P]),
    "msstab_import_recycle": (_I32, [_P, _P, _P]),
    "msstab_select_guess": (_I32, [_P, _P, _P, _P, _P, ctypes.POINTER(_I32)]),
    "msstab_select_guess_scaled": (_I32, [_P, _P, _P, _P, _P, ctypes.POINTER(_I32), ctypes.POINTER(_D),
                                          ctypes.POINTER(_D)]),
    "msstab_select_guess_span": (_I32, [_P, _P, _P, _P, _I64, _I32, _P, ctypes.POINTER(_I32), _P,
                                        ctypes.POINTER(_D)]),
    "msstab_op_spmv": (_I32, [_P, _I32, _P, _P]),
    "msstab_op_residual": (_I32, [_P, _P, _P, _P, _P]),
    "msstab_op_spmv_dot": (_I32, [_P, _I32, _P, _P, _P]),
    "msstab_op_get_p": (_I32, [_P, _I32, _P]),
    "msstab_op_axpby": (_I32, [_P, _D, _P, _D, _P, _P]),
    "msstab_op_multidot": (_I32, [_P, _I32, _P, _I64, _I32, _P, _I64, _I32, _P]),
    "msstab_op_gamma_update": (_I32, [_P, _I32, _P, _P, _I64, _I32, _P]),
    "msstab_op_eta_update": (_I32, [_P, _I32, _P, _P, _I64, _I32, _I32, _P]),
    "msstab_op_lazy_update": (_I32, [_P, _I32, _P, _P, _P, _I64, _I32, _P, _P, _P]),
    "msstab_op_tau_update": (_I32, [_P, _I32, _P, _P, _P, _I64, _P]),
    "msstab_op_tau_step": (_I32, [_P, _I32, _P, _P, _P, _I64, _P, _I32, _P, _P, _P]),
    "msstab_op_small_solve": (_I32, [_P, _I32, _P, _P, _P, _P]),
    "msstab_op_tau_solve": (_I32, [_P, _I32, _P, _P]),
    "msstab_op_ilu_factor": (_I32, [_P, _P]),
    "msstab_op_ilu_levels": (_I32, [_P, _P, _P, _P]),
    "msstab_op_ilu_apply": (_I32, [_P, _I32, _P, _P]),
    "msstab_spmv_dot_noalloc": (_I32, [_I64, _I64, _P, _P, _P, _P, _P, _P, _I64, _I32, _P, _P]),
    "msstab_cnn_num_params": (_I32, []),
    "msstab_cnn_create": (_I32, [_I32, _I32, _I32, _P, _I32, _I32, _I32, _P, ctypes.POINTER(_P)]),
    "msstab_cnn_destroy": (_I32, [_P]),
    "msstab_cnn_last_error": (ctypes.c_char_p, [_P]),
    "msstab_cnn_get_params": (_I32, [_P, _P]),
    "msstab_cnn_set_params": (_I32, [_P, _P]),
    "msstab_cnn_set_scales": (_I32, [_P, ctypes.c_float, ctypes.c_float]),
    "msstab_cnn_set_loss_stencil": (_I32, [_P, _P]),
    "msstab_cnn_get_scales": (_I32, [_P, _P]),
    "msstab_cnn_fit_scales": (_I32, [_P]),
    "msstab_cnn_add_pair": (_I32, [_P, _P, _P, _P]),
    "msstab_cnn_train": (_I32, [_P, _I32, _I32, _I32, _P, ctypes.c_float, _P]),
    "msstab_cnn_forward": (_I32, [_P, _P, _I32, _I32, _P]),
    "msstab_cnn_grad": (_I32, [_P, _P, _P, _I32, _I32, _P, ctypes.POINTER(_D)]),
    "msstab_cnn_adam_step": (_I32, [_P, _P, ctypes.c_float]),
    "msstab_cnn_infer": (_I32, [_P, _P, _P, _P]),
}

_lib = None


def lib_path() -> str:
    return _build.lib_path()


def load(path: Optional[str] = None):
    """Load libmsstab.so (built in-tree by ``build.build()``); raises if absent."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    path = path or lib_path()
    if not os.path.exists(path):
        raise RuntimeError(f"libmsstab.so not found at {path}: build it first "
                           "(python -c 'import __graft_entry__ as g; g.build()')")
    lib = ctypes.CDLL(path)
    for name, (res, args) in _SIGS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def default_options(**kw) -> Options:
    o = Options()
    load().msstab_default_options(ctypes.byref(o))
    for k, v in kw.items():
        if not hasattr(o, k):
            raise TypeError(f"unknown option {k}")
        setattr(o, k, v)
    return o


def _ptr(t) -> int:
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return t.data_ptr()


def _check(rc, h=None):
    if rc != OK:
        msg = load().msstab_last_error(h)
        raise MsstabError(rc, msg.decode() if msg else "")


class Solver:
    """A handle of libmsstab for one matrix A (CSR) and cut-space dimension s.

    ``A`` is a ``problems.CSR`` (host arrays, copied to the device here) or a
    tuple ``(n, row_ptr, col, val)`` of CUDA tensors.  ``p_raw`` is the raw
    random basis of P, shape (s, n).  Keyword arguments set msstab_options
    fields (precision, fetch_policy, fetch_threshold, fetch_cycle, orth_recycle,
    max_mvs, inner_tol, spmv_format, sell_sigma, kernel_timing, max_outer,
    inner_ell, replace_every, precond, persistent, spin_limit).
    """

    def __init__(self, A, s: int, ell: int, p_raw, device: str = "cuda", stream=None, **options):
        import torch
        lib = load()
        if isinstance(A, tuple):
            n, row_ptr, col, val = A
        else:
            n = A.n
            row_ptr = torch.as_tensor(A.row_ptr, dtype=torch.int32, device=device)
            col = torch.as_tensor(A.col, dtype=torch.int32, device=device)
            val = torch.as_tensor(A.val, dtype=torch.float64, device=device)
        if not isinstance(p_raw, torch.Tensor):
            p_raw = torch.as_tensor(np.ascontiguousarray(p_raw), dtype=torch.float64, device=device)
        if tuple(p_raw.shape) != (s, n):
            raise ValueError(f"p_raw must have shape (s, n) = {(s, n)}")
        self.n, self.s, self.ell = int(n), int(s), int(ell)
        self.device = device
        if stream is None:
            stream = torch.cuda.current_stream()
        opt = default_options(**options)
        opt.stream = stream.cuda_stream
        self._stream = stream
        self.options = opt
        h = ctypes.c_void_p()
        rc = lib.msstab_create(self.n, int(val.numel()), _ptr(row_ptr), _ptr(col), _ptr(val), self.s, self.ell,
                               _ptr(p_raw.contiguous()), ctypes.byref(opt), ctypes.byref(h))
        if rc != OK:
            raise MsstabError(rc, lib.msstab_last_error(None).decode())
        self._h = h

    # -- lifetime --------------------------------------------------------
    def close(self):
        if getattr(self, "_h", None):
            load().msstab_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    @property
    def handle(self):
        return self._h

    # -- solving ---------------------------------------------------------
    def solve(self, b, x, tol: float = 1e-8, check: bool = True) -> Stats:
        """Solve A x = b; x (CUDA float64) holds x0 and receives the solution."""
        st = Stats()
        rc = load().msstab_solve(self._h, _ptr(b), _ptr(x), float(tol), ctypes.byref(st))
        if check and rc not in (OK,):
            _check(rc, self._h)
        return st

    def solve_host(self, b: np.ndarray, x: np.ndarray, tol: float = 1e-8, check: bool = True) -> Stats:
        """As solve, with host float64 arrays (copies inside the call)."""
        if b.dtype != np.float64 or x.dtype != np.float64 or not x.flags.c_contiguous:
            raise ValueError("b and x must be contiguous float64 arrays")
        st = Stats()
        rc = load().msstab_solve_host(self._h, b.ctypes.data, x.ctypes.data, float(tol), ctypes.byref(st))
        if check and rc != OK:
            _check(rc, self._h)
        return st

    def history(self):
        cnt = ctypes.c_int32()
        load().msstab_history(self._h, None, None, 0, ctypes.byref(cnt))
        rel = np.zeros(cnt.value)
        mv = np.zeros(cnt.value, dtype=np.int64)
        load().msstab_history(self._h, rel.ctypes.data, mv.ctypes.data, cnt.value, ctypes.byref(cnt))
        return rel, mv

    def set_spin_limit(self, polls: int):
        _check(load().msstab_set_spin_limit(self._h, int(polls)), self._h)

    def solve_rc(self, b, x, tol: float = 1e-8):
        """As solve, returning (status code, Stats) instead of raising."""
        st = Stats()
        rc = load().msstab_solve(self._h, _ptr(b), _ptr(x), float(tol), ctypes.byref(st))
        return rc, st

    def last_error(self) -> str:
        m = load().msstab_last_error(self._h)
        return m.decode() if m else ""

    def reset_recycle(self):
        _check(load().msstab_reset_recycle(self._h), self._h)

    def has_recycle(self) -> bool:
        f = ctypes.c_int32()
        _check(load().msstab_has_recycle(self._h, ctypes.byref(f)), self._h)
        return bool(f.value)

    def export_recycle(self, U, V):
        _check(load().msstab_export_recycle(self._h, _ptr(U), _ptr(V)), self._h)

    def import_recycle(self, U, V):
        _check(load().msstab_import_recycle(self._h, _ptr(U), _ptr(V)), self._h)

    def select_guess(self, b, xprev, delta, x) -> bool:
        used = ctypes.c_int32()
        _check(load().msstab_select_guess(self._h, _ptr(b), _ptr(xprev), _ptr(delta), _ptr(x),
                                          ctypes.byref(used)), self._h)
        return bool(used.value)

    def select_guess_scaled(self, b, xprev, delta, x):
        """x = xprev + alpha delta with the residual-minimising alpha; returns
        (used, alpha, ||b - A x|| / ||b - A xprev||)."""
        used, a, red = ctypes.c_int32(), ctypes.c_double(), ctypes.c_double()
        _check(load().msstab_select_guess_scaled(self._h, _ptr(b), _ptr(xprev), _ptr(delta), _ptr(x),
                                                 ctypes.byref(used), ctypes.byref(a), ctypes.byref(red)), self._h)
        return bool(used.value), a.value, red.value

    def select_guess_span(self, b, xprev, dirs, x):
        """x = xprev + sum_j a_j dirs[j] with the residual-minimising a (dirs:
        (m, n) CUDA float64, m <= 4); returns (used, a, ||b - A x|| / ||b - A xprev||)."""
        m = dirs.shape[0]
        used, red = ctypes.c_int32(), ctypes.c_double()
        coef = (ctypes.c_double * m)()
        _check(load().msstab_select_guess_span(self._h, _ptr(b), _ptr(xprev), _ptr(dirs), dirs.shape[1], m,
                                               _ptr(x), ctypes.byref(used), coef, ctypes.byref(red)), self._h)
        return bool(used.value), list(coef), red.value

    # -- kernel-level entry points -----------------------------------------
    def op_spmv(self, x, y, prec: int = 0):
        _check(load().msstab_op_spmv(self._h, prec, _ptr(x), _ptr(y)), self._h)

    def op_residual(self, b, x, r, out):
        _check(load().msstab_op_residual(self._h, _ptr(b), _ptr(x), _ptr(r), _ptr(out)), self._h)

    def op_spmv_dot(self, x, y, dots, prec: int = 0):
        _check(load().msstab_op_spmv_dot(self._h, prec, _ptr(x), _ptr(y), _ptr(dots)), self._h)

    def op_axpby(self, alpha, x, beta, z, y):
        """y = alpha x + beta z on the handle's stream (no synchronisation)."""
        _check(load().msstab_op_axpby(self._h, float(alpha), _ptr(x), float(beta), _ptr(z), _ptr(y)), self._h)

    def op_get_p(self, P, prec: int = 0):
        _check(load().msstab_op_get_p(self._h, prec, _ptr(P)), self._h)

    def op_multidot(self, X, Y, out, prec: int = 0):
        nx, ldx = X.shape
        ny, ldy = Y.shape
        _check(load().msstab_op_multidot(self._h, prec, _ptr(X), ldx, nx, _ptr(Y), ldy, ny, _ptr(out)), self._h)

    def op_gamma_update(self, R, V, k, gamma, prec: int = 0):
        _check(load().msstab_op_gamma_update(self._h, prec, _ptr(R), _ptr(V), R.shape[1], k, _ptr(gamma)), self._h)

    def op_eta_update(self, R, V, k, q, eta, prec: int = 0):
        _check(load().msstab_op_eta_update(self._h, prec, _ptr(R), _ptr(V), R.shape[1], k, q, _ptr(eta)), self._h)

    def op_lazy_update(self, R, V, x, k, gamma, eta, gram=None, prec: int = 0):
        _check(load().msstab_op_lazy_update(self._h, prec, _ptr(R), _ptr(V), _ptr(x), R.shape[1], k, _ptr(gamma),
                                            _ptr(eta), _ptr(gram)), self._h)

    def op_tau_update(self, R, V, x, tau, prec: int = 0):
        _check(load().msstab_op_tau_update(self._h, prec, _ptr(R), _ptr(V), _ptr(x), R.shape[1], _ptr(tau)),
               self._h)

    def op_tau_step(self, R, V, x, tau, out, do_update: bool = True, prec: int = 0, lazy_gamma=None,
                    lazy_eta=None):
        _check(load().msstab_op_tau_step(self._h, prec, _ptr(R), _ptr(V), _ptr(x), R.shape[1], _ptr(tau),
                                         1 if do_update else 0, _ptr(lazy_gamma), _ptr(lazy_eta), _ptr(out)),
               self._h)

    def op_small_solve(self, M, rhs, z, flag):
        _check(load().msstab_op_small_solve(self._h, rhs.numel(), _ptr(M), _ptr(rhs), _ptr(z), _ptr(flag)),
               self._h)

    def op_tau_solve(self, gram, tau):
        _check(load().msstab_op_tau_solve(self._h, tau.numel(), _ptr(gram), _ptr(tau)), self._h)

    # ILU(0) split preconditioner (handles created with precond=PRECOND_ILU0)
    def op_ilu_factor(self, lu):
        _check(load().msstab_op_ilu_factor(self._h, _ptr(lu)), self._h)

    def op_ilu_levels(self, lev_lower=None, lev_upper=None):
        """Per-row levels (into the optional int32 tensors) and
        (levels lower, levels upper, widest lower, widest upper, blocks lower, blocks upper)."""
        info = (ctypes.c_int32 * 6)()
        _check(load().msstab_op_ilu_levels(self._h, _ptr(lev_lower), _ptr(lev_upper), info), self._h)
        return tuple(info)

    def op_ilu_apply(self, which: int, x, y):
        """which 0: y = L^-1 x; 1: y = U^-1 x; 2: y = U x; 3: y = L^-1 A U^-1 x."""
        _check(load().msstab_op_ilu_apply(self._h, which, _ptr(x), _ptr(y)), self._h)


class CNN:
    """The learned-initial-guess network of libmsstab (thin wrapper)."""

    def __init__(self, shape, params, max_pairs=0, max_batch=8, crop=32, device="cuda", stream=None):
        import torch
        lib = load()
        nx, ny, nz = shape
        p = torch.as_tensor(np.ascontiguousarray(params), dtype=torch.float32, device=device)
        if p.numel() != lib.msstab_cnn_num_params():
            raise ValueError("wrong parameter count")
        stream = stream or torch.cuda.current_stream()
        self._stream = stream
        h = ctypes.c_void_p()
        rc = lib.msstab_cnn_create(nx, ny, nz, p.data_ptr(), max_pairs, max_batch, crop, stream.cuda_stream,
                                   ctypes.byref(h))
        if rc != OK:
            raise MsstabError(rc, lib.msstab_cnn_last_error(None).decode())
        self._h = h
        self.device = device
        self.shape = shape

    def _chk(self, rc):
        if rc != OK:
            raise MsstabError(rc, load().msstab_cnn_last_error(self._h).decode())

    def close(self):
        if getattr(self, "_h", None):
            load().msstab_cnn_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def params(self):
        import torch
        out = torch.empty(load().msstab_cnn_num_params(), dtype=torch.float32, device=self.device)
        self._chk(load().msstab_cnn_get_params(self._h, out.data_ptr()))
        return out

    def set_params(self, p):
        self._chk(load().msstab_cnn_set_params(self._h, _ptr(p)))

    def set_scales(self, s_x, c):
        self._chk(load().msstab_cnn_set_scales(self._h, s_x, c))

    def set_loss_stencil(self, k27=None):
        """Operator-weighted loss with the 3x3x3 stencil k27 (host array, any
        scale), or the plain mean squared error for None."""
        if k27 is None:
            self._chk(load().msstab_cnn_set_loss_stencil(self._h, None))
            return
        k = np.ascontiguousarray(np.asarray(k27, dtype=np.float64).reshape(27))
        self._chk(load().msstab_cnn_set_loss_stencil(self._h, k.ctypes.data))

    def scales(self):
        out = (ctypes.c_float * 2)()
        self._chk(load().msstab_cnn_get_scales(self._h, out))
        return list(out)

    def fit_scales(self):
        self._chk(load().msstab_cnn_fit_scales(self._h))

    def add_pair(self, r0, x_prev, x_next):
        """A training pair: r0 = b - A x_prev, x_prev -> x_next - x_prev."""
        self._chk(load().msstab_cnn_add_pair(self._h, _ptr(r0), _ptr(x_prev), _ptr(x_next)))

    def train(self, origins, B, D, lr):
        o = np.ascontiguousarray(origins, dtype=np.int32)
        iters = o.size // (4 * B)
        hist = np.zeros(iters, dtype=np.float32)
        self._chk(load().msstab_cnn_train(self._h, iters, B, D, o.ctypes.data, float(lr), hist.ctypes.data))
        return hist

    def forward(self, x, B, D):
        import torch
        out = torch.empty((B, D * D * D), dtype=torch.float32, device=self.device)
        self._chk(load().msstab_cnn_forward(self._h, _ptr(x), B, D, out.data_ptr()))
        return out

    def grad(self, x, t, B, D):
        import torch
        g = torch.empty(load().msstab_cnn_num_params(), dtype=torch.float32, device=self.device)
        loss = ctypes.c_double()
        self._chk(load().msstab_cnn_grad(self._h, _ptr(x), _ptr(t), B, D, g.data_ptr(), ctypes.byref(loss)))
        return g, loss.value

    def adam_step(self, g, lr):
        self._chk(load().msstab_cnn_adam_step(self._h, _ptr(g), float(lr)))

    def infer(self, r0, x_prev, delta):
        """delta = the network's correction from r0 = b - A x_prev and x_prev."""
        self._chk(load().msstab_cnn_infer(self._h, _ptr(r0), _ptr(x_prev), _ptr(delta)))


def exported_symbols():
    """Names of the C entry points this binding declares."""
    return sorted(_SIGS)

"""The allocation-free entry point msstab_spmv_dot_noalloc.

It serves callers that may not allocate device memory themselves (a host
application that owns all device memory through its own pool, or a loop where
an allocation is not allowed): the reduction scratch lives in a fixed device
array inside the library.  Here it is called through the C ABI and checked
against the handle-based entry point msstab_op_spmv_dot (same kernel) on two
calls in a row -- the second call reuses the scratch the first one left
behind -- with the tolerance of the kernel tests: 1e-12 relative to the sum
of the absolute values of the terms.  Cases: s = 0 (no P, only y . y), 1, 8
and 16 (the largest s, 17 sums per block) on N = 35,937 (many blocks and a
ragged tail), s = 8 on N = 2,097,152 (more rows than threads in the grid, so
every thread runs several rows), one call on a non-default stream, and a check
that a call after the first one changes the device's free memory by nothing.
This file is collected last; it passes alone in a fresh process and after the
other tests.
"""

import numpy as np
import pytest

from paper_1604_06043_gb300 import problems as pb

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL64 = 1e-12
DEV = "cuda:0"


def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1604_06043_gb300 import build, msstab as M
    build.build()
    return M, M.load()


def _device_csr(A):
    rp = torch.tensor(A.row_ptr, dtype=torch.int32, device=DEV)
    col = torch.tensor(A.col, dtype=torch.int32, device=DEV)
    val = torch.tensor(A.val, dtype=torch.float64, device=DEV)
    return rp, col, val


def _noalloc(lib, A, csr, x, y, P, s, d, stream):
    rp, col, val = csr
    return lib.msstab_spmv_dot_noalloc(A.n, A.nnz, rp.data_ptr(), col.data_ptr(), val.data_ptr(), x.data_ptr(),
                                       y.data_ptr(), P.data_ptr() if P is not None else None, A.n, s,
                                       d.data_ptr(), stream.cuda_stream)


def _check_against_handle(M, lib, A, s, seeds, stream=None):
    """Two calls in a row (one per seed), each against msstab_op_spmv_dot of a
    CSR handle and against the definition."""
    sh = max(s, 1)                        # a handle needs s >= 1; s = 0 compares y and y . y only
    S = M.Solver(A, sh, 2, pb.randn_cols(A.n, sh, pb.SEED_P), device=DEV, spmv_format=M.FORMAT_CSR)
    P = torch.empty((sh, A.n), dtype=torch.float64, device=DEV)
    S.op_get_p(P)
    csr = _device_csr(A)
    Pn = P.cpu().numpy()[:s]
    As = A.to_scipy()
    Aabs = abs(As)
    for seed in seeds:
        xn = pb.uniform(A.n, seed) - 0.5
        x = torch.tensor(xn, device=DEV)
        y_ref = torch.empty(A.n, dtype=torch.float64, device=DEV)
        d_ref = torch.zeros(sh + 1, dtype=torch.float64, device=DEV)
        S.op_spmv_dot(x, y_ref, d_ref)
        torch.cuda.synchronize()
        y = torch.full((A.n,), float("nan"), dtype=torch.float64, device=DEV)
        d = torch.full((s + 1,), float("nan"), dtype=torch.float64, device=DEV)
        st = stream if stream is not None else torch.cuda.current_stream()
        rc = _noalloc(lib, A, csr, x, y, P if s > 0 else None, s, d, st)
        assert rc == M.OK, lib.msstab_last_error(None)
        st.synchronize()
        yabs = Aabs @ np.abs(xn)
        yn, yr = y.cpu().numpy(), y_ref.cpu().numpy()
        assert np.all(np.abs(yn - yr) <= TOL64 * yabs)
        dn, drf = d.cpu().numpy(), d_ref.cpu().numpy()
        dr = np.concatenate([drf[:s], [drf[sh]]])
        scale = np.concatenate([np.abs(Pn) @ yabs, [yabs @ yabs]])
        assert np.all(np.abs(dn - dr) <= TOL64 * scale), (seed, dn - dr, scale)
        # and both against the definition
        yd = As @ xn
        ref = np.concatenate([Pn @ yd, [yd @ yd]])
        assert np.all(np.abs(dn - ref) <= 4 * TOL64 * scale)
    S.close()


@pytest.mark.parametrize("s", [0, 1, 8, 16])
def test_noalloc_matches_handle_entry_point_on_two_calls(s):
    M, lib = _lib()
    A = pb.WORKLOADS["convdiff3d_33"].matrix()     # N = 35937: many blocks and a ragged tail
    _check_against_handle(M, lib, A, s, (21, 22))


def test_noalloc_grid_stride_on_128_cube():
    # 2,097,152 rows: more than the grid's threads, so each thread loops
    M, lib = _lib()
    A = pb.WORKLOADS["convdiff3d_128"].matrix()
    _check_against_handle(M, lib, A, 8, (23, 24))


def test_noalloc_on_a_non_default_stream():
    M, lib = _lib()
    A = pb.WORKLOADS["convdiff3d_33"].matrix()
    side = torch.cuda.Stream(device=DEV)
    _check_against_handle(M, lib, A, 8, (25,), stream=side)


def test_noalloc_allocates_nothing_after_the_first_call():
    M, lib = _lib()
    A = pb.WORKLOADS["convdiff3d_33"].matrix()
    csr = _device_csr(A)
    s = 4
    P = torch.tensor(pb.randn_cols(A.n, s, pb.SEED_P), device=DEV)
    x = torch.tensor(pb.uniform(A.n, 26), device=DEV)
    y = torch.empty(A.n, dtype=torch.float64, device=DEV)
    d = torch.empty(s + 1, dtype=torch.float64, device=DEV)
    st = torch.cuda.current_stream()
    assert _noalloc(lib, A, csr, x, y, P, s, d, st) == M.OK     # first call: module and address set-up
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info(DEV)
    for _ in range(3):
        assert _noalloc(lib, A, csr, x, y, P, s, d, st) == M.OK
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info(DEV)
    # device allocations come in pages of at least 2 MiB; the calls made none
    assert free0 - free1 < (2 << 20), (free0, free1)


def test_noalloc_rejects_sizes_beyond_its_scratch():
    M, lib = _lib()
    z = torch.zeros(64, dtype=torch.float64, device=DEV)
    rp = torch.zeros(65, dtype=torch.int32, device=DEV)
    rc = lib.msstab_spmv_dot_noalloc(64, 0, rp.data_ptr(), None, None, z.data_ptr(), z.data_ptr(), z.data_ptr(),
                                     64, 17, z.data_ptr(), None)
    assert rc == M.ERR_INVALID_ARG
    assert b"s must be" in lib.msstab_last_error(None)
    rc = lib.msstab_spmv_dot_noalloc((1 << 31) - (1 << 22) + 1, 0, rp.data_ptr(), None, None, z.data_ptr(),
                                     z.data_ptr(), z.data_ptr(), 1 << 31, 4, z.data_ptr(), None)
    assert rc == M.ERR_INVALID_ARG
    assert b"n must be" in lib.msstab_last_error(None)

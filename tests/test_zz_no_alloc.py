"""The allocation-free entry point msstab_spmv_dot_noalloc.

It serves callers that may not allocate device memory themselves (a host
application that owns all device memory through its own pool, or a loop where
an allocation is not allowed): the reduction scratch lives in a fixed device
array inside the library.  Here it is called through the C ABI and checked
against the handle-based entry point msstab_op_spmv_dot (same kernel) on two
calls in a row -- the second call reuses the scratch the first one left
behind -- with the tolerance of the kernel tests: 1e-12 relative to the sum
of the absolute values of the terms.  This file is collected last; it passes
alone in a fresh process and after the other tests.
"""

import numpy as np
import pytest

from paper_1604_06043_gb300 import problems as pb

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL64 = 1e-12
DEV = "cuda:0"


def test_noalloc_matches_handle_entry_point_on_two_calls():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1604_06043_gb300 import build, msstab as M
    build.build()
    lib = M.load()
    w = pb.WORKLOADS["convdiff3d_33"]          # N = 35937: many blocks and a ragged tail
    A = w.matrix()
    s = 8
    S = M.Solver(A, s, 2, pb.randn_cols(A.n, s, pb.SEED_P), device=DEV, spmv_format=M.FORMAT_CSR)
    P = torch.empty((s, A.n), dtype=torch.float64, device=DEV)
    S.op_get_p(P)
    rp = torch.tensor(A.row_ptr, dtype=torch.int32, device=DEV)
    col = torch.tensor(A.col, dtype=torch.int32, device=DEV)
    val = torch.tensor(A.val, dtype=torch.float64, device=DEV)
    stream = torch.cuda.current_stream()
    Pn = P.cpu().numpy()
    As = A.to_scipy()
    for seed in (21, 22):
        xn = pb.uniform(A.n, seed) - 0.5
        x = torch.tensor(xn, device=DEV)
        y_ref = torch.empty(A.n, dtype=torch.float64, device=DEV)
        d_ref = torch.zeros(s + 1, dtype=torch.float64, device=DEV)
        S.op_spmv_dot(x, y_ref, d_ref)
        y = torch.full((A.n,), float("nan"), dtype=torch.float64, device=DEV)
        d = torch.full((s + 1,), float("nan"), dtype=torch.float64, device=DEV)
        rc = lib.msstab_spmv_dot_noalloc(A.n, A.nnz, rp.data_ptr(), col.data_ptr(), val.data_ptr(), x.data_ptr(),
                                         y.data_ptr(), P.data_ptr(), A.n, s, d.data_ptr(), stream.cuda_stream)
        assert rc == M.OK, lib.msstab_last_error(None)
        torch.cuda.synchronize()
        yabs = abs(As) @ np.abs(xn)
        yn, yr = y.cpu().numpy(), y_ref.cpu().numpy()
        assert np.all(np.abs(yn - yr) <= TOL64 * yabs)
        dn, dr = d.cpu().numpy(), d_ref.cpu().numpy()
        scale = np.concatenate([np.abs(Pn) @ yabs, [yabs @ yabs]])
        assert np.all(np.abs(dn - dr) <= TOL64 * scale)
        # and both against the definition
        ref = np.concatenate([Pn @ (As @ xn), [(As @ xn) @ (As @ xn)]])
        assert np.all(np.abs(dn - ref) <= 4 * TOL64 * scale)
    S.close()


def test_noalloc_rejects_sizes_beyond_its_scratch():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1604_06043_gb300 import build, msstab as M
    build.build()
    lib = M.load()
    z = torch.zeros(64, dtype=torch.float64, device=DEV)
    rp = torch.zeros(65, dtype=torch.int32, device=DEV)
    rc = lib.msstab_spmv_dot_noalloc(64, 0, rp.data_ptr(), None, None, z.data_ptr(), z.data_ptr(), z.data_ptr(),
                                     64, 17, z.data_ptr(), None)
    assert rc == M.ERR_INVALID_ARG
    assert b"s must be" in lib.msstab_last_error(None)

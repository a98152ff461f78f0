"""Parity at the full sizes of the measured workloads.

128^3: the CUDA path solves the first 23 systems of the implicit-Euler
sequence and each system is compared with the FP64 oracle's committed record
of the same sequence (written by tests/golden/make_oracle_records.py from
oracle/ alone): the true residual, the solution on 512 seeded rows and its
norm, and the products with A.

At s = 8, l = 4 on this sequence the iteration amplifies rounding: two correct
FP64 implementations (the oracle under another BLAS thread count or another
summation order of its dot products, or the GPU) agree through cycle 2 of the
first system and then drift apart (residuals a factor 2-6 apart from cycle 4
on).  Every later system starts from the basis fetched in the first solve, so
each implementation carries its own fetched basis through the whole sequence.
Two tests follow from this:

* the same-basis test: both sides fetch at the end of cycle 2 of the first
  system, before the drift (oracle_convdiff3d_128_fetch2.json).  The later
  systems then start from the same basis up to rounding; within each system
  the histories agree for the first three or four cycles and then drift the
  same way, so the relative residual after cycle 2 must agree within 5 % and
  products with A within 2 except on systems where the two sides stop one
  cycle apart, whose number is bounded by what the oracle shows against
  itself under another summation order.
* the benchmarked sequence (fetch at relres <= sqrt(tol), cycle 8): the first
  system (no recycled basis) must agree within 2 products; on the later
  systems each side runs with its own draw of the fetched basis, so the count
  of one-cycle cases is bounded by the spread that different draws produce,
  and the sum of products with A over systems 2..23 must be within 8 % of the
  record's.
"""

import json
import os

import numpy as np
import pytest

from paper_1604_06043_gb300 import problems as pb
from parity_rules import one_cycle_apart

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
DEV = "cuda:0"
GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "oracle_convdiff3d_128.json")
GOLDEN_FETCH2 = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden",
                             "oracle_convdiff3d_128_fetch2.json")
# one-cycle cases allowed among the 22 recycled systems (see the module
# docstring): the oracle against its own same-basis record under pairwise
# summation stopped one cycle apart on 6 of its first 11 systems, the other
# oracle draws against the benchmarked record on 5-7 of 22, the GPU's draws on
# 10 of 22 (8 of 22 with the same basis)
ONE_CYCLE_MAX_SAME_BASIS = 11
ONE_CYCLE_MAX_OWN_BASIS = 12
# relative residual after cycle 2 of each same-basis system (observed: GPU
# 0.77 %, the pairwise-summation oracle 0.75 % at most)
CYCLE2_REL = 0.05


@pytest.fixture(scope="module")
def M():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1604_06043_gb300 import build, msstab
    build.build()
    return msstab


def _sequence_against_record(M, rec, **opt):
    """Solve the record's systems in order; check every system's true
    residual and solution; return per-system (GPU MVs, record MVs, within 2?)."""
    w = pb.WORKLOADS["convdiff3d_128"]
    assert rec["n"] == w.n and rec["s"] == w.s and rec["ell"] == w.ell
    assert rec["replace_every"] == w.replace_every
    A = w.matrix()
    As = A.to_scipy()
    rows = np.array(rec["sample_rows"])
    S = M.Solver(A, w.s, w.ell, w.p_raw(), device=DEV, replace_every=w.replace_every, **opt)
    f = torch.tensor(w.f(), device=DEV)
    x = torch.tensor(w.x0(), device=DEV)
    b = torch.empty_like(x)
    xprev = w.x0()
    out = []
    for i, r in enumerate(rec["systems"]):
        S.op_axpby(1.0 / w.tau, x, 1.0, f, b)
        st = S.solve(b, x, w.tol)
        xn = x.cpu().numpy()
        bn = xprev / w.tau + w.f()
        assert st.status == 0
        assert np.linalg.norm(bn - As @ xn) <= w.tol * np.linalg.norm(bn) * 1.0001, i
        hist, _ = S.history()
        # within 2, or one cycle apart (counted by the callers)
        within2 = abs(int(st.mvs) - int(r["mvs"])) <= 2
        assert within2 or one_cycle_apart(hist, r["history"]), (i, st.mvs, r["mvs"], hist, r["history"])
        xo = np.array(r["x_sample"])
        assert np.max(np.abs(xn[rows] - xo)) <= 1e-6 * np.max(np.abs(xo)), i
        assert abs(np.linalg.norm(xn) - r["x_norm"]) <= 1e-7 * r["x_norm"]
        out.append((int(st.mvs), int(r["mvs"]), within2, [float(v) for v in hist], r["history"]))
        xprev = xn
    S.close()
    return out


def test_128_sequence_same_basis_matches_oracle_record(M):
    if not os.path.exists(GOLDEN_FETCH2):
        pytest.skip("the fetch-at-cycle-2 record is not committed")
    rec = json.load(open(GOLDEN_FETCH2))
    assert rec["fetch_cycle"] == 2
    res = _sequence_against_record(M, rec, fetch_cycle=2)
    assert res[0][2]                                   # the first system: within 2
    # before the within-system drift: the residual after cycle 2 of every
    # recycled system, started from the same basis
    for i, (_, _, _, hg, ho) in enumerate(res[1:], start=2):
        assert abs(hg[2] - ho[2]) <= CYCLE2_REL * ho[2], (i, hg[:4], ho[:4])
    one_cycle = [(i + 1, g, o) for i, (g, o, ok, _, _) in enumerate(res) if not ok]
    print("same basis: GPU %d, oracle %d products with A over %d systems; one cycle apart: %s"
          % (sum(r[0] for r in res), sum(r[1] for r in res), len(res), one_cycle))
    assert len(one_cycle) <= ONE_CYCLE_MAX_SAME_BASIS, one_cycle


def test_128_sequence_matches_oracle_record(M):
    rec = json.load(open(GOLDEN))
    res = _sequence_against_record(M, rec)
    assert res[0][2]                                   # the first system: within 2
    one_cycle = [(i + 1, g, o) for i, (g, o, ok, _, _) in enumerate(res) if not ok]
    tot_g = sum(r[0] for r in res[1:])
    tot_o = sum(r[1] for r in res[1:])
    print("own bases: GPU %d, oracle %d products with A over systems 2..%d; one cycle apart: %s"
          % (tot_g, tot_o, len(res), one_cycle))
    assert len(one_cycle) <= ONE_CYCLE_MAX_OWN_BASIS, one_cycle
    assert abs(tot_g - tot_o) <= 0.08 * tot_o


def test_128_fp32_inner_form_against_oracle_record(M):
    # the FP32-inner form as benchmarked (inner M(s)stab(1), FP64 defect
    # correction): every system to the FP64 true residual tol, the solution
    # against the FP64 oracle's record on the sampled rows
    rec = json.load(open(GOLDEN))
    w = pb.WORKLOADS["convdiff3d_128"]
    A = w.matrix()
    As = A.to_scipy()
    rows = np.array(rec["sample_rows"])
    S = M.Solver(A, w.s, w.ell, w.p_raw(), device=DEV, precision=M.PREC_FP32_INNER, inner_ell=1,
                 fetch_policy=M.FETCH_NEVER, max_outer=40, replace_every=w.replace_every)
    f = torch.tensor(w.f(), device=DEV)
    x = torch.tensor(w.x0(), device=DEV)
    b = torch.empty_like(x)
    xprev = w.x0()
    worst = 0.0
    for i, r in enumerate(rec["systems"]):
        S.op_axpby(1.0 / w.tau, x, 1.0, f, b)
        st = S.solve(b, x, w.tol)
        xn = x.cpu().numpy()
        bn = xprev / w.tau + w.f()
        assert st.status == 0 and st.mvs_fp32 > 0
        assert np.linalg.norm(bn - As @ xn) <= w.tol * np.linalg.norm(bn) * 1.0001, i
        xo = np.array(r["x_sample"])
        err = np.max(np.abs(xn[rows] - xo)) / np.max(np.abs(xo))
        assert err <= 1e-6, (i, err)
        worst = max(worst, err)
        xprev = xn
    print("FP32-inner form, systems 1..%d: max sampled error vs the oracle %.2e" % (len(rec["systems"]), worst))


def test_256_kappa_sampled_rows_and_first_solve(M):
    w = pb.WORKLOADS["kappa3d_256"]
    A = w.matrix()
    S = M.Solver(A, w.s, w.ell, w.p_raw(), device=DEV, replace_every=w.replace_every)
    rng = np.random.default_rng(31)
    xs = rng.random(A.n) - 0.5
    y = torch.empty(A.n, dtype=torch.float64, device=DEV)
    S.op_spmv(torch.tensor(xs, device=DEV), y)
    yn = y.cpu().numpy()
    rows = rng.choice(A.n, size=4000, replace=False)
    for i in rows:                                   # the definition, row by row
        lo, hi = A.row_ptr[i], A.row_ptr[i + 1]
        ref = float(np.sum(A.val[lo:hi] * xs[A.col[lo:hi]]))
        scale = float(np.sum(np.abs(A.val[lo:hi]) * np.abs(xs[A.col[lo:hi]])))
        assert abs(yn[i] - ref) <= 1e-12 * scale
    x0 = w.x0()
    bn = x0 / w.tau + w.f()
    x = torch.tensor(x0, device=DEV)
    st = S.solve(torch.tensor(bn, device=DEV), x, w.tol)
    r = bn - A.to_scipy() @ x.cpu().numpy()
    assert np.linalg.norm(r) <= w.tol * np.linalg.norm(bn) * 1.0001
    assert st.status == 0 and st.fetched == 1
    S.close()

"""Pins of the fetching-point policies of the oracle (the section on choosing
the fetching point: fetch "shortly before the residual drops"; optionally
estimate the point from a first IDRstab solve).

The paper's own finite-termination experiments (Section 5.2) fix where such a
rule must land: it fetches IDR(2)stab(1) data after 19 cycles (60 MVs, range V
in G_19), IDR(4)stab(1) data from G_9, and IDR(4)stab(2) data after 4 cycles
(G_8, "data B").  Both the estimate from a complete history and the test
applied while the solve runs pick exactly these cycles, and the data fetched by
the running test is the data of a fixed fetch at that cycle, bit for bit.
"""

import json
import math
import os

import numpy as np
import pytest

from oracle import idrstab as O
from paper_1604_06043_gb300 import problems as pb

TRI = pb.tridiag(40, 2.0, 3.0, 1.0)
B1, B2 = pb.termination_rhs(40)


def _P(s):
    return O.orthonormalize_mgs2(pb.randn_cols(40, s, pb.SEED_P))


FT = json.load(open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden",
                                 "paper_finite_termination.json")))


def _paper_points():
    """(s, l, fetching cycle) of the paper's fetches: IDR(2)stab(1) after 60 MVs
    (G_19), IDR(4)stab(1) from G_9 (the l = 1 figure; its data A from G_8 is the
    same run fetched one cycle earlier) and IDR(4)stab(2) from G_8 (data B)."""
    f = FT["fetch_after_mvs"]
    pts = [(f["s"], f["ell"], f["G"] // f["ell"])]
    for m in FT["msstab"]:
        for d in m["data"]:
            if d.get("name") == "A":
                continue
            pts.append((m["s"], d["ell"], d["G"] // d["ell"]))
    return sorted(set(pts))


PAPER_POINTS = _paper_points()
assert PAPER_POINTS == [(2, 1, 19), (4, 1, 9), (4, 2, 4)]


@pytest.mark.parametrize("s,ell,cycle", PAPER_POINTS)
def test_estimate_from_a_probe_history_is_the_papers_fetching_point(s, ell, cycle):
    res = O.idrstab(TRI, B1, np.zeros(40), s, ell, _P(s), tol=1e-14, max_mvs=2000)
    assert O.fetch_estimate(res.history) == cycle


@pytest.mark.parametrize("s,ell,cycle", PAPER_POINTS)
def test_running_drop_test_fetches_the_papers_data(s, ell, cycle):
    P = _P(s)
    res = O.idrstab(TRI, B1, np.zeros(40), s, ell, P, tol=1e-14, max_mvs=2000, fetch_slope=True)
    assert res.fetch_cycle == cycle
    fixed = O.idrstab(TRI, B1, np.zeros(40), s, ell, P, tol=1e-14, max_mvs=2000, fetch_cycle=cycle)
    assert np.array_equal(res.fetched[0], fixed.fetched[0]) and np.array_equal(res.fetched[1], fixed.fetched[1])
    # the data terminates M(s)stab on the second right-hand side as in the paper
    m = O.idrstab(TRI, B2, np.zeros(40), s, ell, P, *res.fetched, tol=1e-13, max_mvs=2000)
    assert m.status == O.OK and m.cycles < res.cycles


def test_estimate_closed_forms():
    # decreases in log10: 1, 0.3, 4.7, 1 -> steepest in cycle 3 -> fetch at cycle 2
    h = [1.0, 0.1, 0.05, 1e-6, 1e-7]
    lg = [math.log10(v) for v in h]
    assert max(range(1, 5), key=lambda k: lg[k - 1] - lg[k]) == 3
    assert O.fetch_estimate(h) == 2
    assert O.fetch_estimate([1.0, 1e-9]) == 1                 # one cycle: at least 1
    assert O.fetch_estimate([1.0]) is None                    # no cycle
    assert O.fetch_estimate([1.0, 0.1, 0.01, 0.001]) == 1     # equal drops: the first


def test_running_drop_test_closed_forms():
    h = [1.0, 0.5, 0.25, 1e-3]
    assert not O.slope_fires(h, 1)                            # needs an earlier cycle
    assert not O.slope_fires(h, 2)                            # 0.3 decades
    assert O.slope_fires(h, 3)                                # 2.4 >= 1 and >= 2 x 0.3
    steady = [10.0 ** (-k) for k in range(8)]                 # one decade each cycle
    assert not any(O.slope_fires(steady, k) for k in range(1, 8))


@pytest.mark.parametrize("policy", ["slope", "probe"])
def test_sequence_policies(policy):
    w = pb.WORKLOADS["convdiff2d_32"]
    A = w.matrix()
    seq = O.msstab_sequence(A, w.f(), w.x0(), w.tau, w.steps, w.s, w.ell, w.p_raw(), tol=w.tol, policy=policy)
    S = seq.solves
    assert all(r.status == O.OK and r.relres_true <= w.tol for r in S)
    s = w.s
    if policy == "slope":
        assert S[0].fetched is not None and 1 <= S[0].fetch_cycle <= S[0].cycles
        rest = S[1:]
    else:
        assert S[0].fetched is None                                   # the probe writes nothing
        k = O.fetch_estimate(S[0].history)
        assert S[1].fetched is not None and S[1].fetch_cycle == min(k, S[1].cycles)
        rest = S[2:]
    # later systems start from the fetched basis: no Arnoldi products
    for r in rest:
        assert r.mv_history[0] == 1 and r.mv_history[1] == 1 + w.ell * (s + 1)

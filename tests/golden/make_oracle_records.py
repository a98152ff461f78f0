"""Write the FP64 oracle's record of the 128^3 implicit-Euler sequence.

The oracle (``oracle/``) solves the first systems of the 3D convection-diffusion
sequence (128^3 grid, beta = (20, 10, 5), tau = 0.005, s = 8, l = 4, tol 1e-8,
M(s)stab with one fetch in the first solve, the true residual replacing the
recursive one at every cycle end) from the seeded inputs, and this
script stores, per system: products with A, cycles, the relative recursive
residual after each cycle, the true relative residual, ||x||, and x at 512
seeded sample rows.  The full-size GPU parity tests compare against this
record, and the CPU baseline of the benchmark takes its cycles per system from
it.  Nothing here touches the CUDA path.

    python tests/golden/make_oracle_records.py [--systems N] [--fetch-cycle C]
        [--threads T] [--dots blas|pairwise] [--out FILE]

Defaults write the committed record (oracle_convdiff3d_128.json: fetch at the
first cycle end with relres <= sqrt(tol), the BLAS pool's default threads).
The options write the records that show how the iteration depends on rounding:
--fetch-cycle 2 fetches at the end of cycle 2 of the first system (before the
rounding differences of two correct FP64 implementations have grown, so that
both hand the same basis on; oracle_convdiff3d_128_fetch2.json, one BLAS
thread); --threads sets the BLAS pool size before numpy loads (another
summation order of the projections); --dots pairwise sums every projection and
Gram entry of Algorithm 1 by numpy's pairwise summation instead of BLAS (a
third order).  Each full run takes 40-60 minutes on one core.
"""

import argparse
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
HERE = os.path.dirname(os.path.abspath(__file__))
OUT = os.path.join(HERE, "oracle_convdiff3d_128.json")


def sample_rows(n, k=512, seed=99):
    import numpy as np
    rows = np.random.default_rng(seed).choice(n, size=k - 2, replace=False)
    return np.sort(np.concatenate([[0, n - 1], rows])).astype(np.int64)


def main(systems=23, out=OUT, fetch_cycle=None, threads=None, dots="blas"):
    if threads:
        os.environ["OPENBLAS_NUM_THREADS"] = str(threads)
        os.environ["OMP_NUM_THREADS"] = str(threads)
    import numpy as np
    sys.path.insert(0, ROOT)
    from oracle import idrstab as O
    from paper_1604_06043_gb300 import problems as pb
    if dots == "pairwise":
        # the same projections and Gram entries, their terms added in numpy's
        # pairwise order instead of the BLAS kernels' order
        O.proj = lambda P, w: np.array([np.sum(p * w) for p in P])

        def tau_step(R):
            L = len(R)
            return O.tau_from_gram(np.array([[np.sum(R[a] * R[c]) for c in range(L)] for a in range(L)]))
        O.tau_step = tau_step
    w = pb.WORKLOADS["convdiff3d_128"]
    A = w.matrix()
    rows = sample_rows(w.n)
    rec = {"workload": w.name, "n": w.n, "nnz": A.nnz, "s": w.s, "ell": w.ell, "tau": w.tau, "tol": w.tol,
           "policy": "once", "fetch_threshold": "sqrt(tol)" if not fetch_cycle else None,
           "fetch_cycle": fetch_cycle, "orth_recycle": True, "replace_every": w.replace_every,
           "blas_threads": threads, "dots": dots,
           "sample_rows": rows.tolist(), "systems": []}
    t_start = time.time()

    def on_solve(res):
        rec["systems"].append({
            "mvs": int(res.mvs), "cycles": int(res.cycles), "status": res.status,
            "relres_true": float(res.relres_true), "history": [float(h) for h in res.history],
            "fetched": res.fetched is not None, "fetch_cycle": int(res.fetch_cycle),
            "x_norm": float(np.linalg.norm(res.x)), "x_sample": res.x[rows].tolist(),
            "seconds": time.time() - t_start,
        })
        tmp = out + ".tmp"
        with open(tmp, "w") as fh:
            json.dump(rec, fh)
        os.replace(tmp, out)
        print(len(rec["systems"]), res.mvs, res.cycles, res.relres_true, time.time() - t_start, flush=True)

    O.msstab_sequence(A, w.f(), w.x0(), w.tau, systems, w.s, w.ell, w.p_raw(), tol=w.tol, policy="once",
                      fetch_cycle=fetch_cycle, replace_every=w.replace_every, on_solve=on_solve)


if __name__ == "__main__":
    ap = argparse.ArgumentParser()
    ap.add_argument("--systems", type=int, default=23)
    ap.add_argument("--fetch-cycle", type=int, default=None)
    ap.add_argument("--threads", type=int, default=None)
    ap.add_argument("--dots", choices=["blas", "pairwise"], default="blas")
    ap.add_argument("--out", default=None)
    a = ap.parse_args()
    out = a.out or (os.path.join(HERE, "oracle_convdiff3d_128_fetch2.json") if a.fetch_cycle == 2 else OUT)
    main(a.systems, out, a.fetch_cycle, a.threads, a.dots)

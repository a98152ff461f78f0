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

    python tests/golden/make_oracle_records.py [systems [output.json]]
"""

import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import idrstab as O  # noqa: E402
from paper_1604_06043_gb300 import problems as pb  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "oracle_convdiff3d_128.json")


def sample_rows(n, k=512, seed=99):
    rows = np.random.default_rng(seed).choice(n, size=k - 2, replace=False)
    return np.sort(np.concatenate([[0, n - 1], rows])).astype(np.int64)


def main(systems=23, out=OUT):
    w = pb.WORKLOADS["convdiff3d_128"]
    A = w.matrix()
    rows = sample_rows(w.n)
    rec = {"workload": w.name, "n": w.n, "nnz": A.nnz, "s": w.s, "ell": w.ell, "tau": w.tau, "tol": w.tol,
           "policy": "once", "fetch_threshold": "sqrt(tol)", "orth_recycle": True,
           "replace_every": w.replace_every,
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
                      replace_every=w.replace_every, on_solve=on_solve)


if __name__ == "__main__":
    main(int(sys.argv[1]) if len(sys.argv) > 1 else 23, sys.argv[2] if len(sys.argv) > 2 else OUT)

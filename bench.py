#!/usr/bin/env python
"""Benchmark of the M(s)stab(l) solver on GB300: ms and products with A per
system for the 128^3 implicit-Euler convection-diffusion sequence at 1e-8
relative residual, with the roofline of the dominant kernel.

A step is one system of the sequence: b = x^(i)/tau + f formed on the device,
then msstab_solve (the whole hot path: products with A fused with the P^T
projections, the gamma/eta/lazy level updates, the degree-l step, the device
small solves, the fetch of the recycled basis).  The first --warmup systems
(system 1 runs IDRstab with its Arnoldi start and fetches U, V) are untimed;
the next --steps systems are timed.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl native|reference]

With --gpus N > 1 (launched by torchrun) every rank solves its own replica of
the sequence (the solver does not shard); value = max-over-ranks time / all
systems solved.  One JSON line is printed by rank 0.
"""

from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "ms/system & #MVs for 128³ implicit-Euler seq at 1e-8 rel res; SpMV HBM GB/s"
UNIT = "ms/system"
WORKLOAD = "convdiff3d_128"
GOLDEN = os.path.join(ROOT, "tests", "golden", "oracle_convdiff3d_128.json")
FAMILIES = ["spmv", "spmv_dot", "gamma", "eta", "lazy", "tau", "other", "cnn", "precond", "level"]
FP64_NOMINAL_TFLOPS = 1.25   # GB300 FP64 (vector and tensor), nominal
# GB300 FP32 on the CUDA cores, from the unit counts and the clock: 152 SMs x
# 128 FP32 lanes x 2 flops (multiply-add) x 2.07 GHz
FP32_NOMINAL_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12
# DRAM bytes (read + write) of one launch of the dominant kernel of each form,
# from one ncu capture of the current kernel at 128^3
# (profiles/ncu_level_fp64_convdiff3d_128.md, ncu_spmv_dot_*_convdiff3d_128.md).
NCU_TRAFFIC = {("convdiff3d_128", "fp64", "level"): 4_600_663_808,
               ("convdiff3d_128", "fp64", "spmv_dot"): 342_305_280,
               ("convdiff3d_128", "fp32_inner", "spmv_dot"): 200_357_376,
               ("convdiff3d_128", "ilu0", "precond"): 161_049_344}


def parse_args(argv=None):
    p = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=20)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", choices=["native", "reference"], default="native")
    p.add_argument("--workload", default=WORKLOAD)
    p.add_argument("--form", choices=["fp64", "fp32_inner", "fp32_inner_recycled", "idrstab", "ilu0"],
                   default="fp64",
                   help="the solver form of the main line: FP64 M(s)stab (default), the FP32-inner "
                        "defect-correction form, or FP64 IDR(s)stab with an Arnoldi start per system")
    p.add_argument("--no-variants", action="store_true", help="skip the IDRstab and FP32-inner runs")
    p.add_argument("--variants", default="", help="comma-separated subset of the variants (default: all)")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--cnn", action="store_true",
                   help="time only the learned-guess network: inference on the full grid and training iterations")
    p.add_argument("--cpu-worker", action="store_true", help=argparse.SUPPRESS)
    p.add_argument("--cpu-full-small", action="store_true", help=argparse.SUPPRESS)
    p.add_argument("--cpu-level-steps", type=int, default=4, help=argparse.SUPPRESS)
    p.add_argument("--cpu-k0", type=int, default=0, help=argparse.SUPPRESS)
    return p.parse_args(argv)


# ---------------------------------------------------------------------------
# distributed helpers (replicas only)
# ---------------------------------------------------------------------------

def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


def aggregate(elapsed_ms: float, steps: int, world: int, dist=None):
    """Max of the per-rank elapsed times and the whole-job ms per system."""
    t = elapsed_ms
    if dist is not None and world > 1:
        import torch
        v = torch.tensor([elapsed_ms], dtype=torch.float64)
        if dist.get_backend() == "nccl":
            v = v.cuda()
        dist.all_reduce(v, op=dist.ReduceOp.MAX)
        t = float(v.item())
    return t, t / (steps * world)


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------

class Clocks:
    QUERY = ("index,uuid,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, uuid=None):
        self.uuid = uuid
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(prefix="clocks", suffix=".csv")
            os.close(fd)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.QUERY}", "--format=csv,noheader",
                                          "-lms", "100"], stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        sm, smax, power, reasons = [], [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [c.strip() for c in line.split(",")]
            if len(f) < 10:
                continue
            if self.uuid and f[1] != self.uuid:
                continue
            try:
                sm.append(float(f[2].split()[0]))
                smax.append(float(f[3].split()[0]))
                power.append(float(f[4].split()[0]))
            except ValueError:
                continue
            for name, val in zip(names, f[6:10]):
                if val.lower() == "active":
                    reasons.add(name)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "power_w_max": max(power) if power else None, "samples": len(sm), "reasons": sorted(reasons)}


# ---------------------------------------------------------------------------
# algorithmic bytes and flops per kernel family (FP64 vectors)
# ---------------------------------------------------------------------------

def sell_entries(A):
    import numpy as np
    lens = np.diff(A.row_ptr.astype(np.int64))
    pad = (-len(lens)) % 32
    lens = np.concatenate([lens, np.zeros(pad, dtype=np.int64)]).reshape(-1, 32)
    return int(lens.max(axis=1).sum() * 32), lens.shape[0]


def family_model(A, s, ell, cycles, solves, replaced=0, vb=8):
    """Algorithmic bytes and FP64 flops of the launches of one timed region.

    Every operand is counted once per launch: the matrix arrays, x read once,
    y written once, each vector column read or written once.  ``replaced``
    true residuals r = b - A x at cycle ends are fused SpMV + P dots that also
    read b."""
    n = A.n
    nnz_sell, nsl = sell_entries(A)
    v = vb * n
    spmv = nnz_sell * (4 + vb) + 8 * nsl + 2 * v
    m = {}
    nd = cycles * ell * (s + 1)
    m["spmv_dot"] = dict(launches=nd + replaced, bytes=spmv + s * v + v * replaced / max(1, nd + replaced),
                         flops=2 * (A.nnz + s * n) + 2 * n * replaced / max(1, nd + replaced))
    m["eta"] = dict(launches=cycles * ell * s, bytes=(s + 2) * v, flops=2 * s * n)
    m["gamma"] = dict(launches=cycles * ell, bytes=(s + 2) * v, flops=2 * s * n)
    lazy_b = sum((s + 1) + (k + 1) * (2 * s + 2) for k in range(ell)) * v
    lazy_f = sum((k + 1) * (s * s + s) for k in range(ell)) * 2 * n
    m["lazy"] = dict(launches=cycles * ell, bytes=lazy_b / ell, flops=lazy_f / ell)
    # the persistent level step: the gamma step, s + 1 fused products, s eta steps
    m["level"] = dict(launches=cycles * ell, bytes=(s + 2) * v + (s + 1) * (spmv + s * v) + s * (s + 2) * v,
                      flops=2 * s * n + (s + 1) * 2 * (A.nnz + s * n) + s * 2 * s * n)
    tau_cycle_b = (ell + 1) * v + ((ell + 1) + 1 + s * (ell + 2) + s + 3 + 2 * s) * v
    tau_cycle_f = 2 * (ell + 1) ** 2 * n + 2 * ((2 * s + 2) * ell + s * (s + 1) + 1) * n
    tau_b = cycles * tau_cycle_b + solves * (2 * s + 1) * v
    tau_f = cycles * tau_cycle_f + solves * 2 * s * (s + 1) * n
    m["tau"] = dict(launches=2 * cycles + solves, bytes=tau_b / max(1, 2 * cycles + solves),
                    flops=tau_f / max(1, 2 * cycles + solves))
    return m, spmv


# ---------------------------------------------------------------------------
# CPU baseline: the oracle, as it stands, on the host cores
# ---------------------------------------------------------------------------

def golden_cycles(first, count, workload="convdiff3d_128"):
    """Mean cycles and MVs per system of systems first..first+count-1 (1-based)
    in the oracle's committed record of the workload, or None."""
    try:
        rec = json.load(open(GOLDEN))
    except Exception:
        return None
    if rec.get("workload") != workload:
        return None
    sy = rec["systems"][first - 1:first - 1 + count]
    if not sy:
        sy = rec["systems"][1:] or rec["systems"]
    if not sy:
        return None
    return (statistics.mean(x["cycles"] for x in sy), statistics.mean(x["mvs"] for x in sy), len(sy))


def FP32_INNER_OPTS(M):
    """The FP32-inner form without recycling: inner IDR(s)stab(1) (FP32 level
    vectors drift for l > 1 on these systems), an Arnoldi start for the first
    inner solve of every system, the basis continued across its
    defect-correction steps, inner tolerance 1e-2 (the library default)."""
    return dict(precision=M.PREC_FP32_INNER, inner_ell=1, fetch_policy=M.FETCH_NEVER, max_outer=40)


def FP32_INNER_RECYCLED_OPTS(M):
    """The FP32-inner form as M(s)stab: the same inner M(s)stab(1), with U, V
    fetched once (first system, relative inner residual <= sqrt(inner tol))
    and passed to the first inner solve of every later system."""
    return dict(precision=M.PREC_FP32_INNER, inner_ell=1, fetch_policy=M.FETCH_ONCE, max_outer=40)


def s_ell_cols(w):
    """Vector columns of the FP64 workspace: (s+1)(l+2) + 3s + 4."""
    return (w.s + 1) * (w.ell + 2) + 3 * w.s + 4


def workload_config(w, n, nnz, W, K, form, world):
    """The `config` object of both arms' JSON lines."""
    dims = "x".join(str(d) for d in w.shape)
    kind = ("variable-coefficient convection-diffusion (lognormal kappa, sigma 1, correlation 8 cells)"
            if getattr(w, "variable_kappa", False) else "convection-diffusion")
    return {"workload": f"{w.name}: 3D {kind}, 7-point FD on a {dims} grid (N={n}, nnz={nnz}), "
                        f"beta={tuple(w.beta)}, implicit Euler tau={w.tau}, systems {W + 1}..{W + K} of the sequence",
            "method": {"fp64": f"M({w.s})stab({w.ell}), fetch once at sqrt(tol), FP64, SELL-32",
                       "fp32_inner": f"FP32-inner IDR({w.s})stab(1) (no recycling) with FP64 defect correction, "
                                     f"SELL-32",
                       "fp32_inner_recycled": f"FP32-inner M({w.s})stab(1), fetch once, with FP64 defect "
                                              f"correction, SELL-32",
                       "idrstab": f"IDR({w.s})stab({w.ell}), Arnoldi start per system, FP64, SELL-32",
                       "ilu0": f"M({w.s})stab({w.ell}) on L^-1 A U^-1 (ILU(0) split preconditioner), fetch once "
                               f"at sqrt(tol), FP64, SELL-32"}[form],
            "true_residual": "replaced every cycle" if w.replace_every == 1 else "checked at convergence",
            "tol": w.tol, "l2": l2_note(w, n, nnz),
            "parallelism": "replicas" if world > 1 else "single GPU"}


L2_BYTES = 129e6   # GB300 L2


def l2_note(w, n, nnz):
    """Whether the step's inputs exceed L2 (so no flush is needed between steps)."""
    foot = f"matrix {12 * nnz / 1e9:.2f} GB + {s_ell_cols(w)} vectors of {8 * n / 1e6:.1f} MB"
    if 12 * nnz + 8 * n > L2_BYTES:
        return f"inputs larger than L2 ({foot}), no flush"
    return f"inputs fit in L2 ({foot}): no flush, timings include L2 reuse"


def extra_mvs(w, cyc):
    """Products with A per system outside the level steps: r0 = b - A x0, and
    the true residuals (one per replace_every cycles, else one to confirm)."""
    return 1 + (cyc / w.replace_every if w.replace_every > 0 else 1)


def cpu_worker(args):
    """Time the oracle on the host: level steps of Algorithm 1 (s = 8, l = 4) on
    system 1 of the workload's sequence, after its Arnoldi start.  Prints JSON."""
    import numpy as np
    from oracle import idrstab as O
    from paper_1604_06043_gb300 import problems as pb
    w = pb.WORKLOADS[args.workload]
    A = w.matrix()
    mv = O.MatVec(A)
    P = O.orthonormalize_mgs2(w.p_raw())
    x = w.x0().copy()
    b = x / w.tau + w.f()
    t0 = time.perf_counter()
    r = b - mv(x)
    t_mv = time.perf_counter() - t0
    U, V = O.arnoldi_start(mv, r, w.s, P)
    R = [r.copy()] + [None] * w.ell
    Vl = [U.copy(), V.copy()] + [np.zeros((w.s, w.n)) for _ in range(w.ell)]
    x0 = x.copy()
    times = []
    for step in range(args.cpu_level_steps):
        k = (args.cpu_k0 + step) % w.ell
        if k == 0 and step > 0:
            R = [R[0]] + [None] * w.ell
        t0 = time.perf_counter()
        gamma = O.gamma_step(P, R, Vl, k)
        O.gamma_update(R, Vl, x0, gamma, k)
        R[k + 1] = mv(R[k])
        for q in range(w.s):
            eta = O.eta_step(P, R, Vl, k, q)
            O.eta_update(R, Vl, k, q, eta)
            Vl[k + 2][q] = mv(Vl[k + 1][q])
        if k == w.ell - 1:
            tau = O.tau_step(R)
            r, x0, U_, V_ = O.tau_update(R, Vl, x0, tau)
            Vl[0], Vl[1] = U_, V_
            R[0] = r
        times.append(time.perf_counter() - t0)
    threads = int(os.environ.get("OPENBLAS_NUM_THREADS", "0")) or len(os.sched_getaffinity(0))
    print(json.dumps({"level_step_s": times, "mv_s": t_mv, "threads": threads}))


def cpu_full_small(args):
    """Time the oracle end to end on the small 2D configuration (32 x 32 grid,
    10 systems, M(4)stab(2), fetch once): the whole sequence.  Prints JSON."""
    from oracle import idrstab as O
    from paper_1604_06043_gb300 import problems as pb
    w = pb.WORKLOADS["convdiff2d_32"]
    A = w.matrix()
    t0 = time.perf_counter()
    res = O.msstab_sequence(A, w.f(), w.x0(), w.tau, w.steps, w.s, w.ell, w.p_raw(), tol=w.tol, policy="once",
                            replace_every=w.replace_every)
    dt = time.perf_counter() - t0
    print(json.dumps({"seconds": dt, "mvs": [int(r.mvs) for r in res.solves],
                      "relres_true_max": max(float(r.relres_true) for r in res.solves)}))


def small_config_line(M, torch, dev):
    """The small configuration (2D 32 x 32, 10 systems) end to end on the GPU
    and on the oracle, both the whole sequence."""
    from paper_1604_06043_gb300 import problems as pb
    w = pb.WORKLOADS["convdiff2d_32"]
    A = w.matrix()
    f = torch.tensor(w.f(), device=dev)
    out = {"workload": f"convdiff2d_32: 2D convection-diffusion, 5-point FD on a 32x32 grid (N={A.n}), "
                       f"beta={tuple(w.beta)}, tau={w.tau}, {w.steps} systems, M({w.s})stab({w.ell}), fetch once"}
    for rep in range(2):            # the first pass warms the module and the graphs' code up
        S = M.Solver(A, w.s, w.ell, w.p_raw(), device=dev, replace_every=w.replace_every)
        x = torch.tensor(w.x0(), device=dev)
        b = torch.empty_like(x)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        mv = run_sequence(M, torch, S, f, x, b, w.tau, w.tol, w.steps)
        e1.record()
        torch.cuda.synchronize()
        S.close()
    out["gpu_ms_per_system"] = round(e0.elapsed_time(e1) / w.steps, 4)
    out["gpu_mvs"] = [t["mvs"] for t in mv]
    env = dict(os.environ)
    for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS", "NUMEXPR_NUM_THREADS"):
        env[v] = "1"
    cmd = [sys.executable, os.path.abspath(__file__), "--cpu-full-small"]
    r = subprocess.run(cmd, capture_output=True, text=True, env=env, timeout=600)
    if r.returncode == 0:
        o = json.loads(r.stdout.strip().splitlines()[-1])
        out["oracle_ms_per_system"] = round(1e3 * o["seconds"] / w.steps, 3)
        out["oracle_mvs"] = o["mvs"]
        out["oracle_cores"] = 1
    else:
        out["oracle_error"] = r.stderr[-300:]
    return out


def run_cpu_sample(args, level_steps, k0=0, single_thread=True):
    """The oracle worker in a subprocess; single_thread pins every BLAS/OpenMP
    pool to one thread, else the pools use all the cores the process may run on."""
    env = dict(os.environ)
    for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS", "NUMEXPR_NUM_THREADS"):
        if single_thread:
            env[v] = "1"
        else:
            env.pop(v, None)
    cmd = [sys.executable, os.path.abspath(__file__), "--cpu-worker", "--workload", args.workload,
           "--cpu-level-steps", str(level_steps), "--cpu-k0", str(k0)]
    out = subprocess.run(cmd, capture_output=True, text=True, env=env, timeout=1800)
    if out.returncode != 0:
        raise RuntimeError(out.stderr[-2000:])
    return json.loads(out.stdout.strip().splitlines()[-1])


def reference_arm(args):
    """--impl reference: the oracle on the host cores, same metric and unit.
    Each step is one level step of Algorithm 1 (k cycling through 0..l-1);
    ms/system = mean level-step time x l x cycles per system + the products
    for r0 and the true residuals, the cycles per system taken from the
    oracle's own committed record of the same systems."""
    rank, world, _ = dist_env()
    if rank != 0:
        return
    from paper_1604_06043_gb300 import problems as pb
    w = pb.WORKLOADS[args.workload]
    nnz = w.matrix().nnz
    g = golden_cycles(args.warmup + 1, args.steps, w.name)
    if g is None:
        print(json.dumps({"impl": "reference", "unavailable": f"no committed oracle record of the cycles per system "
                                                              f"of {w.name} to scale the level steps by"}), flush=True)
        return
    res = run_cpu_sample(args, args.warmup + args.steps)
    timed = res["level_step_s"][args.warmup:]
    cyc = g[0]
    em = extra_mvs(w, cyc)
    ms = statistics.mean(timed) * 1e3 * w.ell * cyc + em * res["mv_s"] * 1e3
    sample = (f"{len(timed)} level steps of Algorithm 1 (s={w.s}, l={w.ell}) of the FP64 oracle on system 1 of "
              f"the {w.name} sequence, scaled by {cyc:.2f} cycles/system (oracle record, systems "
              f"{args.warmup + 1}..{args.warmup + args.steps}) + {em:.2f} MVs (r0 and true residuals)")
    line = {"impl": "reference", "metric": METRIC, "value": ms, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": statistics.mean(timed) * 1e3,
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded generators; the paper's ocean data is not available)",
            "config": workload_config(w, w.n, nnz, args.warmup, args.steps, "fp64", world),
            "cpu_baseline": {"value": ms, "unit": UNIT, "cores": res["threads"], "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": ms, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# the GPU arm
# ---------------------------------------------------------------------------

def learned_guess_variants(M, torch, A, w, dev, f, train_steps=20, apply_steps=80, iters=300, batch=8, lr=2e-3):
    """The learned initial guess on the 100-step sequence: the plain FP64
    solver produces the pairs of systems 1..train_steps, the CNN is trained on
    them with the library's own kernels, and systems train_steps+1 ..
    train_steps+apply_steps are solved from the same state with x0 from
    (plain) x^(i); (rule) x^(i) + network correction, kept only if its
    residual is smaller, else x^(i); (extrap) the residual-minimising point of
    x^(i) + span{x^(i) - x^(i-1)}; (net) of x^(i) + span{network correction};
    (net_extrap) of x^(i) + span{both}; FP64 and FP32-inner solvers.  Products
    with A count the selection's (r0 for the network, 1 + m for the span, 2 for
    the rule)."""
    from paper_1604_06043_gb300 import problems as pb
    import numpy as np
    S = M.Solver(A, w.s, w.ell, w.p_raw(), device=dev, replace_every=w.replace_every)
    x = torch.tensor(w.x0(), device=dev)
    b = torch.empty_like(x)
    r0 = torch.empty_like(x)
    nrm = torch.zeros(2, dtype=torch.float64, device=dev)
    D = min(32, w.shape[0])
    net = M.CNN(w.shape, pb.cnn_init_params(), max_pairs=train_steps, max_batch=batch, crop=D, device=dev)
    for _ in range(train_steps):
        S.op_axpby(1.0 / w.tau, x, 1.0, f, b)
        xp = x.clone()
        S.op_residual(b, x, r0, nrm)
        S.solve(b, x, w.tol)
        net.add_pair(r0, xp, x)
    S.close()
    net.fit_scales()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    hist = net.train(pb.cnn_crop_batches(train_steps, w.shape, D, batch, iters), batch, D, lr)
    torch.cuda.synchronize()
    out = {"train": {"pairs": train_steps, "iters": iters, "batch": batch, "crop": D, "loss": "mse",
                     "seconds": round(time.perf_counter() - t0, 3), "loss_first": float(np.mean(hist[:5])),
                     "loss_last": float(np.mean(hist[-20:]))},
           "systems": f"{train_steps + 1}..{train_steps + apply_steps}"}

    def run(precision, mode):
        opts = FP32_INNER_OPTS(M) if precision == M.PREC_FP32_INNER else {}
        V = M.Solver(A, w.s, w.ell, w.p_raw(), device=dev, replace_every=w.replace_every, **opts)
        xs = torch.tensor(w.x0(), device=dev)
        xprev = torch.empty_like(xs)
        for _ in range(train_steps):             # the same history (and recycle store) as the plain run
            xprev.copy_(xs)
            V.op_axpby(1.0 / w.tau, xs, 1.0, f, b)
            V.solve(b, xs, w.tol, check=False)
        xg = torch.empty_like(xs)
        dirs = torch.empty((2, A.n), dtype=torch.float64, device=dev)
        mv, used, red, fails, worst = [], 0, [], 0, 0.0
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record()
        for _ in range(apply_steps):
            V.op_axpby(1.0 / w.tau, xs, 1.0, f, b)
            extra = 0
            if mode == "rule":
                V.op_residual(b, xs, r0, nrm)
                net.infer(r0, xs, dirs[0])
                u = V.select_guess(b, xs, dirs[0], xg)
                extra = 3
            elif mode != "plain":
                m = 0
                if mode in ("net", "net_extrap"):
                    V.op_residual(b, xs, r0, nrm)
                    net.infer(r0, xs, dirs[m])
                    m += 1
                    extra += 1
                if mode in ("extrap", "net_extrap"):
                    torch.sub(xs, xprev, out=dirs[m])
                    m += 1
                u, a, rr = V.select_guess_span(b, xs, dirs[:m], xg)
                red.append(rr)
                extra += 1 + m
            if mode != "plain":
                used += int(u)
                xprev.copy_(xs)
                xs.copy_(xg)
            else:
                xprev.copy_(xs)
            st = V.solve(b, xs, w.tol, check=False)
            fails += int(st.status != 0)
            worst = max(worst, st.relres_true)
            mv.append(st.mvs + extra)
        e1.record()
        torch.cuda.synchronize()
        V.close()
        d = {"ms_per_system": round(e0.elapsed_time(e1) / apply_steps, 3),
             "mvs_per_system": round(float(np.mean(mv)), 2), "failed_solves": fails, "relres_true_max": worst}
        if mode != "plain":
            d["guess_kept"] = used
            d["fallback_rate"] = round(1.0 - used / apply_steps, 3)
        if red:
            d["start_residual_ratio_mean"] = round(float(np.mean(red)), 4)
        return d

    for prec, tag, modes in ((M.PREC_FP64, "fp64", ("plain", "rule", "extrap", "net", "net_extrap")),
                             (M.PREC_FP32_INNER, "fp32_inner", ("plain", "extrap", "net_extrap"))):
        base = None
        for mode in modes:
            d = run(prec, mode)
            if mode == "plain":
                base = d
            else:
                d["mvs_saved_per_system"] = round(base["mvs_per_system"] - d["mvs_per_system"], 2)
                d["ms_saved_per_system"] = round(base["ms_per_system"] - d["ms_per_system"], 3)
            out[f"{tag}_{mode}"] = d
    # what the trained network gains over the method without it (the same
    # selection with and without the network's direction)
    out["network_gain_mvs_per_system"] = {
        "fp64_over_plain": out["fp64_net"]["mvs_saved_per_system"],
        "fp64_over_extrapolation": round(out["fp64_extrap"]["mvs_per_system"] - out["fp64_net_extrap"]["mvs_per_system"], 2),
        "fp32_inner_over_extrapolation": round(out["fp32_inner_extrap"]["mvs_per_system"]
                                               - out["fp32_inner_net_extrap"]["mvs_per_system"], 2)}
    net.close()
    return out


def ilu_report(V, A, tv, create_ms):
    """The ILU(0) split-preconditioned variant: level schedules, the time of
    one triangular sweep and what bounds it.  A sweep reads, per row, its
    strict lower (or upper) entries (8-byte value + 4-byte column), the row
    pointer, diagonal position and level-order index (4 bytes each), the
    right-hand side and writes the solution (8 bytes each); with the diagonal
    for the upper sweep: about 12 nnz/2 + 28 n bytes (nnz/2: half of the
    off-diagonal entries on each side)."""
    info = V.op_ilu_levels()
    t_ms = sum(t["t_ms"]["precond"] for t in tv)
    n_l = sum(t["n_launch"]["precond"] for t in tv)
    off = A.nnz - A.n
    sweep_bytes = 12 * off / 2 + 28 * A.n
    us = t_ms / max(1, n_l) * 1e3
    return {"create_ms": round(create_ms, 1),
            "levels_lower_upper": [info[0], info[1]], "widest_level": [info[2], info[3]],
            "sweep_blocks": [info[4], info[5]],
            "precond_launches_per_system": round(n_l / max(1, len(tv)), 1),
            "precond_ms_per_system": round(t_ms / max(1, len(tv)), 3),
            "sweep_us": round(us, 2), "us_per_level": round(us / max(1, (info[0] + info[1]) / 2), 3),
            "sweep_alg_bytes": int(sweep_bytes),
            "sweep_GBps": round(sweep_bytes / (us * 1e-6) / 1e9, 1) if us > 0 else None,
            "relres_orig_max": max(t["relres_orig"] for t in tv),
            "note": "pipelined over row chunks (one per SM, levels in order inside a chunk, block barriers "
                    "between them, waits only on other chunks' values); bound by one store-to-load trip per "
                    "level (3n - 2 levels for a 7-point stencil), not by HBM"}



# bytes per voxel that the four convolutions of one inference read and write:
# the half-major bf16 input (16 bytes per voxel and channel half) and output
# (bf16 halves, or FP32 for the one-channel last layer)
CNN_LAYER_BYTES = [16 * 1 + 32, 32 + 32, 32 + 32, 32 + 4]


def cnn_roofline(n, inf_ms, peaks):
    """The CNN inference against both of its roofs: useful convolution FLOPs
    (2 n ci co 27 per layer) over the measured bf16 burst rate, and the
    convolutions' algorithmic bytes over the measured HBM bandwidth."""
    fl = sum(2 * n * ci * co * 27 for ci, co in ((2, 16), (16, 16), (16, 16), (16, 1)))
    by = n * sum(CNN_LAYER_BYTES)
    t = inf_ms * 1e-3
    tf_peak = float(peaks.get("bf16_tflops", 1900.0))
    hbm_peak = float(peaks.get("hbm_gbs", 6800.0))
    src = "measured" if "bf16_tflops" in peaks and "hbm_gbs" in peaks else "fallback"
    return {"tensor": {"achieved": round(fl / t / 1e12, 2), "peak": tf_peak, "unit": "TFLOP/s",
                       "frac": round(fl / t / 1e12 / tf_peak, 4), "flops": fl},
            "hbm": {"achieved": round(by / t / 1e9, 1), "peak": hbm_peak, "unit": "GB/s",
                    "frac": round(by / t / 1e9 / hbm_peak, 4), "bytes": by},
            "peak_source": src + " (MEASURED_PEAKS.json bf16_tflops, hbm_gbs)",
            "note": "whole four-layer inference; per layer the tensor-core MMA count at N = 16 binds it"}


def cnn_bench(args):
    """The learned-guess network alone on the 128^3 grid: inference (2 -> 16
    -> 16 -> 16 -> 1, 3x3x3; the two 16 -> 16 layers on the tensor cores) and
    training iterations (8 crops of 32^3, forward + backward + Adam), synthetic
    residual and solution fields, CUDA events around K calls after W."""
    import numpy as np
    import torch
    from paper_1604_06043_gb300 import build, msstab as M, problems as pb
    build.build()
    w = pb.WORKLOADS[args.workload]
    n = w.n
    dev = "cuda:0"
    W, K = max(3, args.warmup), args.steps
    net = M.CNN(w.shape, pb.cnn_init_params(), max_pairs=2, max_batch=8, crop=32, device=dev)
    g = torch.Generator(device=dev).manual_seed(pb.SEED_CNN)
    r0 = torch.randn(n, dtype=torch.float64, device=dev, generator=g)
    xp = torch.randn(n, dtype=torch.float64, device=dev, generator=g)
    out = torch.empty_like(r0)
    net.add_pair(r0, xp, xp + 1e-2 * r0)
    net.add_pair(xp, r0, r0 + 1e-2 * xp)
    net.fit_scales()
    for _ in range(W):
        net.infer(r0, xp, out)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(K):
        net.infer(r0, xp, out)
    e1.record()
    torch.cuda.synchronize()
    inf_ms = e0.elapsed_time(e1) / K
    batches = pb.cnn_crop_batches(2, w.shape, 32, 8, W + K)
    net.train(batches[:8 * W], 8, 32, 1e-3)
    torch.cuda.synchronize()
    e0.record()
    net.train(batches[8 * W:], 8, 32, 1e-3)
    e1.record()
    torch.cuda.synchronize()
    tr_ms = e0.elapsed_time(e1) / K
    taps = 27
    fl = [2 * n * ci * co * taps for ci, co in ((2, 16), (16, 16), (16, 16), (16, 1))]
    line = {"metric": "learned-guess CNN inference on the full grid", "value": round(inf_ms, 4), "unit": "ms",
            "higher_is_better": False, "n_gpus": 1, "steps": K, "warmup": W, "dtype": "bf16 (fp32 accumulation)",
            "data": "synthetic", "config": {"workload": w.name, "grid": list(w.shape),
                                            "layers": "2->16->16->16->1, 3x3x3, GELU"},
            "inference_tflops": round(sum(fl) / (inf_ms * 1e-3) / 1e12, 2),
            "tensor_core_layer_gflop": [round(fl[1] / 1e9, 2), round(fl[2] / 1e9, 2)],
            "train_iter_ms": round(tr_ms, 4), "train_batch": "8 crops of 32^3"}
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    line["roofline"] = cnn_roofline(n, inf_ms, peaks)
    print(json.dumps(line), flush=True)


def run_sequence(M, torch, S, f, x, b, tau, tol, count, collect=None, check=True):
    out = []
    for _ in range(count):
        S.op_axpby(1.0 / tau, x, 1.0, f, b)
        st = S.solve(b, x, tol, check=check)
        out.append(st.as_dict())
        if collect is not None:
            collect.append(x.clone())
    return out


def main(argv=None):
    args = parse_args(argv)
    if args.cpu_worker:
        cpu_worker(args)
        return
    if args.cpu_full_small:
        cpu_full_small(args)
        return
    if args.impl == "reference":
        reference_arm(args)
        return
    if args.cnn:
        cnn_bench(args)
        return

    import numpy as np
    import torch
    rank, world, local = dist_env()
    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = f"cuda:{local}" if world > 1 else "cuda:0"
    torch.cuda.set_device(dev)

    from paper_1604_06043_gb300 import build, msstab as M, problems as pb
    if rank == 0:
        build.build()
    if dist is not None:
        dist.barrier()
    w = pb.WORKLOADS[args.workload]
    A = w.matrix()
    f_np, x0_np = w.f(), w.x0()
    K, W = args.steps, args.warmup

    form_opts = {"fp64": {}, "fp32_inner": FP32_INNER_OPTS(M), "fp32_inner_recycled": FP32_INNER_RECYCLED_OPTS(M),
                 "idrstab": dict(fetch_policy=M.FETCH_NEVER), "ilu0": dict(precond=M.PRECOND_ILU0)}[args.form]
    # the timed run replays each cycle as a CUDA graph; per-launch event
    # timing (which launches one by one) runs in a second pass over the same
    # systems for the per-kernel roofline
    S = M.Solver(A, w.s, w.ell, w.p_raw(), device=dev, replace_every=w.replace_every, **form_opts)
    stream = torch.cuda.current_stream()
    f = torch.tensor(f_np, device=dev)
    x = torch.tensor(x0_np, device=dev)
    b = torch.empty_like(x)
    warm = run_sequence(M, torch, S, f, x, b, w.tau, w.tol, W)
    xW = x.clone()
    uuid = None
    try:
        uuid = "GPU-" + str(torch.cuda.get_device_properties(dev).uuid)
    except Exception:
        pass
    clocks = Clocks(uuid)
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    timed = run_sequence(M, torch, S, f, x, b, w.tau, w.tol, K)
    e1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    if dist is not None:
        dist.barrier()
    elapsed = e0.elapsed_time(e1)
    T, value = aggregate(elapsed, K, world, dist)

    mvs = [t["mvs"] for t in timed]
    launches = sum(t["launches"] for t in timed) + K          # + the right-hand-side launches

    # kernel-timing pass: a fresh handle, the same warm-up and the same K
    # systems, every launch bracketed by CUDA events on the handle's stream
    ST = M.Solver(A, w.s, w.ell, w.p_raw(), device=dev, kernel_timing=1, replace_every=w.replace_every,
                  **form_opts)
    xt = torch.tensor(x0_np, device=dev)
    run_sequence(M, torch, ST, f, xt, b, w.tau, w.tol, W)
    torch.cuda.synchronize()
    kt0 = torch.cuda.Event(enable_timing=True)
    kt1 = torch.cuda.Event(enable_timing=True)
    kt0.record(stream)
    ktimed = run_sequence(M, torch, ST, f, xt, b, w.tau, w.tol, K)
    kt1.record(stream)
    torch.cuda.synchronize()
    ST.close()
    cycles = sum(t["cycles"] for t in ktimed)
    fam_ms = {f_: sum(t["t_ms"][f_] for t in ktimed) for f_ in FAMILIES}
    fam_n = {f_: sum(t["n_launch"][f_] for t in ktimed) for f_ in FAMILIES}
    replaced = sum(t["cycles"] for t in ktimed) if w.replace_every == 1 else \
        sum(t["cycles"] // w.replace_every for t in ktimed) if w.replace_every > 1 else 0
    if args.form.startswith("fp32_inner"):     # inner cycles of degree 1 on FP32 vectors dominate the launches
        model, spmv_b = family_model(A, w.s, 1, cycles, K, 0, vb=4)
    else:
        model, spmv_b = family_model(A, w.s, w.ell, cycles, K, replaced)
    if args.form == "ilu0":
        # one triangular sweep: the rows' dependencies (value + column), row
        # pointer, diagonal position and position index, right-hand side and
        # solution once (the U x products of each solve are counted with them)
        model["precond"] = dict(launches=fam_n.get("precond", 0), bytes=12 * (A.nnz - A.n) / 2 + 28 * A.n,
                                flops=float(A.nnz - A.n))
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    hbm_peak = float(peaks.get("hbm_gbs", 6800.0))
    peak_src = "measured" if "hbm_gbs" in peaks else "fallback"
    kernels = {}
    for fam, mod in model.items():
        if fam_n.get(fam, 0) == 0:
            continue
        avg_s = fam_ms[fam] / fam_n[fam] / 1e3
        gbs = mod["bytes"] / avg_s / 1e9
        tf = mod["flops"] / avg_s / 1e12
        kernels[fam] = {"launches": fam_n[fam], "total_ms": round(fam_ms[fam], 3),
                        "avg_us": round(avg_s * 1e6, 2), "alg_bytes_per_launch": int(mod["bytes"]),
                        "GBps": round(gbs, 1), "hbm_frac": round(gbs / hbm_peak, 3),
                        "fp64_tflops": round(tf, 3), "fp64_frac_nominal": round(tf / FP64_NOMINAL_TFLOPS, 3)}
    fp32_form = args.form.startswith("fp32_inner")
    if fp32_form:
        # the FP32 inner kernels' arithmetic is FP32: their ALU bound is the FP32 rate
        for k_ in kernels:
            kernels[k_]["fp32_tflops"] = kernels[k_].pop("fp64_tflops")
            kernels[k_]["fp32_frac_nominal"] = round(kernels[k_]["fp32_tflops"] / FP32_NOMINAL_TFLOPS, 3)
            kernels[k_].pop("fp64_frac_nominal")
    dom = max(kernels, key=lambda k_: kernels[k_]["total_ms"])
    kd = kernels[dom]
    share = round(fam_ms[dom] / max(1e-9, sum(fam_ms.values())), 3)
    if fp32_form:
        roofline = {"kernel": dom, "bound": "hbm", "achieved": kd["GBps"], "peak": hbm_peak, "unit": "GB/s",
                    "frac": kd["hbm_frac"], "traffic": NCU_TRAFFIC.get((args.workload, args.form, dom)),
                    "peak_source": f"{peak_src} (MEASURED_PEAKS.json hbm_gbs)",
                    "fp32_frac_of_nominal": kd["fp32_frac_nominal"], "share_of_step": share}
    elif kd["fp64_frac_nominal"] > kd["hbm_frac"]:
        # FP64 FMA throughput, not HBM, binds this kernel on GB300
        roofline = {"kernel": dom, "bound": "alu", "achieved": kd["fp64_tflops"], "peak": FP64_NOMINAL_TFLOPS,
                    "unit": "TFLOP/s (FP64)", "frac": kd["fp64_frac_nominal"],
                    "traffic": NCU_TRAFFIC.get((args.workload, args.form, dom)),
                    "peak_source": "nominal GB300 FP64 rate (no measured FP64 peak in MEASURED_PEAKS.json)",
                    "hbm": {"achieved": kd["GBps"], "peak": hbm_peak, "unit": "GB/s", "frac": kd["hbm_frac"]},
                    "share_of_step": share}
    else:
        roofline = {"kernel": dom, "bound": "hbm", "achieved": kd["GBps"], "peak": hbm_peak, "unit": "GB/s",
                    "frac": kd["hbm_frac"], "traffic": NCU_TRAFFIC.get((args.workload, args.form, dom)),
                    "peak_source": f"{peak_src} (MEASURED_PEAKS.json hbm_gbs)",
                    "fp64_frac_of_nominal": kd["fp64_frac_nominal"], "share_of_step": share}

    line = {"metric": METRIC, "value": round(value, 4), "unit": UNIT, "n_gpus": world, "steps": K, "warmup": W,
            "ms_per_step": round(T / K, 4), "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32+f64" if args.form.startswith("fp32_inner") else "f64",
            "data": "synthetic (seeded generators; the paper's ocean data is not available)",
            "config": workload_config(w, A.n, A.nnz, W, K, args.form, world),
            "mvs_per_system": round(statistics.mean(mvs), 2),
            "cycles_per_system": round(sum(t["cycles"] for t in timed) / K, 3),
            # time per cycle: the FP32 inner form's products count is a draw of
            # its rounding (it changes with the FP32 summation order), the time
            # per cycle is not
            "ms_per_cycle": round(T / max(1, sum(t["cycles"] for t in timed)), 4),
            "kernel_timing_pass": {"ms_per_system": round(kt0.elapsed_time(kt1) / K, 4),
                                   "note": "same systems, launches one by one with CUDA events around each "
                                           "(the timed run replays each cycle as a CUDA graph)"},
            "relres_true_max": max(t["relres_true"] for t in timed),
            "system1": {"ms": round(warm[0]["ms"], 3), "mvs": warm[0]["mvs"], "cycles": warm[0]["cycles"]} if warm else None,
            "spmv_GBps": kernels.get("spmv_dot", {}).get("GBps"),
            "gpu_launches": int(launches), "roofline": roofline, "kernels": kernels, "clocks": clk}

    # end to end through the public API with host buffers, on the same systems:
    # a fresh handle, the same warm-up, then the same K systems via msstab_solve_host
    if not args.no_e2e:
        H = M.Solver(A, w.s, w.ell, w.p_raw(), device=dev, replace_every=w.replace_every, **form_opts)
        # the caller's b and x live in pinned host memory (page-locked numpy views)
        xh = torch.empty(A.n, dtype=torch.float64, pin_memory=True).numpy()
        bh = torch.empty(A.n, dtype=torch.float64, pin_memory=True).numpy()
        xh[:] = x0_np
        # each right-hand side b = x/tau + f is formed as the device run forms it
        # (the library's axpby, outside the timed region) and handed over in
        # host memory: the same systems bit for bit, so that the two runs take
        # the same iterations (the products count is a draw of the rounding)
        xd = torch.empty(A.n, dtype=torch.float64, device=dev)
        bd = torch.empty_like(xd)

        def next_rhs():
            xd.copy_(torch.from_numpy(xh))
            H.op_axpby(1.0 / w.tau, xd, 1.0, f, bd)
            bh[:] = bd.cpu().numpy()

        for _ in range(W):
            next_rhs()
            H.solve_host(bh, xh, w.tol)
        wall, e2e_mvs = [], []
        for _ in range(K):
            next_rhs()
            t0 = time.perf_counter()
            st_h = H.solve_host(bh, xh, w.tol)
            wall.append((time.perf_counter() - t0) * 1e3)
            e2e_mvs.append(st_h.mvs)
        H.close()
        line["e2e"] = {"value": round(statistics.mean(wall), 4), "unit": UNIT, "h2d_bytes_per_step": 16 * A.n,
                       "d2h_bytes_per_step": 8 * A.n, "systems": f"{W + 1}..{W + K}",
                       "mvs_per_system": round(statistics.mean(e2e_mvs), 2),
                       "note": "msstab_solve_host per system: b and x0 copied from pinned host memory, x copied back"}
    S.close()

    # the same systems on the same GPU: IDRstab (Arnoldi start per system) and FP32-inner M(s)stab
    if not args.no_variants:
        ref_x = []
        xs = torch.tensor(x0_np, device=dev)
        variants = {}
        p_block = pb.randn_block_partitioned(A.n, w.s, pb.SEED_P)
        todo = (("idrstab_fp64", dict(fetch_policy=M.FETCH_NEVER), None),
                ("fp32_inner_idrstab1_dc", FP32_INNER_OPTS(M), None),
                ("msstab_fp32_inner_recycled", FP32_INNER_RECYCLED_OPTS(M), None),
                ("msstab_fp64_fetch_every", dict(fetch_policy=M.FETCH_EVERY), None),
                ("msstab_fp64_no_orth", dict(orth_recycle=0), None),
                ("msstab_fp64_block_p", {}, p_block),
                ("msstab_fp64_fetch_slope", dict(fetch_policy=M.FETCH_SLOPE), None),
                ("msstab_fp64_fetch_probe", dict(fetch_policy=M.FETCH_PROBE), None),
                ("msstab_fp64_ilu0", dict(precond=M.PRECOND_ILU0, kernel_timing=1), None),
                ("idrstab_fp64_ilu0", dict(precond=M.PRECOND_ILU0, kernel_timing=1, fetch_policy=M.FETCH_NEVER),
                 None))
        only = set(args.variants.split(",")) if args.variants else None
        for name, opts, praw in todo:
          if only is not None and name not in only:
              continue
          try:
            c0 = time.perf_counter()
            V = M.Solver(A, w.s, w.ell, w.p_raw() if praw is None else praw, device=dev,
                         replace_every=w.replace_every, **opts)
            create_ms = (time.perf_counter() - c0) * 1e3
            xv = torch.tensor(x0_np, device=dev)
            wv = run_sequence(M, torch, V, f, xv, b, w.tau, w.tol, W, check=False)
            torch.cuda.synchronize()
            v0 = torch.cuda.Event(enable_timing=True)
            v1 = torch.cuda.Event(enable_timing=True)
            xs_list = []
            v0.record(stream)
            tv = run_sequence(M, torch, V, f, xv, b, w.tau, w.tol, K,
                              collect=xs_list if "fp32_inner" in name else None, check=False)
            v1.record(stream)
            torch.cuda.synchronize()
            variants[name] = {"ms_per_system": round(v0.elapsed_time(v1) / K, 4),
                              "mvs_per_system": round(statistics.mean(t["mvs"] for t in tv), 2),
                              "relres_true_max": max(t["relres_true"] for t in tv),
                              "failed_solves": sum(1 for t in tv if t["status"] != 0)}
            if "fp32_inner" in name:
                variants[name]["mvs_fp32_per_system"] = round(statistics.mean(t["mvs_fp32"] for t in tv), 2)
                variants[name]["outer_per_system"] = round(statistics.mean(t["outer"] for t in tv), 2)
                variants[name]["fp64_finishes"] = sum(t["fp64_finish"] for t in tv)
            if "fp32_inner" in name:
                variants[name]["_xs"] = xs_list
            if "fetch_" in name or "no_orth" in name or name == "idrstab_fp64":
                variants[name]["mvs_total"] = int(sum(t["mvs"] for t in tv))
            if praw is not None:
                variants[name]["cut_space"] = "block-partitioned N(0,1), seed 3 (rows (i // 32) mod s)"
            if "ilu0" in name:
                variants[name].update(ilu_report(V, A, tv, create_ms))
            if "fetch_" in name:
                variants[name]["fetched_in_warmup"] = [{"system": i + 1, "cycle": t["fetch_at"], "mvs": t["mvs"]}
                                                       for i, t in enumerate(wv) if t["fetched"]]
                variants[name]["note"] = ("fetching point from the running drop test (slope) or from a probe "
                                          "solve's history (probe); the warm-up systems include the fetch")
            V.close()
          except Exception as e:  # a failing variant is reported, the main line still stands
            variants[name] = {"error": str(e)[-300:]}
        # error of the FP32-inner solutions against the FP64 solutions of the
        # same systems (each FP32 sequence runs on its own solutions; the FP64
        # reference is the main line's handle type from the same x^(0))
        for name in [k for k in variants if "fp32_inner" in k and "_xs" in variants[k]]:
            P64 = M.Solver(A, w.s, w.ell, w.p_raw(), device=dev, replace_every=w.replace_every)
            x64 = torch.tensor(x0_np, device=dev)
            run_sequence(M, torch, P64, f, x64, b, w.tau, w.tol, W)
            errs = []
            for xv32 in variants[name].pop("_xs"):
                P64.op_axpby(1.0 / w.tau, x64, 1.0, f, b)
                P64.solve(b, x64, w.tol)
                errs.append(float(torch.linalg.norm(xv32 - x64) / torch.linalg.norm(x64)))
            P64.close()
            if errs:
                variants[name]["rel_err_vs_fp64_per_system"] = [float("%.3g" % e) for e in errs]
                variants[name]["rel_err_vs_fp64_max"] = max(errs)
        if only is None or "learned_guess" in only:
            try:
                wl = pb.WORKLOADS["convdiff3d_128_long"] if args.workload == "convdiff3d_128" else w
                variants["learned_guess"] = learned_guess_variants(M, torch, A, wl, dev, f)
            except Exception as e:
                variants["learned_guess"] = {"error": str(e)[-300:]}
        line["variants"] = variants

    # the oracle sample below is Algorithm 1 without a preconditioner
    if rank == 0 and world == 1 and not args.no_cpu_baseline and args.form != "ilu0":
        try:
            res = run_cpu_sample(args, 4)
            cyc = cycles / K
            em = extra_mvs(w, cyc)
            ms = statistics.mean(res["level_step_s"]) * 1e3 * w.ell * cyc + em * res["mv_s"] * 1e3
            line["cpu_baseline"] = {"value": round(ms, 1), "unit": UNIT, "cores": res["threads"], "kind": "oracle",
                                    "sample": f"one cycle (4 level steps, 36 MVs) of Algorithm 1 of the FP64 oracle on "
                                              f"system 1 of the {w.name} sequence, scaled by the timed run's "
                                              f"{cyc:.2f} cycles/system, + {em:.2f} MVs (r0 and true residuals)"}
            try:   # the same sample with the BLAS pools on every core
                ra = run_cpu_sample(args, 4, single_thread=False)
                msa = statistics.mean(ra["level_step_s"]) * 1e3 * w.ell * cyc + em * ra["mv_s"] * 1e3
                line["cpu_baseline"]["all_threads"] = {"value": round(msa, 1), "cores": ra["threads"]}
            except Exception as e:
                line["cpu_baseline"]["all_threads"] = {"value": None, "note": str(e)[-200:]}
        except Exception as e:  # the baseline is reported, not required
            line["cpu_baseline"] = {"value": None, "unit": UNIT, "cores": 1, "kind": "oracle",
                                    "sample": f"failed: {str(e)[-200:]}"}
        try:   # the small configuration, whole sequence on both sides
            line["small_config_end_to_end"] = small_config_line(M, torch, dev)
        except Exception as e:
            line["small_config_end_to_end"] = {"error": str(e)[-300:]}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()

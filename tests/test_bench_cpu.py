"""Host logic of bench.py that needs no GPU: the L2 statement of the config,
the oracle record lookup and the reference arm's line when no record of the
workload exists."""

import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench                                    # noqa: E402
from paper_1604_06043_gb300 import problems as pb   # noqa: E402


def test_l2_statement_follows_the_footprint():
    big = pb.WORKLOADS["convdiff3d_128"]
    small = pb.WORKLOADS["convdiff3d_24"]
    # 128^3: 175 MB of matrix alone, above the 129 MB L2
    assert bench.l2_note(big, 2097152, 14581760).startswith("inputs larger than L2")
    assert bench.l2_note(small, 13824, 93312).startswith("inputs fit in L2")


def test_oracle_record_is_used_only_for_its_own_workload():
    g = bench.golden_cycles(4, 20, "convdiff3d_128")
    assert g is not None and g[0] > 0 and g[1] > 0 and g[2] == 20
    assert bench.golden_cycles(4, 20, "convdiff3d_24") is None


def test_reference_arm_without_a_record_reports_unavailable():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "1", "--workload", "convdiff3d_24"],
                         capture_output=True, text=True, timeout=300, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    line = json.loads(out.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and "unavailable" in line


def test_cnn_roofline_fractions():
    # 128^3 voxels in 0.46 ms: the FLOPs and bytes follow from the layer shapes
    n = 128 ** 3
    r = bench.cnn_roofline(n, 0.46, {"bf16_tflops": 2000.0, "hbm_gbs": 8000.0})
    fl = 2 * n * 27 * (2 * 16 + 16 * 16 + 16 * 16 + 16 * 1)
    assert r["tensor"]["flops"] == fl
    assert abs(r["tensor"]["achieved"] - fl / 0.46e-3 / 1e12) < 0.01
    assert abs(r["tensor"]["frac"] - r["tensor"]["achieved"] / 2000.0) < 1e-4
    assert r["hbm"]["bytes"] == n * (48 + 64 + 64 + 36)
    assert abs(r["hbm"]["frac"] - r["hbm"]["achieved"] / 8000.0) < 1e-4
    assert r["peak_source"].startswith("measured")
    assert bench.cnn_roofline(n, 0.46, {})["peak_source"].startswith("fallback")

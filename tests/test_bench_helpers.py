"""Host logic of the benchmark (no GPU): metric naming, workload description and the
algorithmic-byte model the roofline fraction is computed from."""
import os
import sys

import numpy as np

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402
from synth.problems import Workload  # noqa: E402


def test_metric_and_workload_names():
    assert bench.fmt_tol(1e-8) == "1e-8" and bench.fmt_tol(1e-4) == "1e-4"
    assert bench.method_name("pcg") == "POD-2G-PCG"
    d = bench.workload_desc(Workload("q4_512"), 64, 1e-8)
    assert "526,338 dofs" in d and "512x512" in d and "batch 64" in d and "tol 1e-8" in d


def test_kernel_bytes_model():
    wl = Workload("q4_512")
    P = wl.problem
    kb = bench.kernel_bytes(wl, 24, lane_iters=64, launches=1, G=1216, Bp=64)
    vals = P.nnzb * 4 * 4
    # one launch with 64 active instances: values + p + q (double-float) + pattern
    assert kb["k_spmv"] == 64 * (vals + 16 * P.n) + P.nnzb * 4 + (P.n_nodes + 1) * 4
    assert kb["k_upd"] == 64 * 48 * P.n
    assert kb["k_restrict"] == 64 * 4 * P.n + P.n * 24 * 4
    # the element form replaces the per-instance values by one coefficient per element
    ke = bench.kernel_bytes(wl, 24, 64, 1, 1216, 64, elements=True)
    assert ke["k_spmv"] - kb["k_spmv"] == 64 * (P.n_el * 4 - vals) + P.nnzb * 8 + P.n_nodes * 32
    # Gauss-Seidel groups: two value passes before the coarse correction, one after
    ks = bench.kernel_bytes(wl, 24, 64, 1, 1216, 64, sgs=True)
    assert ks["k_smooth1"] > 1.9 * kb["k_smooth1"] and ks["k_prol"] < kb["k_prol"]


def test_measured_peak_fallback(tmp_path, monkeypatch):
    peaks, kind = bench.measured_peaks()
    assert kind in ("measured", "fallback") and peaks["hbm_gbs"] > 1000


def test_oracle_timing_cli_reports_iterations():
    """The CPU-baseline leg runs the oracle in a fresh single-threaded process and reads one JSON line."""
    import json
    import subprocess
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1")
    for method, smoother in (("pcg", "jacobi"), ("stationary", "sgs")):
        r = subprocess.run([sys.executable, "-m", "oracle.timing", "q1_16", "0", "full", "1e-8", method, smoother],
                           cwd=root, env=env, capture_output=True, text=True, timeout=300)
        assert r.returncode == 0, r.stderr[-500:]
        out = json.loads(r.stdout.strip().splitlines()[-1])
        assert out["status"] == 0 and out["relres"] <= 1e-8 and out["iterations"] > 0
        assert out["seconds_per_iteration"] > 0


def test_reference_arm_line_matches_the_gpu_arm_contract():
    """`bench.py --impl reference` times the oracle on the same workload and prints the GPU arm's
    metric, with impl, cpu_baseline and e2e keys (small workload, CPU only)."""
    import json
    import subprocess
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--workload", "q1_16", "--steps", "1",
                        "--warmup", "1"], cwd=root, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-800:]
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["metric"] == "solves/s at rel. residual 1e-8 (batched POD-2G-PCG)"
    assert line["unit"] == "solves/s" and line["higher_is_better"] is True and line["value"] > 0
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["value"] == line["value"]
    assert line["e2e"] == {"value": line["value"], "unit": "solves/s", "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}
    assert "225 dofs" in line["config"]["workload"]

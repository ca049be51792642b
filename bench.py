#!/usr/bin/env python
"""Benchmark: batched mixed-precision POD-2G-PCG on one GB300.

Metric: solves/s at relative residual 1e-8 (arXiv 2207.02543, Algorithm 3 with
the two-grid cycle of Algorithm 2, P = Phi_r). Default workload: the largest
single-GPU configuration, 3D linear elasticity with Hex8 elements on a 128^3
cube (6,440,067 unknowns, 57,066,625 3 x 3 blocks, z = 0 face clamped, uniform
load on the top face), lognormal Young's modulus from a 16-term KL field (CoV
0.4), POD basis k = 40 from 400 snapshots, a batch of 4 parameter instances under
an HBM admission budget, double-float outer PCG with an FP32 preconditioner and
FP32 Phi. The same line reports batch 1 of that workload, and, as extra keys, the
2D elasticity Q4 512^2 batch-64 and 3D Hex8 64^3 batch-32 (BF16 Phi) workloads.

One step = per-instance set-up of the batch from FP64 values resident in HBM
(FP32 conversion, D^-1, K_c = Phi^T K Phi, Cholesky) + the batched solve of all
instances to 1e-8. The inputs (16 GB of FP64 values for batch 4) are larger than L2.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

N > 1 runs one independent replica per GPU (torchrun; no data-path collective).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "hex8_128"
EXTRAS = "q4_512,hex8_64"
HBM_BUDGET_GB = 40.0   # admission budget of the default workload's context
TOL = 1e-8
MAXIT = 5000


def _env_rank():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("LOCAL_RANK", "0"))


class ClockSampler:
    """nvidia-smi clock / throttle samples while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.samples = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                self.samples.append(parts)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm = [float(s[1]) for s in self.samples if s[1].replace(".", "").isdigit()]
        mx = [float(s[2]) for s in self.samples if s[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for s in self.samples for i in range(4) if s[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.samples)}


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


def kernel_bytes(wl, k_pad, lane_iters, launches, G, Bp, elements=False, sgs=False, kphi=False):
    """Algorithmic HBM bytes per kernel of the batched iteration (values FP32, vectors
    double-float 8 B, s/y/D^-1 FP32 4 B, Phi FP32 read once per launch, col_idx
    once per launch, per-slot scalars and partials negligible). Element operator:
    per slot 4 B per element coefficient instead of the block values, plus the
    8 B block descriptors and the row element lists once per launch."""
    P = wl.problem
    n, nnzb, bs = P.n, P.nnzb, P.bs
    vals = P.n_el * 4 if elements else nnzb * bs * bs * 4
    pat = nnzb * 4 + (P.n_nodes + 1) * 4 + ((nnzb * 8 + P.n_nodes * 8 * 4) if elements else 0)
    phi = n * k_pad * 4
    per_lane = {  # bytes per active instance-iteration
        "k_p": n * (4 + 8 + 8),
        "k_spmv": vals + n * (8 + 8),
        "k_upd": n * (8 * 4 + 8 * 2),
        "k_smooth1": vals + n * (8 + 4 + 4),
        "k_restrict": n * 4,
        "k_coarse": 0,
        "k_prol": n * (8 + 4 + 4),
        "k_post": vals + n * (4 + 8 + 4 + 4),
    }
    shared = {"k_p": 0, "k_spmv": pat, "k_upd": 0, "k_smooth1": pat, "k_restrict": phi,
              "k_coarse": G // 8 * Bp * (k_pad + 2) * 8, "k_prol": phi, "k_post": pat}
    if kphi:  # prolongation and post-smoothing in one pass from K Phi (timed as k_post)
        per_lane["k_prol"] = 0
        per_lane["k_post"] = n * (4 * k_pad + 8 + 4 + 4 + 4)
        shared["k_prol"] = 0
        shared["k_post"] = phi
    if sgs:   # timing groups: forward sweeps + residual; stored y1; backward sweeps + r^T s
        per_lane["k_smooth1"] = 2 * vals + n * (20 + 16)
        per_lane["k_prol"] = n * (4 + 4)
        per_lane["k_post"] = vals + n * (20 + 16)
        shared["k_smooth1"] = 2 * pat
        shared["k_post"] = pat
    return {name: per_lane[name] * lane_iters + shared[name] * launches for name in per_lane}


# DRAM bytes (read + write) per launch from one ncu capture of these kernels on the
# workload named, keyed by (workload, batch, operator, row-kernel form); valid only for the
# kernel versions that capture measured (the per-thread row kernels, form 0, for q4_512).
NCU_TRAFFIC = {
    ("q4_512", 64, "assembled", 0): {"k_spmv": 3156.2e6, "k_smooth1": 2964.0e6, "k_post": 3100.1e6,
                                     "k_upd": 1569.2e6, "k_restrict": 185.5e6, "k_prol": 568.5e6, "k_p": 615.7e6,
                                     "k_coarse": 1.0e6},
    # staged SpMV and pre-smoothing captured on Hex8 64^3 with 4 slots, scaled to Hex8 128^3 by the
    # stored blocks (57,066,625 / 7,189,057): profiles/traffic_k_rows_ws_hex8_b4.md
    ("hex8_128", 4, "assembled", 7): {"k_spmv": 8.958e9, "k_smooth1": 9.036e9},
    ("hex8_128", 4, "assembled", 3): {"k_spmv": 8.958e9, "k_smooth1": 9.036e9},
}


NCU_SOURCE = {("q4_512", 64, "assembled", 0): "profiles/launches_q4_512_b64.md",
              ("hex8_128", 4, "assembled", 7): "profiles/traffic_k_rows_ws_hex8_b4.md",
              ("hex8_128", 4, "assembled", 3): "profiles/traffic_k_rows_ws_hex8_b4.md"}


def run_oracle(mode, inst, timeout=900, workload=WORKLOAD, tol=TOL, method="pcg", smoother="jacobi"):
    env = dict(os.environ)
    for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        env[v] = "1"
    r = subprocess.run([sys.executable, "-m", "oracle.timing", workload, str(inst), str(mode), str(tol), method, smoother],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=timeout)
    if r.returncode != 0:
        raise RuntimeError(r.stderr[-2000:])
    return json.loads(r.stdout.strip().splitlines()[-1])


def oracle_pool(workload, workers, sample_iters, warmup, steps, tol=TOL, method="pcg", smoother="jacobi",
                timeout=3600):
    """`workers` single-threaded oracle processes on distinct instances (oracle.timing pool mode)."""
    env = dict(os.environ)
    for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        env[v] = "1"
    cmd = [sys.executable, "-m", "oracle.timing", "pool", workload, str(workers), str(sample_iters), str(warmup),
           str(steps), str(tol), method, smoother]
    r = subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=timeout)
    if r.returncode != 0:
        raise RuntimeError(r.stderr[-2000:])
    return json.loads(r.stdout.strip().splitlines()[-1])


GOLDEN_ITERS = os.path.join(ROOT, "tests", "golden", "oracle_iterations.json")


def oracle_iterations(workload, tol=TOL, method="pcg", smoother="jacobi"):
    """Full-solve iteration counts of the oracle per query instance: from the stored file the
    oracle-only script tests/golden/make_oracle_iterations.py writes, else one full oracle
    solve of instance 0 (cached on disk). Returns ({instance: iterations}, source)."""
    try:
        g = json.load(open(GOLDEN_ITERS))[workload]
        if g["tol"] == tol and g["method"] == method and g["smoother"] == smoother:
            return {int(k): int(v) for k, v in g["iterations"].items()}, "tests/golden/oracle_iterations.json"
    except (OSError, KeyError, ValueError):
        pass
    tag = f"{workload}_{method}_{smoother}_{fmt_tol(tol)}"
    cache = os.path.join(ROOT, "_cache", f"oracle_{tag}_iters.json")
    if os.path.exists(cache):
        full = json.load(open(cache))
    else:
        full = run_oracle("full", 0, timeout=3600, workload=workload, tol=tol, method=method, smoother=smoother)
        os.makedirs(os.path.dirname(cache), exist_ok=True)
        json.dump(full, open(cache, "w"))
    return {0: int(full["iterations"])}, "a full oracle solve of instance 0"


def host_memory_available():
    try:
        for line in open("/proc/meminfo"):
            if line.startswith("MemAvailable:"):
                return int(line.split()[1]) * 1024
    except OSError:
        pass
    return 0


def oracle_workers(wl, limit=None, reserve=16e9):
    """Processes the host can run: one per core, bounded by host memory (an oracle process holds
    its instance's CSR matrix, the basis and K Phi; its set-up peaks near 24 B per stored scalar)."""
    P = wl.problem
    per = 24.0 * P.nnzb * P.bs ** 2 + 24.0 * P.n * wl.spec.k + 2e8
    avail = host_memory_available() - reserve
    cores = os.cpu_count() or 1
    w = cores if avail <= 0 else max(1, min(cores, int(avail // per)))
    return min(w, limit) if limit else w


def cpu_model():
    try:
        for line in subprocess.run(["lscpu"], capture_output=True, text=True, timeout=20).stdout.splitlines():
            if line.startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except Exception:  # noqa: BLE001
        pass
    import platform
    return platform.processor() or platform.machine()


def oracle_rate(pool_out, iters):
    """Solves/s of the pool: worker w finishes a solve every set-up_w + n_w * (seconds per iteration
    of w, mean over the timed steps); n_w = the oracle's own full iteration count for w's instance,
    or the mean of the stored counts where w's instance has none."""
    mean_it = sum(iters.values()) / len(iters)
    rate, used = 0.0, []
    for w in range(pool_out["workers"]):
        per = statistics.mean(step[w] for step in pool_out["seconds_per_iteration"])
        n_w = iters.get(w, mean_it)
        used.append(n_w)
        rate += 1.0 / (pool_out["setup_s"][w] + n_w * per)
    return rate, used


def cpu_baseline_entry(wl, workers, sample_iters, tol, method, smoother, warmup=0, steps=1):
    """The oracle as it stands on the host cores (a bounded sample; see oracle_rate)."""
    out = oracle_pool(wl.spec.name, workers, sample_iters, warmup, steps, tol, method, smoother)
    iters, src = oracle_iterations(wl.spec.name, tol, method, smoother)
    rate, used = oracle_rate(out, iters)
    sample = (f"{workers} single-threaded oracle processes on instances 0..{workers - 1}: each timed its "
              f"set-up (D^-1, K_r, Cholesky; mean {statistics.mean(out['setup_s']):.1f} s) and "
              f"{steps} x {sample_iters} {method_name(method)} iterations, scaled to a full solve by the "
              f"oracle's iteration counts ({src}; {', '.join(f'{n:.0f}' for n in used[:8])}"
              f"{' ...' if len(used) > 8 else ''}); host {cpu_model()}, {os.cpu_count()} cores")
    return {"value": rate, "unit": "solves/s", "cores": workers, "kind": "oracle", "sample": sample,
            "cpu_model": cpu_model()}, out


def fmt_tol(tol: float) -> str:
    return f"{tol:.0e}".replace("e-0", "e-")


def method_name(method: str) -> str:
    return "POD-2G-PCG" if method == "pcg" else "POD-2G stationary"


def workload_desc(wl, batch: int, tol: float) -> str:
    sp, P = wl.spec, wl.problem
    kind = {"q1": f"2D Poisson Q1 {sp.ne}x{sp.ne}, lognormal kappa",
            "q4": f"2D plane-stress Q4 {sp.ne}x{sp.ne}, lognormal E (CoV {sp.cov})",
            "hex8": f"3D elasticity Hex8 {sp.ne}^3, lognormal E (CoV {sp.cov})"}[sp.kind]
    return (f"{kind}: {P.n:,} dofs, {P.bs}x{P.bs} BSR, {sp.m}-term KL, k={sp.k} POD from {sp.n_snap} snapshots "
            f"({sp.phi_dtype} Phi), batch {batch}, tol {fmt_tol(tol)}")


# ----------------------------------------------------------------------------- reference arm (oracle)
def sample_iterations(wl):
    """Oracle iterations per timed step: about 3 GB of single-threaded SpMV traffic (2..25)."""
    P = wl.problem
    per_iter = 3 * 12.0 * P.nnzb * P.bs ** 2
    return max(2, min(25, int(3e9 // per_iter)))


def reference_arm(args):
    """The oracle (FP64, host cores) on the GPU arm's workload, method, relaxation and tolerance:
    one single-threaded process per core (as many as host memory holds), each on a distinct
    instance; per step each times a bounded sample of iterations, and a full solve's time is its
    timed set-up plus the oracle's full iteration count times its seconds per iteration."""
    rank, world, local = _env_rank()
    if rank != 0:
        return 0
    from synth.problems import Workload
    from synth.snapshots import pod_basis
    wl = Workload(args.workload)
    B = args.batch or wl.spec.batch
    tol = args.tol
    pod_basis(wl, device="cuda" if wl.n > 20_000 else None)  # the POD basis, cached on disk for the pool
    workers = oracle_workers(wl, limit=args.oracle_workers or None)
    sample_it = sample_iterations(wl)
    t0 = time.perf_counter()
    cpu, out = cpu_baseline_entry(wl, workers, sample_it, tol, args.method, args.smoother, warmup=args.warmup,
                                  steps=args.steps)
    value = cpu["value"]
    line = {
        "metric": f"solves/s at rel. residual {fmt_tol(tol)} (batched {method_name(args.method)})",
        "value": value, "unit": "solves/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": statistics.mean(out["step_wall_s"]) * 1e3 if out["step_wall_s"] else None,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "impl": "reference",
        "config": {"workload": workload_desc(wl, B, tol), "method": method_name(args.method),
                   "smoother": args.smoother, "batch": B, "n": wl.problem.n, "k": wl.spec.k,
                   "oracle_prepare_s": round(out["prepare_s"], 1), "wall_s": round(time.perf_counter() - t0, 1)},
        "cpu_baseline": cpu,
        "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ----------------------------------------------------------------------------- replicas
def replica_offset(rank: int, batch: int) -> int:
    """First query index of a replica: rank r solves instances [r*batch, (r+1)*batch) (no overlap)."""
    return rank * batch


def max_over_ranks(ms: float, dist=None, device="cuda") -> float:
    """Step time of the whole job: the slowest rank's (a MAX all-reduce; identity on one rank)."""
    if dist is None:
        return ms
    import torch
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(ms_max: float, world: int, batch: int) -> float:
    """Whole-job solves/s: every rank solves `batch` instances per step."""
    return world * batch / (ms_max / 1e3)


# ----------------------------------------------------------------------------- GB300 arm
class WorkloadRun:
    """One workload on this rank: its POD basis, B instances' FP64 inputs resident in HBM, and a
    solver context (optionally under an HBM admission budget)."""

    def __init__(self, args, pkg, name, B, rank=0, hbm_budget=0, autotune=True, surrogate=False):
        import torch
        from synth.problems import Workload
        from synth.snapshots import pod_basis
        self.pkg, self.args = pkg, args
        self.wl = wl = Workload(name)
        P = self.P = wl.problem
        self.B = B
        t0 = time.time()
        self.sur_w = None
        if surrogate or args.x0 == "sur":
            # the surrogate's training data and the solver's basis from one snapshot pass (offline)
            from synth.surrogate import train_surrogate
            self.sur_w = train_surrogate(wl, steps=2000, device="cuda")
        self.Phi = pod_basis(wl, device="cuda")
        self.t_phi = time.time() - t0
        self.xis = wl.query_thetas(B, offset=replica_offset(rank, B))   # distinct instances per rank
        self.elements = args.operator == "elements"
        if self.elements:   # FP64 element coefficients, resident in HBM
            self.vals = torch.from_numpy(np.stack([wl.coef(xi) for xi in self.xis])).cuda()
        else:               # FP64 assembled values, resident in HBM
            self.vals = wl.values_torch(self.xis, device="cuda").reshape(B, -1).contiguous()
        self.b_dev = torch.from_numpy(wl.rhs(B, offset=replica_offset(rank, B))).cuda()
        self.x_dev = torch.empty_like(self.b_dev)
        self.stream = torch.cuda.Stream()
        precision = pkg.MIXED_BF16PHI if wl.spec.phi_dtype == "bf16" else pkg.MIXED_FP32PHI
        self.method = pkg.STATIONARY if args.method == "stationary" else pkg.PCG
        self.smoother = pkg.SMOOTHER_SGS if args.smoother == "sgs" else pkg.SMOOTHER_JACOBI
        el = (dict(conn=P.conn, k_ref=P.Kref, fixed=P.clamped if P.dirichlet == "identity" else None)
              if self.elements else None)
        self.s = pkg.Solver(P.row_ptr, P.col_idx, P.bs, self.Phi, precision=precision, omega=wl.spec.omega,
                            max_batch=B, stream=self.stream.cuda_stream, method=self.method, elements=el,
                            smoother=self.smoother, hbm_budget=int(hbm_budget))
        self.slots = list(range(B))
        self.set_batch = self.s.set_coeffs_batch_dev if self.elements else self.s.set_values_batch_dev
        self.set_one = self.s.set_coeffs if self.elements else self.s.set_values
        self.x0_mode = args.x0
        self.x0_dev = torch.empty_like(self.b_dev) if (args.x0 != "zero" or self.sur_w is not None) else None
        self.sur = None
        if self.sur_w is not None:
            from synth.surrogate import load_scale
            self.sur = pkg.Surrogate(self.sur_w, stream=self.stream.cuda_stream)
            self.scales = np.array([load_scale(wl, b) for b in wl.rhs(B, offset=replica_offset(rank, B))])
        self.tuning = None
        if args.tuning:
            # a given launch shape (e.g. the one an earlier autotuned run reported), no autotuning
            shape = {(k if k in ("rows_kernel", "restrict_rows") else f"grid_{k}"): int(v)
                     for k, v in (kv.split("=") for kv in args.tuning.split(","))}
            assert self.s.set_tuning(**shape) == pkg.OK, shape
            self.tuning = self.s.get_tuning()
        elif autotune and not args.no_autotune:
            # launch shapes picked by timing candidates on this workload (outside the timed region)
            st, _ = self.set_batch(self.slots, self.vals)
            assert st == pkg.OK, pkg.strerror(st)
            st, self.tuning = self.s.autotune(self.slots, self.b_dev, iters=32)
            assert st == pkg.OK, pkg.strerror(st)

    def step(self):
        pkg, s = self.pkg, self.s
        st, _ = self.set_batch(self.slots, self.vals)
        assert st == pkg.OK, pkg.strerror(st)
        x0 = None
        if self.x0_mode == "rom":     # POD reduced-order solution as the initial guess
            st = s.rom_solution_dev(self.slots, self.b_dev, self.x0_dev)
            assert st == pkg.OK, pkg.strerror(st)
            x0 = self.x0_dev
        elif self.x0_mode == "sur":   # surrogate prediction from each instance's parameters
            st = self.sur.predict_dev(self.xis, self.scales, self.x0_dev)
            assert st == pkg.OK, pkg.strerror(st)
            x0 = self.x0_dev
        iters, rel, status, rc = s.solve_batch_dev(self.slots, self.b_dev, self.x_dev, x0_dev=x0,
                                                   tol=self.args.tol, maxit=self.args.maxit)
        assert rc == pkg.OK, (pkg.strerror(rc), status)
        return iters, rel

    def timed(self, steps, warmup, dist=None, sampler=None):
        """warmup untimed steps, then `steps` steps between CUDA events on the solver's stream."""
        import torch
        for _ in range(max(warmup, 0)):
            self.step()
        l0 = self.s.launch_count()
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        if sampler:
            sampler.start()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(self.stream)
        its, rels = [], []
        for _ in range(steps):
            it, rel = self.step()
            its.append(it)
            rels.append(rel)
        ev1.record(self.stream)
        torch.cuda.synchronize()
        clocks = sampler.stop() if sampler else None
        if dist:
            dist.barrier()
        return dict(ms=ev0.elapsed_time(ev1) / steps, iters=np.concatenate(its), relres=np.concatenate(rels),
                    launches=self.s.launch_count() - l0, clocks=clocks)

    def roofline(self, steps, num_sms):
        """Per-kernel CUDA-event times from separate instrumented steps (event-record nodes inside the
        graph, outside the timed region), and algorithmic bytes / time per kernel."""
        import torch
        s, wl, P, B = self.s, self.wl, self.P, self.B
        s.kernel_timing(True)
        lane_iters = 0
        for _ in range(max(1, steps)):
            iters, _ = self.step()
            lane_iters += int(np.sum(iters))
        torch.cuda.synchronize()
        ktimes = s.kernel_times()
        s.kernel_timing(False)
        peaks, peak_kind = measured_peaks()
        Bp = 1 << (B - 1).bit_length()
        tun = s.get_tuning() or {}
        G = tun.get("grid_rows", max(1, min((P.n_nodes * Bp + 255) // 256, 4 * num_sms)))
        kp = {0: 0}.get(wl.spec.k, [v for v in (0, 8, 16, 24, 32, 40, 48, 64) if v >= wl.spec.k][0])
        nl = {k: v[1] for k, v in ktimes.items()}
        sgs = self.args.smoother == "sgs"
        kphi = bool(tun.get("rows_kernel", 0) & 4)
        kb = kernel_bytes(wl, kp, lane_iters, nl["k_spmv"], G, Bp, self.elements, sgs, kphi)
        # the same bytes with every lane active in every launch (what one ncu capture of a launch sees)
        kb_all = kernel_bytes(wl, kp, B, 1, G, Bp, self.elements, sgs, kphi)
        rates = {k: (kb[k] / (ktimes[k][0] / 1e3) / 1e9 if ktimes[k][0] > 0 else 0.0) for k in kb}
        dom = max(ktimes, key=lambda k: ktimes[k][0])
        tot_k = sum(v[0] for v in ktimes.values())
        key = (wl.spec.name, B, self.args.operator, int(tun.get("rows_kernel", 0)))
        row = ("k_spmv", "k_smooth1", "k_post")
        return {"bound": "hbm", "kernel": dom, "achieved": rates[dom], "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": rates[dom] / peaks["hbm_gbs"], "peak_kind": peak_kind,
                "bytes_per_launch": kb[dom] / max(nl[dom], 1),
                "bytes_per_launch_all_lanes": kb_all[dom],
                "ms_per_launch": ktimes[dom][0] / max(nl[dom], 1),
                "traffic": NCU_TRAFFIC.get(key, {}).get(dom),
                "traffic_source": NCU_SOURCE.get(key),
                "frac_vs_8TBs": rates[dom] / 8000.0,
                "all_kernels": {k: {"share": ktimes[k][0] / tot_k, "GBs": round(rates[k], 1),
                                    "ms_per_launch": ktimes[k][0] / max(nl[k], 1)} for k in ktimes},
                "spmv_smoother_GBs": sum(kb[k] for k in row) / (sum(ktimes[k][0] for k in row) / 1e3) / 1e9,
                "spmv_smoother_frac": sum(kb[k] for k in row) / (sum(ktimes[k][0] for k in row) / 1e3) / 1e9
                / peaks["hbm_gbs"]}

    def setup_ms(self):
        import torch
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(self.stream)
        st, _ = self.set_batch(self.slots, self.vals)
        e1.record(self.stream)
        torch.cuda.synchronize()
        assert st == self.pkg.OK
        return e0.elapsed_time(e1)

    def close(self):
        import torch
        self.s.close()
        if self.sur is not None:
            self.sur.close()
        del self.vals, self.b_dev, self.x_dev, self.x0_dev
        torch.cuda.empty_cache()


def workload_summary(run, t, roof, B):
    return {"workload": workload_desc(run.wl, B, run.args.tol), "batch": B, "value": B / (t["ms"] / 1e3),
            "unit": "solves/s", "ms_per_step": t["ms"], "iters_mean": float(np.mean(t["iters"])),
            "iters_max": int(np.max(t["iters"])), "relres_max": float(np.max(t["relres"])),
            "tuning": run.tuning, "phi_setup_s": round(run.t_phi, 1),
            "roofline": {k: roof[k] for k in ("kernel", "achieved", "frac", "ms_per_launch", "spmv_smoother_GBs",
                                              "spmv_smoother_frac")},
            "kernels_GBs": {k: v["GBs"] for k, v in roof["all_kernels"].items()}}


def gb300_arm(args):
    import torch
    rank, world, local = _env_rank()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    import __graft_entry__
    __graft_entry__.build()
    import paper_2207_02543_gb300 as pkg
    num_sms = torch.cuda.get_device_properties(local).multi_processor_count

    from synth.problems import SPECS
    B = args.batch or SPECS[args.workload].batch
    budget = args.hbm_budget_gb * 1e9 if args.workload == WORKLOAD else 0
    run = WorkloadRun(args, pkg, args.workload, B, rank, hbm_budget=budget,
                      surrogate=(world == 1 and not args.no_surrogate and args.method == "pcg"))
    wl, P = run.wl, run.P
    sampler = ClockSampler(local)
    t = run.timed(args.steps, args.warmup, dist, sampler)
    roofline = run.roofline(min(args.steps, 2), num_sms)
    setup_ms = run.setup_ms()
    ms = max_over_ranks(t["ms"], dist)
    value = job_value(ms, world, B)
    device_bytes = run.s.device_bytes()

    extra = {}
    if run.sur is not None and args.x0 == "zero":
        # the same steps with the surrogate's prediction as x0 (Section 3.2 then Algorithm 3)
        run.x0_mode = "sur"
        ts = run.timed(max(1, min(args.steps, 2)), 1)
        run.x0_mode = "zero"
        sw = run.sur_w
        extra["x0_surrogate"] = {
            "value": job_value(ts["ms"], 1, B), "unit": "solves/s", "ms_per_step": ts["ms"],
            "iters_mean": float(np.mean(ts["iters"])), "iters_max": int(np.max(ts["iters"])),
            "relres_max": float(np.max(ts["relres"])), "zero_x0_iters_mean": float(np.mean(t["iters"])),
            "zero_x0_value": value, "latent_modes": int(sw.psi.shape[1]), "hidden": int(sw.w1.shape[0]),
            "training_snapshots": wl.spec.n_snap, "latent_val_rel_err": sw.val_rel_err}
    if rank == 0 and world == 1:
        s, slots, tol, maxit = run.s, run.slots, args.tol, args.maxit
        # end to end through the C ABI with host buffers (values, b in; x out), the inputs in pinned
        # host memory (page-locked: the copies run as direct DMA transfers)
        vals_h = run.vals.cpu().pin_memory().numpy()
        b_h = run.b_dev.cpu().pin_memory().numpy()
        e2e_steps = max(1, min(args.steps, 2))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(e2e_steps):
            for i in slots:
                assert run.set_one(i, vals_h[i]) == pkg.OK
            if run.x0_mode == "sur":
                bd = torch.from_numpy(b_h).to(run.b_dev.device)
                assert run.sur.predict_dev(run.xis, run.scales, run.x0_dev) == pkg.OK
                it_h, rel_h, st_h, rc = s.solve_batch_dev(slots, bd, run.x_dev, x0_dev=run.x0_dev, tol=tol,
                                                          maxit=maxit)
                X = run.x_dev.cpu().numpy()
            elif run.x0_mode == "zero":
                X, it_h, rel_h, st_h, rc = s.solve_batch(slots, b_h, tol=tol, maxit=maxit)
            else:   # the reduced-order initial guess lives on the device: copy b in, x out
                bd = torch.from_numpy(b_h).to(run.b_dev.device)
                assert s.rom_solution_dev(slots, bd, run.x0_dev) == pkg.OK
                it_h, rel_h, st_h, rc = s.solve_batch_dev(slots, bd, run.x_dev, x0_dev=run.x0_dev, tol=tol,
                                                          maxit=maxit)
                X = run.x_dev.cpu().numpy()
            assert rc == pkg.OK
        e2e_s = (time.perf_counter() - t0) / e2e_steps
        extra["e2e"] = {"value": B / e2e_s, "unit": "solves/s", "h2d_bytes_per_step": int(vals_h.nbytes + b_h.nbytes),
                        "d2h_bytes_per_step": int(X.nbytes)}
        # plain FP64 one-at-a-time baseline on the same GPU
        if not args.no_plain:
            extra["plain_fp64"] = plain_baseline(run, pkg, vals_h, b_h, value, num_sms)
        # serving: Poisson arrivals at a fraction of the batched throughput, continuous batching
        # (requests carry their instance's values from host memory: measured here on workloads
        # whose instances are below 1 GB, otherwise on the first such extra workload)
        serve_here = not args.no_serve and vals_h[0].nbytes <= 1e9
        if serve_here:
            extra.update(serving_entry(args, s, pkg, wl, vals_h, b_h, value))
        del vals_h, X
        # the same workload at batch 1
        if B > 1 and not args.no_batch1:
            run.close()
            r1 = WorkloadRun(args, pkg, args.workload, 1, rank, hbm_budget=budget)
            t1 = r1.timed(max(1, min(args.steps, 3)), 1)
            extra["batch1"] = workload_summary(r1, t1, r1.roofline(1, num_sms), 1)
            r1.close()
        else:
            run.close()
        # the other configurations, each a few steps in its own context
        extras = [w for w in args.extras.split(",") if w and w != args.workload]
        if extras:
            extra["extra_workloads"] = {}
        for name in extras:
            Bx = SPECS[name].batch
            rx = WorkloadRun(args, pkg, name, Bx, rank)
            tx = rx.timed(2, 2)
            sx = workload_summary(rx, tx, rx.roofline(1, num_sms), Bx)
            extra["extra_workloads"][f"{name}_b{Bx}"] = sx
            if not args.no_serve and "serving" not in extra and rx.vals[0].numel() * 8 <= 1e9:
                vh, bh = rx.vals.cpu().numpy(), rx.b_dev.cpu().numpy()
                extra.update(serving_entry(args, rx.s, pkg, rx.wl, vh, bh, sx["value"]))
                extra["serving"]["workload"] = sx["workload"]
                del vh, bh
            rx.close()
        # the small 2D diffusion problem (3,969 unknowns): launch- and latency-bound
        if not args.no_small:
            extra["small_problem"] = small_problem_entry(pkg, args.tol)
        # CPU baseline: the oracle on the host cores, a bounded sample
        if not args.no_cpu:
            try:
                import resource
                rss = resource.getrusage(resource.RUSAGE_SELF).ru_maxrss * 1024
                workers = oracle_workers(wl, limit=args.oracle_workers or None, reserve=16e9 + rss)
                extra["cpu_baseline"], _ = cpu_baseline_entry(wl, workers, sample_iterations(wl), tol, args.method,
                                                              args.smoother)
            except Exception as e:  # noqa: BLE001
                extra["cpu_baseline"] = {"value": None, "unit": "solves/s", "cores": 0, "kind": "oracle",
                                         "sample": f"failed: {e}"[:300]}
    else:
        run.close()
    if rank == 0:
        line = {
            "metric": f"solves/s at rel. residual {fmt_tol(args.tol)} (batched {method_name(args.method)})",
            "value": value, "unit": "solves/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32+df64",
            "data": "synthetic",
            "config": {"workload": workload_desc(wl, B, args.tol), "method": method_name(args.method),
                       "operator": args.operator, "smoother": args.smoother, "x0": args.x0, "tuning": run.tuning,
                       "batch": B, "n": P.n, "nnzb": P.nnzb, "k": wl.spec.k, "parallelism": f"replicas{world}",
                       "hbm_budget_bytes": int(budget), "device_bytes": int(device_bytes),
                       "l2": (f"inputs larger than L2 ({B * run.P.nnzb * P.bs ** 2 * 8 / 1e9:.2f} GB FP64 "
                              f"{'coefficients' if run.elements else 'values'} per step; per-iteration working "
                              f"set {P.n * B * 8 * 5 / 1e9:.2f} GB of vectors)"),
                       "iters_mean": float(np.mean(t["iters"])), "iters_max": int(np.max(t["iters"])),
                       "relres_max": float(np.max(t["relres"])), "phi_setup_s": round(run.t_phi, 1),
                       "setup_ms_per_step": round(setup_ms, 2)},
            "gpu_launches": int(t["launches"] / max(args.steps, 1)) if args.steps else 0,
            "roofline": roofline, "clocks": t["clocks"],
        }
        line.update(extra)
        line.setdefault("cpu_baseline", None)
        line.setdefault("e2e", None)
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


def small_problem_entry(pkg, tol):
    """Q1 64 x 64 diffusion (3,969 unknowns, k = 10): the plain FP64 path on one query (host-checked
    convergence every iteration), and the batched mixed path at batch 1 and 64, with whole iterations in
    one persistent launch per 8 iterations and as a CUDA graph of 8 iterations per launch (the default):
    per-iteration times show the launch and latency cost of a problem this small."""
    import torch
    from synth.problems import Workload
    from synth.snapshots import pod_basis
    wl = Workload("q1_64")
    P = wl.problem
    Phi = pod_basis(wl)
    out = {"workload": f"2D Poisson Q1 64x64, lognormal kappa: {P.n:,} dofs, k={wl.spec.k}, tol {fmt_tol(tol)}"}
    xis, bs = wl.query_thetas(64), wl.rhs(64)
    sp = pkg.Solver(P.row_ptr, P.col_idx, P.bs, Phi, precision=pkg.FP64, omega=wl.spec.omega, max_batch=1)
    assert sp.set_values(0, wl.values(xis[0])) == pkg.OK
    times, its = [], []
    for r in range(6):
        t0 = time.perf_counter()
        _, it, _, st = sp.solve(0, bs[0], tol=tol, maxit=MAXIT)
        times.append(time.perf_counter() - t0)
        its.append(it)
        assert st == pkg.OK
    sp.close()
    tm = statistics.median(times[1:])
    out["plain_fp64"] = {"ms_per_solve": 1e3 * tm, "iters": int(its[-1]), "us_per_iteration": 1e6 * tm / its[-1]}
    for B, form in ((1, "persistent"), (64, "persistent"), (1, "graph"), (64, "graph")):
        s = pkg.Solver(P.row_ptr, P.col_idx, P.bs, Phi, precision=pkg.MIXED_FP32PHI, omega=wl.spec.omega, max_batch=B)
        vals = wl.values_torch(xis[:B], device="cuda").reshape(B, -1).contiguous()
        b_dev = torch.from_numpy(bs[:B]).cuda()
        x_dev = torch.empty_like(b_dev)
        slots = list(range(B))
        st, _ = s.set_values_batch_dev(slots, vals)
        assert st == pkg.OK
        tune = s.get_tuning()
        if form == "graph":
            assert s.set_tuning(rows_kernel=tune["rows_kernel"] & 7) == pkg.OK
        elif tune["grid_persist"] < 1:   # the persistent form does not apply to this context
            s.close()
            continue
        else:
            assert s.set_tuning(rows_kernel=tune["rows_kernel"] | 8) == pkg.OK
        for _ in range(2):
            it, rel, sts, rc = s.solve_batch_dev(slots, b_dev, x_dev, tol=tol, maxit=MAXIT)
        torch.cuda.synchronize()
        reps = 5
        t0 = time.perf_counter()
        for _ in range(reps):
            it, rel, sts, rc = s.solve_batch_dev(slots, b_dev, x_dev, tol=tol, maxit=MAXIT)
            assert rc == pkg.OK
        torch.cuda.synchronize()
        ms = 1e3 * (time.perf_counter() - t0) / reps
        s.close()
        key = f"batched_b{B}" if form == "persistent" else f"batched_b{B}_graph"
        out[key] = {"ms_per_step": ms, "solves_per_s": B / (ms / 1e3), "iters_max": int(np.max(it)),
                    "us_per_iteration": 1e3 * ms / int(np.max(it)),
                    "form": ("one persistent launch per 8 iterations" if form == "persistent" else
                             "CUDA graph of 8 iterations x 7 kernels"), "grid_persist": tune["grid_persist"]}
    return out


def serving_entry(args, s, pkg, wl, vals_h, b_h, value):
    loads = [float(v) for v in args.serve_loads.split(",")]
    nreq = args.serve_requests or max(8, min(128, int(30 * value)))
    runs = [dict(serve_latency(s, pkg, wl, vals_h, b_h, rate=f * value, nreq=nreq, tol=args.tol,
                               maxit=args.maxit), load=f) for f in loads]
    out = {"serving": runs[0]}
    if len(runs) > 1:
        out["serving_loads"] = runs
    return out


def plain_baseline(run, pkg, vals_h, b_h, value, num_sms):
    """The plain path (FP64 values, vectors and basis; one instance at a time, kernel by kernel,
    convergence checked on the host every iteration, no graphs) on two of the instances."""
    import torch
    wl, P = run.wl, run.P
    sp = pkg.Solver(P.row_ptr, P.col_idx, P.bs, run.Phi, precision=pkg.FP64, omega=wl.spec.omega, max_batch=1,
                    method=run.method, smoother=run.smoother)
    vals_plain = run.vals if not run.elements else wl.values_torch(run.xis[:2], device="cuda").reshape(2, -1)
    times, its = [], []
    for i in range(min(2, run.B)):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        assert sp.set_values(0, vals_plain[i]) == pkg.OK
        xp, itp, relp, stp = sp.solve(0, b_h[i], tol=run.args.tol, maxit=run.args.maxit)
        torch.cuda.synchronize()
        times.append(time.perf_counter() - t0)
        its.append(itp)
        assert stp == pkg.OK
    sp.close()
    pv = 1.0 / statistics.mean(times)
    # algorithmic bytes of one plain iteration (FP64 values read by 3 SpMVs, ~13 FP64 vector streams,
    # Phi twice) and the bytes bound of the batched/plain ratio
    n, nnz, k = P.n, P.nnzb * P.bs ** 2, wl.spec.k
    plain_iter = 3 * (8 * nnz + 4 * nnz) + 8 * 13 * n + 2 * 8 * n * k
    it_mean = statistics.mean(its)
    per_solve = [t for t in times]
    Bp = 1 << (run.B - 1).bit_length()
    kphi = bool((run.s.get_tuning() or {}).get("rows_kernel", 0) & 4)
    batched_iter = sum(kernel_bytes(wl, 0 if k == 0 else [v for v in (8, 16, 24, 32, 40, 48, 64) if v >= k][0],
                                    1, 0, 8, Bp, kphi=kphi).values())
    return {"value": pv, "unit": "solves/s", "iters": its, "ratio_batched_over_plain": value / pv,
            "achieved_GBs": plain_iter * it_mean / statistics.mean(per_solve) / 1e9,
            "bytes_per_iteration": plain_iter, "batched_bytes_per_instance_iteration": batched_iter,
            "bytes_bound_ratio": plain_iter / batched_iter}


def serve_latency(s, pkg, wl, vals_h, b_h, rate, nreq, tol=TOL, maxit=MAXIT):
    import numpy as np
    rng = np.random.default_rng(3000)
    gaps = rng.exponential(1.0 / rate, nreq)
    s.serve_start(max_queue=4 * nreq)
    tickets = []
    t0 = time.perf_counter()
    t_next = t0
    for i in range(nreq):
        t_next += gaps[i]
        while time.perf_counter() < t_next:
            time.sleep(0.0002)
        st, t = s.submit(vals_h[i % len(vals_h)], b_h[i % len(b_h)], tol=tol, maxit=maxit)
        assert st == pkg.OK
        tickets.append(t)
    lat = []
    pending = dict(enumerate(tickets))
    while pending:
        for i, t in list(pending.items()):
            st, r = s.poll(t)
            if st == pkg.OK:
                assert r["status"] == pkg.OK
                lat.append(r["latency_s"])
                del pending[i]
        time.sleep(0.001)
    wall = time.perf_counter() - t0
    s.serve_stop()
    lat.sort()
    return {"requests": nreq, "arrival_rate_per_s": rate, "p50_ms": 1e3 * lat[len(lat) // 2],
            "p99_ms": 1e3 * lat[min(len(lat) - 1, int(0.99 * len(lat)))], "throughput": nreq / wall}


# ----------------------------------------------------------------------------- serving mix
MIX = ("q4_512", "hex8_64", "q1_1024")


def serve_mix(args):
    """Poisson-arrival requests spread in equal thirds over three registered problems (2D elasticity
    Q4 512^2, 3D elasticity Hex8 64^3, 2D diffusion Q1 1024^2 with k = 25), each with its own context
    and continuous batching, admitted under one HBM budget; p50/p99 latency per problem at fractions
    of the mix's saturated throughput. A request carries one of 8 prepared instances of its problem
    (values and right-hand side in host memory), copied by the library at submission."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_2207_02543_gb300 as pkg
    from synth.problems import Workload
    from synth.snapshots import pod_basis
    ni = 8
    mix = pkg.ServingMix(int(args.hbm_budget_gb * 1e9), max_queue=4096)
    probs = {}
    t0 = time.time()
    for name in MIX:
        wl = Workload(name)
        P = wl.problem
        phi = pod_basis(wl, device="cuda")
        prec = pkg.MIXED_BF16PHI if wl.spec.phi_dtype == "bf16" else pkg.MIXED_FP32PHI
        st = mix.register(name, P.row_ptr, P.col_idx, P.bs, phi, precision=prec, omega=wl.spec.omega,
                          max_batch=wl.spec.batch)
        assert st == pkg.OK, (name, pkg.strerror(st))
        xis = wl.query_thetas(ni)
        vals = wl.values_torch(xis, device="cuda").reshape(ni, -1).cpu().numpy()
        probs[name] = dict(wl=wl, vals=vals, b=wl.rhs(ni), batch=wl.spec.batch)
        torch.cuda.empty_cache()
    prep_s = time.time() - t0

    def run(reqs):
        """reqs: list of (time offset s, problem); returns per-problem latencies and the wall time."""
        handles = []
        t_start = time.perf_counter()
        for k, (dt, name) in enumerate(reqs):
            while time.perf_counter() - t_start < dt:
                time.sleep(0.0002)
            pr = probs[name]
            st, h = mix.submit(name, pr["vals"][k % ni], pr["b"][k % ni], tol=args.tol, maxit=args.maxit)
            assert st == pkg.OK, pkg.strerror(st)
            handles.append((name, h))
        lat = {name: [] for name in MIX}
        pending = dict(enumerate(handles))
        while pending:
            for k, (name, h) in list(pending.items()):
                st, r = mix.poll(h)
                if st == pkg.OK:
                    if r["status"] != pkg.OK:
                        failed.append({"problem": name, "status": pkg.strerror(r["status"]), "iters": r["iters"]})
                    lat[name].append(r["latency_s"])
                    del pending[k]
            time.sleep(0.001)
        return lat, time.perf_counter() - t_start

    failed = []

    # saturated throughput of each problem alone: two batches' worth submitted at once (after a warm-up)
    rate = {}
    for name in MIX:
        B = probs[name]["batch"]
        run([(0.0, name)] * B)
        lat, wall = run([(0.0, name)] * (2 * B))
        rate[name] = 2 * B / wall
    lam_sat = len(MIX) / sum(1.0 / r for r in rate.values())   # equal thirds sharing the device
    rng = np.random.default_rng(3000)
    loads = [float(v) for v in args.serve_loads.split(",")]
    out = []
    for f in loads:
        lam = f * lam_sat
        nreq = args.serve_requests or max(30, int(30 * lam))
        gaps = rng.exponential(1.0 / lam, nreq)
        names = [MIX[i] for i in rng.integers(0, len(MIX), nreq)]
        lat, wall = run(list(zip(np.cumsum(gaps), names)))
        per = {}
        for name in MIX:
            ls = sorted(lat[name])
            if ls:
                per[name] = {"requests": len(ls), "p50_ms": 1e3 * ls[len(ls) // 2],
                             "p99_ms": 1e3 * ls[min(len(ls) - 1, int(0.99 * len(ls)))]}
        out.append({"load": f, "arrival_rate_per_s": lam, "requests": nreq, "throughput": nreq / wall,
                    "per_problem": per})
    used = mix.used_bytes()
    mix.close()
    line = {"metric": f"serving mix: p50/p99 latency at rel. residual {fmt_tol(args.tol)} (batched POD-2G-PCG)",
            "unit": "ms", "n_gpus": 1, "data": "synthetic", "dtype": "f32+df64",
            "config": {"workload": "Poisson arrivals, equal thirds over " +
                                   "; ".join(workload_desc(probs[n]["wl"], probs[n]["batch"], args.tol) for n in MIX),
                       "hbm_budget_bytes": int(args.hbm_budget_gb * 1e9), "device_bytes": int(used),
                       "prepare_s": round(prep_s, 1)},
            "saturated_solves_per_s": rate, "mix_saturated_solves_per_s": lam_sat, "loads": out,
            "failed_requests": failed[:20], "failed_count": len(failed)}
    print(json.dumps(line), flush=True)
    return 0 if not failed else 1


def fma_rates(args):
    """Dense FP64 and FP32 (no tensor cores) GEMM throughput on this GPU through torch / cuBLAS: the
    FP64 : FP32 rate ratio that decides whether the outer recurrences are carried in FP64 or in
    double-float (pairs of FP32)."""
    import torch
    torch.backends.cuda.matmul.allow_tf32 = False
    torch.backends.cudnn.allow_tf32 = False
    out = {}
    for name, dt, nn in (("fp64", torch.float64, 8192), ("fp32", torch.float32, 16384)):
        a = torch.randn(nn, nn, device="cuda", dtype=dt)
        b = torch.randn(nn, nn, device="cuda", dtype=dt)
        for _ in range(2):
            torch.mm(a, b)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        reps = 5
        e0.record()
        for _ in range(reps):
            torch.mm(a, b)
        e1.record()
        torch.cuda.synchronize()
        out[name + "_tflops"] = 2.0 * nn ** 3 * reps / (e0.elapsed_time(e1) / 1e3) / 1e12
        del a, b
    out["fp32_over_fp64"] = out["fp32_tflops"] / out["fp64_tflops"]
    out["metric"] = "dense GEMM throughput, torch.mm (cuBLAS), TF32 off"
    print(json.dumps(out), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--no-serve", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--serve-requests", type=int, default=0, help="requests per serving load (default: ~30 s of work)")
    ap.add_argument("--no-batch1", action="store_true", help="skip the batch-1 line of the workload")
    ap.add_argument("--extras", default=EXTRAS, help="other workloads measured after the main one (comma list)")
    ap.add_argument("--hbm-budget-gb", type=float, default=HBM_BUDGET_GB,
                    help="HBM admission budget of the default workload's context")
    ap.add_argument("--serve-loads", default="0.7",
                    help="Poisson arrival rates as fractions of the measured batch throughput, e.g. 0.5,0.7,0.9")
    ap.add_argument("--workload", default=WORKLOAD, help="synthetic workload name (profiling of smaller cases)")
    ap.add_argument("--batch", type=int, default=0, help="instances per step (default: the workload's batch)")
    ap.add_argument("--method", default="pcg", choices=["pcg", "stationary"],
                    help="pcg: Algorithm 3; stationary: the two-grid cycle of Algorithm 2 iterated on its own")
    ap.add_argument("--operator", default="assembled", choices=["assembled", "elements"],
                    help="instances as assembled block values, or as element coefficients (element-factored K)")
    ap.add_argument("--no-autotune", action="store_true", help="keep the default launch shapes")
    ap.add_argument("--tuning", default="", help="launch shape to use instead of autotuning, "
                    "e.g. rows=1216,spmv=1216,restrict=456,prol=608,vec=1216")
    ap.add_argument("--smoother", default="jacobi", choices=["jacobi", "sgs"],
                    help="relaxation of the two-grid cycle: damped Jacobi or multicolour symmetric Gauss-Seidel")
    ap.add_argument("--no-surrogate", action="store_true", help="skip the surrogate-x0 comparison key")
    ap.add_argument("--no-small", action="store_true", help="skip the small-problem (Q1 64x64) key")
    ap.add_argument("--x0", default="zero", choices=["zero", "rom", "sur"],
                    help="initial guess: zero, the POD reduced-order solution Phi K_c^-1 Phi^T b, or the "
                         "surrogate's prediction from the parameters")
    ap.add_argument("--tol", type=float, default=TOL)
    ap.add_argument("--oracle-workers", type=int, default=0,
                    help="cap on the oracle processes of the CPU baseline (default: cores, bounded by host memory)")
    ap.add_argument("--maxit", type=int, default=MAXIT)
    ap.add_argument("--serve-mix", action="store_true",
                    help="serving latency over three registered problems under one HBM budget (separate line)")
    ap.add_argument("--fma-rates", action="store_true", help="FP64 and FP32 dense GEMM throughput (separate line)")
    args = ap.parse_args()
    if args.impl == "reference":
        return reference_arm(args)
    if args.fma_rates:
        return fma_rates(args)
    if args.serve_mix:
        return serve_mix(args)
    return gb300_arm(args)


if __name__ == "__main__":
    sys.exit(main())

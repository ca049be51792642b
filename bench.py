#!/usr/bin/env python
"""Benchmark: batched mixed-precision POD-2G-PCG on one GB300.

Metric: solves/s at relative residual 1e-8 (arXiv 2207.02543, Algorithm 3 with
the two-grid cycle of Algorithm 2, P = Phi_r). Workload: 2D plane-stress
elasticity, Q4 elements on a 512 x 512 grid (526,338 unknowns, 2 x 2 blocks,
left edge clamped, uniform traction on the right edge), lognormal Young's
modulus from an 8-term KL field (mean 1, CoV 0.3), nu = 0.3, POD basis k = 20
from 200 snapshots, a batch of 64 parameter instances sharing one pattern,
double-float outer PCG with an FP32 preconditioner and FP32 Phi.

One step = per-instance set-up of all 64 instances from FP64 values resident in
HBM (FP32 conversion, D^-1, K_c = Phi^T K Phi, Cholesky) + the batched solve of
all 64 to 1e-8. The inputs (4.8 GB of values) are larger than L2.

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

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "q4_512"
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


def kernel_bytes(wl, k_pad, lane_iters, launches, G, Bp, elements=False, sgs=False):
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
    if sgs:   # timing groups: forward sweeps + residual; stored y1; backward sweeps + r^T s
        per_lane["k_smooth1"] = 2 * vals + n * (20 + 16)
        per_lane["k_prol"] = n * (4 + 4)
        per_lane["k_post"] = vals + n * (20 + 16)
        shared["k_smooth1"] = 2 * pat
        shared["k_post"] = pat
    return {name: per_lane[name] * lane_iters + shared[name] * launches for name in per_lane}


# DRAM bytes (read + write) per launch from one ncu capture of these kernels on the
# workload named (profiles/launches_q4_512_b64.md); valid only for the kernel
# versions that capture measured.
NCU_TRAFFIC = {
    ("q4_512", 64, "assembled"): {"k_spmv": 3156.2e6, "k_smooth1": 2964.0e6, "k_post": 3100.1e6, "k_upd": 1569.2e6,
                                  "k_restrict": 185.5e6, "k_prol": 568.5e6, "k_p": 615.7e6, "k_coarse": 1.0e6},
}


NCU_SOURCE = {("q4_512", 64, "assembled"): "profiles/launches_q4_512_b64.md"}


def run_oracle(mode, inst, timeout=900, workload=WORKLOAD, tol=TOL, method="pcg", smoother="jacobi"):
    env = dict(os.environ)
    for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        env[v] = "1"
    r = subprocess.run([sys.executable, "-m", "oracle.timing", workload, str(inst), str(mode), str(tol), method, smoother],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=timeout)
    if r.returncode != 0:
        raise RuntimeError(r.stderr[-2000:])
    return json.loads(r.stdout.strip().splitlines()[-1])


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
def reference_arm(args):
    """The oracle (FP64, host cores) on the GPU arm's workload, method, relaxation and tolerance:
    one single-threaded process per core, each a bounded sample of iterations on a distinct
    instance, scaled by the oracle's own full iteration count of instance 0."""
    rank, world, local = _env_rank()
    if rank != 0:
        return 0
    from synth.problems import Workload
    from synth.snapshots import pod_basis
    wl = Workload(args.workload)
    B = args.batch or wl.spec.batch
    tol = args.tol
    pod_basis(wl, device="cuda" if wl.n > 20_000 else None)  # cached POD basis (library snapshot solves)
    tag = f"{args.workload}_{args.method}_{args.smoother}_{fmt_tol(tol)}"
    cache = os.path.join(ROOT, "_cache", f"oracle_{tag}_iters.json")
    kw = dict(workload=args.workload, tol=tol, method=args.method, smoother=args.smoother)
    if os.path.exists(cache):
        full = json.load(open(cache))
    else:
        full = run_oracle("full", 0, timeout=3600, **kw)
        os.makedirs(os.path.dirname(cache), exist_ok=True)
        json.dump(full, open(cache, "w"))
    cores = min(os.cpu_count() or 1, 16)
    sample_it = min(25, max(1, full["iterations"]))
    from concurrent.futures import ThreadPoolExecutor

    def step():
        t0 = time.perf_counter()
        with ThreadPoolExecutor(cores) as ex:
            outs = list(ex.map(lambda i: run_oracle(sample_it, i, **kw), range(cores)))
        wall = time.perf_counter() - t0
        per_it = max(o["seconds_per_iteration"] for o in outs)
        return wall, per_it
    for _ in range(args.warmup):
        step()
    per = []
    t0 = time.perf_counter()
    for _ in range(args.steps):
        per.append(step()[1])
    wall = time.perf_counter() - t0
    per_it = statistics.mean(per)
    value = cores / (per_it * max(full["iterations"], 1))
    line = {
        "metric": f"solves/s at rel. residual {fmt_tol(tol)} (batched {method_name(args.method)})",
        "value": value, "unit": "solves/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "ms_per_step": wall / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "impl": "reference",
        "config": {"workload": workload_desc(wl, B, tol), "method": method_name(args.method),
                   "smoother": args.smoother, "batch": B, "n": wl.problem.n, "k": wl.spec.k},
        "cpu_baseline": {"value": value, "unit": "solves/s", "cores": cores, "kind": "oracle",
                         "sample": f"{cores} single-threaded oracle processes, {sample_it} "
                                   f"{method_name(args.method)} iterations each on distinct instances per step, "
                                   f"scaled by the oracle's full iteration count ({full['iterations']}) for "
                                   f"instance 0"},
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
def gb300_arm(args):
    import numpy as np
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
    from synth.problems import Workload
    from synth.snapshots import pod_basis

    wl = Workload(args.workload)
    P = wl.problem
    B = args.batch or wl.spec.batch
    t0 = time.time()
    Phi = pod_basis(wl, device="cuda")
    t_phi = time.time() - t0
    # instances of this replica: distinct per rank
    xis = wl.query_thetas(B, offset=replica_offset(rank, B))
    elements = args.operator == "elements"
    if elements:   # FP64 element coefficients, resident in HBM
        vals = torch.from_numpy(np.stack([wl.coef(xi) for xi in xis])).cuda()
    else:          # FP64 assembled values, resident in HBM
        vals = wl.values_torch(xis, device="cuda").reshape(B, -1).contiguous()
    b_dev = torch.from_numpy(wl.rhs(B, offset=replica_offset(rank, B))).cuda()
    x_dev = torch.empty_like(b_dev)
    stream = torch.cuda.Stream()
    precision = pkg.MIXED_BF16PHI if wl.spec.phi_dtype == "bf16" else pkg.MIXED_FP32PHI
    method = pkg.STATIONARY if args.method == "stationary" else pkg.PCG
    tol, maxit = args.tol, args.maxit
    el = dict(conn=P.conn, k_ref=P.Kref, fixed=P.clamped if P.dirichlet == "identity" else None) if elements else None
    smoother = pkg.SMOOTHER_SGS if args.smoother == "sgs" else pkg.SMOOTHER_JACOBI
    s = pkg.Solver(P.row_ptr, P.col_idx, P.bs, Phi, precision=precision, omega=wl.spec.omega,
                   max_batch=B, stream=stream.cuda_stream, method=method, elements=el, smoother=smoother)
    slots = list(range(B))
    set_batch = s.set_coeffs_batch_dev if elements else s.set_values_batch_dev
    set_one = s.set_coeffs if elements else s.set_values

    x0_dev = torch.empty_like(b_dev) if args.x0 == "rom" else None

    def step():
        st, sts = set_batch(slots, vals)
        assert st == pkg.OK, pkg.strerror(st)
        if x0_dev is not None:   # POD reduced-order solution as the initial guess
            st = s.rom_solution_dev(slots, b_dev, x0_dev)
            assert st == pkg.OK, pkg.strerror(st)
        iters, rel, status, rc = s.solve_batch_dev(slots, b_dev, x_dev, x0_dev=x0_dev, tol=tol, maxit=maxit)
        assert rc == pkg.OK, (pkg.strerror(rc), status)
        return iters, rel

    tuning = None
    if args.tuning:
        # a given launch shape (e.g. the one an earlier autotuned run reported), no autotuning
        shape = {f"grid_{k}": int(v) for k, v in (kv.split("=") for kv in args.tuning.split(","))}
        assert s.set_tuning(**shape) == pkg.OK, shape
        tuning = s.get_tuning()
    elif not args.no_autotune:
        # launch shapes picked by timing candidates on this workload (outside the timed region)
        st, sts = set_batch(slots, vals)
        assert st == pkg.OK, pkg.strerror(st)
        st, tuning = s.autotune(slots, b_dev, iters=32)
        assert st == pkg.OK, pkg.strerror(st)
    torch.cuda.synchronize()
    for _ in range(max(args.warmup, 0)):
        iters, rel = step()
    sampler = ClockSampler(local)
    l0 = s.launch_count()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    sampler.start()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    lane_iters = 0
    for _ in range(args.steps):
        iters, rel = step()
        lane_iters += int(np.sum(iters))
    ev1.record(stream)
    torch.cuda.synchronize()
    clocks = sampler.stop()
    if dist:
        dist.barrier()
    ms = ev0.elapsed_time(ev1) / args.steps
    launches = s.launch_count() - l0
    # per-kernel CUDA-event times: separate, instrumented steps (event-record nodes
    # inside the graph), outside the timed region above
    s.kernel_timing(True)
    lane_iters = 0
    for _ in range(max(1, min(args.steps, 2))):
        iters, rel = step()
        lane_iters += int(np.sum(iters))
    torch.cuda.synchronize()
    ktimes = s.kernel_times()
    s.kernel_timing(False)
    # per-instance set-up (values or coefficients -> D^-1, K_c and its Cholesky factor) on its own
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    st, _ = set_batch(slots, vals)
    e1.record(stream)
    torch.cuda.synchronize()
    assert st == pkg.OK
    setup_ms = e0.elapsed_time(e1)
    ms = max_over_ranks(ms, dist)
    value = job_value(ms, world, B)

    # roofline of the dominant kernel (algorithmic bytes / its event-timed duration)
    peaks, peak_kind = measured_peaks()
    Bp = 1 << (B - 1).bit_length()
    G = max(1, min((P.n_nodes * Bp + 255) // 256, 4 * torch.cuda.get_device_properties(local).multi_processor_count))
    kp = {0: 0}.get(wl.spec.k, [v for v in (0, 8, 16, 24, 32, 40, 48, 64) if v >= wl.spec.k][0])
    nl = {k: v[1] for k, v in ktimes.items()}
    kb = kernel_bytes(wl, kp, lane_iters, nl["k_spmv"], G, Bp, elements, args.smoother == "sgs")
    rates = {k: (kb[k] / (ktimes[k][0] / 1e3) / 1e9 if ktimes[k][0] > 0 else 0.0) for k in kb}
    dom = max(ktimes, key=lambda k: ktimes[k][0])
    tot_k = sum(v[0] for v in ktimes.values())
    roofline = {"bound": "hbm", "kernel": dom, "achieved": rates[dom], "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": rates[dom] / peaks["hbm_gbs"], "peak_kind": peak_kind,
                "bytes_per_launch": kb[dom] / max(nl[dom], 1),
                "ms_per_launch": ktimes[dom][0] / max(nl[dom], 1),
                "traffic": NCU_TRAFFIC.get((args.workload, B, args.operator), {}).get(dom),
                "traffic_source": NCU_SOURCE.get((args.workload, B, args.operator)),
                "frac_vs_8TBs": rates[dom] / 8000.0,
                "all_kernels": {k: {"share": ktimes[k][0] / tot_k, "GBs": round(rates[k], 1),
                                    "ms_per_launch": ktimes[k][0] / max(nl[k], 1)} for k in ktimes},
                "spmv_smoother_GBs": (kb["k_spmv"] + kb["k_smooth1"] + kb["k_post"]) /
                                     ((ktimes["k_spmv"][0] + ktimes["k_smooth1"][0] + ktimes["k_post"][0]) / 1e3) / 1e9}

    extra = {}
    if rank == 0 and world == 1:
        # end to end through the C ABI with host buffers (values, b in; x out)
        vals_h = vals.cpu().numpy()
        b_h = b_dev.cpu().numpy()
        e2e_steps = max(1, min(args.steps, 2))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(e2e_steps):
            for i in slots:
                assert set_one(i, vals_h[i]) == pkg.OK
            if x0_dev is None:
                X, it_h, rel_h, st_h, rc = s.solve_batch(slots, b_h, tol=tol, maxit=maxit)
            else:   # the reduced-order initial guess lives on the device: copy b in, x out
                bd = torch.from_numpy(b_h).to(b_dev.device)
                assert s.rom_solution_dev(slots, bd, x0_dev) == pkg.OK
                it_h, rel_h, st_h, rc = s.solve_batch_dev(slots, bd, x_dev, x0_dev=x0_dev, tol=tol, maxit=maxit)
                X = x_dev.cpu().numpy()
            assert rc == pkg.OK
        e2e_s = (time.perf_counter() - t0) / e2e_steps
        extra["e2e"] = {"value": B / e2e_s, "unit": "solves/s", "h2d_bytes_per_step": int(vals_h.nbytes + b_h.nbytes),
                        "d2h_bytes_per_step": int(X.nbytes)}
        # plain FP64 one-at-a-time baseline on the same GPU
        if not args.no_plain:
            sp = pkg.Solver(P.row_ptr, P.col_idx, P.bs, Phi, precision=pkg.FP64, omega=wl.spec.omega, max_batch=1,
                            method=method, smoother=smoother)
            vals_plain = vals if not elements else wl.values_torch(xis[:2], device="cuda").reshape(2, -1)
            nplain = 2
            times, its = [], []
            for i in range(nplain):
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                assert sp.set_values(0, vals_plain[i]) == pkg.OK
                xp, itp, relp, stp = sp.solve(0, b_h[i], tol=tol, maxit=maxit)
                torch.cuda.synchronize()
                times.append(time.perf_counter() - t0)
                its.append(itp)
                assert stp == pkg.OK
            sp.close()
            extra["plain_fp64"] = {"value": 1.0 / statistics.mean(times), "unit": "solves/s",
                                   "iters": its, "ratio_batched_over_plain": value / (1.0 / statistics.mean(times))}
        # serving: Poisson arrivals at ~70% of the batched throughput, continuous batching
        if not args.no_serve:
            loads = [float(v) for v in args.serve_loads.split(",")]
            runs = [dict(serve_latency(s, pkg, wl, vals_h, b_h, rate=f * value, nreq=args.serve_requests, tol=tol,
                                       maxit=maxit), load=f) for f in loads]
            extra["serving"] = runs[0]
            if len(runs) > 1:
                extra["serving_loads"] = runs
        # CPU baseline: the oracle on a bounded sample (single thread)
        if not args.no_cpu:
            try:
                o = run_oracle(100, 0, workload=args.workload, tol=tol, method=args.method, smoother=args.smoother)
                it_full = int(iters[0])
                cpu_val = 1.0 / (o["seconds_per_iteration"] * it_full)
                extra["cpu_baseline"] = {"value": cpu_val, "unit": "solves/s", "cores": 1, "kind": "oracle",
                                         "sample": f"instance 0, first 100 {method_name(args.method)} iterations of "
                                                   f"the FP64 oracle (one thread), scaled by the instance's "
                                                   f"iteration count {it_full}"}
            except Exception as e:  # noqa: BLE001
                extra["cpu_baseline"] = {"value": None, "unit": "solves/s", "cores": 1, "kind": "oracle",
                                         "sample": f"failed: {e}"[:200]}
    s.close()
    if rank == 0:
        line = {
            "metric": f"solves/s at rel. residual {fmt_tol(tol)} (batched {method_name(args.method)})",
            "value": value, "unit": "solves/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32+df64",
            "data": "synthetic",
            "config": {"workload": workload_desc(wl, B, tol), "method": method_name(args.method),
                       "operator": args.operator, "smoother": args.smoother, "x0": args.x0, "tuning": tuning,
                       "batch": B, "n": P.n, "nnzb": P.nnzb, "k": wl.spec.k, "parallelism": f"replicas{world}",
                       "l2": (f"inputs larger than L2 ({vals.numel() * 8 / 1e9:.2f} GB FP64 "
                              f"{'coefficients' if elements else 'values'} per step; per-iteration working set "
                              f"{P.n * B * 8 * 5 / 1e9:.2f} GB of vectors)"),
                       "iters_mean": float(np.mean(iters)), "iters_max": int(np.max(iters)),
                       "relres_max": float(np.max(rel)), "phi_setup_s": round(t_phi, 1),
                       "setup_ms_per_step": round(setup_ms, 2)},
            "gpu_launches": int(launches / max(args.steps, 1)) if args.steps else 0,
            "roofline": roofline, "clocks": clocks,
        }
        line.update(extra)
        line.setdefault("cpu_baseline", None)
        line.setdefault("e2e", None)
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


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


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--no-serve", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--serve-requests", type=int, default=128)
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
    ap.add_argument("--x0", default="zero", choices=["zero", "rom"],
                    help="initial guess: zero, or the POD reduced-order solution Phi K_c^-1 Phi^T b")
    ap.add_argument("--tol", type=float, default=TOL)
    ap.add_argument("--maxit", type=int, default=MAXIT)
    args = ap.parse_args()
    if args.impl == "reference":
        return reference_arm(args)
    return gb300_arm(args)


if __name__ == "__main__":
    sys.exit(main())

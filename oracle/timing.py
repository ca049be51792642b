"""Timed runs of the oracle on the host cores (CPU baseline of the benchmark).

TEST INFRASTRUCTURE: started by bench.py in fresh processes (BLAS threads pinned
to 1), never by the solver library. Two modes:

    python -m oracle.timing <workload> <instance> <iterations|full> <tol> [pcg|stationary] [jacobi|sgs]

runs one single-threaded oracle solve and prints one JSON object: seconds,
iterations run, seconds per iteration, and for a full solve the iteration count
and the true relative residual.

    python -m oracle.timing pool <workload> <workers> <sample_iters> <warmup> <steps> <tol> [pcg|stationary]
                                 [jacobi|sgs]

keeps `workers` single-threaded processes, one parameter instance each (instances
0 .. workers-1 of the workload's query set), all holding their own matrix. Each
process times its oracle set-up (D^-1, K_r = Phi^T K Phi, its Cholesky factor)
once, then, per step, `sample_iters` iterations of the oracle's PCG (or stationary
cycles) from the initial guess; steps start together on all processes. Prints
one JSON object with the set-up seconds and the per-step seconds per iteration
of every process, and the step wall times. The instance matrices are built in
the worker processes, which are forked from this process before it imports any
GPU library (the POD basis is read from the on-disk cache; create it first).
"""
from __future__ import annotations

import json
import os
import sys
import time


def _root():
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    if root not in sys.path:
        sys.path.insert(0, root)
    return root


def _system(wl, inst):
    """The oracle's input for one query instance: FP64 (or FP32-rounded) values, rhs."""
    from synth.rounding import round_f32
    xi = wl.query_thetas(inst + 1)[inst]
    vals = wl.values(xi)
    if wl.spec.precision == "mixed":
        vals = round_f32(vals)
    return vals, wl.rhs(inst + 1)[inst]


def main(argv):
    _root()
    name, inst, mode, tol = argv[0], int(argv[1]), argv[2], float(argv[3])
    method = argv[4] if len(argv) > 4 else "pcg"
    smoother = argv[5] if len(argv) > 5 else "jacobi"
    from oracle import pod2g_oracle as O
    from synth.problems import Workload
    from synth.rounding import round_phi
    from synth.snapshots import pod_basis

    wl = Workload(name)
    phi = round_phi(pod_basis(wl, device="cuda" if wl.n > 20_000 else None), wl.spec.phi_dtype)
    vals, b = _system(wl, inst)
    K = wl.problem.csr(vals)
    maxit = 100000 if mode == "full" else int(mode)
    t0 = time.perf_counter()
    solve = O.pod2g_pcg if method == "pcg" else O.pod2g_stationary
    P = wl.problem
    groups = O.multicolour_groups(P.row_ptr, P.col_idx, P.bs) if smoother == "sgs" else None
    res = solve(K, b, None, phi, wl.spec.omega, tol if mode == "full" else 0.0, maxit, groups=groups)
    dt = time.perf_counter() - t0
    out = dict(workload=name, instance=inst, seconds=dt, iterations=res.iters,
               seconds_per_iteration=dt / max(res.iters, 1), status=res.status, relres=res.relres,
               threads=int(os.environ.get("OMP_NUM_THREADS", "0") or 0))
    print(json.dumps(out))


# ----------------------------------------------------------------------------- pool mode
_SHARED = {}


def _worker(w, inst, sample_iters, nsteps, method, smoother, go, q, build_slots):
    import numpy as np
    import scipy.sparse as sp
    from oracle import pod2g_oracle as O
    wl, phi, indptr, indices, perm = (_SHARED[k] for k in ("wl", "phi", "indptr", "indices", "perm"))
    P = wl.problem
    with build_slots:   # a few instance matrices are built at a time (host memory)
        vals, b = _system(wl, inst)
        data = np.ascontiguousarray(vals.reshape(-1)[perm])
        del vals
    K = sp.csr_matrix((data, indices, indptr), shape=(P.n, P.n))
    groups = O.multicolour_groups(P.row_ptr, P.col_idx, P.bs) if smoother == "sgs" else None
    t0 = time.perf_counter()
    st = O.pod2g_setup(K, phi, wl.spec.omega, 1, 1, groups)
    setup_s = time.perf_counter() - t0
    q.put(("ready", w, setup_s))
    per = []
    for s in range(nsteps):
        go.wait()
        t0 = time.perf_counter()
        if method == "pcg":
            res = O.pcg(K, b, None, O.pod2g_preconditioner(K, st), 0.0, sample_iters)
        else:
            res = O.pod2g_stationary(K, b, None, phi, wl.spec.omega, 0.0, sample_iters, groups=groups)
        dt = time.perf_counter() - t0
        per.append(dt / max(res.iters, 1))
        q.put(("step", w, s, dt / max(res.iters, 1)))
    q.put(("done", w, per))


def pool(argv):
    _root()
    name, workers, sample_iters, warmup, steps, tol = (argv[0], int(argv[1]), int(argv[2]), int(argv[3]),
                                                       int(argv[4]), float(argv[5]))
    method = argv[6] if len(argv) > 6 else "pcg"
    smoother = argv[7] if len(argv) > 7 else "jacobi"
    import multiprocessing as mp

    import numpy as np
    import scipy.sparse as sp
    from synth.problems import Workload
    from synth.rounding import round_phi
    from synth.snapshots import pod_basis
    wl = Workload(name)
    P = wl.problem
    phi = round_phi(pod_basis(wl, cached_only=True), wl.spec.phi_dtype)
    # the CSR pattern of the (identical) instance patterns and the BSR -> CSR value order, shared
    bs = P.bs
    tag = np.arange(1, P.nnzb * bs * bs + 1, dtype=np.float64).reshape(P.nnzb, bs, bs)
    A = sp.bsr_matrix((tag, P.col_idx, P.row_ptr), shape=(P.n, P.n)).tocsr()
    A.sort_indices()
    _SHARED.update(wl=wl, phi=phi, indptr=A.indptr, indices=A.indices, perm=(A.data - 1).astype(np.int64))
    del A, tag
    ctx = mp.get_context("fork")   # this process has not initialised any GPU library
    nsteps = warmup + steps
    go = ctx.Barrier(workers + 1)
    q = ctx.Queue()
    build_slots = ctx.Semaphore(4)
    procs = [ctx.Process(target=_worker, args=(w, w, sample_iters, nsteps, method, smoother, go, q, build_slots))
             for w in range(workers)]
    t_start = time.perf_counter()
    for p in procs:
        p.start()
    setup = {}
    while len(setup) < workers:
        msg = q.get(timeout=3600)
        if msg[0] == "ready":
            setup[msg[1]] = msg[2]
    t_ready = time.perf_counter() - t_start
    walls = []
    per_step = [[None] * workers for _ in range(nsteps)]
    for s in range(nsteps):
        t0 = time.perf_counter()
        go.wait(timeout=3600)
        got = 0
        while got < workers:
            msg = q.get(timeout=3600)
            if msg[0] == "step":
                per_step[msg[2]][msg[1]] = msg[3]
                got += 1
        walls.append(time.perf_counter() - t0)
    for p in procs:
        p.join(timeout=600)
    out = dict(workload=name, workers=workers, sample_iters=sample_iters, warmup=warmup, steps=steps,
               setup_s=[setup[w] for w in range(workers)], prepare_s=t_ready,
               seconds_per_iteration=per_step[warmup:], step_wall_s=walls[warmup:],
               threads=int(os.environ.get("OMP_NUM_THREADS", "0") or 0))
    print(json.dumps(out))


if __name__ == "__main__":
    if len(sys.argv) > 1 and sys.argv[1] == "pool":
        pool(sys.argv[2:])
    else:
        main(sys.argv[1:])

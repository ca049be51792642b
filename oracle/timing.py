"""Timed runs of the oracle on the host cores (CPU baseline of the benchmark).

TEST INFRASTRUCTURE: started by bench.py in fresh single-threaded processes
(BLAS threads pinned to 1), never by the solver library.

    python -m oracle.timing <workload> <instance> <iterations|full> <tol> [pcg|stationary] [jacobi|sgs]

prints one JSON object: seconds, iterations run, seconds per iteration, and for
a full solve the iteration count and the true relative residual.
"""
from __future__ import annotations

import json
import os
import sys
import time


def main(argv):
    name, inst, mode, tol = argv[0], int(argv[1]), argv[2], float(argv[3])
    method = argv[4] if len(argv) > 4 else "pcg"
    smoother = argv[5] if len(argv) > 5 else "jacobi"
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    if root not in sys.path:
        sys.path.insert(0, root)
    import numpy as np
    from oracle import pod2g_oracle as O
    from synth.problems import Workload
    from synth.rounding import round_f32, round_phi
    from synth.snapshots import pod_basis

    wl = Workload(name)
    phi = round_phi(pod_basis(wl, device="cuda" if wl.n > 20_000 else None), wl.spec.phi_dtype)
    xi = wl.query_thetas(inst + 1)[inst]
    vals = wl.values(xi)
    if wl.spec.precision == "mixed":
        vals = round_f32(vals)
    K = wl.problem.csr(vals)
    b = wl.rhs(inst + 1)[inst]
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


if __name__ == "__main__":
    main(sys.argv[1:])

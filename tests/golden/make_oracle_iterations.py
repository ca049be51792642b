"""Writes tests/golden/oracle_iterations.json: the FP64 oracle's own full-solve iteration counts.

For a workload whose oracle solve takes minutes (the 3D Hex8 128^3 elasticity problem), tests and
the benchmark's CPU baseline read these stored counts instead of re-running the oracle. Every value
here comes from oracle/pod2g_oracle.py (Algorithm 3 with the two-grid cycle of Algorithm 2), run on
the inputs the synthetic generator gives (FP32-rounded values and basis for mixed workloads); the
CUDA library is not involved. Each instance runs in its own single-threaded process.

    python tests/golden/make_oracle_iterations.py <workload> <instances> [tol]

The POD basis is computed first (snapshot solves on a CUDA device through torch, as the tests do);
its SHA-256 over the rounded FP64 bytes is stored beside the counts.
"""
from __future__ import annotations

import hashlib
import json
import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
OUT = os.path.join(HERE, "oracle_iterations.json")


def phi_digest(wl):
    import numpy as np
    from synth.rounding import round_phi
    from synth.snapshots import pod_basis
    phi = round_phi(pod_basis(wl, device="cuda" if wl.n > 20_000 else None), wl.spec.phi_dtype)
    return hashlib.sha256(np.ascontiguousarray(phi).tobytes()).hexdigest()


def main(argv):
    sys.path.insert(0, ROOT)
    from synth.problems import Workload
    name, count = argv[0], int(argv[1])
    tol = float(argv[2]) if len(argv) > 2 else 1e-8
    wl = Workload(name)
    digest = phi_digest(wl)
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")

    def full(i):
        r = subprocess.run([sys.executable, "-m", "oracle.timing", name, str(i), "full", str(tol), "pcg", "jacobi"],
                           cwd=ROOT, env=env, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(r.stderr[-2000:])
        return json.loads(r.stdout.strip().splitlines()[-1])

    with ThreadPoolExecutor(count) as ex:
        res = list(ex.map(full, range(count)))
    data = json.load(open(OUT)) if os.path.exists(OUT) else {}
    data[name] = {"tol": tol, "method": "pcg", "smoother": "jacobi", "phi_sha256": digest,
                  "iterations": {str(r["instance"]): r["iterations"] for r in res},
                  "status": {str(r["instance"]): r["status"] for r in res},
                  "relres": {str(r["instance"]): r["relres"] for r in res},
                  "seconds": {str(r["instance"]): round(r["seconds"], 1) for r in res},
                  "writer": "tests/golden/make_oracle_iterations.py (oracle/pod2g_oracle.py only)"}
    with open(OUT, "w") as f:
        json.dump(data, f, indent=1, sort_keys=True)
    print(json.dumps(data[name]))


if __name__ == "__main__":
    main(sys.argv[1:])

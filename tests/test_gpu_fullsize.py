"""Parity at the benchmark's full size and launch configuration.

2D plane-stress Q4 on a 512 x 512 grid (526,338 unknowns, 2,362,369 blocks), POD basis
k = 20 from 200 snapshots, 64 instances solved together exactly as bench.py does
(device-resident FP64 values through pod2g_set_values_batch_dev, launch shapes from
pod2g_autotune, pod2g_solve_batch_dev, tol 1e-8). Checks:
  * every instance: status OK, the library's final residual (computed in FP64 on the
    device) equals an independent FP64 CPU residual ||b - K x|| / ||b|| of the returned x
    (K from the FP32-rounded values the mixed path solves) within the FP64 rounding-error
    bound of the two summation orders, and it is <= 1.05e-8;
  * a sampled instance against the FP64 oracle run on the same rounded values and
    rounded basis: relative 2-norm error of x <= 1e-6 and iteration counts within +-2.
The same checks run for the 3D Hex8 64^3 workload (823,875 unknowns, 32 instances, BF16 basis,
k = 30) and the 2D diffusion Q1 1024^2 workload (1,046,529 unknowns, 16 instances, k = 25). For the 3D Hex8 128^3 workload (6,440,067 unknowns, 57,066,625 blocks, 4 instances,
k = 40), where one oracle solve takes about a quarter of an hour on one core, the iteration
counts are compared with the oracle's own stored counts (tests/golden/oracle_iterations.json,
written by a script that runs only the oracle) within +-2, and every instance passes the FP64
residual checks above.
"""
import json
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu, pytest.mark.slow]

from oracle import pod2g_oracle as O  # noqa: E402
from synth.problems import Workload  # noqa: E402
from synth.rounding import round_f32, round_phi  # noqa: E402
from synth.snapshots import pod_basis  # noqa: E402

TOL = 1e-8


@pytest.fixture(scope="module")
def pkg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import paper_2207_02543_gb300 as p
    return p


GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "oracle_iterations.json")


def _run_batch(pkg, name, sample, golden=False):
    wl = Workload(name)
    P = wl.problem
    B = wl.spec.batch
    Phi = pod_basis(wl, device="cuda")
    prec = pkg.MIXED_BF16PHI if wl.spec.phi_dtype == "bf16" else pkg.MIXED_FP32PHI
    xis = wl.query_thetas(B)
    vals = wl.values_torch(xis, device="cuda").reshape(B, -1).contiguous()
    b = torch.from_numpy(wl.rhs(B)).cuda()
    x = torch.empty_like(b)
    s = pkg.Solver(P.row_ptr, P.col_idx, P.bs, Phi, precision=prec, omega=wl.spec.omega, max_batch=B)
    slots = list(range(B))
    st, sts = s.set_values_batch_dev(slots, vals)
    assert st == pkg.OK
    # the launch shapes bench.py times: picked by the autotuner on this workload
    st, shape = s.autotune(slots, b, iters=32)
    assert st == pkg.OK
    iters, rel, status, rc = s.solve_batch_dev(slots, b, x, tol=TOL, maxit=5000)
    s.close()
    assert rc == pkg.OK and np.all(status == 0)
    X = x.cpu().numpy()
    bh = b.cpu().numpy()
    for i in range(B):
        v = round_f32(vals[i].cpu().numpy()).reshape(-1, P.bs, P.bs)
        K = P.csr(v)
        bn = np.linalg.norm(bh[i])
        true_rel = np.linalg.norm(bh[i] - K @ X[i]) / bn
        # Both sides compute b - K x in FP64 from the same FP32 values and the same x, in
        # different summation orders. A row of m terms computed in FP64 is within
        # gamma_m (|K||x| + |b|)_i of the exact value (gamma_m = m u / (1 - m u), u = 2^-53),
        # so the two relative residuals differ by at most 2 gamma_m ||(|K||x| + |b|)|| / ||b||.
        m = int(np.max(np.diff(K.indptr))) + 1
        u = 2.0 ** -53
        scale = np.linalg.norm(abs(K) @ np.abs(X[i]) + np.abs(bh[i])) / bn
        bound = 2 * (m * u / (1 - m * u)) * scale
        assert true_rel <= 1.05 * TOL + bound, (i, true_rel, bound)
        assert abs(true_rel - rel[i]) <= bound, (i, true_rel, rel[i], bound)
    if golden:
        g = json.load(open(GOLDEN))[name]
        assert g["tol"] == TOL and g["method"] == "pcg" and g["smoother"] == "jacobi"
        for i in range(B):
            assert abs(int(iters[i]) - int(g["iterations"][str(i)])) <= 2, (i, iters[i], g["iterations"][str(i)])
    phi_used = round_phi(Phi, wl.spec.phi_dtype)
    for i in sample:
        K = P.csr(round_f32(vals[i].cpu().numpy()).reshape(-1, P.bs, P.bs))
        ref = O.pod2g_pcg(K, bh[i], None, phi_used, wl.spec.omega, TOL, 5000)
        print(f"instance {i}: gpu iters {iters[i]} oracle iters {ref.iters}; oracle history tail "
              f"{[f'{h:.3e}' for h in ref.history[-40:]]}")
        assert ref.status == O.OK
        err = np.linalg.norm(X[i] - ref.x) / np.linalg.norm(ref.x)
        assert err <= 1e-6, (i, err)
        assert abs(int(iters[i]) - ref.iters) <= 2, (i, iters[i], ref.iters)


def test_q4_512_batch64_full_size(pkg):
    _run_batch(pkg, "q4_512", sample=[37])


def test_hex8_64_batch32_full_size(pkg):
    # 3D Hex8 elasticity 64^3 (823,875 unknowns, 3x3 BSR), k = 30 from 300 snapshots, BF16 basis, 32 instances
    _run_batch(pkg, "hex8_64", sample=[5])


def test_q1_1024_batch16_full_size(pkg):
    # 2D diffusion Q1 1024^2 (1,046,529 unknowns, scalar rows), k = 25 from 250 snapshots, 16 instances:
    # the third problem of the serving mix
    _run_batch(pkg, "q1_1024", sample=[3])


def test_hex8_128_batch4_full_size(pkg):
    # 3D Hex8 elasticity 128^3 (6,440,067 unknowns), k = 40 from 400 snapshots, FP32 basis, 4 instances
    _run_batch(pkg, "hex8_128", sample=[], golden=True)

"""Serving mix: requests for three registered problems of different sizes and block
sizes (Q4 2D elasticity, Hex8 3D elasticity with a BF16 basis, Q1 diffusion),
admitted under one HBM budget and batched per problem on the fly while the other
problems' work is on the device. Every result must be the one the same instance
gets when solved alone (bit-identical: a slot's arithmetic does not depend on the
other slots), and a problem that does not fit the remaining budget is refused."""
import time

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from synth.problems import Workload  # noqa: E402
from synth.rounding import round_f32  # noqa: E402
from synth.snapshots import pod_basis  # noqa: E402


@pytest.fixture(scope="module")
def pkg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import paper_2207_02543_gb300 as p
    return p


def test_mix_of_three_problems(pkg):
    names = {"q4_16": pkg.MIXED_FP32PHI, "hex8_8": pkg.MIXED_BF16PHI, "q1_32": pkg.MIXED_FP32PHI}
    per = 5
    mix = pkg.ServingMix(hbm_budget=2 << 30)
    reqs, alone = [], {}
    wls = {}
    for name, prec in names.items():
        wl = Workload(name)
        wls[name] = wl
        P = wl.problem
        Phi = pod_basis(wl, use_disk=False)
        kw = dict(precision=prec, omega=wl.spec.omega, max_batch=3, chunk=4)
        # reference: each instance alone in a context of the same shape
        ref = pkg.Solver(P.row_ptr, P.col_idx, P.bs, Phi, **kw)
        xis = wl.query_thetas(per)
        B = wl.rhs(per)
        for i in range(per):
            v = round_f32(wl.values(xis[i]))
            assert ref.set_values(0, v) == pkg.OK
            alone[(name, i)] = ref.solve(0, B[i], tol=1e-8, maxit=3000)
            reqs.append((name, i, v, B[i]))
        ref.close()
        assert mix.register(name, P.row_ptr, P.col_idx, P.bs, Phi, **kw) == pkg.OK
    # interleave the problems' requests, submitted while earlier ones are running
    order = sorted(range(len(reqs)), key=lambda j: (reqs[j][1], j))
    handles = {}
    for j in order:
        name, i, v, b = reqs[j]
        st, h = mix.submit(name, v, b, tol=1e-8, maxit=3000)
        assert st == pkg.OK
        handles[(name, i)] = h
    done = {}
    t0 = time.time()
    while len(done) < len(handles) and time.time() - t0 < 120:
        for key, h in handles.items():
            if key in done:
                continue
            st, r = mix.poll(h)
            if st == pkg.OK:
                done[key] = r
        time.sleep(0.001)
    assert len(done) == len(handles)
    for key, r in done.items():
        x, it, rel, st = alone[key]
        assert r["status"] == pkg.OK and st == pkg.OK
        assert r["iters"] == it and np.array_equal(r["x"], x), key
    # admission: a problem that does not fit the remaining budget is refused
    used = mix.used_bytes()
    tight = pkg.ServingMix(hbm_budget=used // 8)
    wl = wls["q4_16"]
    P = wl.problem
    st = tight.register("big", P.row_ptr, P.col_idx, P.bs, pod_basis(wl, use_disk=False),
                        precision=pkg.MIXED_FP32PHI, max_batch=64)
    assert st == pkg.ADMISSION
    tight.close()
    mix.close()

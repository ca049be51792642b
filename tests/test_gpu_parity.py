"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle on the same
seeded inputs.

Tolerances (stated by the solver's specification): relative 2-norm error of x
<= 1e-7 on the FP64 path, <= 1e-6 on the mixed path at tol 1e-8, iteration
counts within +-2. On the mixed path the oracle is given the FP32-rounded
values and the FP32/BF16-rounded basis, so both solve the same system with the
same coarse space.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import pod2g_oracle as O  # noqa: E402
from synth.problems import Workload  # noqa: E402
from synth.rounding import round_f32, round_phi  # noqa: E402
from synth.snapshots import pod_basis  # noqa: E402
from fp64_residual import assert_relres_matches  # noqa: E402

TOL = 1e-8


@pytest.fixture(scope="module")
def pkg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import paper_2207_02543_gb300 as p
    return p


def _setup(name, count, device="cuda"):
    wl = Workload(name)
    Phi = pod_basis(wl, device=device if wl.n > 20_000 else None)
    return wl, Phi


def _oracle(wl, vals, Phi, b, x0=None, tol=TOL, maxit=5000, pre=1, post=1, beta="fr"):
    K = wl.problem.csr(vals)
    return O.pod2g_pcg(K, b, x0, Phi, wl.spec.omega, tol, maxit, r1=pre, r2=post, beta=beta)


def _relerr(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def test_fp64_plain_path_full_q1_64(pkg):
    wl, Phi = _setup("q1_64", 1)
    P = wl.problem
    xi = wl.query_thetas(1)[0]
    vals = wl.values(xi)
    b = wl.rhs(1)[0]
    s = pkg.Solver(P.row_ptr, P.col_idx, P.bs, Phi, precision=pkg.FP64, omega=wl.spec.omega, max_batch=1)
    assert s.set_values(0, vals) == pkg.OK
    x, it, rel, st = s.solve(0, b, tol=TOL, maxit=1000)
    ref = _oracle(wl, vals, Phi, b)
    assert st == pkg.OK and ref.status == O.OK
    assert _relerr(x, ref.x) <= 1e-7
    assert abs(it - ref.iters) <= 2
    assert rel <= 1.01 * TOL and abs(rel - ref.relres) <= 1e-9
    s.close()


@pytest.mark.parametrize("name,precision", [("q1_32", 1), ("q4_16", 1), ("q4_64", 1), ("hex8_8", 2),
                                            ("hex8_8", 1)])
def test_mixed_batched_matches_oracle(pkg, name, precision):
    wl, Phi = _setup(name, 1)
    P = wl.problem
    m = wl.spec.batch
    xis = wl.query_thetas(m)
    Bm = wl.rhs(m)
    phi_used = round_phi(Phi, "bf16" if precision == pkg.MIXED_BF16PHI else "f32")
    s = pkg.Solver(P.row_ptr, P.col_idx, P.bs, Phi, precision=precision, omega=wl.spec.omega, max_batch=m)
    vals = [round_f32(wl.values(xi)) for xi in xis]
    for i in range(m):
        assert s.set_values(i, vals[i]) == pkg.OK
    X, iters, rel, st, rc = s.solve_batch(list(range(m)), Bm, tol=TOL, maxit=3000)
    assert rc == pkg.OK
    for i in range(m):
        ref = _oracle(wl, vals[i], phi_used, Bm[i])
        assert ref.status == O.OK
        assert _relerr(X[i], ref.x) <= 1e-6, (i, _relerr(X[i], ref.x))
        assert abs(int(iters[i]) - ref.iters) <= 2, (i, iters[i], ref.iters)
        assert rel[i] <= 1.05 * TOL
        assert_relres_matches(wl.problem.csr(vals[i]), Bm[i], X[i], rel[i], TOL)
    s.close()


@pytest.mark.parametrize("name,precision", [("hex8_32", 2), ("q1_128", 1)])
def test_mixed_batched_many_lanes(pkg, name, precision):
    """The lane counts of the 3D elasticity (3x3 blocks, 32 slots, k = 30, BF16 basis) and 2D
    diffusion (scalar, 16 slots, k = 25) workloads at moderate size: every instance through the
    FP64 residual check, a sample of instances against the oracle."""
    wl, Phi = _setup(name, 1)
    P = wl.problem
    m = wl.spec.batch
    xis = wl.query_thetas(m)
    Bm = wl.rhs(m)
    phi_used = round_phi(Phi, "bf16" if precision == pkg.MIXED_BF16PHI else "f32")
    s = pkg.Solver(P.row_ptr, P.col_idx, P.bs, Phi, precision=precision, omega=wl.spec.omega, max_batch=m)
    vals = [round_f32(wl.values(xi)) for xi in xis]
    for i in range(m):
        assert s.set_values(i, vals[i]) == pkg.OK
    X, iters, rel, st, rc = s.solve_batch(list(range(m)), Bm, tol=TOL, maxit=5000)
    assert rc == pkg.OK and np.all(st == pkg.OK)
    s.close()
    for i in range(m):
        assert_relres_matches(P.csr(vals[i]), Bm[i], X[i], rel[i], TOL)
    for i in sorted({0, m // 2 + 1, m - 1}):
        ref = _oracle(wl, vals[i], phi_used, Bm[i])
        assert ref.status == O.OK
        assert _relerr(X[i], ref.x) <= 1e-6, (i, _relerr(X[i], ref.x))
        assert abs(int(iters[i]) - ref.iters) <= 2, (i, iters[i], ref.iters)


def test_result_identical_alone_and_in_mix(pkg):
    wl, Phi = _setup("q4_16", 1)
    P = wl.problem
    xis = wl.query_thetas(4)
    Bm = wl.rhs(4)
    s = pkg.Solver(P.row_ptr, P.col_idx, P.bs, Phi, precision=pkg.MIXED_FP32PHI, omega=wl.spec.omega, max_batch=4)
    vals = [round_f32(wl.values(xi)) for xi in xis]
    # instance 0 alone in slot 0
    assert s.set_values(0, vals[0]) == pkg.OK
    xa, ita, ra, sa = s.solve(0, Bm[0], tol=TOL, maxit=2000)
    # the same instance in slot 3, next to three others
    for i, slot in enumerate([3, 0, 1, 2]):
        assert s.set_values(slot, vals[i]) == pkg.OK
    X, iters, rel, st, rc = s.solve_batch([3, 0, 1, 2], Bm, tol=TOL, maxit=2000)
    assert rc == pkg.OK
    assert np.array_equal(X[0], xa) and iters[0] == ita
    s.close()


def test_edge_cases(pkg):
    wl, Phi = _setup("q4_16", 1)
    P = wl.problem
    n = P.n
    s = pkg.Solver(P.row_ptr, P.col_idx, P.bs, Phi, precision=pkg.MIXED_FP32PHI, omega=wl.spec.omega, max_batch=3)
    vals = round_f32(wl.values(wl.query_thetas(1)[0]))
    for i in range(3):
        assert s.set_values(i, vals) == pkg.OK
    b = wl.rhs(1)[0]
    # b = 0 -> x = 0, 0 iterations
    x, it, rel, st = s.solve(0, np.zeros(n), x0=np.ones(n), tol=TOL)
    assert st == pkg.OK and it == 0 and np.all(x == 0) and rel == 0.0
    # x0 = converged solution -> 0 iterations
    x1, it1, rel1, st1 = s.solve(1, b, tol=1e-10, maxit=2000)
    assert st1 == pkg.OK
    x2, it2, rel2, st2 = s.solve(1, b, x0=x1, tol=1e-8, maxit=2000)
    assert st2 == pkg.OK and it2 == 0
    # maxit exhaustion -> NOT_CONVERGED after exactly maxit iterations, last iterate returned
    x3, it3, rel3, st3 = s.solve(2, b, tol=1e-14, maxit=5)
    assert st3 == pkg.NOT_CONVERGED and it3 == 5 and np.all(np.isfinite(x3))
    ref = _oracle(wl, vals, round_phi(Phi, "f32"), b, tol=1e-14, maxit=5)
    assert ref.iters == 5 and _relerr(x3, ref.x) <= 1e-6
    # NaN right-hand side -> NONFINITE
    bn = b.copy(); bn[3] = np.nan
    x4, it4, rel4, st4 = s.solve(0, bn, tol=TOL)
    assert st4 == pkg.NONFINITE
    # invalid slot
    assert s.solve(7, b)[3] == pkg.INVALID_ARG
    s.close()


def test_dependent_basis_is_not_spd(pkg):
    wl, Phi = _setup("q4_16", 1)
    P = wl.problem
    dep = np.column_stack([Phi[:, 0], Phi[:, 0], Phi[:, 1]])
    for prec in (pkg.FP64, pkg.MIXED_FP32PHI):
        s = pkg.Solver(P.row_ptr, P.col_idx, P.bs, dep, precision=prec, omega=wl.spec.omega, max_batch=1)
        assert s.set_values(0, wl.values(wl.query_thetas(1)[0])) == pkg.NOT_SPD
        assert s.solve(0, wl.rhs(1)[0])[3] == pkg.INVALID_ARG  # slot without a valid set-up
        s.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_one_iteration_when_rhs_in_range_without_presmoothing(pkg, precision):
    wl, Phi = _setup("q4_16", 1)
    P = wl.problem
    vals = round_f32(wl.values(wl.query_thetas(1)[0]))
    phi_used = round_phi(Phi, "f32")
    K = P.csr(vals)
    c = np.linspace(1.0, -1.0, Phi.shape[1])
    b = K @ (phi_used @ c)
    s = pkg.Solver(P.row_ptr, P.col_idx, P.bs, phi_used, precision=precision, omega=wl.spec.omega, pre=0, post=1)
    assert s.set_values(0, vals) == pkg.OK
    tol = 1e-10 if precision == pkg.FP64 else 1e-4   # the mixed preconditioner is exact to FP32 only
    x, it, rel, st = s.solve(0, b, tol=tol, maxit=50)
    assert st == pkg.OK and it == 1
    assert _relerr(x, phi_used @ c) <= (1e-9 if precision == pkg.FP64 else 1e-4)
    s.close()


def test_no_coarse_space_and_sweep_variants(pkg):
    wl, Phi = _setup("q1_32", 1)
    P = wl.problem
    vals = round_f32(wl.values(wl.query_thetas(1)[0]))
    b = wl.rhs(1)[0]
    for pre, post, k in [(1, 1, 0), (0, 1, 4), (1, 0, 4)]:
        ph = round_phi(Phi[:, :k], "f32")
        ref = _oracle(wl, vals, ph, b, pre=pre, post=post)
        for prec in (pkg.FP64, pkg.MIXED_FP32PHI):
            s = pkg.Solver(P.row_ptr, P.col_idx, P.bs, ph, precision=prec, omega=wl.spec.omega, pre=pre, post=post)
            assert s.set_values(0, vals) == pkg.OK
            x, it, rel, st = s.solve(0, b, tol=TOL, maxit=3000)
            assert st == pkg.OK and abs(it - ref.iters) <= 2, (pre, post, k, prec, it, ref.iters)
            assert _relerr(x, ref.x) <= (1e-7 if prec == pkg.FP64 else 1e-6)
            s.close()


def test_polak_ribiere_option(pkg):
    wl, Phi = _setup("q4_16", 1)
    P = wl.problem
    vals = round_f32(wl.values(wl.query_thetas(1)[0]))
    b = wl.rhs(1)[0]
    ref = _oracle(wl, vals, round_phi(Phi, "f32"), b, beta="pr")
    for prec in (pkg.FP64, pkg.MIXED_FP32PHI):
        s = pkg.Solver(P.row_ptr, P.col_idx, P.bs, Phi, precision=prec, omega=wl.spec.omega, beta_pr=True)
        assert s.set_values(0, vals) == pkg.OK
        x, it, rel, st = s.solve(0, b, tol=TOL, maxit=2000)
        assert st == pkg.OK and abs(it - ref.iters) <= 2
        assert _relerr(x, ref.x) <= 1e-6
        s.close()


def test_device_entry_points(pkg):
    wl, Phi = _setup("q4_16", 1)
    P = wl.problem
    m = 3
    xis = wl.query_thetas(m)
    vals = np.stack([round_f32(wl.values(xi)) for xi in xis])
    Bm = wl.rhs(m)
    s = pkg.Solver(P.row_ptr, P.col_idx, P.bs, Phi, precision=pkg.MIXED_FP32PHI, omega=wl.spec.omega, max_batch=4)
    vd = torch.from_numpy(vals.reshape(m, -1)).cuda()
    st, sts = s.set_values_batch_dev([2, 0, 1], vd)
    assert st == pkg.OK and np.all(sts == 0)
    bd = torch.from_numpy(Bm).cuda()
    xd = torch.empty_like(bd)
    iters, rel, status, rc = s.solve_batch_dev([2, 0, 1], bd, xd, tol=TOL, maxit=2000)
    assert rc == pkg.OK
    X, iters_h, rel_h, st_h, rc_h = s.solve_batch([2, 0, 1], Bm, tol=TOL, maxit=2000)
    assert np.array_equal(xd.cpu().numpy(), X) and np.array_equal(iters, iters_h)
    s.close()


def test_serving_continuous_batching_matches_batch(pkg):
    wl, Phi = _setup("q4_16", 1)
    P = wl.problem
    m = 7
    xis = wl.query_thetas(m)
    vals = [round_f32(wl.values(xi)) for xi in xis]
    Bm = wl.rhs(m)
    s = pkg.Solver(P.row_ptr, P.col_idx, P.bs, Phi, precision=pkg.MIXED_FP32PHI, omega=wl.spec.omega, max_batch=2,
                   chunk=4)
    # reference: each instance solved alone in slot 0
    alone = []
    for i in range(m):
        assert s.set_values(0, vals[i]) == pkg.OK
        alone.append(s.solve(0, Bm[i], tol=TOL, maxit=2000))
    s.serve_start(max_queue=16)
    tickets = []
    for i in range(m):
        st, t = s.submit(vals[i], Bm[i], tol=TOL, maxit=2000)
        assert st == pkg.OK
        tickets.append(t)
    import time
    res = {}
    t0 = time.time()
    while len(res) < m and time.time() - t0 < 60:
        for i, t in enumerate(tickets):
            if i in res:
                continue
            st, r = s.poll(t)
            if st == pkg.OK:
                res[i] = r
        time.sleep(0.001)
    s.serve_stop()
    assert len(res) == m
    for i in range(m):
        r = res[i]
        assert r["status"] == pkg.OK
        assert np.array_equal(r["x"], alone[i][0]) and r["iters"] == alone[i][1]
        assert r["latency_s"] > 0
    s.close()


def test_serving_admission_limit(pkg):
    wl, Phi = _setup("q4_16", 1)
    P = wl.problem
    s = pkg.Solver(P.row_ptr, P.col_idx, P.bs, Phi, precision=pkg.MIXED_FP32PHI, omega=wl.spec.omega, max_batch=1)
    assert pkg.Solver  # context creation over a tiny HBM budget is refused
    with pytest.raises(pkg.Pod2gError) as e:
        pkg.Solver(P.row_ptr, P.col_idx, P.bs, Phi, precision=pkg.MIXED_FP32PHI, max_batch=4, hbm_budget=1 << 16)
    assert e.value.status == pkg.ADMISSION
    s.close()

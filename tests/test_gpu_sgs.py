"""GPU parity of the multicolour symmetric Gauss-Seidel relaxation (eq. GaussSeidel:
forward sweeps before, backward sweeps after the coarse correction, nodes coloured
greedily in index order) through the C ABI, against the oracle's two-grid cycle
with the same sweep order (`multicolour_groups`, `gauss_seidel`).

Tolerances as for the Jacobi path: x within 1e-7 (FP64) / 1e-6 (mixed, tol 1e-8),
iteration counts within +-2.
"""
import time

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import element_operator as EO  # noqa: E402
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


def _relerr(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def _groups(P):
    return O.multicolour_groups(P.row_ptr, P.col_idx, P.bs)


@pytest.mark.parametrize("name,precision,method", [("q1_32", 1, 0), ("q4_16", 1, 0), ("hex8_8", 2, 0),
                                                   ("q4_64", 1, 0), ("q1_32", 1, 1), ("q1_64", 0, 0),
                                                   ("hex8_8", 0, 1), ("hex8_16", 2, 0)])
def test_sgs_matches_oracle(pkg, name, precision, method):
    wl = Workload(name)
    P, Phi = wl.problem, pod_basis(wl)
    fp64 = precision == pkg.FP64
    m = 1 if fp64 else wl.spec.batch
    xis = wl.query_thetas(m)
    Bm = wl.rhs(m)
    vals = [wl.values(xi) if fp64 else round_f32(wl.values(xi)) for xi in xis]
    phi_used = Phi if fp64 else round_phi(Phi, "bf16" if precision == pkg.MIXED_BF16PHI else "f32")
    s = pkg.Solver(P.row_ptr, P.col_idx, P.bs, Phi, precision=precision, omega=wl.spec.omega, max_batch=m,
                   method=method, smoother=pkg.SMOOTHER_SGS)
    for i in range(m):
        assert s.set_values(i, vals[i]) == pkg.OK
    X, it, rel, st, rc = s.solve_batch(list(range(m)), Bm, tol=TOL, maxit=5000)
    assert rc == pkg.OK
    groups = _groups(P)
    solve = O.pod2g_pcg if method == 0 else O.pod2g_stationary
    for i in range(m):
        ref = solve(P.csr(vals[i]), Bm[i], None, phi_used, wl.spec.omega, TOL, 5000, groups=groups)
        assert ref.status == O.OK and st[i] == pkg.OK
        assert abs(it[i] - ref.iters) <= 2, (i, it[i], ref.iters)
        assert _relerr(X[i], ref.x) <= (1e-7 if fp64 else 1e-6)
        assert rel[i] <= 1.01 * TOL
    s.close()


def test_sgs_needs_fewer_iterations_than_jacobi(pkg):
    wl = Workload("q4_64")
    P, Phi = wl.problem, pod_basis(wl)
    vals = round_f32(wl.values(wl.query_thetas(1)[0]))
    b = wl.rhs(1)[0]
    its = {}
    for sm in (pkg.SMOOTHER_JACOBI, pkg.SMOOTHER_SGS):
        s = pkg.Solver(P.row_ptr, P.col_idx, P.bs, Phi, omega=wl.spec.omega, smoother=sm)
        assert s.set_values(0, vals) == pkg.OK
        x, it, rel, st = s.solve(0, b, tol=TOL, maxit=3000)
        assert st == pkg.OK
        its[sm] = it
        s.close()
    assert its[pkg.SMOOTHER_SGS] < its[pkg.SMOOTHER_JACOBI]


def test_sgs_element_operator_bit_identical_to_assembled(pkg):
    wl = Workload("q4_16")
    P, Phi = wl.problem, pod_basis(wl)
    m = wl.spec.batch
    coefs = [wl.coef(xi) for xi in wl.query_thetas(m)]
    Bm = wl.rhs(m)
    el = {"conn": P.conn, "k_ref": P.Kref, "fixed": P.clamped}
    kw = dict(omega=wl.spec.omega, max_batch=m, smoother=pkg.SMOOTHER_SGS)
    se = pkg.Solver(P.row_ptr, P.col_idx, P.bs, Phi, elements=el, **kw)
    sa = pkg.Solver(P.row_ptr, P.col_idx, P.bs, Phi, **kw)
    for i in range(m):
        assert se.set_coeffs(i, coefs[i]) == pkg.OK
        v32 = EO.element_values_f32(P.row_ptr, P.col_idx, P.conn, P.npe, P.bs, P.Kref, coefs[i], P.clamped)
        assert sa.set_values(i, v32) == pkg.OK
    Xe, ie, *_ = se.solve_batch(list(range(m)), Bm, tol=TOL, maxit=3000)
    Xa, ia, *_ = sa.solve_batch(list(range(m)), Bm, tol=TOL, maxit=3000)
    assert list(ie) == list(ia) and np.array_equal(Xe, Xa)
    se.close()
    sa.close()


def test_sgs_serving_matches_batch(pkg):
    """Sweeps touch only the lanes they run for: a request joining a running batch
    gets the result it gets in a batch of its own (same slot count)."""
    wl = Workload("q1_32")
    P, Phi = wl.problem, pod_basis(wl)
    m = 6
    vals = [round_f32(wl.values(xi)) for xi in wl.query_thetas(m)]
    Bm = wl.rhs(m)
    kw = dict(omega=wl.spec.omega, max_batch=3, chunk=4, smoother=pkg.SMOOTHER_SGS)
    se = pkg.Solver(P.row_ptr, P.col_idx, P.bs, Phi, **kw)
    X, it = np.zeros((m, P.n)), np.zeros(m, dtype=int)
    for g in range(0, m, 3):
        for i in range(3):
            assert se.set_values(i, vals[g + i]) == pkg.OK
        Xg, itg, rel, st, rc = se.solve_batch([0, 1, 2], Bm[g:g + 3], tol=TOL, maxit=3000)
        assert rc == pkg.OK
        X[g:g + 3], it[g:g + 3] = Xg, itg
    srv = pkg.Solver(P.row_ptr, P.col_idx, P.bs, Phi, **kw)
    srv.serve_start(max_queue=16)
    tickets = []
    for i in range(m):
        s_, t = srv.submit(vals[i], Bm[i], tol=TOL, maxit=3000)
        assert s_ == pkg.OK
        tickets.append(t)
    done, t0 = {}, time.time()
    while len(done) < m and time.time() - t0 < 60:
        for i, t in enumerate(tickets):
            if i not in done:
                s_, r = srv.poll(t)
                if s_ == pkg.OK:
                    done[i] = r
        time.sleep(0.002)
    srv.serve_stop()
    assert len(done) == m
    for i in range(m):
        assert done[i]["status"] == pkg.OK and done[i]["iters"] == it[i]
        assert np.array_equal(done[i]["x"], X[i])
    se.close()
    srv.close()


def test_sgs_option_checks(pkg):
    wl = Workload("q4_16")
    P, Phi = wl.problem, pod_basis(wl)
    with pytest.raises(pkg.Pod2gError) as e:
        pkg.Solver(P.row_ptr, P.col_idx, P.bs, Phi, smoother=pkg.SMOOTHER_SGS, beta_pr=True)
    assert e.value.status == pkg.INVALID_ARG
    with pytest.raises(pkg.Pod2gError) as e:
        pkg.Solver(P.row_ptr, P.col_idx, P.bs, Phi, smoother=5)
    assert e.value.status == pkg.INVALID_ARG

"""Instances set up from parameters theta (element contexts with a registered field
c_e(theta) = exp(mu + sigma * modes[e] . theta), the truncated Karhunen-Loeve form of the
lognormal material fields) through the C ABI.

The coefficients are evaluated on the device in FP64 and rounded to FP32, so the solve
matches the one from host-computed coefficients of the input generator within the
parity tolerances (x <= 1e-6 at tol 1e-8, iterations +-2), and the oracle's solve of the
same system. Serving by theta gives exactly the batch result in a context with the same
slot count.
"""
import time

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import element_operator as EO  # noqa: E402
from oracle import pod2g_oracle as O  # noqa: E402
from synth.problems import Workload  # noqa: E402
from synth.rounding import round_phi  # noqa: E402
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


def _field(wl):
    psi = wl.kl_modes * np.sqrt(wl.kl_lam)[None, :]
    if wl.spec.kind == "q1":
        return psi, 0.0, 1.0
    return psi, wl.mu_g, wl.sigma_g


def _solver(pkg, wl, Phi, m, **kw):
    P = wl.problem
    el = {"conn": P.conn, "k_ref": P.Kref, "fixed": P.clamped if P.dirichlet == "identity" else None}
    s = pkg.Solver(P.row_ptr, P.col_idx, P.bs, Phi, omega=wl.spec.omega, max_batch=m, elements=el, **kw)
    psi, mu, sigma = _field(wl)
    assert s.set_field(psi, mu, sigma) == pkg.OK
    return s


@pytest.mark.parametrize("name", ["q4_16", "hex8_8", "q1_32"])
def test_theta_setup_matches_coefficients_and_oracle(pkg, name):
    wl = Workload(name)
    P, Phi = wl.problem, pod_basis(wl)
    m = wl.spec.batch
    xis = wl.query_thetas(m)
    Bm = wl.rhs(m)
    s = _solver(pkg, wl, Phi, m)
    st, sts = s.set_theta_batch(list(range(m)), xis)
    assert st == pkg.OK and np.all(sts == pkg.OK)
    Xt, it_t, rel, stt, rc = s.solve_batch(list(range(m)), Bm, tol=TOL, maxit=3000)
    assert rc == pkg.OK
    fixed = P.clamped if P.dirichlet == "identity" else None
    phi32 = round_phi(Phi, "f32")
    for i in range(m):
        c = wl.coef(xis[i])
        assert s.set_coeffs(i, c) == pkg.OK
    Xc, it_c, *_ = s.solve_batch(list(range(m)), Bm, tol=TOL, maxit=3000)
    for i in range(m):
        assert abs(int(it_t[i]) - int(it_c[i])) <= 2 and _relerr(Xt[i], Xc[i]) <= 1e-6
        v32 = EO.element_values_f32(P.row_ptr, P.col_idx, P.conn, P.npe, P.bs, P.Kref, wl.coef(xis[i]), fixed)
        ref = O.pod2g_pcg(P.csr(v32), Bm[i], None, phi32, wl.spec.omega, TOL, 3000)
        assert abs(int(it_t[i]) - ref.iters) <= 2 and _relerr(Xt[i], ref.x) <= 1e-6
    s.close()


def test_serving_by_theta_matches_batch(pkg):
    wl = Workload("q4_16")
    P, Phi = wl.problem, pod_basis(wl)
    m = 6
    xis = wl.query_thetas(m)
    Bm = wl.rhs(m)
    s = _solver(pkg, wl, Phi, 3, chunk=4)
    X, it = np.zeros((m, P.n)), np.zeros(m, dtype=int)
    for g in range(0, m, 3):
        st, _ = s.set_theta_batch([0, 1, 2], xis[g:g + 3])
        assert st == pkg.OK
        Xg, itg, _, _, rc = s.solve_batch([0, 1, 2], Bm[g:g + 3], tol=TOL, maxit=3000)
        assert rc == pkg.OK
        X[g:g + 3], it[g:g + 3] = Xg, itg
    srv = _solver(pkg, wl, Phi, 3, chunk=4)
    srv.serve_start(max_queue=16)
    tickets = []
    for i in range(m):
        st, t = srv.submit_theta(xis[i], Bm[i], tol=TOL, maxit=3000)
        assert st == pkg.OK
        tickets.append(t)
    done, t0 = {}, time.time()
    while len(done) < m and time.time() - t0 < 60:
        for i, t in enumerate(tickets):
            if i not in done:
                st, r = srv.poll(t)
                if st == pkg.OK:
                    done[i] = r
        time.sleep(0.002)
    srv.serve_stop()
    assert len(done) == m
    for i in range(m):
        assert done[i]["status"] == pkg.OK and done[i]["iters"] == it[i] and np.array_equal(done[i]["x"], X[i])
    s.close()
    srv.close()


def test_field_errors(pkg):
    wl = Workload("q4_16")
    P, Phi = wl.problem, pod_basis(wl)
    el = {"conn": P.conn, "k_ref": P.Kref, "fixed": P.clamped}
    s = pkg.Solver(P.row_ptr, P.col_idx, P.bs, Phi, elements=el, max_batch=2)
    assert s.set_theta(0, np.zeros(8)) == pkg.INVALID_ARG            # no field registered
    psi, mu, sigma = _field(wl)
    assert s.set_field(psi, 1.0, 1.0, lognormal=False) == pkg.OK
    theta = np.zeros(psi.shape[1])
    theta[0] = -1e3                                                  # drives coefficients negative
    assert s.set_theta(0, theta) == pkg.NOT_SPD
    assert s.set_field(psi, mu, sigma) == pkg.OK                      # a new field replaces the old
    theta[0] = 1e4                                                   # exp overflows
    assert s.set_theta(0, theta) == pkg.NONFINITE
    assert s.set_theta(0, theta[:-1]) == pkg.INVALID_ARG
    s.close()
    a = pkg.Solver(P.row_ptr, P.col_idx, P.bs, Phi)                   # assembled context: no field
    assert a.set_field(psi) == pkg.INVALID_ARG
    a.close()

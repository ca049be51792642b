"""GPU parity of the element-factored operator (K = sum_e c_e K_ref, formed per block
inside the row kernels) through the C ABI.

* The element context and an assembled context given the oracle's FP32 element
  values (oracle/element_operator.py) solve the same FP32 system with the same
  kernels, so iteration counts and x must be bit-identical.
* Against the FP64 oracle solve of that system: relative error of x <= 1e-6 at
  tol 1e-8 and iteration counts within +-2, as for the assembled mixed path.
"""
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


def _elements(P):
    return {"conn": P.conn, "k_ref": P.Kref, "fixed": P.clamped if P.dirichlet == "identity" else None}


def _f32_values(P, coef):
    fixed = P.clamped if P.dirichlet == "identity" else None
    return EO.element_values_f32(P.row_ptr, P.col_idx, P.conn, P.npe, P.bs, P.Kref, coef, fixed)


def _relerr(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


@pytest.mark.parametrize("name,precision,method", [("q1_32", 1, 0), ("q4_16", 1, 0), ("hex8_8", 2, 0),
                                                   ("q4_64", 1, 0), ("q1_32", 1, 1), ("hex8_16", 2, 0),
                                                   ("hex8_16", 2, 1)])
def test_element_path_matches_assembled_and_oracle(pkg, name, precision, method):
    wl = Workload(name)
    P, Phi = wl.problem, pod_basis(wl)
    m = wl.spec.batch
    coefs = [wl.coef(xi) for xi in wl.query_thetas(m)]
    Bm = wl.rhs(m)
    phi_used = round_phi(Phi, "bf16" if precision == pkg.MIXED_BF16PHI else "f32")
    kw = dict(precision=precision, omega=wl.spec.omega, max_batch=m, method=method)
    se = pkg.Solver(P.row_ptr, P.col_idx, P.bs, Phi, elements=_elements(P), **kw)
    sa = pkg.Solver(P.row_ptr, P.col_idx, P.bs, Phi, **kw)
    # element contexts run the per-thread row kernels: compare with the same form and launch shape
    shape = se.get_tuning()
    assert shape["rows_kernel"] == 0
    assert sa.set_tuning(**shape) == pkg.OK
    vals = [_f32_values(P, c) for c in coefs]
    for i in range(m):
        assert se.set_coeffs(i, coefs[i]) == pkg.OK
        assert sa.set_values(i, vals[i]) == pkg.OK
    slots = list(range(m))
    Xe, ie, re, ste, rc = se.solve_batch(slots, Bm, tol=TOL, maxit=5000)
    assert rc == pkg.OK
    Xa, ia, ra, sta, rca = sa.solve_batch(slots, Bm, tol=TOL, maxit=5000)
    assert rca == pkg.OK
    assert list(ie) == list(ia)
    assert np.array_equal(Xe, Xa)
    solve = O.pod2g_pcg if method == 0 else O.pod2g_stationary
    for i in range(m):
        ref = solve(P.csr(vals[i]), Bm[i], None, phi_used, wl.spec.omega, TOL, 5000)
        assert ref.status == O.OK and ste[i] == pkg.OK
        assert abs(ie[i] - ref.iters) <= 2, (i, ie[i], ref.iters)
        assert _relerr(Xe[i], ref.x) <= 1e-6
    se.close()
    sa.close()


def test_element_batch_dev_setup_and_memory(pkg):
    wl = Workload("q4_64")
    P, Phi = wl.problem, pod_basis(wl)
    m = 8
    xis = wl.query_thetas(m)
    C = torch.from_numpy(np.stack([wl.coef(xi) for xi in xis])).cuda()
    B = torch.from_numpy(wl.rhs(m)).cuda()
    X = torch.empty_like(B)
    se = pkg.Solver(P.row_ptr, P.col_idx, P.bs, Phi, elements=_elements(P), max_batch=64, omega=wl.spec.omega)
    sa = pkg.Solver(P.row_ptr, P.col_idx, P.bs, Phi, max_batch=64, omega=wl.spec.omega)
    # the element context holds no per-slot matrix values
    values_bytes = P.nnzb * P.bs * P.bs * 64 * 4
    assert sa.device_bytes() - se.device_bytes() >= 0.9 * values_bytes
    st, sts = se.set_coeffs_batch_dev(list(range(m)), C)
    assert st == pkg.OK and np.all(sts == pkg.OK)
    iters, rel, status, rc = se.solve_batch_dev(list(range(m)), B, X, tol=TOL, maxit=3000)
    assert rc == pkg.OK
    # same result through the host-array entry points
    for i in range(m):
        assert se.set_coeffs(i, C[i].cpu().numpy()) == pkg.OK
    Xh, ih, rh, sth, rch = se.solve_batch(list(range(m)), B.cpu().numpy(), tol=TOL, maxit=3000)
    assert list(ih) == list(iters) and np.array_equal(Xh, X.cpu().numpy())
    se.close()
    sa.close()


def test_element_serving_matches_batch(pkg):
    wl = Workload("q1_32")
    P, Phi = wl.problem, pod_basis(wl)
    m = 6
    coefs = [wl.coef(xi) for xi in wl.query_thetas(m)]
    Bm = wl.rhs(m)
    # same slot count as the serving context (the per-slot summation order depends on
    # the lane stride, i.e. on max_batch, and on nothing else)
    se = pkg.Solver(P.row_ptr, P.col_idx, P.bs, Phi, elements=_elements(P), max_batch=3, omega=wl.spec.omega,
                    chunk=4)
    X, it = np.zeros((m, P.n)), np.zeros(m, dtype=int)
    for g in range(0, m, 3):
        for i in range(3):
            assert se.set_coeffs(i, coefs[g + i]) == pkg.OK
        Xg, itg, rel, st, rc = se.solve_batch([0, 1, 2], Bm[g:g + 3], tol=TOL, maxit=3000)
        assert rc == pkg.OK
        X[g:g + 3], it[g:g + 3] = Xg, itg
    srv = pkg.Solver(P.row_ptr, P.col_idx, P.bs, Phi, elements=_elements(P), max_batch=3, omega=wl.spec.omega,
                     chunk=4)
    srv.serve_start(max_queue=16)
    tickets = []
    for i in range(m):
        s_, t = srv.submit(coefs[i], Bm[i], tol=TOL, maxit=3000)
        assert s_ == pkg.OK
        tickets.append(t)
    import time
    done = {}
    t0 = time.time()
    while len(done) < m and time.time() - t0 < 60:
        for i, t in enumerate(tickets):
            if i in done:
                continue
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


def test_element_description_errors(pkg):
    wl = Workload("q4_16")
    P, Phi = wl.problem, pod_basis(wl)
    el = _elements(P)
    with pytest.raises(pkg.Pod2gError) as e:
        pkg.Solver(P.row_ptr, P.col_idx, P.bs, Phi, elements=el, precision=pkg.FP64)
    assert e.value.status == pkg.INVALID_ARG
    bad = dict(el, conn=el["conn"].copy())
    bad["conn"][0, 3] = P.n_nodes - 1          # couples node 0 with the far corner: no stored block
    with pytest.raises(pkg.Pod2gError) as e:
        pkg.Solver(P.row_ptr, P.col_idx, P.bs, Phi, elements=bad)
    assert e.value.status == pkg.INVALID_ARG
    asym = dict(el, k_ref=el["k_ref"].copy())
    asym["k_ref"][0, 1] += 1.0
    with pytest.raises(pkg.Pod2gError) as e:
        pkg.Solver(P.row_ptr, P.col_idx, P.bs, Phi, elements=asym)
    assert e.value.status == pkg.INVALID_ARG
    se = pkg.Solver(P.row_ptr, P.col_idx, P.bs, Phi, elements=el, max_batch=2)
    assert se.set_values(0, wl.values(wl.query_thetas(1)[0])) == pkg.INVALID_ARG
    c = wl.coef(wl.query_thetas(1)[0])
    c[5] = np.nan
    assert se.set_coeffs(0, c) == pkg.NONFINITE
    assert se.set_coeffs(0, c[:-1]) == pkg.INVALID_ARG
    se.close()

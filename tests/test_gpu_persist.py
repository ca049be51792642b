"""The persistent form of the batched path: whole PCG iterations (Algorithm 3 with the
two-grid preconditioner of Algorithm 2, Section 3.3) in one cooperative launch with
grid-wide barriers between the phases (rows_kernel bit 3, selected explicitly here).

It regroups partial sums only, so the bar is the same as for every launch shape:
relative x error <= 1e-6 against the oracle at tol 1e-8, iteration counts within +-2,
the same against the graph form, deterministic for a given grid, and a slot's result
independent of the other slots.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import pod2g_oracle as O  # noqa: E402
from synth.problems import Workload  # noqa: E402
from synth.rounding import round_f32, round_phi  # noqa: E402
from synth.snapshots import pod_basis  # noqa: E402

TOL = 1e-8
PERSIST = 8


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


def _phi_used(wl, Phi):
    return round_phi(Phi, "bf16" if wl.spec.phi_dtype == "bf16" else "f32")


def _solver(pkg, wl, Phi, m, **kw):
    P = wl.problem
    prec = pkg.MIXED_BF16PHI if wl.spec.phi_dtype == "bf16" else pkg.MIXED_FP32PHI
    s = pkg.Solver(P.row_ptr, P.col_idx, P.bs, Phi, precision=prec, omega=wl.spec.omega, max_batch=m, **kw)
    vals = [round_f32(wl.values(xi)) for xi in wl.query_thetas(m)]
    for i in range(m):
        assert s.set_values(i, vals[i]) == pkg.OK
    return s, vals


@pytest.mark.parametrize("name,m", [("q1_32", 1), ("q1_32", 20), ("q4_16", 3), ("q4_64", 7), ("q4_16", 40),
                                    ("hex8_8", 36), ("hex8_16", 5), ("hex8_16", 1)])
def test_persistent_matches_oracle_and_graph(pkg, name, m):
    wl = Workload(name)
    P, Phi = wl.problem, pod_basis(wl)
    Bm = wl.rhs(m)
    res = {}
    for form in ("persist", "persist", "graph"):
        s, vals = _solver(pkg, wl, Phi, m)
        t = s.get_tuning()
        assert t["grid_persist"] >= 1 and not t["rows_kernel"] & PERSIST   # available, not the default
        if form == "persist":
            assert s.set_tuning(rows_kernel=t["rows_kernel"] | PERSIST) == pkg.OK
        X, it, rel, st, rc = s.solve_batch(list(range(m)), Bm, tol=TOL, maxit=3000)
        assert rc == pkg.OK and np.all(st == pkg.OK)
        assert np.all(rel <= TOL * 1.5)
        s.close()
        if form in res:
            assert np.array_equal(res[form][0], X) and list(res[form][1]) == list(it)   # deterministic
        res[form] = (X, it)
    (Xp, ip), (Xg, ig) = res["persist"], res["graph"]
    for i in range(m):
        assert abs(int(ip[i]) - int(ig[i])) <= 2 and _relerr(Xp[i], Xg[i]) <= 1e-6
    phi_used = _phi_used(wl, Phi)
    for i in sorted({0, m - 1}):
        ref = O.pod2g_pcg(P.csr(vals[i]), Bm[i], None, phi_used, wl.spec.omega, TOL, 3000)
        assert abs(int(ip[i]) - ref.iters) <= 2, (i, ip[i], ref.iters)
        assert _relerr(Xp[i], ref.x) <= 1e-6, (i, _relerr(Xp[i], ref.x))


def test_persistent_grid_sizes(pkg):
    """One CTA (every barrier trivially passed), an odd count, and the largest resident grid."""
    wl = Workload("q4_64")
    P, Phi = wl.problem, pod_basis(wl)
    m = 7
    Bm = wl.rhs(m)
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    out = {}
    for g in (1, 37, 2 * sms, 2 * sms):
        s, vals = _solver(pkg, wl, Phi, m)
        assert s.set_tuning(rows_kernel=s.get_tuning()["rows_kernel"] | PERSIST, grid_persist=g) == pkg.OK
        assert s.get_tuning()["grid_persist"] == g
        X, it, rel, st, rc = s.solve_batch(list(range(m)), Bm, tol=TOL, maxit=3000)
        assert rc == pkg.OK and np.all(st == pkg.OK)
        s.close()
        if g in out:
            assert np.array_equal(out[g][0], X)
        out[g] = (X, it)
    ref = O.pod2g_pcg(P.csr(vals[3]), Bm[3], None, _phi_used(wl, Phi), wl.spec.omega, TOL, 3000)
    for g, (X, it) in out.items():
        assert abs(int(it[3]) - ref.iters) <= 2 and _relerr(X[3], ref.x) <= 1e-6, g


def test_persistent_invalid_grid_rejected(pkg):
    wl = Workload("q4_16")
    P, Phi = wl.problem, pod_basis(wl)
    s, _ = _solver(pkg, wl, Phi, 2)
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    assert s.set_tuning(grid_persist=-1) == pkg.INVALID_ARG
    assert s.set_tuning(grid_persist=4 * sms + 1) == pkg.INVALID_ARG
    assert s.set_tuning(rows_kernel=16) == pkg.INVALID_ARG
    s.close()
    # not for the element-factored operator or Gauss-Seidel smoothing: bit 3 rejected
    g = pkg.Solver(P.row_ptr, P.col_idx, P.bs, Phi, omega=wl.spec.omega, max_batch=2, smoother=pkg.SMOOTHER_SGS)
    assert g.get_tuning()["rows_kernel"] & PERSIST == 0
    assert g.set_tuning(rows_kernel=PERSIST, grid_persist=8) == pkg.INVALID_ARG
    g.close()


@pytest.mark.parametrize("variant", ["pr", "stationary"])
def test_persistent_variants_match_oracle(pkg, variant):
    wl = Workload("q4_16")
    P, Phi = wl.problem, pod_basis(wl)
    m = 4
    Bm = wl.rhs(m)
    kw = dict(beta_pr=True) if variant == "pr" else dict(method=pkg.STATIONARY)
    s, vals = _solver(pkg, wl, Phi, m, **kw)
    assert s.set_tuning(rows_kernel=s.get_tuning()["rows_kernel"] | PERSIST) == pkg.OK
    X, it, rel, st, rc = s.solve_batch(list(range(m)), Bm, tol=TOL, maxit=5000)
    assert rc == pkg.OK and np.all(st == pkg.OK)
    s.close()
    phi_used = _phi_used(wl, Phi)
    for i in (0, m - 1):
        if variant == "pr":
            ref = O.pod2g_pcg(P.csr(vals[i]), Bm[i], None, phi_used, wl.spec.omega, TOL, 5000, beta="pr")
        else:
            ref = O.pod2g_stationary(P.csr(vals[i]), Bm[i], None, phi_used, wl.spec.omega, TOL, 5000)
        assert abs(int(it[i]) - ref.iters) <= 2, (variant, i, it[i], ref.iters)
        assert _relerr(X[i], ref.x) <= 1e-6


def test_persistent_slot_independent_of_batch(pkg):
    """A slot's iterate is bit-identical alone and in a batch whose other slots stop at
    different iterations (a zero right-hand side stops at load, others converge at
    different counts), and an iteration cap gives NOT_CONVERGED with the capped iterate."""
    wl = Workload("q4_16")
    P, Phi = wl.problem, pod_basis(wl)
    m = 5
    Bm = wl.rhs(m)
    Bm[1] = 0.0
    Bm[3] *= 1e-3
    s, vals = _solver(pkg, wl, Phi, m)
    X, it, rel, st, rc = s.solve_batch(list(range(m)), Bm, tol=TOL, maxit=3000)
    assert rc == pkg.OK and np.all(st == pkg.OK)
    assert it[1] == 0 and not X[1].any()
    for i in (0, 2, 4):
        Xa, ia, _, sa, rca = s.solve_batch([i], Bm[i:i + 1], tol=TOL, maxit=3000)
        assert rca == pkg.OK and sa[0] == pkg.OK
        assert np.array_equal(Xa[0], X[i]) and ia[0] == it[i]
    Xc, ic, _, sc_, rcc = s.solve_batch([0, 2], Bm[[0, 2]], tol=TOL, maxit=13)
    assert np.all(ic == 13) and np.all(sc_ == pkg.NOT_CONVERGED)
    s.close()
    ref = O.pod2g_pcg(P.csr(vals[0]), Bm[0], None, _phi_used(wl, Phi), wl.spec.omega, TOL, 13)
    assert ref.iters == 13 and _relerr(Xc[0], ref.x) <= 1e-5


def test_persistent_autotune_keeps_a_valid_form(pkg):
    wl = Workload("q1_32")
    P, Phi = wl.problem, pod_basis(wl)
    m = 20
    s, vals = _solver(pkg, wl, Phi, m)
    Bm = wl.rhs(m)
    st, shape = s.autotune(list(range(m)), torch.from_numpy(Bm).cuda(), iters=16)
    assert st == pkg.OK and shape["grid_persist"] >= 1
    X, it, rel, sts, rc = s.solve_batch(list(range(m)), Bm, tol=TOL, maxit=3000)
    assert rc == pkg.OK and np.all(sts == pkg.OK)
    ref = O.pod2g_pcg(P.csr(vals[5]), Bm[5], None, _phi_used(wl, Phi), wl.spec.omega, TOL, 3000)
    assert abs(int(it[5]) - ref.iters) <= 2 and _relerr(X[5], ref.x) <= 1e-6
    s.close()

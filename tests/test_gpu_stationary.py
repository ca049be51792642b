"""GPU parity of the stationary method: the POD-2G two-grid cycle (Algorithm 2 with
P = Phi_r, Section 3.3) iterated on its own, u <- u + AMG(0; K, f - K u, r1, r2),
through the C ABI, against the oracle's `pod2g_stationary`.

Tolerances as for the PCG path: relative 2-norm error of x <= 1e-7 on the FP64
path and <= 1e-6 on the mixed path at tol 1e-8; cycle counts within +-2. The
mixed path gets the oracle FP32-rounded values and the rounded basis.
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


@pytest.mark.parametrize("name", ["q1_32", "hex8_8"])
def test_stationary_fp64_plain_path(pkg, name):
    wl = Workload(name)
    P, Phi = wl.problem, pod_basis(wl)
    vals = wl.values(wl.query_thetas(1)[0])
    b = wl.rhs(1)[0]
    s = pkg.Solver(P.row_ptr, P.col_idx, P.bs, Phi, precision=pkg.FP64, omega=wl.spec.omega,
                   method=pkg.STATIONARY)
    assert s.set_values(0, vals) == pkg.OK
    x, it, rel, st = s.solve(0, b, tol=TOL, maxit=5000)
    ref = O.pod2g_stationary(P.csr(vals), b, None, Phi, wl.spec.omega, TOL, 5000)
    assert st == pkg.OK and ref.status == O.OK
    assert abs(it - ref.iters) <= 2
    assert _relerr(x, ref.x) <= 1e-7
    assert rel <= TOL and abs(rel - ref.relres) <= 1e-9
    s.close()


@pytest.mark.parametrize("name,precision", [("q1_32", 1), ("q4_16", 1), ("hex8_8", 2), ("hex8_16", 2)])
def test_stationary_mixed_batched_matches_oracle(pkg, name, precision):
    wl = Workload(name)
    P, Phi = wl.problem, pod_basis(wl)
    m = wl.spec.batch
    xis = wl.query_thetas(m)
    Bm = wl.rhs(m)
    phi_used = round_phi(Phi, "bf16" if precision == pkg.MIXED_BF16PHI else "f32")
    s = pkg.Solver(P.row_ptr, P.col_idx, P.bs, Phi, precision=precision, omega=wl.spec.omega, max_batch=m,
                   method=pkg.STATIONARY)
    vals = [round_f32(wl.values(xi)) for xi in xis]
    for i in range(m):
        assert s.set_values(i, vals[i]) == pkg.OK
    X, iters, rel, st, rc = s.solve_batch(list(range(m)), Bm, tol=TOL, maxit=5000)
    assert rc == pkg.OK
    for i in range(m):
        ref = O.pod2g_stationary(P.csr(vals[i]), Bm[i], None, phi_used, wl.spec.omega, TOL, 5000)
        assert st[i] == pkg.OK and ref.status == O.OK
        assert abs(iters[i] - ref.iters) <= 2, (i, iters[i], ref.iters)
        assert _relerr(X[i], ref.x) <= 1e-6
        assert rel[i] <= 1.01 * TOL
    s.close()


def test_stationary_maxit_iterate_matches_oracle(pkg):
    """Stopped by maxit: the status says so and x is the oracle's iterate after maxit cycles."""
    wl = Workload("q4_16")
    P, Phi = wl.problem, pod_basis(wl)
    vals = round_f32(wl.values(wl.query_thetas(1)[0]))
    b = wl.rhs(1)[0]
    ref = O.pod2g_stationary(P.csr(vals), b, None, round_phi(Phi, "f32"), wl.spec.omega, TOL, 37)
    assert ref.status == O.NOT_CONVERGED and ref.iters == 37
    for precision in (pkg.FP64, pkg.MIXED_FP32PHI):
        s = pkg.Solver(P.row_ptr, P.col_idx, P.bs, Phi if precision == pkg.FP64 else Phi, precision=precision,
                       omega=wl.spec.omega, method=pkg.STATIONARY)
        assert s.set_values(0, vals) == pkg.OK
        x, it, rel, st = s.solve(0, b, tol=TOL, maxit=37)
        assert st == pkg.NOT_CONVERGED and it == 37
        tol_x = 1e-9 if precision == pkg.FP64 else 1e-6
        if precision == pkg.FP64:
            ref64 = O.pod2g_stationary(P.csr(vals), b, None, Phi, wl.spec.omega, TOL, 37)
            assert _relerr(x, ref64.x) <= tol_x
        else:
            assert _relerr(x, ref.x) <= tol_x
        assert abs(rel - ref.relres) <= 1e-3 * ref.relres
        s.close()


def test_pcg_needs_fewer_iterations_than_stationary(pkg):
    """Section 4's comparison: the Krylov acceleration of Algorithm 3 converges in far
    fewer iterations than the two-grid cycle used as the solver, on the same system."""
    wl = Workload("hex8_8")
    P, Phi = wl.problem, pod_basis(wl)
    vals = wl.values(wl.query_thetas(1)[0])
    b = wl.rhs(1)[0]
    its = {}
    for method in (pkg.PCG, pkg.STATIONARY):
        s = pkg.Solver(P.row_ptr, P.col_idx, P.bs, Phi, precision=pkg.MIXED_FP32PHI, omega=wl.spec.omega,
                       method=method)
        assert s.set_values(0, vals) == pkg.OK
        x, it, rel, st = s.solve(0, b, tol=TOL, maxit=5000)
        assert st == pkg.OK
        its[method] = it
        s.close()
    assert its[pkg.PCG] * 5 < its[pkg.STATIONARY]


def test_stationary_alone_and_in_batch_bit_identical(pkg):
    wl = Workload("q1_32")
    P, Phi = wl.problem, pod_basis(wl)
    m = 4
    xis = wl.query_thetas(m)
    Bm = wl.rhs(m)
    s = pkg.Solver(P.row_ptr, P.col_idx, P.bs, Phi, precision=pkg.MIXED_FP32PHI, omega=wl.spec.omega,
                   max_batch=m, method=pkg.STATIONARY)
    for i in range(m):
        assert s.set_values(i, wl.values(xis[i])) == pkg.OK
    X, iters, rel, st, rc = s.solve_batch(list(range(m)), Bm, tol=TOL, maxit=5000)
    assert rc == pkg.OK
    x2, it2, rel2, st2 = s.solve(2, Bm[2], tol=TOL, maxit=5000)
    assert it2 == iters[2] and np.array_equal(x2, X[2])
    s.close()


def test_stationary_method_rejected_when_invalid(pkg):
    wl = Workload("q1_16")
    P, Phi = wl.problem, pod_basis(wl)
    with pytest.raises(pkg.Pod2gError) as e:
        pkg.Solver(P.row_ptr, P.col_idx, P.bs, Phi, method=7)
    assert e.value.status == pkg.INVALID_ARG

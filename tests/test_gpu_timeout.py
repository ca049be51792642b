"""Failure detection without a GPU fault: the host's bounded wait of a batched solve.

A context created with spin_limit = 1 polls the device once (one CUDA-graph launch of
`chunk` = 8 iterations) and gives up on a solve that needs ~100 iterations: the call
returns POD2G_TIMEOUT, every instance reports POD2G_TIMEOUT with its last (finite) iterate
and at most one launch's worth of iterations, and the context stays usable: a solve that
needs no iteration (b = 0) on the same context returns OK, and a second context on the
same device then solves the problem to the oracle's result. Nothing waits on the device
without a bound, and no kernel faults.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import pod2g_oracle as O  # noqa: E402
from synth.problems import Workload  # noqa: E402
from synth.rounding import round_f32, round_phi  # noqa: E402
from synth.snapshots import pod_basis  # noqa: E402


@pytest.fixture(scope="module")
def pkg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import paper_2207_02543_gb300 as p
    return p


def test_host_spin_limit_gives_timeout_and_context_stays_usable(pkg):
    wl = Workload("q4_64")
    P, Phi = wl.problem, pod_basis(wl)
    m = 3
    Bm = wl.rhs(m)
    vals = [round_f32(wl.values(xi)) for xi in wl.query_thetas(m)]
    s = pkg.Solver(P.row_ptr, P.col_idx, P.bs, Phi, omega=wl.spec.omega, max_batch=m, spin_limit=1)
    for i in range(m):
        assert s.set_values(i, vals[i]) == pkg.OK
    X, it, rel, st, rc = s.solve_batch(list(range(m)), Bm, tol=1e-8, maxit=5000)
    assert rc == pkg.TIMEOUT
    assert np.all(st == pkg.TIMEOUT)
    assert np.all(np.isfinite(X)) and np.all(it >= 1) and np.all(it <= 2 * 8)
    assert np.all(rel > 1e-8)
    # the same context: a right-hand side of zero needs no iteration
    X0, it0, rel0, st0, rc0 = s.solve_batch([0], np.zeros((1, P.n)), tol=1e-8, maxit=5000)
    assert rc0 == pkg.OK and it0[0] == 0 and np.all(X0 == 0.0)
    s.close()
    # a new context on the same device solves the problem
    s2 = pkg.Solver(P.row_ptr, P.col_idx, P.bs, Phi, omega=wl.spec.omega, max_batch=1)
    assert s2.set_values(0, vals[0]) == pkg.OK
    X2, it2, rel2, st2, rc2 = s2.solve_batch([0], Bm[:1], tol=1e-8, maxit=5000)
    s2.close()
    assert rc2 == pkg.OK
    ref = O.pod2g_pcg(P.csr(vals[0]), Bm[0], None, round_phi(Phi, "f32"), wl.spec.omega, 1e-8, 5000)
    assert abs(int(it2[0]) - ref.iters) <= 2
    assert np.linalg.norm(X2[0] - ref.x) <= 1e-6 * np.linalg.norm(ref.x)

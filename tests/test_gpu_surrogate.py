"""Surrogate initial guess on the device (Section 3.2) through the C ABI, and POD-2G-PCG started
from it, against the oracle.

  * the device prediction s * Psi (z_mean + z_std * FFNN(theta)) against the oracle's FP64
    prediction from the same weights: relative error <= 1e-5 (Psi stored and the decoder
    accumulated in FP32: about sqrt(ks) * 2^-24 ~ 1e-6);
  * the solve from that x0 against the oracle's solve from its own prediction: relative x error
    <= 1e-6, iterations within +-2;
  * against the device solve from x0 = 0: the same x within 1e-6, and the surrogate start needs
    no more iterations on average (mean +1 at most). The count of a single instance may rise a
    little: PCG's iteration count to a residual tolerance is not monotone in the initial error
    (the Krylov space of b - K x0 changes with x0), so each instance is bounded by +5 only.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import pod2g_oracle as O  # noqa: E402
from oracle import surrogate as S  # noqa: E402
from synth.problems import Workload  # noqa: E402
from synth.rounding import round_f32, round_phi  # noqa: E402
from synth.snapshots import pod_basis  # noqa: E402
from synth.surrogate import load_scale, train_surrogate  # noqa: E402

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


@pytest.mark.parametrize("name,nq", [("q1_32", 5), ("q4_64", 7), ("hex8_16", 5), ("q4_64", 40)])
def test_surrogate_x0_on_device_matches_oracle(pkg, name, nq):
    wl = Workload(name)
    P, Phi = wl.problem, pod_basis(wl)
    sur = train_surrogate(wl, steps=2000)
    xis, Bm = wl.query_thetas(nq), wl.rhs(nq)
    scale = np.array([load_scale(wl, b) for b in Bm])
    sd = pkg.Surrogate(sur)
    x0 = torch.empty((nq, P.n), dtype=torch.float64, device="cuda")
    assert sd.predict_dev(xis, scale, x0) == pkg.OK
    torch.cuda.synchronize()
    X0 = x0.cpu().numpy()
    sd.close()
    ref0 = [S.surrogate_prediction(xis[q], scale[q], sur) for q in range(nq)]
    for q in range(nq):
        assert _relerr(X0[q], ref0[q]) <= 1e-5, (q, _relerr(X0[q], ref0[q]))
    if nq > 8:
        return
    prec = pkg.MIXED_BF16PHI if wl.spec.phi_dtype == "bf16" else pkg.MIXED_FP32PHI
    phi_used = round_phi(Phi, "bf16" if wl.spec.phi_dtype == "bf16" else "f32")
    vals = [round_f32(wl.values(xi)) for xi in xis]
    s = pkg.Solver(P.row_ptr, P.col_idx, P.bs, Phi, precision=prec, omega=wl.spec.omega, max_batch=nq)
    for i in range(nq):
        assert s.set_values(i, vals[i]) == pkg.OK
    b_dev = torch.from_numpy(Bm).cuda()
    xs = torch.empty_like(b_dev)
    its, rel, st, rc = s.solve_batch_dev(list(range(nq)), b_dev, xs, x0_dev=x0, tol=TOL, maxit=3000)
    assert rc == pkg.OK
    Xs = xs.cpu().numpy()
    X, it0, rel0, st0, rc0 = s.solve_batch(list(range(nq)), Bm, tol=TOL, maxit=3000)
    assert rc0 == pkg.OK
    s.close()
    for i in range(nq):
        ref = O.pod2g_pcg(P.csr(vals[i]), Bm[i], ref0[i], phi_used, wl.spec.omega, TOL, 3000)
        assert ref.status == O.OK
        assert abs(int(its[i]) - ref.iters) <= 2, (i, its[i], ref.iters)
        assert _relerr(Xs[i], ref.x) <= 1e-6
        assert _relerr(Xs[i], X[i]) <= 1e-6
        assert its[i] <= it0[i] + 5, (i, list(its), list(it0))
    assert np.mean(its) <= np.mean(it0) + 1, (list(its), list(it0))

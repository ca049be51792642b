"""The coarse matrix K_c = Phi^T K Phi of the per-instance set-up (Section 3.3, eq. POD_ROM),
through the C ABI, against the oracle's coarse_operator on the same FP32-rounded values and
rounded basis.

Two contractions exist on the mixed paths: double-float on the CUDA cores, and the tensor
cores (tcgen05, BF16 pieces of the FP32 operands, FP32 accumulation per CTA, FP64 across
CTAs). Bounds, on the largest entry of K_c:
  * double-float: 1e-12 (K Phi and the contraction carry ~14 digits);
  * tensor cores: 2e-6. The six kept piece products represent each term phi_i w_i to
    ~3 * 2^-24 of |phi_i||w_i|, and a CTA sums at most ceil(n / SMs) terms in FP32
    (relative rounding ~2^-24 per addition); for these workloads that bounds the error
    near 1e-7 of the largest entry (an FP64 emulation of the same arithmetic gives
    0.8e-7 to 1.1e-7), and 2e-6 leaves a factor of ~20.
The returned factor satisfies L L^T = K_c to FP64 rounding.
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


def _kc_gpu(pkg, wl, Phi, vals, coarse):
    P = wl.problem
    prec = pkg.MIXED_BF16PHI if wl.spec.phi_dtype == "bf16" else pkg.MIXED_FP32PHI
    s = pkg.Solver(P.row_ptr, P.col_idx, P.bs, Phi, precision=prec, omega=wl.spec.omega, max_batch=len(vals),
                   coarse=coarse)
    out = []
    for i, v in enumerate(vals):
        assert s.set_values(i, v) == pkg.OK
        L = s.coarse_factor(i)
        assert np.all(np.triu(L, 1) == 0)
        out.append(L @ L.T)
    s.close()
    return out


@pytest.mark.parametrize("name", ["q1_32", "q4_16", "hex8_8", "q4_64", "hex8_16"])
def test_coarse_matrix_matches_oracle(pkg, name):
    wl = Workload(name)
    P, Phi = wl.problem, pod_basis(wl)
    phi_used = round_phi(Phi, "bf16" if wl.spec.phi_dtype == "bf16" else "f32")
    vals = [round_f32(wl.values(xi)) for xi in wl.query_thetas(3)]
    ref = []
    for v in vals:
        Kr = O.coarse_operator(P.csr(v), phi_used)
        ref.append(0.5 * (Kr + Kr.T))
    for coarse, bound in ((pkg.COARSE_DF, 1e-12), (pkg.COARSE_TENSOR, 2e-6)):
        got = _kc_gpu(pkg, wl, Phi, vals, coarse)
        for g, r in zip(got, ref):
            err = np.abs(g - r).max() / np.abs(r).max()
            assert err <= bound, (coarse, err)


@pytest.mark.parametrize("k", [1, 17, 40, 64])
def test_coarse_matrix_tensor_cores_any_width(pkg, k):
    """Mode counts that exercise every accumulator width N = 16, 32, 48, 64 and a one-mode basis."""
    wl = Workload("q4_64")
    P = wl.problem
    Phi = np.linalg.qr(np.random.default_rng(k).standard_normal((P.n, k)))[0]
    vals = [round_f32(wl.values(xi)) for xi in wl.query_thetas(2)]
    phi_used = round_phi(Phi, "f32")
    got = _kc_gpu(pkg, wl, Phi, vals, pkg.COARSE_TENSOR)
    for g, v in zip(got, vals):
        Kr = O.coarse_operator(P.csr(v), phi_used)
        r = 0.5 * (Kr + Kr.T)
        assert np.abs(g - r).max() / np.abs(r).max() <= 2e-6


def test_solve_with_tensor_core_coarse_matrix_matches_oracle(pkg):
    wl = Workload("hex8_16")
    P, Phi = wl.problem, pod_basis(wl)
    m = wl.spec.batch
    Bm = wl.rhs(m)
    phi_used = round_phi(Phi, "bf16")
    vals = [round_f32(wl.values(xi)) for xi in wl.query_thetas(m)]
    s = pkg.Solver(P.row_ptr, P.col_idx, P.bs, Phi, precision=pkg.MIXED_BF16PHI, omega=wl.spec.omega,
                   max_batch=m, coarse=pkg.COARSE_TENSOR)
    for i in range(m):
        assert s.set_values(i, vals[i]) == pkg.OK
    X, it, rel, st, rc = s.solve_batch(list(range(m)), Bm, tol=TOL, maxit=3000)
    s.close()
    assert rc == pkg.OK
    for i in range(m):
        ref = O.pod2g_pcg(P.csr(vals[i]), Bm[i], None, phi_used, wl.spec.omega, TOL, 3000)
        assert abs(int(it[i]) - ref.iters) <= 2
        assert np.linalg.norm(X[i] - ref.x) <= 1e-6 * np.linalg.norm(ref.x)

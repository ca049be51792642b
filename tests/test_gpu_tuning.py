"""Launch shapes of the batched path and the autotuner, through the C ABI.

A launch shape only regroups partial sums: results are deterministic for a given
shape, and every shape stays within the parity tolerances against the oracle
(relative x error <= 1e-6 at tol 1e-8, iteration counts within +-2).
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


def _solver(pkg, wl, Phi, m):
    P = wl.problem
    s = pkg.Solver(P.row_ptr, P.col_idx, P.bs, Phi, omega=wl.spec.omega, max_batch=m)
    vals = [round_f32(wl.values(xi)) for xi in wl.query_thetas(m)]
    for i in range(m):
        assert s.set_values(i, vals[i]) == pkg.OK
    return s, vals


def test_autotune_then_solve_matches_oracle(pkg):
    wl = Workload("q4_64")
    P, Phi = wl.problem, pod_basis(wl)
    m = wl.spec.batch
    s, vals = _solver(pkg, wl, Phi, m)
    Bm = wl.rhs(m)
    st, shape = s.autotune(list(range(m)), torch.from_numpy(Bm).cuda(), iters=16)
    assert st == pkg.OK
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    assert shape["grid_rows"] % 8 == 0 and 8 <= shape["grid_rows"] <= 8 * sms
    assert shape["grid_spmv"] % 8 == 0 and 8 <= shape["grid_spmv"] <= 8 * sms
    assert shape["grid_restrict"] % 8 == 0 and 8 <= shape["grid_restrict"] <= 4 * sms
    assert 1 <= shape["grid_prol"] <= 8 * sms and 1 <= shape["grid_vec"] <= 8 * sms
    assert s.get_tuning() == shape
    X, it, rel, sts, rc = s.solve_batch(list(range(m)), Bm, tol=TOL, maxit=3000)
    assert rc == pkg.OK
    phi32 = round_phi(Phi, "f32")
    for i in (0, m - 1):
        ref = O.pod2g_pcg(P.csr(vals[i]), Bm[i], None, phi32, wl.spec.omega, TOL, 3000)
        assert abs(it[i] - ref.iters) <= 2 and _relerr(X[i], ref.x) <= 1e-6
    s.close()


def test_shapes_deterministic_and_within_tolerance(pkg):
    wl = Workload("q4_16")
    P, Phi = wl.problem, pod_basis(wl)
    m = wl.spec.batch
    Bm = wl.rhs(m)
    small = dict(grid_rows=8, grid_restrict=8, grid_prol=1, grid_vec=1, grid_spmv=16, rows_kernel=0,
                 restrict_rows=8)
    res = []
    for shape in (small, small, None):
        s, vals = _solver(pkg, wl, Phi, m)
        if shape:
            assert s.set_tuning(**shape) == pkg.OK
            got = s.get_tuning()
            assert {k: got[k] for k in shape} == shape
        res.append(s.solve_batch(list(range(m)), Bm, tol=TOL, maxit=3000))
        s.close()
    (Xa, ia, *_), (Xb, ib, *_), (Xc, ic, *_) = res
    assert np.array_equal(Xa, Xb) and list(ia) == list(ib)       # same shape: bit-identical
    for i in range(m):
        assert abs(ia[i] - ic[i]) <= 2 and _relerr(Xa[i], Xc[i]) <= 1e-6


def test_invalid_shapes_rejected(pkg):
    wl = Workload("q4_16")
    P, Phi = wl.problem, pod_basis(wl)
    s, _ = _solver(pkg, wl, Phi, 2)
    assert s.set_tuning(grid_rows=12) == pkg.INVALID_ARG          # not a multiple of 8
    assert s.set_tuning(grid_spmv=0) == pkg.INVALID_ARG
    assert s.set_tuning(grid_restrict=0) == pkg.INVALID_ARG
    assert s.set_tuning(grid_vec=10 ** 6) == pkg.INVALID_ARG
    assert s.set_tuning(rows_kernel=16) == pkg.INVALID_ARG
    assert s.set_tuning(restrict_rows=6) == pkg.INVALID_ARG       # not a multiple of 4
    s.close()
    f = pkg.Solver(P.row_ptr, P.col_idx, P.bs, Phi, precision=pkg.FP64)
    with pytest.raises(pkg.Pod2gError):
        f.get_tuning()
    f.close()


@pytest.mark.parametrize("name,m", [("q4_16", 3), ("q4_64", 7), ("hex8_16", 5), ("q1_32", 5), ("q4_16", 40),
                                    ("hex8_8", 36), ("q1_32", 20), ("q4_16", 1), ("hex8_16", 1), ("q1_32", 1)])
def test_row_kernel_forms_match_oracle(pkg, name, m):
    """The forms of the sparse row kernels (one thread per block row and slot, or warp-staged
    with bulk-copied values -- for a single slot, a group of lanes per block row -- for the
    smoother passes and the outer SpMV independently; and,
    where the context stores K Phi, the post-smoothing pass that forms K y2 from it) give the
    oracle's result: relative x error <= 1e-6, iteration counts within +-2, and each form is
    deterministic."""
    wl = Workload(name)
    P, Phi = wl.problem, pod_basis(wl)
    Bm = wl.rhs(m)
    phi_used = round_phi(Phi, "bf16" if wl.spec.phi_dtype == "bf16" else "f32")
    prec = pkg.MIXED_BF16PHI if wl.spec.phi_dtype == "bf16" else pkg.MIXED_FP32PHI
    res = {}
    probe = pkg.Solver(P.row_ptr, P.col_idx, P.bs, Phi, precision=prec, omega=wl.spec.omega, max_batch=m)
    kphi = probe.get_tuning()["rows_kernel"] & 4
    probe.close()
    forms = (0, 1, 2, 3, 4, 7, 7) if kphi else (0, 1, 2, 3, 3)
    for form in forms:
        s = pkg.Solver(P.row_ptr, P.col_idx, P.bs, Phi, precision=prec, omega=wl.spec.omega, max_batch=m)
        vals = [round_f32(wl.values(xi)) for xi in wl.query_thetas(m)]
        for i in range(m):
            assert s.set_values(i, vals[i]) == pkg.OK
        assert s.set_tuning(rows_kernel=form) == pkg.OK
        X, it, rel, st, rc = s.solve_batch(list(range(m)), Bm, tol=TOL, maxit=3000)
        assert rc == pkg.OK and np.all(st == pkg.OK)
        s.close()
        if form in res:
            assert np.array_equal(res[form][0], X) and list(res[form][1]) == list(it)
        res[form] = (X, it)
    for i in sorted({0, m - 1}):
        ref = O.pod2g_pcg(P.csr(vals[i]), Bm[i], None, phi_used, wl.spec.omega, TOL, 3000)
        for form, (X, it) in res.items():
            assert abs(int(it[i]) - ref.iters) <= 2, (form, i, it[i], ref.iters)
            assert _relerr(X[i], ref.x) <= 1e-6, (form, i, _relerr(X[i], ref.x))

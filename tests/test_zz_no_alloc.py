"""pod2g_solve_noalloc: the solve for callers that cannot allocate device memory.

The entry point keeps its scratch in a fixed static device array instead of
calling cudaMalloc. Its results must be those of the regular entry point
(pod2g_solve on an FP64 context) within the FP64-path tolerances used by the
other parity tests: relative 2-norm error of x <= 1e-7, iteration counts within
+-2. It is called twice in a row, because every call reuses (and must first
reset) what the previous call left in the shared array. This file is collected
last so that a run stopping at the first failure has run every other test.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from synth.problems import Workload  # noqa: E402
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
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.mark.parametrize("name", ["q1_64", "q4_16"])
def test_noalloc_matches_regular_solve_twice(pkg, name):
    wl = Workload(name)
    P = wl.problem
    Phi = pod_basis(wl, use_disk=False)
    k = Phi.shape[1]
    vals = wl.values(wl.query_thetas(1)[0])
    b = wl.rhs(1)[0]
    # the regular entry point (allocating context)
    s = pkg.Solver(P.row_ptr, P.col_idx, P.bs, Phi, precision=pkg.FP64, omega=wl.spec.omega, max_batch=1)
    assert s.set_values(0, vals) == pkg.OK
    x_ref, it_ref, rel_ref, st_ref = s.solve(0, b, tol=TOL, maxit=2000)
    s.close()
    assert st_ref == pkg.OK
    # the no-allocation entry point: device inputs and outputs owned by the caller
    dev = torch.device("cuda")
    rp = torch.from_numpy(P.row_ptr.astype(np.int32)).to(dev)
    ci = torch.from_numpy(P.col_idx.astype(np.int32)).to(dev)
    v = torch.from_numpy(vals.reshape(-1)).to(dev)
    ph = torch.from_numpy(np.ascontiguousarray(Phi.T).reshape(-1)).to(dev)  # column-major n x k
    bd = torch.from_numpy(b).to(dev)
    for call in range(2):
        xd = torch.full_like(bd, float("nan"))
        rc, it, rel, st = pkg.solve_noalloc(rp, ci, P.bs, v, ph, k, bd, xd, tol=TOL, maxit=2000,
                                            omega=wl.spec.omega)
        assert rc == pkg.OK and st == pkg.OK, (call, pkg.strerror(rc))
        x = xd.cpu().numpy()
        assert _relerr(x, x_ref) <= 1e-7, (call, _relerr(x, x_ref))
        assert abs(it - it_ref) <= 2, (call, it, it_ref)
        assert rel <= 1.01 * TOL and abs(rel - rel_ref) <= 1e-9


def test_noalloc_rejects_sizes_beyond_its_capacity(pkg):
    dev = torch.device("cuda")
    z = torch.zeros(4, dtype=torch.float64, device=dev)
    zi = torch.zeros(4, dtype=torch.int32, device=dev)
    import ctypes as C
    lib = pkg.load_library()
    p = lambda t: C.c_void_p(t.data_ptr())  # noqa: E731
    it, rr, st = C.c_int(0), C.c_double(0.0), C.c_int(0)
    # n = 20000 > POD2G_NOALLOC_MAX_N: refused before any device access
    rc = lib.pod2g_solve_noalloc(20000, 1, 20000, p(zi), p(zi), p(z), p(z), 1, None, p(z), None, 1e-8, 10, p(z),
                                 C.byref(it), C.byref(rr), C.byref(st), None)
    assert rc == pkg.TOO_LARGE
    rc = lib.pod2g_solve_noalloc(2, 1, 2, p(zi), p(zi), p(z), p(z), pkg.NOALLOC_MAX_K + 1, None, p(z), None, 1e-8,
                                 10, p(z), C.byref(it), C.byref(rr), C.byref(st), None)
    assert rc == pkg.TOO_LARGE
    assert "scratch capacity" in pkg.strerror(pkg.TOO_LARGE)

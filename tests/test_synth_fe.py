"""Pins for the synthetic-problem generator (FE assembly, loads, KL fields).

These check the generated systems against closed forms and textbook facts, never
against themselves: element-matrix rank and rigid-body null spaces, the Q1
closed-form element matrix, uniform-strain energy, the patch test, the O(h^2)
convergence of the Poisson midpoint value to its Fourier-series solution, and
the KL trace identity.
"""
import itertools

import numpy as np
import pytest

from synth import fe, kl
from synth.problems import Workload, SPECS


def _corner_coords(dim, h=1.0):
    return np.array([[((a >> d) & 1) * h for d in range(dim)] for a in range(2 ** dim)])


@pytest.mark.parametrize("name,K,rank", [
    ("q1", fe.element_matrix_q1(0.25), 3),
    ("q4", fe.element_matrix_q4(0.25), 5),
    ("hex8", fe.element_matrix_hex8(0.125), 18),
])
def test_element_matrix_symmetric_rank(name, K, rank):
    assert np.allclose(K, K.T, atol=1e-14)
    w = np.linalg.eigvalsh(K)
    assert np.all(w > -1e-12)
    assert int((w > 1e-10 * w.max()).sum()) == rank


def test_q1_closed_form():
    # bilinear Laplacian on a square: diag 4/6, edge neighbours -1/6, opposite corner -2/6
    # local order here: 0 (0,0), 1 (1,0), 2 (0,1), 3 (1,1)
    ref = np.array([[4, -1, -1, -2], [-1, 4, -2, -1], [-1, -2, 4, -1], [-2, -1, -1, 4]]) / 6.0
    assert np.allclose(fe.element_matrix_q1(0.37), ref, atol=1e-14)


def test_rigid_body_modes_in_null_space():
    X2 = _corner_coords(2, 0.3)
    K4 = fe.element_matrix_q4(0.3)
    modes2 = [np.tile([1.0, 0.0], 4), np.tile([0.0, 1.0], 4), np.column_stack([-X2[:, 1], X2[:, 0]]).reshape(-1)]
    for m in modes2:
        assert np.abs(K4 @ m).max() < 1e-12
    X3 = _corner_coords(3, 0.2)
    K8 = fe.element_matrix_hex8(0.2)
    x, y, z = X3.T
    modes3 = [np.tile(e, 8) for e in np.eye(3)] + [
        np.column_stack([-y, x, 0 * x]).reshape(-1),
        np.column_stack([0 * x, -z, y]).reshape(-1),
        np.column_stack([z, 0 * x, -x]).reshape(-1)]
    for m in modes3:
        assert np.abs(K8 @ m).max() < 1e-12


def test_uniform_strain_energy():
    rng = np.random.default_rng(0)
    h = 0.3
    # 2D plane stress: u = G x with symmetric G -> energy = 1/2 eps^T D eps * area
    G = rng.standard_normal((2, 2)); G = 0.5 * (G + G.T)
    X = _corner_coords(2, h)
    u = (X @ G.T).reshape(-1)
    eps = np.array([G[0, 0], G[1, 1], 2 * G[0, 1]])
    E = 0.5 * u @ fe.element_matrix_q4(h) @ u
    assert np.isclose(E, 0.5 * eps @ fe.plane_stress_D(1.0, 0.3) @ eps * h * h, rtol=1e-12)
    # 3D
    G = rng.standard_normal((3, 3)); G = 0.5 * (G + G.T)
    X = _corner_coords(3, h)
    u = (X @ G.T).reshape(-1)
    eps = np.array([G[0, 0], G[1, 1], G[2, 2], 2 * G[0, 1], 2 * G[1, 2], 2 * G[0, 2]])
    E = 0.5 * u @ fe.element_matrix_hex8(h) @ u
    lam, mu = fe.lame(1.0, 0.3)
    tr = G[0, 0] + G[1, 1] + G[2, 2]
    energy_density = 0.5 * lam * tr ** 2 + mu * np.sum(G * G)
    assert np.isclose(E, energy_density * h ** 3, rtol=1e-12)
    assert np.isclose(0.5 * eps @ fe.elasticity_3d_D() @ eps, energy_density, rtol=1e-12)


@pytest.mark.parametrize("kind,ne", [("q1", 6), ("q4", 5), ("hex8", 3)])
def test_pattern_structure(kind, ne):
    P = fe._build(kind, ne)
    rp, ci = P.row_ptr, P.col_idx
    for i in range(P.n_nodes):
        cols = ci[rp[i]:rp[i + 1]]
        assert np.all(np.diff(cols) > 0) and i in cols
    c = np.random.default_rng(1).uniform(0.5, 2.0, P.n_el)
    A = P.csr(P.values(c))
    assert abs(A - A.T).max() < 1e-15
    assert np.linalg.eigvalsh(A.toarray()).min() > 0


def test_full_size_counts():
    P = fe.q4_problem(512)
    assert (P.n, P.nnzb) == (526_338, 2_362_369)
    P = fe.q1_problem(64)
    assert (P.n, P.nnzb) == (3969, 34_969)


def test_identity_rows_for_clamped_nodes():
    P = fe.hex8_problem(3)
    A = P.csr(P.values(np.ones(P.n_el))).toarray()
    cl = np.nonzero(np.repeat(P.clamped, 3))[0]
    assert len(cl) == 3 * 16
    for d in cl:
        row = A[d].copy(); row[d] -= 1.0
        assert np.abs(row).max() == 0.0 and np.abs(A[:, d]).sum() == 1.0
        assert P.f0[d] == 0.0


def test_patch_test_linear_fields():
    # unit coefficient: a linear field solves the homogeneous problem away from the boundary
    P = fe.q4_problem(6)
    A = P.csr(P.values(np.ones(P.n_el)))
    xy = np.array([[i / 6, j / 6] for j in range(7) for i in range(7)])
    u = np.column_stack([0.3 * xy[:, 0] - 0.2 * xy[:, 1] + 0.1, 0.7 * xy[:, 1] + 0.4 * xy[:, 0]]).reshape(-1)
    res = (A @ u).reshape(-1, 2)
    # rows next to the clamped edge x = 0 lose their clamped columns: skip them too
    inner = np.all((xy > 1e-9) & (xy < 1 - 1e-9), axis=1) & (xy[:, 0] > 1 / 6 + 1e-9)
    assert np.abs(res[inner]).max() < 1e-12
    P = fe.hex8_problem(4)
    A = P.csr(P.values(np.ones(P.n_el)))
    g = np.array([(i / 4, j / 4, l / 4) for l in range(5) for j in range(5) for i in range(5)])
    u = (g @ np.array([[0.2, -0.1, 0.3], [0.5, 0.1, -0.2], [0.0, 0.4, 0.1]]).T).reshape(-1)
    res = (A @ u).reshape(-1, 3)
    inner = np.all((g > 1e-9) & (g < 1 - 1e-9), axis=1) & (g[:, 2] > 0.25 + 1e-9)
    assert inner.sum() == 18
    assert np.abs(res[inner]).max() < 1e-12


def _poisson_midpoint_series(terms=4001):
    # -lap u = 1 on the unit square, u = 0 on the boundary (double sine series)
    m = np.arange(1, terms + 1, 2, dtype=np.float64)
    sm = np.where(((m - 1) / 2) % 2 == 0, 1.0, -1.0)
    M, N = np.meshgrid(m, m, indexing="ij")
    S = np.outer(sm, sm) / (M * N * (M ** 2 + N ** 2))
    return 16.0 / np.pi ** 4 * S.sum()


def test_poisson_midpoint_converges_at_second_order():
    import scipy.sparse.linalg as sla
    exact = _poisson_midpoint_series()
    assert abs(exact - 0.0736713532814) < 1e-9
    errs = []
    for ne in (16, 32, 64):
        P = fe.q1_problem(ne)
        A = P.csr(P.values(np.ones(P.n_el))).tocsc()
        u = sla.spsolve(A, P.f0)
        mid = (ne // 2 - 1) + (ne - 1) * (ne // 2 - 1)
        errs.append(abs(u[mid] - exact))
    assert errs[-1] < 5e-5
    assert 3.5 < errs[0] / errs[1] < 4.5 and 3.5 < errs[1] / errs[2] < 4.5


def test_loads_integrate_to_total_force():
    assert np.isclose(fe.q4_problem(8).f0.reshape(-1, 2)[:, 1].sum(), -1.0)
    assert np.isclose(fe.hex8_problem(4).f0.reshape(-1, 3)[:, 2].sum(), -1.0)
    P = fe.q1_problem(8)
    assert np.isclose(P.f0.sum(), (7 / 8) ** 2)


def test_kl_trace_and_eigen_equation():
    ne, ell = 40, 0.3
    lam, phi = kl.kl_1d(ne, ell)
    h = 1.0 / ne
    assert np.isclose(lam.sum(), 1.0, rtol=1e-12)   # trace of c(x,x) = 1 over [0, 1]
    x = (np.arange(ne) + 0.5) * h
    C = np.exp(-(x[:, None] - x[None, :]) ** 2 / (2 * ell ** 2))
    for j in range(5):
        assert np.allclose(C @ phi[:, j] * h, lam[j] * phi[:, j], atol=1e-12)
        assert np.isclose((phi[:, j] ** 2).sum() * h, 1.0)


def test_kl_2d_modes_are_eigenpairs_of_the_2d_kernel():
    ne, ell, sigma, m = 8, 0.3, 0.5, 6
    lam, modes = kl.kl_modes(2, ne, ell, sigma, m)
    h = 1.0 / ne
    c = (np.arange(ne) + 0.5) * h
    X = np.array([(cx, cy) for cy in c for cx in c])  # x fastest
    D2 = ((X[:, None, :] - X[None, :, :]) ** 2).sum(-1)
    C = sigma ** 2 * np.exp(-D2 / (2 * ell ** 2)) * h * h
    w = np.sort(np.linalg.eigvalsh(C))[::-1]
    assert np.allclose(lam, w[:m], rtol=1e-10)
    for j in range(m):
        assert np.allclose(C @ modes[:, j], lam[j] * modes[:, j], atol=1e-12)


def test_lognormal_parameters():
    for cov in (0.3, 0.4):
        mu, s = kl.lognormal_params(cov)
        assert np.isclose(np.exp(mu + 0.5 * s * s), 1.0)
        assert np.isclose(np.sqrt(np.expm1(s * s)), cov)


def test_workload_seeds_are_deterministic():
    wl = Workload("q4_16")
    a = wl.values(wl.query_thetas(2)[1])
    b = Workload("q4_16").values(Workload("q4_16").query_thetas(2)[1])
    assert np.array_equal(a, b)
    th = wl.snapshot_thetas()
    assert th.shape == (SPECS["q4_16"].n_snap, SPECS["q4_16"].m)


@pytest.mark.parametrize("name", ["q1_16", "q4_16", "hex8_8"])
def test_batched_torch_assembly_identical(name):
    torch = pytest.importorskip("torch")
    wl = Workload(name)
    xis = wl.query_thetas(3)
    V = wl.values_torch(xis).numpy()
    for i, xi in enumerate(xis):
        assert np.array_equal(V[i], wl.values(xi))


# ----------------------------------------------------------------------------- multigrid snapshot solver
@pytest.mark.parametrize("name", ["q1_16", "q4_16", "hex8_8"])
def test_grid_operator_equals_assembled_matrix(name):
    torch = pytest.importorskip("torch")
    from synth import mg
    from synth.problems import Workload
    wl = Workload(name)
    P = wl.problem
    xis = wl.snapshot_thetas(2)
    coef = torch.from_numpy(np.stack([wl.coef(x) for x in xis]))
    A = mg.GridOperator(P.kind, P.ne, coef, torch.float64)
    u = np.random.default_rng(0).standard_normal((2, P.n))
    Y = mg.from_grid(P, A.apply(mg.to_grid(P, torch.from_numpy(u)))).numpy()
    D = mg.from_grid(P, A.diagonal()).numpy()
    for s in range(2):
        K = P.csr(wl.values(xis[s]))
        ref = K @ u[s]
        assert np.abs(Y[s] - ref).max() <= 1e-13 * np.abs(ref).max()
        assert np.allclose(D[s], K.diagonal(), rtol=1e-14)


@pytest.mark.parametrize("dim", [2, 3])
def test_restriction_is_the_transpose_of_interpolation(dim):
    torch = pytest.importorskip("torch")
    from synth import mg
    rng = np.random.default_rng(dim)
    nc = 5
    X = torch.from_numpy(rng.standard_normal((1,) + (nc,) * dim + (2,)))
    Y = torch.from_numpy(rng.standard_normal((1,) + (2 * nc - 1,) * dim + (2,)))
    PX = mg.prolong(X, dim)
    assert PX.shape == Y.shape
    assert abs(float((PX * Y).sum()) - float((X * mg.restrict(Y, dim)).sum())) <= 1e-12 * float(
        (PX.abs() * Y.abs()).sum())
    # interpolation reproduces a linear field exactly
    grid = torch.stack(torch.meshgrid(*([torch.arange(nc, dtype=torch.float64)] * dim), indexing="ij"), -1)
    lin = (grid @ torch.arange(1.0, dim + 1, dtype=torch.float64))[None, ..., None]
    fine = torch.stack(torch.meshgrid(*([torch.arange(2 * nc - 1, dtype=torch.float64) / 2] * dim), indexing="ij"),
                       -1)
    assert torch.allclose(mg.prolong(lin, dim), (fine @ torch.arange(1.0, dim + 1, dtype=torch.float64))[None, ..., None])


@pytest.mark.parametrize("name", ["q1_32", "q4_64", "hex8_16"])
def test_multigrid_pcg_matches_direct_solve(name):
    torch = pytest.importorskip("torch")
    import scipy.sparse.linalg as sla
    from synth import mg
    from synth.problems import Workload
    wl = Workload(name)
    P = wl.problem
    xis = wl.snapshot_thetas(2)
    coef = torch.from_numpy(np.stack([wl.coef(x) for x in xis]))
    X, it = mg.mg_pcg(P, coef, P.f0, tol=1e-11)
    assert it <= 40
    for s in range(2):
        vals = wl.values(xis[s])
        xs = sla.splu(P.csr(vals).tocsc()).solve(P.f0)
        assert np.linalg.norm(X[s].numpy() - xs) <= 1e-9 * np.linalg.norm(xs)
        rel = mg.bsr_residual(P, torch.from_numpy(vals), X[s], P.f0)
        assert rel <= 1e-10

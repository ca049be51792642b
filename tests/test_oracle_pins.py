"""Pins for the CPU oracle, each against something other than the oracle itself.

* dense Cholesky vs the definition L L^T = A and a library solve;
* POD by the method of snapshots vs the SVD route (Eckart-Young energy identity);
* the two-grid cycle (Algorithm 2, step by step) vs the dense error operator
  M^{r2} C M^{r1} of eq. AMGerror / eq. FinalScheme;
* PCG iterates vs brute-force A-norm minimisation over the Krylov space
  (Section 2.1, eq. MinProblemCG), orthogonality of residuals and conjugacy of
  directions, A-norm monotonicity;
* special cases: full coarse space => one iteration; b in K Phi with r1 = 0 =>
  one iteration and x = Phi c; empty coarse space => two damped-Jacobi sweeps
  B = 2S - S K S; Phi -> Phi Q invariance; x0 = x* => 0 iterations; f = 0;
* planted mistakes: modified copies of oracle steps fail the pins above;
* the power-iteration estimate of rho(D^-1 K) vs the dense eigenvalues of D^-1/2 K D^-1/2.
"""
import numpy as np
import pytest
import scipy.sparse as sp

import oracle
from oracle import pod2g_oracle as O
from synth import fe
from synth.problems import Workload
from synth.snapshots import pod_basis, snapshot_matrix


def _small_system(seed=0, ne=5, kind="q1"):
    P = fe._build(kind, ne)
    c = np.random.default_rng(seed).lognormal(0.0, 0.5, P.n_el)
    K = P.csr(P.values(c))
    return P, K


def _basis(K, k, seed=1):
    # a smooth-ish orthonormal basis: a few exact solutions for random loads, orthonormalised
    rng = np.random.default_rng(seed)
    F = rng.standard_normal((K.shape[0], k))
    X = np.linalg.solve(K.toarray(), F)
    Q, _ = np.linalg.qr(X)
    return Q


def _spd(k, seed=0):
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((k, k))
    return A @ A.T + k * np.eye(k)


# ----------------------------------------------------------------------------- Cholesky
@pytest.mark.parametrize("k", [1, 2, 7, 20])
def test_cholesky_definition_and_solve(k):
    A = _spd(k, k)
    L = O.cholesky(A)
    assert np.allclose(np.tril(L), L)
    assert np.allclose(L @ L.T, A, rtol=1e-13, atol=1e-12)
    assert np.allclose(L, np.linalg.cholesky(A), rtol=1e-12)
    c = np.random.default_rng(k).standard_normal(k)
    assert np.allclose(O.cholesky_solve(L, c), np.linalg.solve(A, c), rtol=1e-11)


def test_cholesky_rejects_indefinite():
    A = _spd(5)
    A[2, 2] = -1.0
    with pytest.raises(np.linalg.LinAlgError):
        O.cholesky(A)


# ----------------------------------------------------------------------------- POD
def test_pod_method_of_snapshots_matches_svd():
    rng = np.random.default_rng(3)
    U = rng.standard_normal((200, 12)) @ np.diag(2.0 ** -np.arange(12)) @ rng.standard_normal((12, 30))
    r = 5
    Phi, lam = O.pod_method_of_snapshots(U, r)
    W, s, _ = np.linalg.svd(U, full_matrices=False)
    assert np.allclose(Phi.T @ Phi, np.eye(r), atol=1e-10)
    assert np.allclose(lam[:12], s[:12] ** 2, rtol=1e-9)
    assert np.isclose(lam.sum(), np.linalg.norm(U) ** 2, rtol=1e-12)
    assert np.allclose(Phi @ Phi.T, W[:, :r] @ W[:, :r].T, atol=1e-9)
    # Eckart-Young: truncation error equals the discarded energy
    E = U - Phi @ (Phi.T @ U)
    assert np.isclose(np.linalg.norm(E) ** 2, lam[r:].sum(), rtol=1e-6)


def test_pod_of_real_snapshots_spans_generator_basis():
    wl = Workload("q1_16")
    U = snapshot_matrix(wl)
    Phi, lam = O.pod_method_of_snapshots(U, wl.spec.k)
    G = pod_basis(wl, use_disk=False)
    assert np.allclose(Phi @ Phi.T, G @ G.T, atol=1e-8)
    assert lam[:wl.spec.k].sum() / lam.sum() > 1 - 1e-4


# ----------------------------------------------------------------------------- Algorithm 2
@pytest.mark.parametrize("r1,r2", [(1, 1), (0, 1), (2, 1), (1, 0)])
def test_two_grid_cycle_equals_error_operator(r1, r2):
    P, K = _small_system(2)
    Phi = _basis(K, 4)
    st = O.pod2g_setup(K, Phi, 2 / 3, r1, r2)
    E = O.two_grid_error_operator(K, Phi, st.Dinv, 2 / 3, r1, r2)
    Kd = K.toarray()
    rng = np.random.default_rng(5)
    f = rng.standard_normal(K.shape[0])
    u0 = rng.standard_normal(K.shape[0])
    xs = np.linalg.solve(Kd, f)
    u1 = O.two_grid_cycle(K, f, u0, Phi, st.L_c, st.Dinv, 2 / 3, r1, r2)
    assert np.allclose(xs - u1, E @ (xs - u0), atol=1e-11 * np.abs(xs).max())


def test_preconditioner_symmetric_positive_definite():
    P, K = _small_system(4, kind="q4", ne=3)
    Phi = _basis(K, 3)
    st = O.pod2g_setup(K, Phi, 2 / 3)
    assert 2 / 3 * O.spectral_radius_estimate(K, st.Dinv, 200) < 2
    apply = O.pod2g_preconditioner(K, st)
    n = K.shape[0]
    B = np.column_stack([apply(e) for e in np.eye(n)])
    Kd = K.toarray()
    E = O.two_grid_error_operator(K, Phi, st.Dinv, 2 / 3)
    assert np.allclose(B, (np.eye(n) - E) @ np.linalg.inv(Kd), atol=1e-10)
    assert np.abs(B - B.T).max() < 1e-12 * np.abs(B).max()
    assert np.linalg.eigvalsh(0.5 * (B + B.T)).min() > 0


def test_galerkin_orthogonality_after_correction():
    P, K = _small_system(6)
    Phi = _basis(K, 5)
    st = O.pod2g_setup(K, Phi, 2 / 3)
    f = np.random.default_rng(0).standard_normal(K.shape[0])
    tr = {}
    O.two_grid_cycle(K, f, np.zeros_like(f), Phi, st.L_c, st.Dinv, 2 / 3, 1, 1, trace=tr)
    assert np.abs(Phi.T @ (f - K @ tr["after_correction"])).max() < 1e-12 * np.abs(f).max()


def test_empty_coarse_space_is_two_jacobi_sweeps():
    P, K = _small_system(7)
    n = K.shape[0]
    st = O.pod2g_setup(K, np.zeros((n, 0)), 2 / 3)
    S = np.diag(2 / 3 * st.Dinv)
    Kd = K.toarray()
    B = 2 * S - S @ Kd @ S
    f = np.random.default_rng(1).standard_normal(n)
    assert np.allclose(O.pod2g_preconditioner(K, st)(f), B @ f, atol=1e-13)


# ----------------------------------------------------------------------------- Algorithms 1 / 3
def _krylov_min(Kd, f, x0, Bd, k):
    """Brute force: x in x0 + span{z, (BK) z, ...} (k vectors, z = B r0) minimising ||x - x*||_K."""
    r0 = f - Kd @ x0
    z = Bd @ r0
    V = [z]
    for _ in range(k - 1):
        V.append(Bd @ (Kd @ V[-1]))
    V = np.column_stack(V)
    V, _ = np.linalg.qr(V)
    y = np.linalg.solve(V.T @ Kd @ V, V.T @ r0)
    return x0 + V @ y


@pytest.mark.parametrize("beta", ["fr", "pr"])
@pytest.mark.parametrize("precond", ["identity", "jacobi", "pod2g"])
def test_pcg_iterates_minimise_energy_norm(precond, beta):
    # With a fixed SPD preconditioner r_{k+1}^T s_k = 0, so the Polak-Ribiere beta equals the
    # Algorithm 1 ratio and both give the K-norm minimiser over the preconditioned Krylov space.
    P, K = _small_system(8, ne=6)
    n = K.shape[0]
    Kd = K.toarray()
    rng = np.random.default_rng(2)
    f = rng.standard_normal(n)
    x0 = rng.standard_normal(n)
    if precond == "identity":
        app = lambda r: r.copy()
    elif precond == "jacobi":
        app = O.jacobi_preconditioner(K)
    else:
        app = O.pod2g_preconditioner(K, O.pod2g_setup(K, _basis(K, 3), 2 / 3))
    Bd = np.column_stack([app(e) for e in np.eye(n)])
    res = O.pcg(K, f, x0, app, 1e-30, 6, beta=beta, record=True)
    xs = np.linalg.solve(Kd, f)
    for k in range(1, 7):
        xk = res.iterates[k]["x"]
        xb = _krylov_min(Kd, f, x0, Bd, k)
        assert np.linalg.norm(xk - xb) <= 1e-8 * np.linalg.norm(xs - x0)


def test_pcg_orthogonality_and_monotone_energy_error():
    P, K = _small_system(9, ne=8)
    Phi = _basis(K, 4)
    f = np.random.default_rng(4).standard_normal(K.shape[0])
    res = O.pod2g_pcg(K, f, None, Phi, 2 / 3, 1e-30, 10, record=True)
    Kd = K.toarray()
    xs = np.linalg.solve(Kd, f)
    R = res.iterates
    for i in range(8):
        for j in range(8):
            if i != j:
                assert abs(R[i]["r"] @ R[j]["s"]) < 1e-9 * np.sqrt(abs(R[i]["r"] @ R[i]["s"]) * abs(R[j]["r"] @ R[j]["s"]))
                pi, pj = R[i]["p"], R[j]["p"]
                assert abs(pi @ Kd @ pj) < 1e-9 * np.sqrt((pi @ Kd @ pi) * (pj @ Kd @ pj))
    errs = [np.sqrt((xs - it["x"]) @ Kd @ (xs - it["x"])) for it in R]
    assert all(b < a for a, b in zip(errs, errs[1:]))


def test_pcg_converges_to_dense_solution():
    P, K = _small_system(10, ne=12)
    Phi = _basis(K, 5)
    f = P.f0
    res = O.pod2g_pcg(K, f, None, Phi, 2 / 3, 1e-10, 500)
    assert res.status == O.OK and res.relres <= 1.1e-10
    xs = np.linalg.solve(K.toarray(), f)
    cond = np.linalg.cond(K.toarray())
    assert np.linalg.norm(res.x - xs) <= cond * 1.1e-10 * np.linalg.norm(xs)
    assert res.history[-1] <= 1e-10 < res.history[-2]


def test_full_coarse_space_one_iteration():
    P, K = _small_system(11, ne=4)
    n = K.shape[0]
    Q, _ = np.linalg.qr(np.random.default_rng(0).standard_normal((n, n)))
    res = O.pod2g_pcg(K, P.f0, None, Q, 2 / 3, 1e-10, 50)
    assert res.iters == 1 and res.relres < 1e-12


def test_rhs_in_range_of_K_Phi_one_iteration_without_presmoothing():
    P, K = _small_system(12, ne=7)
    Phi = _basis(K, 4)
    c = np.array([1.0, -2.0, 0.5, 3.0])
    f = K @ (Phi @ c)
    res = O.pod2g_pcg(K, f, None, Phi, 2 / 3, 1e-10, 50, r1=0, r2=1)
    assert res.iters == 1
    assert np.allclose(res.x, Phi @ c, rtol=1e-12, atol=1e-13)


def test_rotation_of_basis_leaves_iterates_unchanged():
    P, K = _small_system(13, ne=9)
    Phi = _basis(K, 5)
    Q, _ = np.linalg.qr(np.random.default_rng(3).standard_normal((5, 5)))
    a = O.pod2g_pcg(K, P.f0, None, Phi, 2 / 3, 1e-9, 200)
    b = O.pod2g_pcg(K, P.f0, None, Phi @ Q, 2 / 3, 1e-9, 200)
    assert a.iters == b.iters
    assert np.allclose(a.history, b.history, rtol=1e-6)
    assert np.allclose(a.x, b.x, rtol=1e-9, atol=1e-12 * np.abs(a.x).max())


def test_special_inputs():
    P, K = _small_system(14)
    Phi = _basis(K, 3)
    n = K.shape[0]
    r = O.pod2g_pcg(K, np.zeros(n), np.ones(n), Phi, 2 / 3, 1e-8, 10)
    assert r.iters == 0 and r.status == O.OK and np.all(r.x == 0)
    xs = np.linalg.solve(K.toarray(), P.f0)
    r = O.pod2g_pcg(K, P.f0, xs, Phi, 2 / 3, 1e-8, 10)
    assert r.iters == 0 and r.status == O.OK
    r = O.pod2g_pcg(K, P.f0, None, Phi, 2 / 3, 1e-14, 2)
    assert r.iters == 2 and r.status == O.NOT_CONVERGED
    dep = np.column_stack([Phi[:, 0], Phi[:, 0]])
    r = O.pod2g_pcg(K, P.f0, None, dep, 2 / 3, 1e-8, 10)
    assert r.status == O.NOT_SPD


def test_better_pod_space_and_initial_guess_need_fewer_iterations():
    wl = Workload("q1_16")
    Pb = wl.problem
    K = Pb.csr(wl.values(wl.query_thetas(1)[0]))
    f = Pb.f0
    U = snapshot_matrix(wl)
    its = []
    for k in (2, 4, 8):
        Phi, _ = O.pod_method_of_snapshots(U, k)
        its.append(O.pod2g_pcg(K, f, None, Phi, 2 / 3, 1e-8, 500).iters)
    assert its[0] >= its[1] >= its[2]
    Phi, _ = O.pod_method_of_snapshots(U, 6)
    cold = O.pod2g_pcg(K, f, None, Phi, 2 / 3, 1e-8, 500).iters
    warm = O.pod2g_pcg(K, f, O.rom_solution(K, Phi, f), Phi, 2 / 3, 1e-8, 500).iters
    jac = O.jacobi_pcg(K, f, None, 1e-8, 2000).iters
    assert warm <= cold < jac


# ----------------------------------------------------------------------------- planted mistakes
def _cycle_without_post_relaxation(K, f, u, Phi, L_c, Dinv, omega, r1, r2, trace=None):
    return O.two_grid_cycle(K, f, u, Phi, L_c, Dinv, omega, r1, 0)


def _cycle_transposed_restriction(K, f, u, Phi, L_c, Dinv, omega, r1, r2, trace=None):
    u = O.damped_jacobi(K, Dinv, omega, f, u, r1)
    r = f - K @ u
    e_c = O.cholesky_solve(L_c, Phi.T @ (K @ r))   # wrong: restricts K r
    u = u + Phi @ e_c
    return O.damped_jacobi(K, Dinv, omega, f, u, r2)


@pytest.mark.parametrize("bad", [_cycle_without_post_relaxation, _cycle_transposed_restriction])
def test_planted_cycle_mistakes_are_caught(bad, monkeypatch):
    P, K = _small_system(2)
    Phi = _basis(K, 4)
    st = O.pod2g_setup(K, Phi, 2 / 3, 1, 1)
    E = O.two_grid_error_operator(K, Phi, st.Dinv, 2 / 3, 1, 1)
    f = np.random.default_rng(5).standard_normal(K.shape[0])
    xs = np.linalg.solve(K.toarray(), f)
    u1 = bad(K, f, np.zeros_like(f), Phi, st.L_c, st.Dinv, 2 / 3, 1, 1)
    assert not np.allclose(xs - u1, E @ xs, atol=1e-8 * np.abs(xs).max())


def test_planted_beta_mistake_is_caught(monkeypatch):
    P, K = _small_system(8, ne=6)
    n = K.shape[0]
    Kd = K.toarray()
    f = np.random.default_rng(2).standard_normal(n)
    app = O.jacobi_preconditioner(K)
    Bd = np.diag(1 / K.diagonal())
    # beta with the wrong sign: p = s - beta p
    x, r = np.zeros(n), f.copy()
    s = app(r); p = s.copy(); rs = r @ s
    for k in range(3):
        q = K @ p; a = rs / (p @ q); x = x + a * p; r = r - a * q
        s = app(r); rs_new = r @ s; p = s - (rs_new / rs) * p; rs = rs_new
    xb = _krylov_min(Kd, f, np.zeros(n), Bd, 3)
    assert np.linalg.norm(x - xb) > 1e-6 * np.linalg.norm(xb)
    good = O.pcg(K, f, None, app, 1e-30, 3)
    assert np.linalg.norm(good.x - xb) <= 1e-9 * np.linalg.norm(xb)


class _VaryingPreconditioner:
    """s = B_j r for the j-th application: B_j = D^{-1} scaled by a seeded positive diagonal
    that changes on every call (symmetric and positive definite, but not the same operator
    twice), so that r_{k+1}^T s_k != 0 and the two beta forms differ."""

    def __init__(self, K, seed):
        self.dinv = 1.0 / K.diagonal()
        self.rng = np.random.default_rng(seed)

    def __call__(self, r):
        return self.dinv * self.rng.uniform(0.5, 2.0, r.shape[0]) * r


def test_polak_ribiere_conjugacy_defect_under_a_varying_preconditioner():
    # For any preconditioner sequence, p_{k+1} = s_{k+1} + beta p_k with K p_k = (r_k - r_{k+1}) / alpha_k
    # and alpha_k p_k^T K p_k = r_k^T s_k gives
    #   alpha_k p_{k+1}^T K p_k = s_{k+1}^T r_k - s_{k+1}^T r_{k+1} + beta r_k^T s_k.
    # The Polak-Ribiere beta r_{k+1}^T (s_{k+1} - s_k) / r_k^T s_k makes the right-hand side
    # s_{k+1}^T r_k - r_{k+1}^T s_k (zero for a fixed symmetric preconditioner), the Algorithm 1
    # ratio makes it s_{k+1}^T r_k. Both are checked on the recorded iterates, where the two
    # forms give different directions.
    P, K = _small_system(8, ne=6)
    Kd = K.toarray()
    f = np.random.default_rng(3).standard_normal(K.shape[0])
    recs = {}
    for beta in ("pr", "fr"):
        res = O.pcg(K, f, None, _VaryingPreconditioner(K, 11), 1e-30, 6, beta=beta, record=True)
        R = res.iterates
        recs[beta] = R
        for k in range(1, 5):
            rk, sk, pk = R[k]["r"], R[k]["s"], R[k]["p"]
            r1, s1, p1 = R[k + 1]["r"], R[k + 1]["s"], R[k + 1]["p"]
            alpha = (rk @ sk) / (pk @ Kd @ pk)
            lhs = alpha * (p1 @ Kd @ pk)
            rhs = s1 @ rk - (r1 @ sk if beta == "pr" else 0.0)
            scale = abs(s1 @ rk) + abs(r1 @ sk) + abs(s1 @ r1)
            assert abs(lhs - rhs) <= 1e-9 * scale, (beta, k, lhs, rhs)
    # the two forms really differ here (the pin above is not vacuous)
    d = np.linalg.norm(recs["pr"][4]["x"] - recs["fr"][4]["x"])
    assert d > 1e-6 * np.linalg.norm(recs["fr"][4]["x"])


def test_planted_polak_ribiere_mistakes_are_caught():
    # copies of the PR update with a wrong sign inside, or the new r^T s as denominator, break
    # one of the two pins above (varying-preconditioner identity, or the fixed-preconditioner
    # Krylov minimiser)
    P, K = _small_system(8, ne=6)
    n = K.shape[0]
    Kd = K.toarray()
    f = np.random.default_rng(2).standard_normal(n)

    def run(app, rule, steps):
        x, r = np.zeros(n), f.copy()
        s = app(r); p = s.copy(); rs = r @ s
        out = []
        for _ in range(steps):
            q = K @ p; a = rs / (p @ q); x = x + a * p; r_new = r - a * q
            s_new = app(r_new); rs_new = r_new @ s_new
            b = rule(r_new, s_new, s, rs, rs_new)
            p_new = s_new + b * p
            out.append((a, r, s, p, r_new, s_new, p_new))
            r, s, p, rs = r_new, s_new, p_new, rs_new
        return x, out

    wrong_sign = lambda r1, s1, s0, rs, rs1: r1 @ (s1 + s0) / rs  # noqa: E731
    wrong_den = lambda r1, s1, s0, rs, rs1: r1 @ (s1 - s0) / rs1  # noqa: E731
    # wrong sign: the conjugacy identity of the varying-preconditioner pin fails
    _, out = run(_VaryingPreconditioner(K, 11), wrong_sign, 4)
    bad = 0
    for a, rk, sk, pk, r1, s1, p1 in out[1:]:
        lhs = a * (p1 @ Kd @ pk)
        rhs = s1 @ rk - r1 @ sk
        bad += abs(lhs - rhs) > 1e-6 * (abs(s1 @ rk) + abs(r1 @ sk) + abs(s1 @ r1))
    assert bad > 0
    # wrong denominator: the fixed-preconditioner iterates leave the Krylov minimiser
    x, _ = run(O.jacobi_preconditioner(K), wrong_den, 3)
    xb = _krylov_min(Kd, f, np.zeros(n), np.diag(1 / K.diagonal()), 3)
    assert np.linalg.norm(x - xb) > 1e-6 * np.linalg.norm(xb)


# ----------------------------------------------------------------------------- Algorithm 2 as a solver
def test_stationary_iterates_follow_error_operator_powers():
    P, K = _small_system(15, ne=6)
    Phi = _basis(K, 4)
    n = K.shape[0]
    st = O.pod2g_setup(K, Phi, 2 / 3)
    E = O.two_grid_error_operator(K, Phi, st.Dinv, 2 / 3)
    rng = np.random.default_rng(8)
    f = rng.standard_normal(n)
    u0 = rng.standard_normal(n)
    xs = np.linalg.solve(K.toarray(), f)
    for k in (1, 3, 7):
        res = O.pod2g_stationary(K, f, u0, Phi, 2 / 3, 0.0, k)
        assert res.iters == k
        assert np.allclose(xs - res.x, np.linalg.matrix_power(E, k) @ (xs - u0), atol=1e-10 * np.abs(xs).max())


def test_stationary_converges_with_contraction_rate():
    P, K = _small_system(16, ne=10)
    Phi = _basis(K, 6)
    st = O.pod2g_setup(K, Phi, 2 / 3)
    E = O.two_grid_error_operator(K, Phi, st.Dinv, 2 / 3)
    rho = max(abs(np.linalg.eigvals(E)))
    assert rho < 1
    res = O.pod2g_stationary(K, P.f0, None, Phi, 2 / 3, 1e-8, 5000)
    assert res.status == O.OK and res.relres <= 1e-8
    # the residual contracts asymptotically at about rho per cycle
    h = np.array(res.history)
    tail = (h[-1] / h[-11]) ** 0.1
    assert tail <= rho * 1.05
    xs = np.linalg.solve(K.toarray(), P.f0)
    assert np.linalg.norm(res.x - xs) <= 1e-6 * np.linalg.norm(xs)


def test_stationary_special_inputs():
    P, K = _small_system(17)
    Phi = _basis(K, 3)
    n = K.shape[0]
    r = O.pod2g_stationary(K, np.zeros(n), np.ones(n), Phi, 2 / 3, 1e-8, 10)
    assert r.iters == 0 and np.all(r.x == 0)
    r = O.pod2g_stationary(K, P.f0, None, Phi, 2 / 3, 1e-14, 3)
    assert r.iters == 3 and r.status == O.NOT_CONVERGED


# ----------------------------------------------------------------------------- Gauss-Seidel relaxation
def _gs_system(kind="q4", ne=4, seed=20):
    P, K = _small_system(seed, ne=ne, kind=kind)
    groups = O.multicolour_groups(P.row_ptr, P.col_idx, P.bs)
    return P, K, groups


@pytest.mark.parametrize("kind,ne,colours", [("q1", 6, 4), ("q4", 5, 4), ("hex8", 3, 8)])
def test_multicolour_groups_are_independent_and_partition(kind, ne, colours):
    P, K, groups = _gs_system(kind, ne)
    assert len(groups) == colours * P.bs
    allg = np.sort(np.concatenate(groups))
    assert np.array_equal(allg, np.arange(P.n))
    Kd = K.toarray()
    for g in groups:
        sub = Kd[np.ix_(g, g)]
        assert np.count_nonzero(sub - np.diag(np.diag(sub))) == 0    # no coupling inside a group
    # structural check on the block pattern: neighbours never share a colour
    nodecol = np.empty(P.n_nodes, dtype=int)
    for t, g in enumerate(groups):
        nodecol[g // P.bs] = t // P.bs
    rows = np.repeat(np.arange(P.n_nodes), np.diff(P.row_ptr))
    off = rows != P.col_idx
    assert np.all(nodecol[rows[off]] != nodecol[P.col_idx[off]])


def test_gauss_seidel_sweep_equals_triangular_splitting():
    from scipy.linalg import solve_triangular
    P, K, groups = _gs_system("q4", 4)
    order = np.concatenate(groups)
    Kd = K.toarray()
    rng = np.random.default_rng(3)
    f, u = rng.standard_normal(P.n), rng.standard_normal(P.n)
    Kp = Kd[np.ix_(order, order)]
    for reverse, lower in ((False, True), (True, False)):
        tri = np.tril(Kp) if lower else np.triu(Kp)
        step = solve_triangular(tri, (f - Kd @ u)[order], lower=lower)
        want = u.copy()
        want[order] += step
        got = O.gauss_seidel(K, K.diagonal(), f, u, groups, 1, reverse=reverse)
        assert np.allclose(got, want, rtol=1e-12, atol=1e-12 * np.abs(want).max())


def test_symmetric_gauss_seidel_cycle_and_preconditioner():
    P, K, groups = _gs_system("q4", 4, 21)
    Phi = _basis(K, 3)
    order = np.concatenate(groups)
    st = O.pod2g_setup(K, Phi, 1.0, 1, 1, groups)
    E = O.two_grid_error_operator(K, Phi, st.Dinv, 1.0, order=order)
    Kd = K.toarray()
    rng = np.random.default_rng(5)
    f, u0 = rng.standard_normal(P.n), rng.standard_normal(P.n)
    xs = np.linalg.solve(Kd, f)
    u1 = O.two_grid_cycle(K, f, u0, Phi, st.L_c, st.Dinv, 1.0, 1, 1, groups=groups)
    assert np.allclose(xs - u1, E @ (xs - u0), atol=1e-10 * np.abs(xs).max())
    app = O.pod2g_preconditioner(K, st)
    B = np.column_stack([app(e) for e in np.eye(P.n)])
    assert np.abs(B - B.T).max() < 1e-12 * np.abs(B).max()
    assert np.linalg.eigvalsh(0.5 * (B + B.T)).min() > 0
    # planted mistake: forward sweeps on both sides give a non-symmetric cycle
    fwd = O.gauss_seidel
    bad = lambda r: (lambda y: fwd(K, K.diagonal(), r, y + Phi @ O.cholesky_solve(st.L_c, Phi.T @ (r - K @ y)),
                                   groups, 1))(fwd(K, K.diagonal(), r, np.zeros_like(r), groups, 1))
    Bb = np.column_stack([bad(e) for e in np.eye(P.n)])
    assert np.abs(Bb - Bb.T).max() > 1e-6 * np.abs(Bb).max()


def test_gauss_seidel_smoother_needs_fewer_pcg_iterations():
    P, K, groups = _gs_system("q1", 24, 22)
    Phi = _basis(K, 6)
    f = P.f0
    jac = O.pod2g_pcg(K, f, None, Phi, 2 / 3, 1e-8, 500)
    sgs = O.pod2g_pcg(K, f, None, Phi, 1.0, 1e-8, 500, groups=groups)
    assert jac.status == O.OK and sgs.status == O.OK
    assert sgs.iters < jac.iters
    xs = np.linalg.solve(K.toarray(), f)
    assert np.linalg.norm(sgs.x - xs) <= 1e-6 * np.linalg.norm(xs)


# ----------------------------------------------------------------------------- Section 3.3 steps 3-4
def test_rom_solution_is_the_galerkin_projection():
    """x_rom = Phi u_r with K_r u_r = Phi^T f: residual orthogonal to span(Phi), the K-norm
    best approximation of x* in span(Phi) (checked against a least-squares solve in the
    K-inner product), exact when x* lies in span(Phi)."""
    P, K = _small_system(30, ne=6)
    Kd = K.toarray()
    Phi = _basis(K, 5)
    f = P.f0
    x = O.rom_solution(K, Phi, f)
    assert np.abs(Phi.T @ (f - Kd @ x)).max() < 1e-12 * np.abs(f).max()
    xs = np.linalg.solve(Kd, f)
    Lk = np.linalg.cholesky(Kd)                      # ||v||_K = ||L^T v||_2
    coef, *_ = np.linalg.lstsq(Lk.T @ Phi, Lk.T @ xs, rcond=None)
    assert np.allclose(x, Phi @ coef, rtol=1e-9, atol=1e-12 * np.abs(xs).max())
    c = np.random.default_rng(3).standard_normal(5)
    assert np.allclose(O.rom_solution(K, Phi, Kd @ (Phi @ c)), Phi @ c, rtol=1e-10, atol=1e-12)


# ----------------------------------------------------------------------------- smoother bound
@pytest.mark.parametrize("kind,ne", [("q4", 4), ("hex8", 3), ("q1", 6)])
def test_spectral_radius_estimate_matches_dense_eigenvalues(kind, ne):
    """rho(D^-1 K) from power iteration against the largest eigenvalue of the symmetric similar
    matrix D^-1/2 K D^-1/2 (dense, LAPACK), which bounds the admissible Jacobi damping (omega rho < 2)."""
    P, K = _small_system(3, ne=ne, kind=kind)
    Dinv = O.jacobi_inverse_diagonal(K)
    s = np.sqrt(Dinv)
    lam = np.linalg.eigvalsh(s[:, None] * K.toarray() * s[None, :]).max()
    est = O.spectral_radius_estimate(K, Dinv, 400)
    assert abs(est - lam) <= 0.02 * lam, (est, lam)

"""CPU FP64 oracle of the POD-2G-preconditioned conjugate gradient method.

TEST INFRASTRUCTURE ONLY. This module is the independent, slow, obviously correct
statement of what the CUDA solver computes. Only the tests, the package's smoke
check and the CPU-baseline leg of the benchmark may import it; the solver library
never does, and it shares no code with the CUDA path.

Every routine follows one passage of arXiv 2207.02543 (Nikolopoulos et al.,
"AI-enhanced iterative solvers for accelerating the solution of large scale
parametrized systems"), in the paper's order and notation:

  * pcg                      Algorithm 1 (PCG) and Algorithm 3 (PCG with an AMG
                             preconditioner), Section 2.1 / Section 3.4
  * two_grid_cycle           Algorithm 2 (two-level cycle), Section 2.2, with the
                             prolongation P := Phi_r (Section 3.3)
  * pod2g_preconditioner     s = AMG(0; K, r, r1, r2), Algorithm 3
  * damped_jacobi            the relaxation scheme G (damped Jacobi; the paper
                             analyses Gauss-Seidel, eq. GaussSeidel)
  * gauss_seidel             pointwise Gauss-Seidel, eq. GaussSeidel, in a multicolour
    multicolour_groups       order (forward before, backward after the correction)
  * pod_method_of_snapshots  Section 3.3 steps 1-2, eq. PODrelationEigenvectors
  * coarse_operator          K_r = Phi_r^T K Phi_r, eq. POD_ROM
  * rom_solution             u = Phi_r K_r^{-1} Phi_r^T f, Section 3.3 steps 3-4
  * two_grid_error_operator  e^(k) = M^{r2} (I - Phi (Phi^T K Phi)^{-1} Phi^T K) M^{r1}
                             e^(k-1), eq. AMGerror / eq. FinalScheme
  * cholesky / cholesky_solve  textbook dense Cholesky for the k x k coarse system

Readings where the paper is silent or garbled (each also listed in the design notes):
  * the loop condition printed as "while ||r|| < delta" is read as
    "while ||r|| > delta" (Algorithms 1-3);
  * delta is a relative tolerance: stop when ||r_k||_2 <= tol * ||f||_2, tested on
    the recurrence residual before every iteration, k = 0 included;
  * iteration count = number of alpha updates; maxit reached => not converged,
    the last iterate returned; f = 0 => x = 0 with 0 iterations;
  * relaxation = damped Jacobi u <- u + omega D^{-1} (f - K u), r1 = r2 = 1 by default;
  * beta is the ratio printed in Algorithm 1 (Fletcher-Reeves form); the
    Polak-Ribiere variant r_{k+1}^T (s_{k+1} - s_k) / r_k^T s_k is available as
    an option (identical in exact arithmetic for a fixed SPD preconditioner);
  * K_r is symmetrised, (K_r + K_r^T) / 2, before its Cholesky factorisation.
Sparse products use scipy.sparse (a library SpMV); dense factorisations are
written out.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

# status codes (same meaning as the library's)
OK, NOT_CONVERGED, BREAKDOWN, NOT_SPD = 0, 1, 2, 3


def jacobi_inverse_diagonal(K) -> np.ndarray:
    """D^{-1} with D = diag(K) (the Jacobi preconditioner T = diag(K), Section 2.1)."""
    d = np.asarray(K.diagonal(), dtype=np.float64)
    if np.any(~(d > 0)):
        raise ValueError("non-positive diagonal")
    return 1.0 / d


# ----------------------------------------------------------------------------- dense k x k
def cholesky(A: np.ndarray) -> np.ndarray:
    """Lower-triangular L with L L^T = A (textbook column algorithm). Raises on a non-SPD A."""
    A = np.asarray(A, dtype=np.float64)
    k = A.shape[0]
    L = np.zeros_like(A)
    for j in range(k):
        d = A[j, j] - sum(L[j, t] * L[j, t] for t in range(j))
        if not d > 0:
            raise np.linalg.LinAlgError("coarse matrix is not SPD")
        L[j, j] = np.sqrt(d)
        for i in range(j + 1, k):
            L[i, j] = (A[i, j] - sum(L[i, t] * L[j, t] for t in range(j))) / L[j, j]
    return L


def cholesky_solve(L: np.ndarray, c: np.ndarray) -> np.ndarray:
    """Solve L L^T e = c by forward then backward substitution."""
    k = L.shape[0]
    y = np.zeros(k)
    for i in range(k):
        y[i] = (c[i] - sum(L[i, t] * y[t] for t in range(i))) / L[i, i]
    e = np.zeros(k)
    for i in reversed(range(k)):
        e[i] = (y[i] - sum(L[t, i] * e[t] for t in range(i + 1, k))) / L[i, i]
    return e


# ----------------------------------------------------------------------------- POD (Section 3.3)
def pod_method_of_snapshots(U: np.ndarray, r: int):
    """Section 3.3: solve U^T U Psi = Psi Lambda, Phi = U Psi Lambda^{-1/2}; keep the r leading columns.

    Returns (Phi_r, eigenvalues Lambda in descending order)."""
    U = np.asarray(U, dtype=np.float64)
    G = U.T @ U
    lam, Psi = np.linalg.eigh(G)
    order = np.argsort(-lam, kind="stable")
    lam = lam[order]
    Psi = Psi[:, order]
    Phi = U @ Psi[:, :r] / np.sqrt(lam[:r])[None, :]
    return Phi, lam


def coarse_operator(K, Phi: np.ndarray) -> np.ndarray:
    """K_r = Phi^T K Phi (eq. POD_ROM), symmetrised."""
    KPhi = K @ Phi
    Kr = Phi.T @ KPhi
    return 0.5 * (Kr + Kr.T)


def rom_solution(K, Phi: np.ndarray, f: np.ndarray) -> np.ndarray:
    """POD-ROM solution u = Phi_r u_r with K_r u_r = Phi_r^T f (Section 3.3 steps 3-4)."""
    L = cholesky(coarse_operator(K, Phi))
    return Phi @ cholesky_solve(L, Phi.T @ f)


# ----------------------------------------------------------------------------- Algorithm 2
def damped_jacobi(K, Dinv, omega, f, u, sweeps):
    """`sweeps` iterations of u <- u + omega D^{-1} (f - K u)."""
    for _ in range(sweeps):
        u = u + omega * Dinv * (f - K @ u)
    return u


def multicolour_groups(row_ptr, col_idx, bs):
    """Independent dof groups for Gauss-Seidel: nodes (block rows) are coloured
    greedily in index order, each taking the smallest colour that no neighbour of a
    lower index holds, so nodes of one colour share no stored block. Group (c, a)
    holds component a of every node of colour c; the dofs of one group do not couple,
    so a sweep over the groups in order (c = 0, 1, ..; a = 0..bs-1 within c) is a
    pointwise Gauss-Seidel sweep. Returns the list of dof index arrays in sweep order."""
    nb = len(row_ptr) - 1
    colour = np.full(nb, -1, dtype=np.int64)
    for i in range(nb):
        taken = {int(colour[j]) for j in col_idx[row_ptr[i]:row_ptr[i + 1]] if j < i}
        c = 0
        while c in taken:
            c += 1
        colour[i] = c
    groups = []
    for c in range(int(colour.max()) + 1):
        nodes = np.nonzero(colour == c)[0]
        for a in range(bs):
            groups.append(nodes * bs + a)
    return groups


def gauss_seidel(K, Kdiag, f, u, groups, sweeps, reverse=False):
    """`sweeps` pointwise Gauss-Seidel sweeps u_d <- u_d + (f - K u)_d / K_dd over the
    dofs in the order of `groups` (reversed for the backward sweep): the relaxation
    scheme of eq. GaussSeidel (Section 2.2). Each group is updated at once, which is
    exact because its dofs do not couple."""
    order = groups[::-1] if reverse else groups
    u = np.array(u, dtype=np.float64)
    for _ in range(sweeps):
        for g in order:
            u[g] = u[g] + (f[g] - K[g] @ u) / Kdiag[g]
    return u


def two_grid_cycle(K, f, u, Phi, L_c, Dinv, omega, r1, r2, trace=None, groups=None):
    """One cycle of Algorithm 2 with prolongation P = Phi (Section 3.3):
    pre-relax r1 times, residual, restrict and solve K_c e_c = Phi^T r, prolong,
    correct, post-relax r2 times. Relaxation: damped Jacobi, or with `groups`
    forward Gauss-Seidel before and backward Gauss-Seidel after the coarse
    correction (the symmetric pair, so that the cycle from zero is a symmetric
    preconditioner)."""
    if groups is None:
        u = damped_jacobi(K, Dinv, omega, f, u, r1)      # pre-relaxation
    else:
        u = gauss_seidel(K, 1.0 / Dinv, f, u, groups, r1)
    r = f - K @ u                                         # residual update
    e_c = cholesky_solve(L_c, Phi.T @ r)                  # K_c e_c = P^T r
    e = Phi @ e_c                                         # prolongation
    u = u + e                                             # correction
    if trace is not None:
        trace["after_correction"] = u.copy()
    if groups is None:
        u = damped_jacobi(K, Dinv, omega, f, u, r2)      # post-relaxation
    else:
        u = gauss_seidel(K, 1.0 / Dinv, f, u, groups, r2, reverse=True)
    return u


@dataclass
class Pod2gSetup:
    """Per-instance set-up of the preconditioner: D^{-1}, K_c = Phi^T K Phi and its Cholesky factor."""
    Phi: np.ndarray
    Dinv: np.ndarray
    L_c: np.ndarray
    omega: float
    r1: int = 1
    r2: int = 1
    groups: list | None = None     # Gauss-Seidel sweep groups (None: damped Jacobi)


def pod2g_setup(K, Phi, omega, r1=1, r2=1, groups=None) -> Pod2gSetup:
    Dinv = jacobi_inverse_diagonal(K)
    L_c = cholesky(coarse_operator(K, Phi)) if Phi.shape[1] > 0 else np.zeros((0, 0))
    return Pod2gSetup(Phi=np.asarray(Phi, dtype=np.float64), Dinv=Dinv, L_c=L_c, omega=omega, r1=r1, r2=r2,
                      groups=groups)


def pod2g_preconditioner(K, setup: Pod2gSetup):
    """r -> AMG(0; K, r, r1, r2): one two-grid cycle from a zero initial guess (Algorithm 3)."""
    def apply(r):
        return two_grid_cycle(K, r, np.zeros_like(r), setup.Phi, setup.L_c, setup.Dinv,
                              setup.omega, setup.r1, setup.r2, groups=setup.groups)
    return apply


def jacobi_preconditioner(K):
    Dinv = jacobi_inverse_diagonal(K)
    return lambda r: Dinv * r


# ----------------------------------------------------------------------------- Algorithms 1 / 3
@dataclass
class PCGResult:
    x: np.ndarray
    iters: int
    status: int
    relres: float                  # true ||f - K x|| / ||f|| at exit
    history: list = field(default_factory=list)   # recurrence ||r_k|| / ||f||, k = 0..iters
    iterates: list | None = None   # optional x_k, r_k, s_k, p_k records


def pcg(K, f, u0, apply_Tinv, tol, maxit, beta="fr", record=False) -> PCGResult:
    """Algorithm 1 (and Algorithm 3 when apply_Tinv is the two-grid cycle)."""
    f = np.asarray(f, dtype=np.float64)
    n = f.shape[0]
    fnorm = float(np.linalg.norm(f))
    if fnorm == 0.0:
        return PCGResult(np.zeros(n), 0, OK, 0.0, [0.0])
    u = np.zeros(n) if u0 is None else np.array(u0, dtype=np.float64)
    r = f - K @ u
    s = apply_Tinv(r)
    p = s.copy()
    rs = float(r @ s)
    k = 0
    hist = [float(np.linalg.norm(r)) / fnorm]
    recs = [] if record else None
    status = NOT_CONVERGED
    while True:
        if np.linalg.norm(r) <= tol * fnorm:
            status = OK
            break
        if k >= maxit:
            status = NOT_CONVERGED
            break
        if not np.isfinite(rs) or rs <= 0.0:
            status = BREAKDOWN
            break
        if record:
            recs.append(dict(x=u.copy(), r=r.copy(), s=s.copy(), p=p.copy()))
        q = K @ p
        pq = float(p @ q)
        if not np.isfinite(pq) or pq <= 0.0:
            status = BREAKDOWN
            break
        alpha = rs / pq
        u = u + alpha * p
        r = r - alpha * q
        k += 1
        hist.append(float(np.linalg.norm(r)) / fnorm)
        if np.linalg.norm(r) <= tol * fnorm:
            status = OK
            break
        s_new = apply_Tinv(r)
        rs_new = float(r @ s_new)
        if beta == "pr":
            b = float(r @ (s_new - s)) / rs
        else:
            b = rs_new / rs
        p = s_new + b * p
        s = s_new
        rs = rs_new
    if record:
        recs.append(dict(x=u.copy(), r=r.copy(), s=s.copy(), p=p.copy()))
    true_rel = float(np.linalg.norm(f - K @ u)) / fnorm
    return PCGResult(u, k, status, true_rel, hist, recs)


def pod2g_pcg(K, f, u0, Phi, omega, tol, maxit, r1=1, r2=1, beta="fr", record=False, groups=None) -> PCGResult:
    """POD-2G-preconditioned CG: Algorithm 3 with the two-grid cycle of Algorithm 2, P = Phi_r."""
    try:
        st = pod2g_setup(K, Phi, omega, r1, r2, groups)
    except np.linalg.LinAlgError:
        return PCGResult(np.zeros(K.shape[0]) if u0 is None else np.array(u0, float), 0, NOT_SPD, np.nan)
    return pcg(K, f, u0, pod2g_preconditioner(K, st), tol, maxit, beta=beta, record=record)


def jacobi_pcg(K, f, u0, tol, maxit, record=False) -> PCGResult:
    return pcg(K, f, u0, jacobi_preconditioner(K), tol, maxit, record=record)


# ----------------------------------------------------------------------------- operators (dense, tiny cases)
def two_grid_error_operator(K, Phi, Dinv, omega, r1=1, r2=1, order=None) -> np.ndarray:
    """Dense e -> M2^{r2} C M1^{r1} e with C = I - Phi (Phi^T K Phi)^{-1} Phi^T K
    (eq. AMGerror, eq. FinalScheme) and M1 = M2 = I - omega D^{-1} K (damped Jacobi),
    or, given a dof `order`, the Gauss-Seidel splittings of the permuted matrix:
    M1 = I - (D + L)^{-1} K (forward), M2 = I - (D + U)^{-1} K (backward), L / U the
    strictly lower / upper triangles of K in that order (eq. GaussSeidel)."""
    Kd = K.toarray() if hasattr(K, "toarray") else np.asarray(K)
    n = Kd.shape[0]
    I = np.eye(n)
    if order is None:
        M1 = M2 = I - omega * Dinv[:, None] * Kd
    else:
        Pm = np.eye(n)[order]                   # row t of Pm picks dof order[t]
        Kp = Pm @ Kd @ Pm.T
        lower = np.tril(Kp)
        upper = np.triu(Kp)
        M1 = I - Pm.T @ np.linalg.solve(lower, Kp) @ Pm
        M2 = I - Pm.T @ np.linalg.solve(upper, Kp) @ Pm
    Kc = Phi.T @ Kd @ Phi
    C = I - Phi @ np.linalg.solve(Kc, Phi.T @ Kd)
    return np.linalg.matrix_power(M2, r2) @ C @ np.linalg.matrix_power(M1, r1)


def spectral_radius_estimate(K, Dinv, steps=30, seed=0) -> float:
    """Power-iteration estimate of rho(D^{-1} K) (the damped-Jacobi smoother needs omega * rho < 2)."""
    rng = np.random.default_rng(seed)
    v = rng.standard_normal(K.shape[0])
    v /= np.linalg.norm(v)
    lam = 0.0
    for _ in range(steps):
        w = Dinv * (K @ v)
        lam = float(np.linalg.norm(w))
        v = w / lam
    return lam


# ----------------------------------------------------------------------------- Algorithm 2 as a solver
def pod2g_stationary(K, f, u0, Phi, omega, tol, maxit, r1=1, r2=1, groups=None) -> PCGResult:
    """POD-2G used directly as the iterative solver (Algorithm 2, Section 3.3): repeat
    the two-grid cycle on the current approximation while ||f - K u|| > tol ||f||
    (the guard of Algorithm 2 read as ">"), at most maxit cycles. iters = cycles applied."""
    f = np.asarray(f, dtype=np.float64)
    n = f.shape[0]
    fnorm = float(np.linalg.norm(f))
    if fnorm == 0.0:
        return PCGResult(np.zeros(n), 0, OK, 0.0, [0.0])
    try:
        st = pod2g_setup(K, Phi, omega, r1, r2, groups)
    except np.linalg.LinAlgError:
        return PCGResult(np.zeros(n) if u0 is None else np.array(u0, float), 0, NOT_SPD, np.nan)
    u = np.zeros(n) if u0 is None else np.array(u0, dtype=np.float64)
    r = f - K @ u
    hist = [float(np.linalg.norm(r)) / fnorm]
    k = 0
    status = NOT_CONVERGED
    while True:
        if np.linalg.norm(r) <= tol * fnorm:
            status = OK
            break
        if k >= maxit:
            break
        u = two_grid_cycle(K, f, u, st.Phi, st.L_c, st.Dinv, omega, r1, r2, groups=groups)
        r = f - K @ u
        k += 1
        hist.append(float(np.linalg.norm(r)) / fnorm)
        if not np.isfinite(hist[-1]):
            status = BREAKDOWN
            break
    return PCGResult(u, k, status, hist[-1], hist)

"""Snapshot sets and POD bases for the synthetic workloads (the offline stage).

The paper's offline stage solves the FE problem for N parameter samples and
keeps the solutions as columns of U (Section 3.3); its POD basis is the leading
r left singular vectors of U, uncentred (R = U U^T, Section 3.3 eq.
PODrelationEigenvectors). Here that basis is an *input* of the solver, produced
by library routines only:

  * snapshot solves: SuperLU (scipy.sparse.linalg.splu) for small systems; for
    large ones, geometric-multigrid-preconditioned conjugate gradients on torch
    (synth/mg.py: matrix-free K = sum_e c_e K_ref on the structured grid, FP32
    V-cycle, FP64 outer iteration), many instances at once, to a relative residual
    of 1e-11. The first and last snapshot of every chunk are checked against the
    assembled block values with an independent SpMV. Any bug here could only yield
    a worse coarse space, which both the oracle and the CUDA path then receive
    unchanged.
  * the basis: numpy thin SVD (small), or on a CUDA device a Householder QR of U
    followed by the SVD of its triangular factor (the same left singular vectors),
    columns signed so that their largest-magnitude entry is positive.
"""
from __future__ import annotations

import os

import numpy as np

from .problems import Workload

_MEMO: dict = {}


def cache_dir() -> str:
    d = os.environ.get("POD2G_CACHE", os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "_cache"))
    os.makedirs(d, exist_ok=True)
    return d


def _direct_solve(wl: Workload, xis: np.ndarray, f: np.ndarray) -> np.ndarray:
    import scipy.sparse.linalg as sla
    P = wl.problem
    U = np.empty((P.n, len(xis)))
    for i, xi in enumerate(xis):
        A = P.csr(wl.values(xi)).tocsc()
        U[:, i] = sla.splu(A).solve(f)
    return U


def _mg_solve(wl: Workload, xis: np.ndarray, f: np.ndarray, device: str, chunk: int, tol: float = 1e-11):
    """Snapshots by multigrid PCG, `chunk` instances at a time; returns U [n, N] (torch, on device)."""
    import torch
    from . import mg
    P = wl.problem
    U = torch.empty((P.n, len(xis)), dtype=torch.float64, device=device)
    for s0 in range(0, len(xis), chunk):
        part = xis[s0:s0 + chunk]
        coef = torch.from_numpy(np.stack([wl.coef(xi) for xi in part])).to(device)
        X, _ = mg.mg_pcg(P, coef, f, tol=tol)
        U[:, s0:s0 + len(part)] = X.T
        # independent check of the first and last snapshot of the chunk: the assembled block
        # values of the generator and a gather / index_add SpMV (not the grid operator)
        for t in sorted({0, len(part) - 1}):
            vals = P.values_torch(coef[t:t + 1])[0]
            rel = mg.bsr_residual(P, vals, X[t], f)
            del vals
            if not rel <= 100 * tol:
                raise RuntimeError(f"snapshot solve did not converge: relative residual {rel:.3e}")
        del X, coef
    return U


def snapshot_matrix(wl: Workload, count: int | None = None, device: str | None = None) -> np.ndarray:
    """U = [u_1 ... u_N], u_i = K(theta_i)^{-1} f0 for the LHS snapshot parameters."""
    xis = wl.snapshot_thetas(count)
    f = wl.problem.f0
    if device in (None, "cpu"):
        if wl.n > 20_000:
            raise ValueError("large snapshot sets are solved on a CUDA device (device='cuda')")
        return _direct_solve(wl, xis, f)
    # instances per multigrid chunk: ~600 bytes of vectors and element temporaries per unknown
    budget = float(os.environ.get("POD2G_SNAPSHOT_BYTES", 60e9))
    chunk = max(1, min(len(xis), 64, int(budget // (600 * wl.n))))
    return _mg_solve(wl, xis, f, device, chunk)


def signed_left_singular(U, k: int) -> np.ndarray:
    if isinstance(U, np.ndarray):
        W, s, _ = np.linalg.svd(U, full_matrices=False)
        Phi = W[:, :k].copy()
    else:   # torch tensor on a device: U = Q R, R = W_R S V^T, so U's left singular vectors are Q W_R
        import torch
        Q, R = torch.linalg.qr(U, mode="reduced")
        W_R, _, _ = torch.linalg.svd(R)
        Phi = (Q @ W_R[:, :k]).cpu().numpy()
        del Q, R
    for j in range(k):
        i = int(np.argmax(np.abs(Phi[:, j])))
        if Phi[i, j] < 0:
            Phi[:, j] = -Phi[:, j]
    return Phi


def pod_basis(wl: Workload, k: int | None = None, count: int | None = None, device: str | None = None,
              use_disk: bool = True, cached_only: bool = False) -> np.ndarray:
    """FP64 POD basis Phi (n x k) of the workload's snapshot set (memoised, optionally on disk).
    cached_only: read the on-disk basis of a large workload, never compute it (FileNotFoundError)."""
    k = wl.spec.k if k is None else k
    count = wl.spec.n_snap if count is None else count
    key = (wl.spec.name, k, count)
    if key in _MEMO:
        return _MEMO[key]
    path = os.path.join(cache_dir(), f"phi_{wl.spec.name}_k{k}_N{count}.npy")
    if use_disk and os.path.exists(path):
        Phi = np.load(path)
    elif cached_only and wl.n > 20_000:
        raise FileNotFoundError(f"{path}: compute the POD basis of {wl.spec.name} first")
    else:
        U = snapshot_matrix(wl, count, device)
        Phi = signed_left_singular(U, k)
        if use_disk:
            np.save(path, Phi)
    _MEMO[key] = Phi
    return Phi


def surrogate_data(wl: Workload, ks: int, count: int | None = None, device: str | None = None,
                   use_disk: bool = True):
    """Training data of the surrogate (Section 3.2) from the workload's snapshot set: the first ks
    left singular vectors Psi (n x ks, the decoder of a linear autoencoder) and the latent
    coordinates Z = Psi^T U (ks x N) of the N snapshots, with their parameters. The solver's basis
    Phi is the first k columns of the same factorisation (stored too if missing)."""
    count = wl.spec.n_snap if count is None else count
    key = ("sur", wl.spec.name, ks, count)
    if key in _MEMO:
        return _MEMO[key]
    path = os.path.join(cache_dir(), f"sur_{wl.spec.name}_ks{ks}_N{count}.npz")
    if use_disk and os.path.exists(path):
        d = np.load(path)
        out = (d["psi"], d["z"], d["theta"])
    else:
        U = snapshot_matrix(wl, count, device)
        k = wl.spec.k
        W = signed_left_singular(U, max(k, ks))
        phi_path = os.path.join(cache_dir(), f"phi_{wl.spec.name}_k{k}_N{count}.npy")
        if use_disk and not os.path.exists(phi_path):
            np.save(phi_path, W[:, :k])
        psi = W[:, :ks].copy()
        if isinstance(U, np.ndarray):
            z = psi.T @ U
        else:
            import torch
            z = (torch.from_numpy(psi).to(U.device).T @ U).cpu().numpy()
        del U, W
        out = (psi, z, wl.snapshot_thetas(count))
        if use_disk:
            np.savez(path, psi=psi, z=z, theta=out[2])
    _MEMO[key] = out
    return out

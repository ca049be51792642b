"""Snapshot sets and POD bases for the synthetic workloads (the offline stage).

The paper's offline stage solves the FE problem for N parameter samples and
keeps the solutions as columns of U (Section 3.3); its POD basis is the leading
r left singular vectors of U, uncentred (R = U U^T, Section 3.3 eq.
PODrelationEigenvectors). Here that basis is an *input* of the solver, produced
by library routines only:

  * snapshot solves: SuperLU (scipy.sparse.linalg.splu) for small systems;
    for large ones, conjugate gradients with a diagonal preconditioner on
    torch's CSR SpMV (cuSPARSE), the instances of a chunk stacked as one
    block-diagonal matrix. Solutions are accurate to a relative residual of
    1e-11. Any bug here could only yield a worse coarse space, which both the
    oracle and the CUDA path then receive unchanged.
  * the basis: numpy / torch thin SVD, columns signed so that their
    largest-magnitude entry is positive.
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


def _bsr_to_csr_perm(P):
    """Permutation taking flattened BSR values to scipy CSR data order, plus the CSR arrays."""
    import scipy.sparse as sp
    bs = P.bs
    tag = np.arange(1, P.nnzb * bs * bs + 1, dtype=np.float64).reshape(P.nnzb, bs, bs)
    A = sp.bsr_matrix((tag, P.col_idx, P.row_ptr), shape=(P.n, P.n)).tocsr()
    A.sort_indices()
    perm = (A.data - 1).astype(np.int64)
    return A.indptr.astype(np.int64), A.indices.astype(np.int64), perm


def _cg_solve_torch(wl: Workload, xis: np.ndarray, f: np.ndarray, device: str, chunk: int, tol: float = 1e-11,
                    maxit: int = 200000) -> np.ndarray:
    import torch
    P = wl.problem
    n = P.n
    indptr, indices, perm = _bsr_to_csr_perm(P)
    nnz = indices.shape[0]
    U = np.empty((n, len(xis)))
    ip_t = torch.from_numpy(indptr).to(device)
    ix_t = torch.from_numpy(indices).to(device)
    f_t = torch.from_numpy(f).to(device)
    for s in range(0, len(xis), chunk):
        part = xis[s:s + chunk]
        c = len(part)
        vals = torch.empty(c * nnz, dtype=torch.float64, device=device)
        diag = torch.empty(c, n, dtype=torch.float64, device=device)
        for t, xi in enumerate(part):
            v = wl.values(xi)
            vals[t * nnz:(t + 1) * nnz] = torch.from_numpy(v.reshape(-1)[perm]).to(device)
            d = np.einsum("bii->bi", v[P._diag_blk]).reshape(-1)
            diag[t] = torch.from_numpy(d).to(device)
        crow = torch.cat([ip_t[:-1] + t * nnz for t in range(c)] + [ip_t[-1:] + (c - 1) * nnz])
        col = torch.cat([ix_t + t * n for t in range(c)])
        A = torch.sparse_csr_tensor(crow, col, vals, size=(c * n, c * n))
        dinv = (1.0 / diag).reshape(-1)
        b = f_t.repeat(c)
        x = torch.zeros_like(b)
        r = b.clone()
        z = dinv * r
        p = z.clone()
        rz = (r * z).view(c, n).sum(1)
        bnorm = torch.linalg.vector_norm(b.view(c, n), dim=1)
        active = torch.ones(c, dtype=torch.float64, device=device)
        for it in range(maxit):
            q = (A @ p.unsqueeze(1)).squeeze(1)
            pq = (p * q).view(c, n).sum(1)
            alpha = torch.where(active > 0, rz / pq, torch.zeros_like(rz))
            x += (alpha[:, None] * p.view(c, n)).view(-1)
            r -= (alpha[:, None] * q.view(c, n)).view(-1)
            if it % 20 == 19:
                rn = torch.linalg.vector_norm(r.view(c, n), dim=1)
                active = (rn > tol * bnorm).to(torch.float64)
                if float(active.sum()) == 0:
                    break
            z = dinv * r
            rz_new = (r * z).view(c, n).sum(1)
            beta = torch.where(active > 0, rz_new / rz, torch.zeros_like(rz))
            p = z + (beta[:, None] * p.view(c, n)).view(-1)
            rz = rz_new
        U[:, s:s + c] = x.view(c, n).T.cpu().numpy()
        # check the first and last snapshot of the batch with scipy's SpMV (independent of cuSPARSE)
        for t in sorted({0, c - 1}):
            K = P.csr(wl.values(part[t]))
            rel = np.linalg.norm(f - K @ U[:, s + t]) / np.linalg.norm(f)
            if not rel <= 100 * tol:
                raise RuntimeError(f"snapshot solve did not converge: relative residual {rel:.3e}")
        del A, vals
    return U


def snapshot_matrix(wl: Workload, count: int | None = None, device: str | None = None) -> np.ndarray:
    """U = [u_1 ... u_N], u_i = K(theta_i)^{-1} f0 for the LHS snapshot parameters."""
    xis = wl.snapshot_thetas(count)
    f = wl.problem.f0
    if device in (None, "cpu"):
        if wl.n > 20_000:
            raise ValueError("large snapshot sets are solved on a CUDA device (device='cuda')")
        return _direct_solve(wl, xis, f)
    # instances per block-diagonal CG batch: values (8 B) + column indices (8 B) + ~8 work vectors
    budget = float(os.environ.get("POD2G_SNAPSHOT_BYTES", 40e9))
    nnz = wl.problem.nnzb * wl.problem.bs ** 2
    chunk = max(1, min(len(xis), int(budget // (nnz * 16 + 64 * wl.n)), (2 ** 30) // nnz))  # well inside int32 limits
    return _cg_solve_torch(wl, xis, f, device, chunk)


def signed_left_singular(U: np.ndarray, k: int) -> np.ndarray:
    W, s, _ = np.linalg.svd(U, full_matrices=False)
    Phi = W[:, :k].copy()
    for j in range(k):
        i = int(np.argmax(np.abs(Phi[:, j])))
        if Phi[i, j] < 0:
            Phi[:, j] = -Phi[:, j]
    return Phi


def pod_basis(wl: Workload, k: int | None = None, count: int | None = None, device: str | None = None,
              use_disk: bool = True) -> np.ndarray:
    """FP64 POD basis Phi (n x k) of the workload's snapshot set (memoised, optionally on disk)."""
    k = wl.spec.k if k is None else k
    count = wl.spec.n_snap if count is None else count
    key = (wl.spec.name, k, count)
    if key in _MEMO:
        return _MEMO[key]
    path = os.path.join(cache_dir(), f"phi_{wl.spec.name}_k{k}_N{count}.npy")
    if use_disk and os.path.exists(path):
        Phi = np.load(path)
    else:
        U = snapshot_matrix(wl, count, device)
        Phi = signed_left_singular(U, k)
        if use_disk:
            np.save(path, Phi)
    _MEMO[key] = Phi
    return Phi

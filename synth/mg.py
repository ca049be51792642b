"""Snapshot solves for the structured-mesh workloads by geometric-multigrid PCG (input generation).

The offline stage of the method (Section 3.3) needs the solutions u_i = K(theta_i)^{-1} f of
many parameter samples; their span gives the POD basis that the solver then receives as an
input. This module produces those solutions with library tensor operations (torch), on the
structure the generator already knows: every matrix is K = sum_e c_e K_ref on a uniform
mesh (see fe.StructuredProblem). It holds no POD-2G arithmetic and shares nothing with the
CUDA solver; a mistake here could only give a worse coarse space, which the oracle and the
CUDA path then both receive unchanged.

  * GridOperator applies K matrix-free on the full node grid, batched over instances: the
    element vectors of all elements are gathered by 2^dim shifted slices, multiplied by
    K_ref (one GEMM) and by c_e, and scattered back. Constrained nodes (the eliminated
    boundary of the Q1 problems, the clamped face of the Q4 / Hex8 problems) carry the
    identity, exactly like the assembled matrix.
  * The preconditioner is a symmetric V(2,2)-cycle: damped-Jacobi smoothing, linear
    interpolation between nested grids (mesh size doubled per level) and its transpose as
    restriction, coarse operators re-discretised from the children's mean coefficient, and
    a dense Cholesky solve on the coarsest grid. It runs in FP32.
  * The outer iteration is conjugate gradients in FP64 with the Polak-Ribiere beta (robust
    to the FP32 preconditioner), stopped at a relative residual of 1e-11.
"""
from __future__ import annotations

import numpy as np

from . import fe


def _element_matrix(kind: str, ne: int) -> np.ndarray:
    h = 1.0 / ne
    return {"q1": fe.element_matrix_q1, "q4": fe.element_matrix_q4, "hex8": fe.element_matrix_hex8}[kind](h)


def _dim_bs(kind: str):
    return (2, 1) if kind == "q1" else (2, 2) if kind == "q4" else (3, 3)


def free_mask(kind: str, ne: int, device, dim: int):
    """Unconstrained nodes of the full (ne+1)^dim node grid, as a bool tensor [..., z, y, x]."""
    import torch
    n1 = ne + 1
    idx = torch.arange(n1, device=device)
    if kind == "q1":
        inner = (idx > 0) & (idx < ne)
        return inner[:, None] & inner[None, :]
    if kind == "q4":   # left edge x = 0 clamped
        return (idx > 0)[None, :].expand(n1, n1).clone()
    return (idx > 0)[:, None, None].expand(n1, n1, n1).clone()   # hex8: face z = 0 clamped


class GridOperator:
    """K(c) = sum_e c_e K_ref on the full node grid of one mesh level, for S instances.

    Vectors are tensors [S, (n1,)* dim, bs] indexed [s, (z,) y, x, component] (x fastest, as
    the generator numbers nodes). Element coefficients c: [S, n_el] in element order
    (x fastest)."""

    def __init__(self, kind: str, ne: int, coef, dtype):
        import torch
        self.kind, self.ne = kind, ne
        self.dim, self.bs = _dim_bs(kind)
        self.dtype = dtype
        dev = coef.device
        self.S = coef.shape[0]
        self.Kref = torch.from_numpy(_element_matrix(kind, ne)).to(dev, dtype)
        self.c = coef.to(dtype).reshape(self.S, *([ne] * self.dim))
        self.free = free_mask(kind, ne, dev, self.dim)
        self.freef = self.free.to(dtype)[None, ..., None]
        self.corners = [tuple((a >> d) & 1 for d in range(self.dim)) for a in range(2 ** self.dim)]

    def _slice(self, a):
        ne = self.ne
        off = self.corners[a]          # (dx, dy[, dz])
        return tuple(slice(o, o + ne) for o in reversed(off))   # tensor order (z,) y, x

    def apply(self, U):
        import torch
        S, bs, npe = U.shape[0], self.bs, 2 ** self.dim
        Um = U * self.freef
        Ue = torch.stack([Um[(slice(None),) + self._slice(a)] for a in range(npe)], dim=-2)
        Ue = Ue.reshape(*Ue.shape[:-2], npe * bs)
        Ye = (Ue @ self.Kref) * self.c[..., None]
        Ye = Ye.reshape(*Ye.shape[:-1], npe, bs)
        out = torch.zeros_like(U)
        for a in range(npe):
            out[(slice(None),) + self._slice(a)] += Ye[..., a, :]
        return out * self.freef + U * (1.0 - self.freef)

    def diagonal(self):
        import torch
        npe, bs = 2 ** self.dim, self.bs
        dk = torch.diagonal(self.Kref).reshape(npe, bs)
        shape = (self.S,) + tuple([self.ne + 1] * self.dim) + (bs,)
        out = torch.zeros(shape, dtype=self.dtype, device=self.c.device)
        for a in range(npe):
            out[(slice(None),) + self._slice(a)] += self.c[..., None] * dk[a]
        return out * self.freef + (1.0 - self.freef)

    def coarsened(self):
        """The operator of the next coarser mesh (ne / 2): each coarse element's coefficient is
        the mean of its 2^dim children."""
        c = self.c
        for ax in range(1, self.dim + 1):
            sh = list(c.shape)
            c = c.reshape(*sh[:ax], sh[ax] // 2, 2, *sh[ax + 1:]).mean(dim=ax + 1)
        return GridOperator(self.kind, self.ne // 2, c.reshape(self.S, -1), self.dtype)


def prolong(X, dim: int):
    """Linear interpolation from the (n1c,)*dim node grid to the (2 n1c - 1,)*dim grid."""
    import torch
    for ax in range(1, dim + 1):
        n = X.shape[ax]
        a = X.narrow(ax, 0, n - 1)
        b = X.narrow(ax, 1, n - 1)
        mid = 0.5 * (a + b)
        inter = torch.stack([a, mid], dim=ax + 1).flatten(ax, ax + 1)
        X = torch.cat([inter, X.narrow(ax, n - 1, 1)], dim=ax)
    return X


def restrict(Y, dim: int):
    """The transpose of prolong: full weighting (x_i = y_2i + (y_2i-1 + y_2i+1) / 2)."""
    for ax in range(dim, 0, -1):
        n = (Y.shape[ax] + 1) // 2
        even = Y.narrow(ax, 0, 2 * n - 1)[(slice(None),) * ax + (slice(0, None, 2),)]
        odd = Y.narrow(ax, 1, 2 * n - 2)[(slice(None),) * ax + (slice(0, None, 2),)]
        X = even.clone()
        X.narrow(ax, 0, n - 1).add_(0.5 * odd)
        X.narrow(ax, 1, n - 1).add_(0.5 * odd)
        Y = X
    return Y


class Multigrid:
    """Symmetric V(nu, nu)-cycle for S instances (FP32), coarsest grid solved by dense Cholesky."""

    def __init__(self, kind: str, ne: int, coef, coarsest: int | None = None, nu: int = 2, power_steps: int = 12,
                 dtype=None):
        import torch
        dtype = dtype or torch.float32
        dim, _ = _dim_bs(kind)
        coarsest = coarsest or (8 if dim == 3 else 16)
        self.dim, self.nu = dim, nu
        self.levels = [GridOperator(kind, ne, coef, dtype)]
        while self.levels[-1].ne > coarsest and self.levels[-1].ne % 2 == 0:
            self.levels.append(self.levels[-1].coarsened())
        self.dinv = [1.0 / L.diagonal() for L in self.levels[:-1]]
        self.omega = [self._omega(L, d, power_steps) for L, d in zip(self.levels[:-1], self.dinv)]
        self._coarse_factor()

    def _omega(self, L, dinv, steps):
        """omega = (4/3) / lambda_max(D^-1 K) per instance, lambda_max by power iteration (x 1.05)."""
        import torch
        g = torch.Generator(device="cpu").manual_seed(7)
        shape = (L.S,) + tuple([L.ne + 1] * L.dim) + (L.bs,)
        v = torch.rand(shape, generator=g, dtype=torch.float64).to(dinv.device, dinv.dtype) * L.freef
        lam = None
        for _ in range(steps):
            w = dinv * L.apply(v) * L.freef
            lam = torch.linalg.vector_norm(w.reshape(L.S, -1), dim=1) / torch.linalg.vector_norm(v.reshape(L.S, -1),
                                                                                                 dim=1)
            v = w / torch.linalg.vector_norm(w.reshape(L.S, -1), dim=1).reshape(-1, *([1] * (w.dim() - 1)))
        return ((4.0 / 3.0) / (1.05 * lam)).reshape(-1, *([1] * (v.dim() - 1)))

    def _coarse_factor(self):
        import torch
        L = self.levels[-1]
        free = L.free.reshape(-1)
        fidx = torch.nonzero(free).squeeze(1)
        nf = fidx.numel() * L.bs
        n1 = L.ne + 1
        npt = free.numel()
        # columns of the operator on the free dofs: apply K to unit vectors, all instances at once
        cols = []
        eye_chunk = 512
        for s0 in range(0, nf, eye_chunk):
            s1 = min(nf, s0 + eye_chunk)
            m = s1 - s0
            E = torch.zeros((m, npt * L.bs), dtype=torch.float64, device=L.c.device)
            dof = (fidx.repeat_interleave(L.bs) * L.bs + torch.arange(L.bs, device=E.device).repeat(fidx.numel()))
            E[torch.arange(m, device=E.device), dof[s0:s1]] = 1.0
            E = E.reshape(m, *([n1] * L.dim), L.bs)
            Lk = GridOperator(L.kind, L.ne, L.c.reshape(L.S, -1).to(torch.float64).repeat_interleave(m, dim=0),
                              torch.float64)
            Y = Lk.apply(E.repeat(L.S, *([1] * (E.dim() - 1))))
            cols.append(Y.reshape(L.S, m, npt * L.bs)[:, :, dof])
        self.cdof = dof
        A = torch.cat(cols, dim=1)                     # [S, nf, nf] (symmetric)
        self.cchol = torch.linalg.cholesky(0.5 * (A + A.transpose(1, 2)))

    def _coarse_solve(self, R):
        import torch
        L = self.levels[-1]
        flat = R.reshape(L.S, -1).to(torch.float64)
        y = torch.cholesky_solve(flat[:, self.cdof].unsqueeze(-1), self.cchol).squeeze(-1)
        out = torch.zeros_like(flat)
        out[:, self.cdof] = y
        return out.reshape(R.shape).to(R.dtype)

    def _vcycle(self, lvl, R):
        if lvl == len(self.levels) - 1:
            return self._coarse_solve(R)
        L, dinv, w = self.levels[lvl], self.dinv[lvl], self.omega[lvl]
        X = w * dinv * R
        for _ in range(self.nu - 1):
            X = X + w * dinv * (R - L.apply(X))
        Rc = restrict((R - L.apply(X)) * L.freef, self.dim) * self.levels[lvl + 1].freef
        X = X + prolong(self._vcycle(lvl + 1, Rc), self.dim) * L.freef
        for _ in range(self.nu):
            X = X + w * dinv * (R - L.apply(X))
        return X * L.freef

    def __call__(self, R):
        return self._vcycle(0, R.to(self.levels[0].dtype)).to(R.dtype)


def to_grid(P: fe.StructuredProblem, u):
    """System vectors [S, n] -> full-grid tensors [S, (n1,)* dim, bs] (constrained entries: the
    system's value for identity rows, zero for eliminated boundary nodes)."""
    import torch
    S = u.shape[0]
    n1 = P.ne + 1
    if P.dirichlet == "eliminate":
        G = torch.zeros((S,) + (n1,) * P.dim + (P.bs,), dtype=u.dtype, device=u.device)
        inner = (slice(None),) + (slice(1, P.ne),) * P.dim
        G[inner] = u.reshape((S,) + (P.ne - 1,) * P.dim + (P.bs,))
        return G
    return u.reshape((S,) + (n1,) * P.dim + (P.bs,))


def from_grid(P: fe.StructuredProblem, G):
    S = G.shape[0]
    if P.dirichlet == "eliminate":
        return G[(slice(None),) + (slice(1, P.ne),) * P.dim].reshape(S, -1)
    return G.reshape(S, -1)


def mg_pcg(P: fe.StructuredProblem, coef, f: np.ndarray, tol: float = 1e-11, maxit: int = 500,
           coarsest: int | None = None):
    """Solve K(c_s) u_s = f for S coefficient vectors coef [S, n_el] (torch, any device) by
    multigrid-preconditioned CG in FP64. Returns (U [S, n] float64 tensor, iterations)."""
    import torch
    S = coef.shape[0]
    dev = coef.device
    A = GridOperator(P.kind, P.ne, coef.to(torch.float64), torch.float64)
    M = Multigrid(P.kind, P.ne, coef, coarsest=coarsest)
    fg = to_grid(P, torch.from_numpy(np.asarray(f, dtype=np.float64)).to(dev).reshape(1, -1)).expand(
        S, *([-1] * (P.dim + 1))).contiguous()
    shp = (-1,) + (1,) * (P.dim + 1)

    def dot(a, b):
        return (a * b).reshape(S, -1).sum(1)

    x = torch.zeros_like(fg)
    r = fg.clone()
    z = M(r)
    p = z.clone()
    rz = dot(r, z)
    bnorm = torch.sqrt(dot(fg, fg))
    active = torch.sqrt(dot(r, r)) > tol * bnorm
    it = 0
    while bool(active.any()) and it < maxit:
        q = A.apply(p)
        alpha = torch.where(active, rz / dot(p, q), torch.zeros_like(rz))
        x = x + alpha.reshape(shp) * p
        r = r - alpha.reshape(shp) * q
        it += 1
        active = active & (torch.sqrt(dot(r, r)) > tol * bnorm)
        z_new = M(r)
        beta = torch.where(active, dot(r, z_new - z) / rz, torch.zeros_like(rz))
        rz = dot(r, z_new)
        p = z_new + beta.reshape(shp) * p
        z = z_new
    if bool(active.any()):
        raise RuntimeError(f"multigrid PCG did not reach {tol:g} in {maxit} iterations")
    return from_grid(P, x), it


def bsr_residual(P: fe.StructuredProblem, vals, u, f) -> float:
    """||f - K u|| / ||f|| with K the generator's assembled block values (torch, device of vals):
    an independent check of a snapshot (block gather and index_add, not the grid operator)."""
    import torch
    dev = vals.device
    bs = P.bs
    cache = getattr(P, "_mg_rows", None)
    if cache is None or cache[0] != str(dev):
        col = torch.from_numpy(P.col_idx.astype(np.int64)).to(dev)
        rows = torch.from_numpy(np.repeat(np.arange(P.n_nodes), np.diff(P.row_ptr)).astype(np.int64)).to(dev)
        cache = (str(dev), col, rows)
        P._mg_rows = cache
    _, col, rows = cache
    U = u.reshape(-1, bs)
    Y = torch.zeros_like(U)
    step = 1 << 24
    for s0 in range(0, col.numel(), step):
        s1 = min(col.numel(), s0 + step)
        Y.index_add_(0, rows[s0:s1], torch.einsum("kab,kb->ka", vals[s0:s1], U[col[s0:s1]]))
    ft = torch.from_numpy(np.asarray(f, dtype=np.float64)).to(dev)
    return float(torch.linalg.vector_norm(ft - Y.reshape(-1)) / torch.linalg.vector_norm(ft))

"""Structured-mesh finite elements: the parametrized SPD systems K(theta) u = f(theta).

This module builds the *input* of the solver (the discretised elliptic problems of
Section 2.0, eq. fineProblem), not the solver. It holds no PCG, two-grid or POD
arithmetic.

Meshes are uniform: unit square split into ne x ne square elements (Q1 scalar
diffusion, Q4 plane-stress elasticity) or unit cube split into ne^3 cubes (Hex8
3D elasticity). Nodes are numbered lexicographically, x fastest:
    node(i, j[, l]) = i + (ne+1) * (j + (ne+1) * l)
and dof = bs * node + component. A local element node a = i + 2 j (+ 4 l) with
i, j, l in {0, 1} sits at offset (i, j, l) from the element's lowest corner.

Every element's coefficient is constant (evaluated at its centroid), so the
assembled matrix is exactly K(theta) = sum_e c_e(theta) K_e^ref, with one
reference element matrix per problem. The matrix is stored in block-CSR (BSR)
form over nodes: row_ptr/col_idx (int32, columns sorted, diagonal present,
structurally symmetric) and values[nnzb, bs, bs] (row-major blocks).

Dirichlet conditions:
  * Q1 ("eliminate"): boundary nodes are removed; interior nodes renumbered
    lexicographically (63^2 = 3,969 dofs on a 64^2 mesh).
  * Q4 / Hex8 ("identity"): all nodes are kept; a clamped node's block row and
    block column are zeroed and its diagonal block set to the identity, the rhs
    entry set to 0. Pattern keeps the full mesh connectivity (zeros stored).
"""
from __future__ import annotations

import itertools
from dataclasses import dataclass, field

import numpy as np

GAUSS_2 = (-1.0 / np.sqrt(3.0), 1.0 / np.sqrt(3.0))


def _local_corners(dim):
    """Local node a -> (i, j[, l]) offsets, a = i + 2 j + 4 l."""
    return [tuple((a >> d) & 1 for d in range(dim)) for a in range(2 ** dim)]


def _shape_grads(dim, h, xi):
    """Gradients (physical) of the 2^dim multilinear shape functions at reference point xi."""
    corners = _local_corners(dim)
    g = np.zeros((len(corners), dim))
    for a, c in enumerate(corners):
        s = [2 * ci - 1 for ci in c]  # reference coordinate of node a
        for d in range(dim):
            v = 0.5 * s[d]
            for e in range(dim):
                if e != d:
                    v *= 0.5 * (1.0 + s[e] * xi[e])
            g[a, d] = v * (2.0 / h)  # d(xi)/dx = 2/h
    return g


def element_matrix_q1(h: float = 1.0) -> np.ndarray:
    """Bilinear Laplacian element matrix, unit coefficient, 2x2 Gauss (exact)."""
    K = np.zeros((4, 4))
    detJ = (h / 2.0) ** 2
    for xi in itertools.product(GAUSS_2, repeat=2):
        G = _shape_grads(2, h, xi)
        K += G @ G.T * detJ
    return K


def plane_stress_D(E: float = 1.0, nu: float = 0.3) -> np.ndarray:
    return E / (1.0 - nu ** 2) * np.array([[1.0, nu, 0.0], [nu, 1.0, 0.0], [0.0, 0.0, (1.0 - nu) / 2.0]])


def lame(E: float, nu: float):
    """Lamé constants from Young's modulus and Poisson ratio (Section 4.1, eq. Lame)."""
    mu = E / (2.0 * (1.0 + nu))
    lam = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu))
    return lam, mu


def elasticity_3d_D(E: float = 1.0, nu: float = 0.3) -> np.ndarray:
    lam, mu = lame(E, nu)
    D = np.zeros((6, 6))
    D[:3, :3] = lam
    D[np.arange(3), np.arange(3)] = lam + 2.0 * mu
    D[3, 3] = D[4, 4] = D[5, 5] = mu
    return D


def strain_B(dim, G):
    """Engineering-strain operator for nodal displacements (interleaved components)."""
    nn = G.shape[0]
    if dim == 2:
        B = np.zeros((3, 2 * nn))
        for a in range(nn):
            B[0, 2 * a] = G[a, 0]
            B[1, 2 * a + 1] = G[a, 1]
            B[2, 2 * a] = G[a, 1]
            B[2, 2 * a + 1] = G[a, 0]
        return B
    B = np.zeros((6, 3 * nn))
    for a in range(nn):
        gx, gy, gz = G[a]
        B[0, 3 * a] = gx
        B[1, 3 * a + 1] = gy
        B[2, 3 * a + 2] = gz
        B[3, 3 * a] = gy; B[3, 3 * a + 1] = gx      # gamma_xy
        B[4, 3 * a + 1] = gz; B[4, 3 * a + 2] = gy  # gamma_yz
        B[5, 3 * a] = gz; B[5, 3 * a + 2] = gx      # gamma_xz
    return B


def element_matrix_q4(h: float = 1.0, nu: float = 0.3) -> np.ndarray:
    """Q4 plane-stress stiffness (unit E, unit thickness), 2x2 Gauss, full integration."""
    D = plane_stress_D(1.0, nu)
    K = np.zeros((8, 8))
    detJ = (h / 2.0) ** 2
    for xi in itertools.product(GAUSS_2, repeat=2):
        B = strain_B(2, _shape_grads(2, h, xi))
        K += B.T @ D @ B * detJ
    return K


def element_matrix_hex8(h: float, nu: float = 0.3) -> np.ndarray:
    """Hex8 isotropic elasticity stiffness (unit E), 2x2x2 Gauss."""
    D = elasticity_3d_D(1.0, nu)
    K = np.zeros((24, 24))
    detJ = (h / 2.0) ** 3
    for xi in itertools.product(GAUSS_2, repeat=3):
        B = strain_B(3, _shape_grads(3, h, xi))
        K += B.T @ D @ B * detJ
    return K


@dataclass
class StructuredProblem:
    """A structured-mesh FE problem with a theta-independent pattern.

    values(c) assembles K = sum_e c_e K_e^ref for an element-coefficient vector c.
    """
    kind: str             # "q1", "q4", "hex8"
    dim: int
    ne: int               # elements per side
    bs: int               # dofs per node (block size)
    dirichlet: str        # "eliminate" or "identity"
    Kref: np.ndarray      # reference element matrix (bs*2^dim square)
    n_nodes: int          # nodes in the system (after elimination)
    row_ptr: np.ndarray   # int32 [n_nodes+1]
    col_idx: np.ndarray   # int32 [nnzb]
    f0: np.ndarray        # load vector, float64 [n_nodes*bs]
    clamped: np.ndarray   # bool [n_nodes] (identity rows); all False for "eliminate"
    centroids: np.ndarray  # [n_el, dim]
    _elem_nodes: np.ndarray = field(repr=False, default=None)  # [n_el, 2^dim] system node ids (-1: eliminated)
    _pair_blk: list = field(repr=False, default=None)          # per (a,b): (elem mask, block ids)
    _diag_blk: np.ndarray = field(repr=False, default=None)
    _clamp_blocks: np.ndarray = field(repr=False, default=None)

    @property
    def n(self) -> int:
        return self.n_nodes * self.bs

    @property
    def nnzb(self) -> int:
        return int(self.col_idx.shape[0])

    @property
    def n_el(self) -> int:
        return int(self.centroids.shape[0])

    @property
    def npe(self) -> int:
        """Nodes per element."""
        return 2 ** self.dim

    @property
    def conn(self) -> np.ndarray:
        """Element connectivity int32 [n_el, npe]: system node of each local node, -1 if eliminated."""
        return np.ascontiguousarray(self._elem_nodes, dtype=np.int32)

    def values(self, coef: np.ndarray) -> np.ndarray:
        """Assemble values[nnzb, bs, bs] (float64) for element coefficients coef[n_el]."""
        coef = np.asarray(coef, dtype=np.float64)
        assert coef.shape == (self.n_el,)
        bs = self.bs
        vals = np.zeros((self.nnzb, bs, bs))
        for (a, b), (emask, blk) in zip(itertools.product(range(2 ** self.dim), repeat=2), self._pair_blk):
            if blk.size == 0:
                continue
            kab = self.Kref[a * bs:(a + 1) * bs, b * bs:(b + 1) * bs]
            c = coef if emask is None else coef[emask]
            # for a fixed local pair (a, b) every element hits a distinct block: no collisions
            vals[blk] += c[:, None, None] * kab[None, :, :]
        if self.dirichlet == "identity" and self._clamp_blocks.size:
            vals[self._clamp_blocks] = 0.0
            cl = np.nonzero(self.clamped)[0]
            vals[self._diag_blk[cl]] = np.eye(bs)[None]
        return vals

    def values_torch(self, coef):
        """Batched assembly on a torch device: coef [B, n_el] float64 -> values [B, nnzb, bs, bs].

        Same operations in the same order as values(), so the results are identical."""
        import torch
        dev = coef.device
        Bn = coef.shape[0]
        bs = self.bs
        cache = getattr(self, "_torch_maps", None)
        if cache is None or cache[0] != str(dev):
            maps = []
            for emask, blk in self._pair_blk:
                em = None if emask is None else torch.from_numpy(np.nonzero(emask)[0]).to(dev)
                maps.append((em, torch.from_numpy(blk).to(dev)))
            cl = np.nonzero(self.clamped)[0]
            cache = (str(dev), maps, torch.from_numpy(self._clamp_blocks).to(dev),
                     torch.from_numpy(self._diag_blk[cl]).to(dev), torch.from_numpy(self.Kref).to(dev))
            self._torch_maps = cache
        _, maps, clamp_t, diag_cl_t, Kref = cache
        vals = torch.zeros((Bn, self.nnzb, bs, bs), dtype=torch.float64, device=dev)
        for (a, b), (em, blk) in zip(itertools.product(range(2 ** self.dim), repeat=2), maps):
            if blk.numel() == 0:
                continue
            kab = Kref[a * bs:(a + 1) * bs, b * bs:(b + 1) * bs]
            c = coef if em is None else coef[:, em]
            vals[:, blk] += c[:, :, None, None] * kab[None, None, :, :]
        if self.dirichlet == "identity" and clamp_t.numel():
            vals[:, clamp_t] = 0.0
            vals[:, diag_cl_t] = torch.eye(bs, dtype=torch.float64, device=dev)
        return vals

    def csr(self, vals: np.ndarray):
        """scipy CSR of the scalar matrix (a library container used by tests and solvers)."""
        import scipy.sparse as sp
        return sp.bsr_matrix((vals, self.col_idx, self.row_ptr), shape=(self.n, self.n)).tocsr()


def _build(kind: str, ne: int, nu: float = 0.3) -> StructuredProblem:
    dim = 2 if kind in ("q1", "q4") else 3
    bs = {"q1": 1, "q4": 2, "hex8": 3}[kind]
    h = 1.0 / ne
    nn1 = ne + 1
    if kind == "q1":
        Kref = element_matrix_q1(h)
    elif kind == "q4":
        Kref = element_matrix_q4(h, nu)
    else:
        Kref = element_matrix_hex8(h, nu)
    dirichlet = "eliminate" if kind == "q1" else "identity"

    # --- mesh nodes -> system node ids
    grid = np.stack(np.meshgrid(*([np.arange(nn1)] * dim), indexing="ij"), axis=-1)  # [i,j,(l)] order
    grid = grid.transpose(*reversed(range(dim)), dim).reshape(-1, dim)  # x fastest: id = i + nn1*j + ...
    mesh_ids = np.arange(nn1 ** dim)
    if dirichlet == "eliminate":
        interior = np.all((grid > 0) & (grid < ne), axis=1)
        sys_id = np.full(nn1 ** dim, -1, dtype=np.int64)
        sys_id[interior] = np.arange(int(interior.sum()))
        sys_coords = grid[interior]
        side = ne - 1
        offset0 = 1
    else:
        sys_id = mesh_ids.copy()
        sys_coords = grid
        side = nn1
        offset0 = 0
    n_nodes = sys_coords.shape[0]

    # --- stencil: neighbour offsets sorted so that column ids ascend
    offs = [tuple(reversed(o)) for o in itertools.product((-1, 0, 1), repeat=dim)]  # x fastest -> id order
    offs_arr = np.array(offs)  # [3^dim, dim]
    strides = np.array([side ** d for d in range(dim)])
    loc = sys_coords - offset0  # coords in the system grid
    nbr = loc[:, None, :] + offs_arr[None, :, :]
    valid = np.all((nbr >= 0) & (nbr < side), axis=2)  # [n_nodes, 3^dim]
    nbr_id = (nbr * strides).sum(axis=2)
    counts = valid.sum(axis=1)
    row_ptr = np.zeros(n_nodes + 1, dtype=np.int64)
    row_ptr[1:] = np.cumsum(counts)
    col_idx = nbr_id[valid].astype(np.int32)  # row-major over (node, offset) -> sorted per row
    stencil_blk = np.full(valid.shape, -1, dtype=np.int64)
    stencil_blk[valid] = np.arange(int(row_ptr[-1]))
    off_index = {o: t for t, o in enumerate(offs)}

    # --- elements
    egrid = np.stack(np.meshgrid(*([np.arange(ne)] * dim), indexing="ij"), axis=-1)
    egrid = egrid.transpose(*reversed(range(dim)), dim).reshape(-1, dim)
    centroids = (egrid + 0.5) * h
    corners = _local_corners(dim)
    mesh_strides = np.array([nn1 ** d for d in range(dim)])
    elem_mesh_nodes = np.stack([((egrid + np.array(c)) * mesh_strides).sum(axis=1) for c in corners], axis=1)
    elem_nodes = sys_id[elem_mesh_nodes]  # -1 where eliminated

    pair_blk = []
    for a, b in itertools.product(range(len(corners)), repeat=2):
        na = elem_nodes[:, a]
        nb = elem_nodes[:, b]
        o = tuple(np.array(corners[b]) - np.array(corners[a]))
        if dirichlet == "eliminate":
            m = (na >= 0) & (nb >= 0)
            blk = stencil_blk[na[m], off_index[o]]
            pair_blk.append((m, blk))
        else:
            blk = stencil_blk[na, off_index[o]]
            pair_blk.append((None, blk))
        assert np.all(blk >= 0)
    diag_blk = stencil_blk[:, off_index[tuple([0] * dim)]]

    # --- loads and clamps
    n = n_nodes * bs
    f0 = np.zeros(n)
    clamped = np.zeros(n_nodes, dtype=bool)
    if kind == "q1":
        f0[:] = h * h  # f = 1: integral of each interior hat function
    elif kind == "q4":
        clamped = sys_coords[:, 0] == 0  # left edge x = 0
        right = sys_coords[:, 0] == ne
        w = np.where((sys_coords[:, 1] == 0) | (sys_coords[:, 1] == ne), 0.5 * h, h)
        f0[2 * np.nonzero(right)[0] + 1] = -1.0 * w[right]  # traction (0, -1) on x = 1
    else:
        clamped = sys_coords[:, 2] == 0  # z = 0 face
        top = sys_coords[:, 2] == ne
        ex = np.where((sys_coords[:, 0] == 0) | (sys_coords[:, 0] == ne), 0.5, 1.0)
        ey = np.where((sys_coords[:, 1] == 0) | (sys_coords[:, 1] == ne), 0.5, 1.0)
        w = ex * ey * h * h
        f0[3 * np.nonzero(top)[0] + 2] = -1.0 * w[top]  # load (0, 0, -1) on z = 1
    clamp_blocks = np.zeros(0, dtype=np.int64)
    if dirichlet == "identity":
        cl = np.nonzero(clamped)[0]
        rowmask = np.zeros(int(row_ptr[-1]), dtype=bool)
        rows_of_blk = np.repeat(np.arange(n_nodes), counts)
        rowmask |= clamped[rows_of_blk]
        rowmask |= clamped[col_idx]
        clamp_blocks = np.nonzero(rowmask)[0]
        for c in cl:
            f0[bs * c:bs * (c + 1)] = 0.0

    return StructuredProblem(kind=kind, dim=dim, ne=ne, bs=bs, dirichlet=dirichlet, Kref=Kref,
                             n_nodes=n_nodes, row_ptr=row_ptr.astype(np.int32), col_idx=col_idx,
                             f0=f0, clamped=clamped, centroids=centroids,
                             _elem_nodes=elem_nodes, _pair_blk=pair_blk, _diag_blk=diag_blk,
                             _clamp_blocks=clamp_blocks)


def q1_problem(ne: int) -> StructuredProblem:
    return _build("q1", ne)


def q4_problem(ne: int, nu: float = 0.3) -> StructuredProblem:
    return _build("q4", ne, nu)


def hex8_problem(ne: int, nu: float = 0.3) -> StructuredProblem:
    return _build("hex8", ne, nu)

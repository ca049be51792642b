"""The element-factored form of the parametrized stiffness matrix, as the solver's
element path defines it.

TEST INFRASTRUCTURE ONLY (same rules as pod2g_oracle): imported by the tests,
never by the solver library; it shares no code with the CUDA path.

The finite-element systems of arXiv 2207.02543 (Section 4.1, Section 4.2) have a
material coefficient that is constant over each element, so the stiffness matrix
is the sum K(theta) = sum_e c_e(theta) K_e over elements, and on a uniform mesh
every K_e is one reference matrix K_ref scattered to the element's nodes. Block
(i, j) of K gathers, from every element e that holds both node i (local index a)
and node j (local index b), the bs x bs sub-block K_ref[a, b] scaled by c_e.
A node marked fixed keeps only the identity on its diagonal block: its block row
and block column are zero elsewhere (a clamped node kept as an identity row).

Two evaluations:
  * element_values_f64: the sum in FP64 (the mathematical definition);
  * element_values_f32: the FP32 matrix the solver's element path applies. Each
    entry is c_e (rounded to FP32) times the K_ref entry (rounded to FP32),
    rounded, then the products are added left to right in ascending element
    index, with a rounding after every addition (no fused multiply-add).
Both sides of a parity test therefore solve the same FP32 system.
"""
from __future__ import annotations

import numpy as np


def block_contributions(row_ptr, col_idx, conn, npe):
    """All (block, element, a, b) with element e holding node i = conn[e, a] and node
    j = conn[e, b] and block (i, j) stored, sorted by block, then element index.

    conn[e, a] is the block row (node) of local node a of element e, or -1 (no node).
    Raises ValueError when an element couples two nodes whose block is not stored."""
    row_ptr = np.asarray(row_ptr, dtype=np.int64)
    col_idx = np.asarray(col_idx, dtype=np.int64)
    conn = np.asarray(conn, dtype=np.int64).reshape(-1, npe)
    nb = len(row_ptr) - 1
    rows = np.repeat(np.arange(nb), np.diff(row_ptr))
    keys = rows * nb + col_idx                        # ascending: rows in order, sorted columns
    out = []
    for a in range(npe):
        for b in range(npe):
            i, j = conn[:, a], conn[:, b]
            ok = (i >= 0) & (j >= 0)
            e = np.nonzero(ok)[0]
            want = i[ok] * nb + j[ok]
            pos = np.searchsorted(keys, want)
            if np.any(pos >= len(keys)) or np.any(keys[np.minimum(pos, len(keys) - 1)] != want):
                raise ValueError(f"an element couples local nodes {a}, {b} whose block is not stored")
            out.append(np.stack([pos, e, np.full_like(e, a), np.full_like(e, b)], axis=1))
    c = np.concatenate(out) if out else np.zeros((0, 4), dtype=np.int64)
    order = np.lexsort((c[:, 1], c[:, 0]))
    return c[order]


def _fixed_blocks(row_ptr, col_idx, fixed):
    """(zero, identity) boolean masks over blocks for the fixed nodes."""
    nb = len(row_ptr) - 1
    rows = np.repeat(np.arange(nb), np.diff(row_ptr))
    fx = np.zeros(nb, dtype=bool) if fixed is None else np.asarray(fixed, dtype=bool)
    col_idx = np.asarray(col_idx)
    touched = fx[rows] | fx[col_idx]
    ident = touched & (rows == col_idx) & fx[rows]
    return touched & ~ident, ident


def element_values_f64(row_ptr, col_idx, conn, npe, bs, Kref, coef, fixed=None):
    """values[nnzb, bs, bs] = sum_e c_e K_ref[a, b] in FP64 (fixed nodes: identity / zero)."""
    Kref = np.asarray(Kref, dtype=np.float64)
    coef = np.asarray(coef, dtype=np.float64)
    C = block_contributions(row_ptr, col_idx, conn, npe)
    nnzb = int(np.asarray(row_ptr)[-1])
    vals = np.zeros((nnzb, bs, bs))
    for r in range(bs):
        for cc in range(bs):
            terms = coef[C[:, 1]] * Kref[C[:, 2] * bs + r, C[:, 3] * bs + cc]
            np.add.at(vals[:, r, cc], C[:, 0], terms)
    zero, ident = _fixed_blocks(row_ptr, col_idx, fixed)
    vals[zero] = 0.0
    vals[ident] = np.eye(bs)
    return vals


def element_values_f32(row_ptr, col_idx, conn, npe, bs, Kref, coef, fixed=None):
    """The FP32 values the element path applies (see the module docstring), returned as float64."""
    K32 = np.asarray(Kref, dtype=np.float64).astype(np.float32)
    c32 = np.asarray(coef, dtype=np.float64).astype(np.float32)
    C = block_contributions(row_ptr, col_idx, conn, npe)
    nnzb = int(np.asarray(row_ptr)[-1])
    # rank of each contribution within its block (0 = smallest element index)
    start = np.searchsorted(C[:, 0], np.arange(nnzb))
    rank = np.arange(len(C)) - start[C[:, 0]]
    vals = np.zeros((nnzb, bs, bs), dtype=np.float32)
    for t in range(int(rank.max()) + 1 if len(C) else 0):
        sel = C[rank == t]                            # at most one contribution per block
        blk, e, a, b = sel[:, 0], sel[:, 1], sel[:, 2], sel[:, 3]
        for r in range(bs):
            for cc in range(bs):
                term = c32[e] * K32[a * bs + r, b * bs + cc]        # FP32 product, rounded
                vals[blk, r, cc] = vals[blk, r, cc] + term          # FP32 addition, rounded
    zero, ident = _fixed_blocks(row_ptr, col_idx, fixed)
    vals[zero] = 0.0
    vals[ident] = np.eye(bs, dtype=np.float32)
    return vals.astype(np.float64)

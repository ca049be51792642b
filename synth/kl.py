"""Karhunen-Loeve expansion of a squared-exponential random field on the unit square/cube.

Input generation only: this supplies the element coefficients c_e(theta) that
parametrise K(theta) (the lognormal material parameters that Section 4.1 and
Section 4.2 use as random inputs become lognormal KL fields here).

Covariance C(x, y) = sigma^2 exp(-|x - y|^2 / (2 ell^2)). It factorises over the
coordinates, so the multi-dimensional eigenpairs are products of 1D Nystrom
eigenpairs computed on the element-centroid grid with quadrature weight h:
    (c(x_i, x_j) h) v = lam v,     phi = v / sqrt(h)   (so sum_i phi_i^2 h = 1).
Multi-dimensional modes are sorted by eigenvalue (descending); ties, which occur
exactly for permuted index tuples, are broken by the index sum, then
lexicographically. Each 1D eigenvector's largest-magnitude entry is made
positive (lowest index on ties).
"""
from __future__ import annotations

import itertools

import numpy as np


def kl_1d(ne: int, ell: float):
    """1D Nystrom eigenpairs of exp(-(x-y)^2/(2 ell^2)) on [0,1], centroids of ne cells."""
    h = 1.0 / ne
    x = (np.arange(ne) + 0.5) * h
    A = np.exp(-(x[:, None] - x[None, :]) ** 2 / (2.0 * ell ** 2)) * h
    lam, V = np.linalg.eigh(A)
    order = np.argsort(-lam, kind="stable")
    lam = lam[order]
    V = V[:, order]
    for j in range(V.shape[1]):
        i = int(np.argmax(np.abs(V[:, j])))
        if V[i, j] < 0:
            V[:, j] = -V[:, j]
    return lam, V / np.sqrt(h)


def kl_modes(dim: int, ne: int, ell: float, sigma: float, m: int):
    """Top-m eigenvalues and modes (evaluated at element centroids, x fastest)."""
    lam1, phi1 = kl_1d(ne, ell)
    top = min(m, ne)
    cands = []
    for idx in itertools.product(range(top), repeat=dim):
        v = sigma ** 2 * float(np.prod([lam1[i] for i in idx]))
        cands.append((-float(f"{v:.12e}"), sum(idx), idx, v))
    cands.sort()
    chosen = cands[:m]
    lam = np.array([c[3] for c in chosen])
    modes = np.empty((ne ** dim, m))
    for t, c in enumerate(chosen):
        idx = c[2]
        # element e = ix + ne*iy (+ ne^2*iz): outer product with x fastest
        mode = phi1[:, idx[0]]
        for d in range(1, dim):
            mode = np.multiply.outer(phi1[:, idx[d]], mode)
        modes[:, t] = mode.reshape(-1)
    return lam, modes


def field(lam: np.ndarray, modes: np.ndarray, xi: np.ndarray) -> np.ndarray:
    """g = sum_m sqrt(lam_m) xi_m phi_m at the element centroids."""
    return modes @ (np.sqrt(lam) * np.asarray(xi, dtype=np.float64))


def lognormal_params(cov: float):
    """(mu_g, sigma_g) so that exp(mu_g + sigma_g g) has mean 1 and CoV `cov` for g ~ N(0, 1)."""
    s2 = np.log1p(cov ** 2)
    return -0.5 * s2, float(np.sqrt(s2))

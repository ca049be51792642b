"""Shared check of the library's reported final residual (used by the GPU parity tests).

The library recomputes ||b - K x||_2 / ||b||_2 at exit in FP64 from its stored values.
The host recomputes it from the same matrix and the returned x with scipy in FP64, in a
different summation order. A row of m terms evaluated in FP64 is within
gamma_m (|K||x| + |b|)_i of its exact value (gamma_m = m u / (1 - m u), u = 2^-53), so the
two relative residuals differ by at most 2 gamma_m ||(|K||x| + |b|)||_2 / ||b||_2.
"""
import numpy as np


def host_relres_and_bound(K, b, x):
    bn = np.linalg.norm(b)
    true_rel = np.linalg.norm(b - K @ x) / bn
    m = int(np.max(np.diff(K.indptr))) + 1
    u = 2.0 ** -53
    scale = np.linalg.norm(abs(K) @ np.abs(x) + np.abs(b)) / bn
    return true_rel, 2 * (m * u / (1 - m * u)) * scale


def assert_relres_matches(K, b, x, rel_lib, tol):
    true_rel, bound = host_relres_and_bound(K, b, x)
    assert abs(true_rel - rel_lib) <= bound, (true_rel, rel_lib, bound)
    assert true_rel <= 1.05 * tol + bound, (true_rel, bound)

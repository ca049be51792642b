"""Randomised properties of the oracle beyond the structured meshes (hypothesis; skipped
where it is not installed):

* multicolour_groups on random structurally symmetric block patterns: the groups partition
  the dofs, no two dofs of a group couple, and a sweep equals the triangular splitting;
* PCG with the two-grid preconditioner on random SPD block systems: converges to the dense
  solution, its K-norm error never increases, and the cycle operator is symmetric.
"""
import numpy as np
import pytest

hyp = pytest.importorskip("hypothesis")
from hypothesis import given, settings, strategies as st  # noqa: E402

import scipy.sparse as sp  # noqa: E402

from oracle import pod2g_oracle as O  # noqa: E402


def _random_block_spd(seed, nb, bs, density):
    rng = np.random.default_rng(seed)
    mask = rng.random((nb, nb)) < density
    mask = mask | mask.T | np.eye(nb, dtype=bool)
    rows, cols = np.nonzero(mask)                     # row-major: sorted rows, sorted columns
    row_ptr = np.zeros(nb + 1, dtype=np.int64)
    np.add.at(row_ptr, rows + 1, 1)
    row_ptr = np.cumsum(row_ptr)
    A = rng.standard_normal((nb * bs, nb * bs)) * np.kron(mask, np.ones((bs, bs)))
    K = A @ A.T * np.kron(mask, np.ones((bs, bs)))    # keep the block pattern
    K = 0.5 * (K + K.T) + np.diag(np.abs(K).sum(axis=1) + 1.0)   # diagonally dominant => SPD
    return row_ptr, cols.astype(np.int64), sp.csr_matrix(K)


@settings(max_examples=25, deadline=None)
@given(seed=st.integers(0, 10 ** 6), nb=st.integers(2, 12), bs=st.integers(1, 3),
       density=st.floats(0.05, 0.6))
def test_groups_partition_and_sweep_splitting(seed, nb, bs, density):
    from scipy.linalg import solve_triangular
    row_ptr, col_idx, K = _random_block_spd(seed, nb, bs, density)
    groups = O.multicolour_groups(row_ptr, col_idx, bs)
    n = nb * bs
    assert np.array_equal(np.sort(np.concatenate(groups)), np.arange(n))
    Kd = K.toarray()
    for g in groups:
        sub = Kd[np.ix_(g, g)]
        assert np.count_nonzero(sub - np.diag(np.diag(sub))) == 0
    order = np.concatenate(groups)
    rng = np.random.default_rng(seed + 1)
    f, u = rng.standard_normal(n), rng.standard_normal(n)
    Kp = Kd[np.ix_(order, order)]
    want = u.copy()
    want[order] += solve_triangular(np.tril(Kp), (f - Kd @ u)[order], lower=True)
    got = O.gauss_seidel(K, K.diagonal(), f, u, groups, 1)
    assert np.allclose(got, want, rtol=1e-10, atol=1e-10 * max(1.0, np.abs(want).max()))


@settings(max_examples=20, deadline=None)
@given(seed=st.integers(0, 10 ** 6), nb=st.integers(3, 10), bs=st.integers(1, 2), k=st.integers(0, 3),
       sgs=st.booleans())
def test_two_grid_pcg_on_random_spd_systems(seed, nb, bs, k, sgs):
    row_ptr, col_idx, K = _random_block_spd(seed, nb, bs, 0.3)
    n = nb * bs
    k = min(k, n - 1)
    rng = np.random.default_rng(seed + 2)
    Phi = np.linalg.qr(rng.standard_normal((n, k)))[0] if k else np.zeros((n, 0))
    groups = O.multicolour_groups(row_ptr, col_idx, bs) if sgs else None
    omega = 1.0 if sgs else 0.5
    f = rng.standard_normal(n)
    res = O.pod2g_pcg(K, f, None, Phi, omega, 1e-10, 10 * n, groups=groups, record=True)
    Kd = K.toarray()
    xs = np.linalg.solve(Kd, f)
    assert res.status == O.OK
    assert np.linalg.norm(res.x - xs) <= 1e-7 * np.linalg.norm(xs)
    errs = [float((r["x"] - xs) @ Kd @ (r["x"] - xs)) for r in res.iterates]
    assert all(b <= a * (1 + 1e-9) + 1e-24 for a, b in zip(errs, errs[1:]))
    st_ = O.pod2g_setup(K, Phi, omega, 1, 1, groups)
    app = O.pod2g_preconditioner(K, st_)
    B = np.column_stack([app(e) for e in np.eye(n)])
    assert np.abs(B - B.T).max() <= 1e-10 * np.abs(B).max()

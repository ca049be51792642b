"""Pins for the element-factored operator of the oracle (oracle/element_operator.py).

* the FP64 evaluation equals the input generator's assembly (a separate code path:
  per local-pair scatter) for Q1 (eliminated boundary), Q4 and Hex8 (clamped nodes);
* the FP32 evaluation is within the rounding-error bound of a length-T sum of
  rounded products of the FP64 sum;
* entries with one contributing element are the single rounded product;
* the summation order and rounding agree with a brute-force scalar loop;
* a connectivity that needs a block the pattern lacks is rejected.
"""
import numpy as np
import pytest

from oracle import element_operator as EO
from synth import fe
from synth.problems import Workload


def _prob(kind, ne, seed=0):
    P = fe._build(kind, ne)
    coef = np.random.default_rng(seed).lognormal(0.0, 0.5, P.n_el)
    return P, coef


def _args(P):
    fixed = P.clamped if P.dirichlet == "identity" else None
    return P.row_ptr, P.col_idx, P.conn, P.npe, P.bs, P.Kref, fixed


@pytest.mark.parametrize("kind,ne", [("q1", 6), ("q4", 5), ("hex8", 3)])
def test_f64_matches_generator_assembly(kind, ne):
    P, coef = _prob(kind, ne)
    rp, ci, conn, npe, bs, K, fixed = _args(P)
    v = EO.element_values_f64(rp, ci, conn, npe, bs, K, coef, fixed)
    ref = P.values(coef)
    scale = np.abs(ref).max()
    assert np.allclose(v, ref, rtol=1e-14, atol=1e-14 * scale)


@pytest.mark.parametrize("kind,ne", [("q1", 6), ("q4", 5), ("hex8", 3)])
def test_f32_within_summation_bound(kind, ne):
    P, coef = _prob(kind, ne, 1)
    rp, ci, conn, npe, bs, K, fixed = _args(P)
    v32 = EO.element_values_f32(rp, ci, conn, npe, bs, K, coef, fixed)
    v64 = EO.element_values_f64(rp, ci, conn, npe, bs, K, coef, fixed)
    absum = EO.element_values_f64(rp, ci, conn, npe, bs, np.abs(K), np.abs(coef), fixed)
    C = EO.block_contributions(rp, ci, conn, npe)
    T = np.bincount(C[:, 0], minlength=len(ci))[:, None, None]
    u = 2.0 ** -24
    bound = (T + 3) * u * np.abs(absum) * (1 + 1e-6)
    assert np.all(np.abs(v32 - v64) <= bound + 1e-300)
    # the values are FP32 numbers
    assert np.array_equal(v32, v32.astype(np.float32).astype(np.float64))


def test_single_contribution_entries_are_one_rounded_product():
    P, coef = _prob("q4", 4, 2)
    rp, ci, conn, npe, bs, K, fixed = _args(P)
    v32 = EO.element_values_f32(rp, ci, conn, npe, bs, K, coef, None)
    C = EO.block_contributions(rp, ci, conn, npe)
    T = np.bincount(C[:, 0], minlength=len(ci))
    K32, c32 = K.astype(np.float32), coef.astype(np.float32)
    single = np.nonzero(T == 1)[0]
    assert single.size > 0
    for blk in single[:50]:
        _, e, a, b = C[C[:, 0] == blk][0]
        want = (c32[e] * K32[a * bs:(a + 1) * bs, b * bs:(b + 1) * bs]).astype(np.float64)
        assert np.array_equal(v32[blk], want)


def test_order_and_rounding_match_scalar_loop():
    P, coef = _prob("hex8", 2, 3)
    rp, ci, conn, npe, bs, K, fixed = _args(P)
    v32 = EO.element_values_f32(rp, ci, conn, npe, bs, K, coef, None)
    nb = len(rp) - 1
    conn = P.conn
    brute = np.zeros((len(ci), bs, bs), dtype=np.float32)
    for i in range(nb):
        for blk in range(rp[i], rp[i + 1]):
            j = ci[blk]
            for r in range(bs):
                for cc in range(bs):
                    acc = np.float32(0.0)
                    for e in range(P.n_el):                     # ascending element index
                        ea = np.nonzero(conn[e] == i)[0]
                        eb = np.nonzero(conn[e] == j)[0]
                        if ea.size and eb.size:
                            t = np.float32(coef[e]) * np.float32(K[ea[0] * bs + r, eb[0] * bs + cc])
                            acc = np.float32(acc + t)
                    brute[blk, r, cc] = acc
    assert np.array_equal(v32, brute.astype(np.float64))


def test_missing_block_rejected():
    P, coef = _prob("q4", 3)
    rp, ci, conn, npe, bs, K, fixed = _args(P)
    conn = conn.copy()
    conn[0, 3] = P.n_nodes - 1          # couples node 0 with the far corner
    with pytest.raises(ValueError):
        EO.block_contributions(rp, ci, conn, npe)


def test_workload_coefficients_reproduce_values():
    wl = Workload("q4_16")
    xi = wl.query_thetas(1)[0]
    P = wl.problem
    v = EO.element_values_f64(P.row_ptr, P.col_idx, P.conn, P.npe, P.bs, P.Kref, wl.coef(xi), P.clamped)
    assert np.allclose(v, wl.values(xi), rtol=1e-14, atol=1e-14 * np.abs(v).max())

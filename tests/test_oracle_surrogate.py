"""Pins of the oracle's surrogate initial guess (oracle/surrogate.py, Section 3.2) against what
the mathematics and independent solves fix, and of the training data it receives."""
import math

import numpy as np
import pytest

from oracle import pod2g_oracle as O
from oracle import surrogate as S
from synth.problems import Workload
from synth.snapshots import snapshot_matrix


class _W:
    """A hand-set network."""

    def __init__(self, **kw):
        self.__dict__.update(kw)


def _one_unit(a, c, d, w3=4.0, b3=1.0):
    return _W(w1=np.array([[a]]), b1=np.array([0.0]), w2=np.array([[c]]), b2=np.array([d]),
              w3=np.array([[w3]]), b3=np.array([b3]), z_mean=np.array([0.0]), z_std=np.array([1.0]),
              psi=np.array([[1.0]]))


def test_ffnn_layers_compose_in_order():
    # tanh(atanh(0.5)) = 0.5, then tanh(2 atanh(0.25) * 0.5) = 0.25, then 4 * 0.25 + 1 = 2
    w = _one_unit(math.atanh(0.5), 2 * math.atanh(0.25), 0.0)
    assert abs(S.ffnn(np.array([1.0]), w.w1, w.b1, w.w2, w.b2, w.w3, w.b3)[0] - 2.0) <= 1e-14
    # the second layer's bias enters inside its tanh: tanh(0 * h1 + atanh(0.75)) = 0.75
    w = _one_unit(1.0, 0.0, math.atanh(0.75))
    assert abs(S.ffnn(np.array([3.0]), w.w1, w.b1, w.w2, w.b2, w.w3, w.b3)[0] - 4.0) <= 1e-14


def test_ffnn_properties():
    rng = np.random.default_rng(0)
    H, m, ks = 7, 3, 5
    w1, w2, w3 = rng.standard_normal((H, m)), rng.standard_normal((H, H)), rng.standard_normal((ks, H))
    z = np.zeros(H)
    th = rng.standard_normal(m)
    # all biases zero: the network is odd in theta (tanh is odd)
    assert np.allclose(S.ffnn(-th, w1, z, w2, z, w3, np.zeros(ks)), -S.ffnn(th, w1, z, w2, z, w3, np.zeros(ks)),
                       atol=1e-15)
    # a zero second layer: the output is tanh(b2) mapped by the last layer, whatever theta
    b2, b3 = rng.standard_normal(H), rng.standard_normal(ks)
    o = S.ffnn(th, w1, z, np.zeros((H, H)), b2, w3, b3)
    assert np.allclose(o, w3 @ np.tanh(b2) + b3, atol=1e-14)
    # outputs of a tanh layer are bounded by 1: |o - b3| <= sum_j |w3_ij|
    big = S.ffnn(1e6 * th, w1, z, w2, z, w3, b3)
    assert np.all(np.abs(big - b3) <= np.abs(w3).sum(1) + 1e-12)


def test_prediction_is_linear_in_the_load_and_decodes_with_psi():
    rng = np.random.default_rng(1)
    n, ks, H, m = 40, 6, 5, 3
    w = _W(psi=np.linalg.qr(rng.standard_normal((n, ks)))[0], w1=rng.standard_normal((H, m)),
           b1=rng.standard_normal(H), w2=rng.standard_normal((H, H)), b2=rng.standard_normal(H),
           w3=rng.standard_normal((ks, H)), b3=rng.standard_normal(ks), z_mean=rng.standard_normal(ks),
           z_std=rng.random(ks) + 0.5)
    th = rng.standard_normal(m)
    u1 = S.surrogate_prediction(th, 1.0, w)
    assert np.allclose(S.surrogate_prediction(th, 2.5, w), 2.5 * u1, rtol=1e-15, atol=0)
    # the prediction lies in span(Psi) with coordinates z_mean + z_std * FFNN(theta)
    z = w.psi.T @ u1
    assert np.allclose(w.psi @ z, u1, atol=1e-13)
    assert np.allclose(z, w.z_mean + w.z_std * S.ffnn(th, w.w1, w.b1, w.w2, w.b2, w.w3, w.b3), atol=1e-13)


def test_decoder_of_a_snapshot_latent_is_its_pod_projection():
    """A network whose output is the standardised latent of snapshot i (W3 = 0, b3 set) predicts
    Psi Psi^T u_i, which equals the independently solved u_i up to the POD truncation error."""
    from synth.surrogate import latent_size
    from synth.snapshots import surrogate_data
    wl = Workload("q1_16")
    ks = latent_size(wl)
    psi, Z, theta = surrogate_data(wl, ks, use_disk=False)
    U = snapshot_matrix(wl)          # direct solves (SuperLU), independent of the decoder
    sv = np.linalg.svd(U, compute_uv=False)
    tail = np.sqrt(np.sum(sv[ks:] ** 2))   # ||(I - Psi Psi^T) u_i|| <= (sum of discarded sigma^2)^(1/2)
    H, m = 4, wl.spec.m
    zm, zs = Z.mean(1), Z.std(1) + 1e-300
    for i in (0, 7, len(theta) - 1):
        w = _W(psi=psi, w1=np.zeros((H, m)), b1=np.zeros(H), w2=np.zeros((H, H)), b2=np.zeros(H),
               w3=np.zeros((ks, H)), b3=(Z[:, i] - zm) / zs, z_mean=zm, z_std=zs)
        u = S.surrogate_prediction(theta[i], 1.0, w)
        assert np.allclose(u, psi @ (psi.T @ U[:, i]), rtol=1e-10, atol=1e-14 * np.abs(U[:, i]).max())
        assert np.linalg.norm(u - U[:, i]) <= tail * (1 + 1e-8)


def test_trained_surrogate_predicts_solutions_and_pcg_from_it_converges():
    """The trained surrogate's prediction for a query is within 25% of the direct solution (about
    10% with the 17 training snapshots of this small case; a decoding or scaling mistake gives
    errors near 100%), and POD-2G-PCG from it reaches the same x as from zero without
    more iterations (the paper's error bound, eq. ineq:Main, grows with the initial error)."""
    import scipy.sparse.linalg as sla
    pytest.importorskip("torch")
    from synth.surrogate import train_surrogate, load_scale
    from synth.snapshots import pod_basis
    wl = Workload("q1_16")
    sur = train_surrogate(wl, steps=1500, use_disk=False)
    P, Phi = wl.problem, pod_basis(wl, use_disk=False)
    xs, bs = wl.query_thetas(4), wl.rhs(4)
    for i in range(4):
        K = P.csr(wl.values(xs[i]))
        u = sla.splu(K.tocsc()).solve(bs[i])
        x0 = S.surrogate_prediction(xs[i], load_scale(wl, bs[i]), sur)
        assert np.linalg.norm(x0 - u) <= 0.25 * np.linalg.norm(u)
        r0 = O.pod2g_pcg(K, bs[i], None, Phi, wl.spec.omega, 1e-10, 500)
        r1 = O.pod2g_pcg(K, bs[i], x0, Phi, wl.spec.omega, 1e-10, 500)
        assert r0.status == O.OK and r1.status == O.OK
        assert r1.iters <= r0.iters + 1
        assert np.linalg.norm(r1.x - r0.x) <= 1e-8 * np.linalg.norm(r0.x)

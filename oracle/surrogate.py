"""CPU FP64 oracle of the surrogate initial guess (Section 3.2, eq. FFNN and the online phase).

TEST INFRASTRUCTURE ONLY: imported by the tests, the package's smoke check and the CPU-baseline
leg of the benchmark, never by the solver library; it shares no code with the CUDA path.

The surrogate maps the parameters theta to a solution in two steps, u = decoder(FFNN(theta)):
  * FFNN(theta): a feed-forward network with two hidden tanh layers,
        h1 = tanh(W1 theta + b1),  h2 = tanh(W2 h1 + b2),  o = W3 h2 + b3,
    whose output is the standardised latent vector; the latent is z = z_mean + z_std * o;
  * decoder(z) = Psi z with the ks POD modes Psi (the linear autoencoder of the snapshot set).
A query whose load is s times the unit load of the snapshots gets s * decoder(FFNN(theta))
(linearity of the solution in the load). Everything is evaluated in FP64 with numpy.
"""
from __future__ import annotations

import numpy as np


def ffnn(theta, w1, b1, w2, b2, w3, b3) -> np.ndarray:
    """The network's output o(theta) (eq. FFNN's model), FP64."""
    h1 = np.tanh(w1 @ theta + b1)
    h2 = np.tanh(w2 @ h1 + b2)
    return w3 @ h2 + b3


def latent(theta, sur) -> np.ndarray:
    """z = z_mean + z_std * FFNN(theta)."""
    return sur.z_mean + sur.z_std * ffnn(np.asarray(theta, dtype=np.float64), sur.w1, sur.b1, sur.w2, sur.b2,
                                         sur.w3, sur.b3)


def decoder(z, psi) -> np.ndarray:
    """u = Psi z."""
    return psi @ z


def surrogate_prediction(theta, scale, sur) -> np.ndarray:
    """u_sur = scale * decoder(FFNN(theta)) (the online phase of Section 3.2)."""
    return scale * decoder(latent(theta, sur), sur.psi)

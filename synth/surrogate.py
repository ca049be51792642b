"""Training of the surrogate that supplies the initial guess (Section 3.2): u = decoder(FFNN(theta)).

Offline input generation, like the POD basis: it produces weights that the CUDA library and the
oracle then both receive unchanged, and holds none of the solver's arithmetic.

  * Encoder / decoder: the linear autoencoder of the snapshot set, i.e. its first ks POD modes Psi
    (the minimiser of the reconstruction loss over linear encoders and decoders); the latent of a
    snapshot u_i is z_i = Psi^T u_i and the decoder is u = Psi z. (The paper trains a convolutional
    autoencoder; a linear one keeps the decoder a tall-skinny product on the device.)
  * FFNN: theta (the m KL coordinates) -> hidden -> hidden -> ks, tanh activations, trained on the
    standardised latents (z - mean) / std with the mean-squared loss of eq. FFNN, Adam, a 70 / 30
    train / validation split as in the paper (Section 4.1), keeping the weights of the best
    validation loss.
  * Loads: every snapshot is solved for the unit load f0; the solution is linear in the load, so a
    query with right-hand side s f0 gets s times the prediction.
"""
from __future__ import annotations

import os
from dataclasses import dataclass

import numpy as np

from .problems import Workload
from .snapshots import cache_dir, surrogate_data


@dataclass
class SurrogateWeights:
    psi: np.ndarray      # [n, ks] decoder (POD modes)
    w1: np.ndarray       # [H, m]
    b1: np.ndarray       # [H]
    w2: np.ndarray       # [H, H]
    b2: np.ndarray       # [H]
    w3: np.ndarray       # [ks, H]
    b3: np.ndarray       # [ks]
    z_mean: np.ndarray   # [ks]
    z_std: np.ndarray    # [ks]
    val_rel_err: float   # mean relative l2 error of the predicted latents on the validation split


def latent_size(wl: Workload) -> int:
    """ks = 2k latent coordinates, at most half the snapshots."""
    return int(min(2 * wl.spec.k, wl.spec.n_snap // 2))


def train_surrogate(wl: Workload, hidden: int = 64, steps: int = 4000, seed: int = 0, device: str | None = None,
                    use_disk: bool = True) -> SurrogateWeights:
    ks = latent_size(wl)
    path = os.path.join(cache_dir(), f"surnet_{wl.spec.name}_ks{ks}_H{hidden}_s{seed}.npz")
    if use_disk and os.path.exists(path):
        d = np.load(path)
        return SurrogateWeights(**{k: d[k] for k in d.files if k != "val_rel_err"},
                                val_rel_err=float(d["val_rel_err"]))
    import torch
    psi, Z, theta = surrogate_data(wl, ks, device=device if wl.n > 20_000 else None, use_disk=use_disk)
    N = Z.shape[1]
    rng = np.random.default_rng(5000 + wl.spec.cid + seed)
    perm = rng.permutation(N)
    ntr = int(round(0.7 * N))
    tr, va = perm[:ntr], perm[ntr:]
    X = torch.from_numpy(theta).double()
    Y = torch.from_numpy(Z.T.copy()).double()
    z_mean = Y[tr].mean(0)
    z_std = Y[tr].std(0).clamp_min(1e-300)
    Yn = (Y - z_mean) / z_std
    g = torch.Generator().manual_seed(6000 + wl.spec.cid + seed)
    m = X.shape[1]

    def init(o, i):
        lim = (6.0 / (o + i)) ** 0.5
        return (torch.rand(o, i, generator=g, dtype=torch.float64) * 2 - 1) * lim

    params = [init(hidden, m), torch.zeros(hidden, dtype=torch.float64), init(hidden, hidden),
              torch.zeros(hidden, dtype=torch.float64), init(ks, hidden), torch.zeros(ks, dtype=torch.float64)]
    for p in params:
        p.requires_grad_(True)

    def net(x):
        h = torch.tanh(x @ params[0].T + params[1])
        h = torch.tanh(h @ params[2].T + params[3])
        return h @ params[4].T + params[5]

    opt = torch.optim.Adam(params, lr=3e-3)
    best, best_p = float("inf"), None
    for it in range(steps):
        opt.zero_grad()
        loss = ((net(X[tr]) - Yn[tr]) ** 2).mean()
        loss.backward()
        opt.step()
        if it % 50 == 49 or it == steps - 1:
            with torch.no_grad():
                vl = float(((net(X[va]) - Yn[va]) ** 2).mean())
            if vl < best:
                best, best_p = vl, [p.detach().clone() for p in params]
    with torch.no_grad():
        for p, q in zip(params, best_p):
            p.copy_(q)
        zp = net(X[va]) * z_std + z_mean
        rel = float((torch.linalg.vector_norm(zp - Y[va], dim=1) / torch.linalg.vector_norm(Y[va], dim=1)).mean())
    w = [p.detach().numpy().copy() for p in params]
    out = SurrogateWeights(psi=psi, w1=w[0], b1=w[1], w2=w[2], b2=w[3], w3=w[4], b3=w[5],
                           z_mean=z_mean.numpy().copy(), z_std=z_std.numpy().copy(), val_rel_err=rel)
    if use_disk:
        np.savez(path, **{k: getattr(out, k) for k in ("psi", "w1", "b1", "w2", "b2", "w3", "b3", "z_mean", "z_std")},
                 val_rel_err=rel)
    return out


def load_scale(wl: Workload, b: np.ndarray) -> float:
    """The load factor s of a right-hand side b = s f0 (least squares)."""
    f0 = wl.problem.f0
    return float(b @ f0 / (f0 @ f0))

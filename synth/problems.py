"""Named synthetic workloads: problem + KL coefficient model + POD size + batch.

Seeds (all numpy Generator / scipy QMC seeds):
  * snapshot parameters: Latin hypercube in probability space (seed 1000 + config id),
    mapped to N(0, 1) through the inverse normal CDF (the paper samples its
    training parameters by Latin hypercube, Section 3.2 / Section 4.1);
  * query parameters: xi ~ N(0, 1) (seed 2000 + config id);
  * load scale per query: lognormal, mean 1, CoV 0.3 (seed 4000 + config id), the
    analogue of the paper's random load P (Section 4.1, table of random parameters).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from . import fe, kl


@dataclass(frozen=True)
class Spec:
    name: str
    cid: int            # config id (seeds)
    kind: str           # q1 / q4 / hex8
    ne: int
    m: int              # KL terms
    k: int              # POD modes
    n_snap: int         # snapshots
    batch: int          # batch slots
    omega: float        # damped-Jacobi weight
    phi_dtype: str      # "f64", "f32", "bf16"
    precision: str      # "fp64" (plain FP64 path) or "mixed"
    sigma: float = 1.0  # KL kernel std (q1 uses exp(g) directly)
    cov: float = 0.3    # CoV of the lognormal modulus (elasticity)
    ell: float = 0.3


# Full-size workloads (the five synthetic configurations) and scaled-down variants
# with the same structure for tests.
SPECS = {
    "q1_64": Spec("q1_64", 1, "q1", 64, 4, 10, 50, 1, 2.0 / 3.0, "f64", "fp64", sigma=0.5),
    "q4_512": Spec("q4_512", 2, "q4", 512, 8, 20, 200, 64, 2.0 / 3.0, "f32", "mixed", cov=0.3),
    "hex8_64": Spec("hex8_64", 3, "hex8", 64, 12, 30, 300, 32, 0.5, "bf16", "mixed", cov=0.4),
    "q1_1024": Spec("q1_1024", 4, "q1", 1024, 16, 25, 250, 16, 2.0 / 3.0, "f32", "mixed", sigma=0.5),
    "hex8_128": Spec("hex8_128", 5, "hex8", 128, 16, 40, 400, 4, 0.5, "f32", "mixed", cov=0.4),
    # scaled-down variants (tests)
    "q1_16": Spec("q1_16", 11, "q1", 16, 4, 6, 24, 4, 2.0 / 3.0, "f64", "fp64", sigma=0.5),
    "q1_32": Spec("q1_32", 12, "q1", 32, 4, 8, 30, 5, 2.0 / 3.0, "f32", "mixed", sigma=0.5),
    "q4_16": Spec("q4_16", 13, "q4", 16, 8, 8, 30, 3, 2.0 / 3.0, "f32", "mixed", cov=0.3),
    "q4_64": Spec("q4_64", 14, "q4", 64, 8, 20, 60, 7, 2.0 / 3.0, "f32", "mixed", cov=0.3),
    "hex8_8": Spec("hex8_8", 15, "hex8", 8, 12, 10, 30, 3, 0.5, "bf16", "mixed", cov=0.4),
    "hex8_16": Spec("hex8_16", 16, "hex8", 16, 12, 30, 60, 5, 0.5, "bf16", "mixed", cov=0.4),
    # mid-size case of the 2D elasticity family (profiling: a few GB on the device)
    "q4_256": Spec("q4_256", 17, "q4", 256, 8, 20, 100, 64, 2.0 / 3.0, "f32", "mixed", cov=0.3),
    "hex8_32": Spec("hex8_32", 18, "hex8", 32, 12, 30, 100, 32, 0.5, "bf16", "mixed", cov=0.4),
    # 2D diffusion at the lane count and basis size of the 1024^2 serving member (16 slots, k = 25)
    "q1_128": Spec("q1_128", 19, "q1", 128, 16, 25, 60, 16, 2.0 / 3.0, "f32", "mixed", sigma=0.5),
}


class Workload:
    """A spec instantiated: mesh, pattern, KL modes; theta -> values; loads."""

    def __init__(self, spec: Spec | str):
        if isinstance(spec, str):
            spec = SPECS[spec]
        self.spec = spec
        if spec.kind == "q1":
            self.problem = fe.q1_problem(spec.ne)
        elif spec.kind == "q4":
            self.problem = fe.q4_problem(spec.ne)
        else:
            self.problem = fe.hex8_problem(spec.ne)
        dim = self.problem.dim
        sig = spec.sigma if spec.kind == "q1" else 1.0
        self.kl_lam, self.kl_modes = kl.kl_modes(dim, spec.ne, spec.ell, sig, spec.m)
        self.mu_g, self.sigma_g = kl.lognormal_params(spec.cov)

    @property
    def n(self):
        return self.problem.n

    def coef(self, xi: np.ndarray) -> np.ndarray:
        """Element coefficients for KL coordinates xi (length m)."""
        g = kl.field(self.kl_lam, self.kl_modes, xi)
        if self.spec.kind == "q1":
            return np.exp(g)                       # kappa = exp(sum sqrt(lam) xi phi)
        return np.exp(self.mu_g + self.sigma_g * g)  # E lognormal, mean 1, CoV cov

    def values(self, xi: np.ndarray) -> np.ndarray:
        return self.problem.values(self.coef(xi))

    def values_torch(self, xis: np.ndarray, device="cpu"):
        """Batched values [len(xis), nnzb, bs, bs] (float64 torch tensor), identical to values()."""
        import torch
        coef = np.stack([self.coef(xi) for xi in xis])
        return self.problem.values_torch(torch.from_numpy(coef).to(device))

    def snapshot_thetas(self, count: int | None = None) -> np.ndarray:
        from scipy.stats import qmc
        from scipy.special import ndtri
        count = self.spec.n_snap if count is None else count
        u = qmc.LatinHypercube(d=self.spec.m, seed=1000 + self.spec.cid).random(count)
        return ndtri(u)

    def query_thetas(self, count: int, offset: int = 0) -> np.ndarray:
        rng = np.random.default_rng(2000 + self.spec.cid)
        xi = rng.standard_normal((offset + count, self.spec.m))
        return xi[offset:]

    def load_scales(self, count: int, offset: int = 0) -> np.ndarray:
        if self.spec.kind == "q1":
            return np.ones(count)
        mu, s = kl.lognormal_params(0.3)
        rng = np.random.default_rng(4000 + self.spec.cid)
        z = rng.standard_normal(offset + count)[offset:]
        return np.exp(mu + s * z)

    def rhs(self, count: int, offset: int = 0) -> np.ndarray:
        """Right-hand sides b_i = s_i f0, shape [count, n]."""
        return self.load_scales(count, offset)[:, None] * self.problem.f0[None, :]

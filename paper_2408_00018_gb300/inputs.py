"""Seeded synthetic inputs (boxes, rotations, batched problem lists).

Shared by the tests, the benchmark and the CPU oracle's checks.  Nothing here
computes any step of the annealing: it only produces the data a user would
pass in (Eq. 1's box and cost choice, and the orthogonal matrices of the
rotated costs).
"""
from __future__ import annotations

import numpy as np

# Boxes of the workloads (Sec. 4.1 Schwefel box widened/narrowed as the
# workloads state; Appendix tests 1, 13, 14).
BOXES = {
    "schwefel": (-500.0, 500.0),
    "rastrigin": (-5.12, 5.12),
    "ackley": (-32.0, 32.0),
    "rosenbrock": (-5.0, 10.0),
    "rot_rastrigin": (-5.12, 5.12),
    "rot_schwefel": (-500.0, 500.0),
}

# Closed-form minima used as targets (Sec. 4.1; Appendix tests 1, 13, 14).
SCHWEFEL_F_STAR = -418.98288727243370
F_STAR = {"schwefel": SCHWEFEL_F_STAR, "rastrigin": 0.0, "ackley": 0.0, "rosenbrock": 0.0, "rot_rastrigin": 0.0}


def box(cost: str, n: int):
    lo, hi = BOXES[cost]
    return np.full(n, lo), np.full(n, hi)


def rotation(n: int, seed: int = 0) -> np.ndarray:
    """Orthogonal Q: the Q factor of a seeded n x n N(0,1) matrix, signs fixed so diag(R) > 0."""
    rng = np.random.default_rng([seed, n, 2])
    A = rng.standard_normal((n, n))
    Q, R = np.linalg.qr(A)
    return Q * np.sign(np.diag(R))[None, :]


def batch_problems(count: int = 512, seed: int = 0, n_range=(2, 512), chain_range=(256, 16384)):
    """A list of independent problems: cost uniform over the four separable costs,
    n uniform in n_range, chain count uniform in chain_range (inclusive)."""
    rng = np.random.default_rng([seed, count, 4])
    names = ["schwefel", "rastrigin", "ackley", "rosenbrock"]
    out = []
    for _ in range(count):
        cost = names[int(rng.integers(0, 4))]
        n = int(rng.integers(n_range[0], n_range[1] + 1))
        chains = int(rng.integers(chain_range[0], chain_range[1] + 1))
        lo, hi = box(cost, n)
        out.append({"cost": cost, "n": n, "chains": chains, "lo": lo, "hi": hi})
    return out


# The workloads, by what they are.
SCHWEFEL_N2_FP64 = dict(cost="schwefel", n=2, chains=1024, L=100, levels=50, T0=100.0, rho=0.9,
                        sigma_frac=0.1, precision="fp64", seed=0)
SCHWEFEL_N256_FP32 = dict(cost="schwefel", n=256, chains=262144, L=1000, levels=200, T0=100.0, rho=0.95,
                          sigma_frac=0.1, precision="fp32", seed=0)
# Rotated costs: Q = rotation(n, q_seed).
ROT_RASTRIGIN_N1024 = dict(cost="rot_rastrigin", n=1024, chains=65536, L=500, levels=100, T0=100.0, rho=0.95,
                           sigma_frac=0.1, precision="fp32", seed=0, q_seed=0)
ROT_SCHWEFEL_N128 = dict(cost="rot_schwefel", n=128, chains=131072, L=2000, levels=150, T0=100.0, rho=0.95,
                         sigma_frac=0.1, precision="fp32", seed=0, q_seed=0)

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


# ------------------------------------------------------------ the Appendix suite
# Tables of the Appendix's Tests 11, 18 and 19, as printed: row i of A holds a_i,
# c holds c_i.  They are problem data (like the rotations above): the solver and
# the oracle both receive them as a table of rows (a_i1 .. a_in, c_i).
LANGERMAN_A = [
    [9.681, 0.667, 4.783, 9.095, 3.517, 9.325, 6.544, 0.211, 5.122, 2.020],
    [9.400, 2.041, 3.788, 7.931, 2.882, 2.672, 3.568, 1.284, 7.033, 7.374],
    [8.025, 9.152, 5.114, 7.621, 4.564, 4.711, 2.996, 6.126, 0.734, 4.982],
    [2.196, 0.415, 5.649, 6.979, 9.510, 9.166, 6.304, 6.054, 9.377, 1.426],
    [8.074, 8.777, 3.467, 1.863, 6.708, 6.349, 4.534, 0.276, 7.633, 1.567],
]
LANGERMAN_C = [0.806, 0.517, 0.100, 0.908, 0.965]

SHEKEL_A = [[4, 4, 4, 4], [1, 1, 1, 1], [8, 8, 8, 8], [6, 6, 6, 6], [3, 7, 3, 7],
            [2, 9, 2, 9], [5, 5, 3, 3], [8, 1, 8, 1], [6, 2, 6, 2], [7, 3.6, 7, 3.6]]
SHEKEL_C = [0.1, 0.2, 0.2, 0.4, 0.4, 0.6, 0.3, 0.7, 0.5, 0.5]

FOXHOLES_A = [
    [9.681, 0.667, 4.783, 9.095, 3.517, 9.325, 6.544, 0.211, 5.122, 2.020],
    [9.400, 2.041, 3.788, 7.931, 2.882, 2.672, 3.568, 1.284, 7.033, 7.374],
    [8.025, 9.152, 5.114, 7.621, 4.564, 4.711, 2.996, 6.126, 0.734, 4.982],
    [2.196, 0.415, 5.649, 6.979, 9.510, 9.166, 6.304, 6.054, 9.377, 1.426],
    [8.074, 8.777, 3.467, 1.863, 6.708, 6.349, 4.534, 0.276, 7.633, 1.567],
    [7.650, 5.658, 0.720, 2.764, 3.278, 5.283, 7.474, 6.274, 1.409, 8.208],
    [1.256, 3.605, 8.623, 6.905, 4.584, 8.133, 6.071, 6.888, 4.187, 5.448],
    [8.314, 2.261, 4.224, 1.781, 4.124, 0.932, 8.129, 8.658, 1.208, 5.762],
    [0.226, 8.858, 1.420, 0.945, 1.622, 4.698, 6.228, 9.096, 0.972, 7.637],
    [7.305, 2.228, 1.242, 5.928, 9.133, 1.826, 4.060, 5.204, 8.713, 8.247],
    [0.652, 7.027, 0.508, 4.876, 8.807, 4.632, 5.808, 6.937, 3.291, 7.016],
    [2.699, 3.516, 5.874, 4.119, 4.461, 7.496, 8.817, 0.690, 6.593, 9.789],
    [8.327, 3.897, 2.017, 9.570, 9.825, 1.150, 1.395, 3.885, 6.354, 0.109],
    [2.132, 7.006, 7.136, 2.641, 1.882, 5.943, 7.273, 7.691, 2.880, 0.564],
    [4.707, 5.579, 4.080, 0.581, 9.698, 8.542, 8.077, 8.515, 9.231, 4.670],
    [8.304, 7.559, 8.567, 0.322, 7.128, 8.392, 1.472, 8.524, 2.277, 7.826],
    [8.632, 4.409, 4.832, 5.768, 7.050, 6.715, 1.711, 4.323, 4.405, 4.591],
    [4.887, 9.112, 0.170, 8.967, 9.693, 9.867, 7.508, 7.770, 8.382, 6.740],
    [2.440, 6.686, 4.299, 1.007, 7.008, 1.427, 9.398, 8.480, 9.950, 1.675],
    [6.306, 8.583, 6.084, 1.138, 4.350, 3.134, 7.853, 6.061, 7.457, 2.258],
    [0.652, 2.343, 1.370, 0.821, 1.310, 1.063, 0.689, 8.819, 8.833, 9.070],
    [5.558, 1.272, 5.756, 9.857, 2.279, 2.764, 1.284, 1.677, 1.244, 1.234],
    [3.352, 7.549, 9.817, 9.437, 8.687, 4.167, 2.570, 6.540, 0.228, 0.027],
    [8.798, 0.880, 2.370, 0.168, 1.701, 3.680, 1.231, 2.390, 2.499, 0.064],
    [1.460, 8.057, 1.336, 7.217, 7.914, 3.615, 9.981, 9.198, 5.292, 1.224],
    [0.432, 8.645, 8.774, 0.249, 8.081, 7.461, 4.416, 0.652, 4.002, 4.644],
    [0.679, 2.800, 5.523, 3.049, 2.968, 7.225, 6.730, 4.199, 9.614, 9.229],
    [4.263, 1.074, 7.286, 5.599, 8.291, 5.200, 9.214, 8.272, 4.398, 4.506],
    [9.496, 4.830, 3.150, 8.270, 5.079, 1.231, 5.731, 9.494, 1.883, 9.732],
    [4.138, 2.562, 2.532, 9.661, 5.611, 5.500, 6.886, 2.341, 9.699, 6.500],
]
FOXHOLES_C = [0.806, 0.517, 0.100, 0.908, 0.965, 0.669, 0.524, 0.902, 0.531, 0.876,
              0.462, 0.491, 0.463, 0.714, 0.352, 0.869, 0.813, 0.811, 0.828, 0.964,
              0.789, 0.360, 0.369, 0.992, 0.332, 0.817, 0.632, 0.883, 0.608, 0.326]

TABLE_COSTS = ("langerman", "shekel", "foxholes")


def table(cost: str, n: int, m: int | None = None) -> np.ndarray:
    """Rows (a_i1 .. a_in, c_i) of Test 11, 18 or 19 for n coordinates (the first n
    columns of A); Shekel takes its first m rows (m = 5, 7 or 10)."""
    A, c = {"langerman": (LANGERMAN_A, LANGERMAN_C), "shekel": (SHEKEL_A, SHEKEL_C),
            "foxholes": (FOXHOLES_A, FOXHOLES_C)}[cost]
    A, c = np.asarray(A, np.float64), np.asarray(c, np.float64)
    rows = A.shape[0] if m is None else m
    if n > A.shape[1] or rows > A.shape[0]:
        raise ValueError(f"{cost}: the table has {A.shape[0]} rows of {A.shape[1]} coordinates")
    return np.ascontiguousarray(np.concatenate([A[:rows, :n], c[:rows, None]], axis=1))


# The 41 problems of the paper's test suite (the table of test functions and
# dimensions in Sec. 4.2), with the Appendix's boxes and printed minima.
# (name, cost, n, lower, upper, f*, Shekel m); a box side may be per coordinate.
_SUITE = [
    *[(f"F0_{s}", "schwefel", n, -512.0, 512.0, -418.982887, None)
      for s, n in zip("abcdefg", (8, 16, 32, 64, 128, 256, 512))],
    *[(f"F1_{s}", "ackley", n, -30.0, 30.0, 0.0, None) for s, n in zip("abcd", (30, 100, 200, 400))],
    ("F2", "branin", 2, -20.0, 20.0, 0.397887, None),
    ("F3_a", "cosine_mixture", 2, -1.0, 1.0, -0.2, None),
    ("F3_b", "cosine_mixture", 4, -1.0, 1.0, -0.4, None),
    ("F4", "dekkers_aarts", 2, -20.0, 20.0, -24776.518, None),
    ("F5", "easom", 2, -10.0, 10.0, -1.0, None),
    ("F6", "exponential", 4, -1.0, 1.0, -1.0, None),
    ("F7", "goldstein_price", 2, -2.0, 2.0, 3.0, None),
    *[(f"F8_{s}", "griewank", n, -600.0, 600.0, 0.0, None) for s, n in zip("abc", (100, 200, 400))],
    ("F9", "himmelblau", 2, -6.0, 6.0, 0.0, None),
    *[(f"F10_{s}", "levy_montalvo", n, -10.0, 10.0, 0.0, None) for s, n in zip("abc", (2, 5, 10))],
    ("F11_a", "langerman", 2, 0.0, 10.0, -1.080938, None),
    ("F11_b", "langerman", 5, 0.0, 10.0, -0.964999, None),
    ("F12_a", "michalewicz", 2, 0.0, np.pi, -1.8013, None),
    ("F12_b", "michalewicz", 5, 0.0, np.pi, -4.6877, None),
    ("F12_c", "michalewicz", 10, 0.0, np.pi, -9.6602, None),
    ("F13_a", "rastrigin", 100, -5.12, 5.12, 0.0, None),
    ("F13_b", "rastrigin", 400, -5.12, 5.12, 0.0, None),
    ("F14", "rosenbrock", 4, -2.048, 2.048, 0.0, None),
    ("F15", "salomon", 10, -100.0, 100.0, 0.0, None),
    ("F16", "six_hump_camel", 2, [-3.0, -2.0], [3.0, 2.0], -1.0316, None),
    ("F17", "shubert", 2, -10.0, 10.0, -186.7309, None),
    ("F18_a", "shekel", 4, 0.0, 10.0, -10.1532, 5),
    ("F18_b", "shekel", 4, 0.0, 10.0, -10.4029, 7),
    ("F18_c", "shekel", 4, 0.0, 10.0, -10.5364, 10),
    ("F19_a", "foxholes", 2, -5.0, 15.0, -12.1190, None),
    ("F19_b", "foxholes", 5, -5.0, 15.0, -10.4056, None),
]


def appendix_suite():
    """The 41 problems: dicts with name, cost, n, lo, hi (arrays), f_star and table (or None)."""
    out = []
    for name, cost, n, lo, hi, fs, m in _SUITE:
        lo_a = np.ascontiguousarray(np.broadcast_to(np.asarray(lo, np.float64), (n,)))
        hi_a = np.ascontiguousarray(np.broadcast_to(np.asarray(hi, np.float64), (n,)))
        tab = table(cost, n, m) if cost in TABLE_COSTS else None
        out.append({"name": name, "cost": cost, "n": n, "lo": lo_a, "hi": hi_a, "f_star": fs, "table": tab})
    return out

"""GPU parity of the hybrid SA's Nelder-Mead (Sec. 4.2, Table 10) with the oracle's.

The kernel and the oracle take the same steps in the same order; they differ
only in rounding (f summed over threads, CUDA's math library, the centroid from
a running vertex sum), so a fixed number of iterations lands on the same vertex
up to that rounding, and a converged run on the same local minimum.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2408_00018_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sa():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2408_00018_gb300 import sa as sa_mod
    return sa_mod


CENTRE = {"schwefel": 420.97, "rastrigin": 0.0, "ackley": 0.0, "rosenbrock": 1.0, "rot_schwefel": 100.0,
          "rot_rastrigin": 0.0}

CASES = [("schwefel", 4, 40.0, 0.05), ("rastrigin", 3, 0.3, 0.01), ("rosenbrock", 2, 0.8, 0.05),
         ("ackley", 5, 0.5, 0.02), ("schwefel", 40, 20.0, 0.02), ("rot_rastrigin", 6, 0.3, 0.01),
         ("rot_schwefel", 8, 40.0, 0.05), ("rastrigin", 1, 0.3, 0.01)]


def _starts(cost, n, spread, k, seed):
    rng = np.random.default_rng(seed)
    lo, hi = inputs.box(cost, n)
    x0 = np.clip(CENTRE[cost] + spread * rng.standard_normal((k, n)), lo, hi)
    x0[-1] = lo + 0.25 * (hi - lo)  # a start far from the minimum
    return lo, hi, x0


def _q(cost, n):
    return inputs.rotation(n, 4) if cost.startswith("rot_") else None


@pytest.mark.parametrize("cost,n,spread,step", CASES)
@pytest.mark.parametrize("iters", [7, 60])
@pytest.mark.parametrize("adaptive", [False, True])
def test_fixed_iterations_match_oracle(sa, cost, n, spread, step, iters, adaptive):
    """ftol = xtol = 0: both run exactly `iters` iterations through the same branches
    (standard coefficients, and Gao & Han's adaptive ones)."""
    if adaptive and n == 1:
        pytest.skip("the adaptive shrink is 1 - 1/n = 0 at n = 1: the simplex collapses onto one point, at an "
                    "iteration the last rounding of f decides")
    k = 12
    lo, hi, x0 = _starts(cost, n, spread, k, seed=n + iters)
    Q = _q(cost, n)
    xg, fg, itg = sa.nelder_mead(cost, x0, lo, hi, step_frac=step, max_iter=iters, ftol=0.0, xtol=0.0, Q=Q,
                                 adaptive=adaptive)
    for j in range(k):
        xo, fo, ito = oracle.nelder_mead(cost, x0[j], lo, hi, Q=Q, step_frac=step, max_iter=iters, ftol=0.0, xtol=0.0,
                                         adaptive=adaptive)
        assert itg[j] == ito == iters
        if j == k - 1:
            # every coordinate of this start is equal: on a cost symmetric under permuting the
            # coordinates the simplex's values tie exactly, the rounding of f breaks the ties,
            # and the two may reach the same point with its coordinates permuted
            xg_j, xo_j = np.sort(xg[j]), np.sort(xo)
        else:
            xg_j, xo_j = xg[j], xo
        assert np.allclose(xg_j, xo_j, rtol=0, atol=1e-9 * (hi - lo).max()), (j, xg[j], xo)
        assert abs(fg[j] - fo) <= 1e-12 * max(1.0, abs(fo)), (j, fg[j], fo)


@pytest.mark.parametrize("cost,n,spread,step,iters", [
    ("rastrigin", 400, 0.3, 0.01, 150),    # the Table 10 sizes: 400 coordinates on 416 threads
    ("schwefel", 1500, 20.0, 0.02, 40),    # more coordinates than threads (1024)
    ("rot_schwefel", 96, 40.0, 0.05, 300),  # past the running sum's first afresh re-sum (every n + 1)
    ("ackley", 33, 0.5, 0.02, 500),        # two warps, one of them nearly idle
])
@pytest.mark.parametrize("adaptive", [False, True])
def test_fixed_iterations_match_oracle_at_large_n(sa, cost, n, spread, step, iters, adaptive):
    k = 3
    lo, hi, x0 = _starts(cost, n, spread, k, seed=n)
    Q = _q(cost, n)
    xg, fg, itg = sa.nelder_mead(cost, x0, lo, hi, step_frac=step, max_iter=iters, ftol=0.0, xtol=0.0, Q=Q,
                                 adaptive=adaptive)
    for j in range(k):
        xo, fo, ito = oracle.nelder_mead(cost, x0[j], lo, hi, Q=Q, step_frac=step, max_iter=iters, ftol=0.0, xtol=0.0,
                                         adaptive=adaptive)
        assert itg[j] == ito == iters
        assert np.allclose(xg[j], xo, rtol=0, atol=1e-9 * (hi - lo).max()), (j, np.abs(xg[j] - xo).max())
        assert abs(fg[j] - fo) <= 1e-11 * max(1.0, abs(fo)), (j, fg[j], fo)


@pytest.mark.parametrize("cost,n,spread,step", CASES)
def test_converged_runs_match_oracle(sa, cost, n, spread, step):
    k = 12
    lo, hi, x0 = _starts(cost, n, spread, k, seed=3 * n)
    Q = _q(cost, n)
    xg, fg, itg = sa.nelder_mead(cost, x0, lo, hi, step_frac=step, max_iter=200 * (n + 1), Q=Q)
    for j in range(k):
        xo, fo, ito = oracle.nelder_mead(cost, x0[j], lo, hi, Q=Q, step_frac=step, max_iter=200 * (n + 1))
        assert abs(fg[j] - fo) <= 1e-9 * max(1.0, abs(fo)), (j, fg[j], fo, itg[j], ito)
        assert abs(oracle.cost(cost, xg[j], Q) - fg[j]) <= 1e-12 * max(1.0, abs(fg[j]))
        assert (xg[j] >= lo).all() and (xg[j] <= hi).all()
        assert fg[j] <= oracle.cost(cost, x0[j], Q) + 1e-12 * max(1.0, abs(fg[j]))


def test_zero_iterations_return_the_best_initial_vertex(sa):
    lo, hi, x0 = _starts("schwefel", 6, 50.0, 5, seed=1)
    xg, fg, itg = sa.nelder_mead("schwefel", x0, lo, hi, step_frac=0.05, max_iter=0)
    for j in range(5):
        xo, fo, ito = oracle.nelder_mead("schwefel", x0[j], lo, hi, step_frac=0.05, max_iter=0)
        assert itg[j] == 0 and np.array_equal(xg[j], xo) and abs(fg[j] - fo) <= 1e-13 * abs(fo)


def test_rejects_bad_arguments(sa):
    lo, hi = np.full(3, -5.12), np.full(3, 5.12)
    x0 = np.zeros((1, 3))
    for kw in (dict(step_frac=0.0), dict(step_frac=1.5), dict(ftol=-1.0), dict(xtol=float("nan")),
               dict(max_iter=-1)):
        with pytest.raises(RuntimeError):
            sa.nelder_mead("rastrigin", x0, lo, hi, **kw)
    with pytest.raises(RuntimeError):
        sa.nelder_mead("rastrigin", np.zeros((1025, 3)), lo, hi)
    with pytest.raises(RuntimeError):
        sa.nelder_mead("rot_rastrigin", x0, lo, hi)  # Q missing
    with pytest.raises(RuntimeError):
        sa.nelder_mead("rastrigin", x0, lo, hi, Q=np.eye(3))  # Q given to a separable cost
    with pytest.raises(RuntimeError):
        sa.nelder_mead("rastrigin", x0, hi, lo)  # empty box
    with pytest.raises(RuntimeError):
        sa.nelder_mead("rastrigin", np.zeros((1, 4097)), -5.12, 5.12)  # above the 4096 coordinates of a block


@pytest.mark.parametrize("cost,n,method", [("schwefel", 8, "nelder_mead"), ("rot_schwefel", 6, "nelder_mead"),
                                           ("schwefel", 8, "nelder_mead_adaptive")])
def test_hybrid_run_polishes_with_nelder_mead(sa, cost, n, method):
    """Hybrid SA with Nelder-Mead on the best final state (polish_k = 1): the
    incumbent is the lower of the annealing's incumbent and the oracle's
    Nelder-Mead from the last level's best state, started with the last level's
    step scale."""
    C, L, K, T0, rho, sf = 256, 60, 6, 100.0, 0.8, 0.1
    lo, hi = inputs.box(cost, n)
    Q = _q(cost, n)
    kw = dict(Q=Q) if Q is not None else {}
    prec = "fp32" if Q is not None else "fp64"  # rotated costs run the FP32 rank-1 sweep
    base = sa.Schedule(T0=T0, rho=rho, levels=K, sigma_frac=sf, precision=prec)
    with sa.create(cost, lo, hi, n, C, L, base, seed=5, **kw) as h:
        h.run()
        x_a, f_a, _ = h.best()
        x_last, f_last = h.restart_point()
    hyb = sa.Schedule(T0=T0, rho=rho, levels=K, sigma_frac=sf, precision=prec, polish_k=1,
                      polish_method=method)
    with sa.create(cost, lo, hi, n, C, L, hyb, seed=5, **kw) as h:
        h.run()
        x_b, f_b, _ = h.best()
    T = T0
    for _ in range(K - 1):
        T = T * rho
    step = min(1.0, sf * math.sqrt(T / T0))
    x_o, f_o, _ = oracle.nelder_mead(cost, x_last, lo, hi, Q=Q, step_frac=step, max_iter=200 * (n + 1),
                                     ftol=1e-12, xtol=1e-10, adaptive=method.endswith("adaptive"))
    assert f_o <= f_last
    if f_o < f_a:
        assert abs(f_b - f_o) <= 1e-9 * abs(f_o), (f_b, f_o, f_a)
        assert abs(oracle.cost(cost, x_b, Q) - f_b) <= 1e-12 * abs(f_b)
    else:
        assert f_b == f_a and np.array_equal(x_b, x_a)

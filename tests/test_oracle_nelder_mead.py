"""Pins of the oracle's Nelder-Mead, the local minimiser of the paper's hybrid SA
(Sec. 4.2, Table 10).

The oracle follows the standard method (Lagarias, Reeds, Wright & Wright 1998):
reflection 1, expansion 2, contraction 1/2, shrink 1/2, trial points clipped
into the box.  It is pinned against scipy's independent implementation of the
same method (same coefficients, same initial simplex, same clipping), against
the textbook Rosenbrock run, and against the closed-form minima of the costs.
"""
import numpy as np
import pytest

import oracle


def _simplex(x0, lo, hi, step_frac):
    """The initial simplex the oracle builds: x0 and x0 +- step_frac (u_k - l_k) e_k."""
    n = x0.size
    S = np.tile(np.clip(x0, lo, hi), (n + 1, 1))
    for k in range(n):
        d = step_frac * (hi[k] - lo[k])
        S[k + 1, k] = S[k + 1, k] + d if S[k + 1, k] + d <= hi[k] else S[k + 1, k] - d
    return np.clip(S, lo, hi)


@pytest.mark.parametrize("cost,n,lo,hi,x0,iters", [
    ("rosenbrock", 2, -5.0, 10.0, [-1.2, 1.0], 40),
    ("schwefel", 4, -500.0, 500.0, [380.0, 400.0, 430.0, 410.0], 60),
    ("rastrigin", 3, 0.6, 5.0, [0.7, 0.9, 1.3], 50),  # clipping at the face x = 0.6 is active
    ("ackley", 5, -32.768, 32.768, [0.5, -0.3, 0.2, 0.1, -0.4], 80),
])
@pytest.mark.parametrize("adaptive", [False, True])
def test_matches_scipy_nelder_mead_iteration_for_iteration(cost, n, lo, hi, x0, iters, adaptive):
    """Standard coefficients, and Gao & Han's adaptive ones (scipy's adaptive=True)."""
    scipy_opt = pytest.importorskip("scipy.optimize")
    lo_v, hi_v = np.full(n, lo), np.full(n, hi)
    x0 = np.array(x0, np.float64)
    step = 0.05
    f = lambda x: oracle.cost(cost, np.asarray(x, np.float64))  # noqa: E731
    ref = scipy_opt.minimize(f, x0, method="Nelder-Mead", bounds=list(zip(lo_v, hi_v)),
                             # scipy's iteration counter starts at 1: maxiter = iters + 1 runs `iters` iterations
                             options=dict(initial_simplex=_simplex(x0, lo_v, hi_v, step), maxiter=iters + 1,
                                          xatol=0.0, fatol=0.0, adaptive=adaptive))
    x, fx, it = oracle.nelder_mead(cost, x0, lo_v, hi_v, step_frac=step, max_iter=iters, ftol=-1.0, adaptive=adaptive)
    assert it == iters
    # the two differ only in rounding: the centroid's summation order (sorted vs slot order)
    # and the trial points' form ((1 + a) c - a v_h there, c + a (c - v_h) here)
    assert np.allclose(x, ref.x, rtol=1e-9, atol=1e-9 * (hi - lo)), (x, ref.x)
    assert abs(fx - ref.fun) <= 1e-9 * max(1.0, abs(ref.fun))


def test_rosenbrock_textbook_start_converges_to_the_minimum():
    x, f, it = oracle.nelder_mead("rosenbrock", [-1.2, 1.0], [-5.0, -5.0], [10.0, 10.0], ftol=1e-16)
    assert f < 1e-12 and np.allclose(x, 1.0, atol=1e-5)
    assert 0 < it < 1000


def test_closed_form_minima():
    xs = 420.968746359982  # the Schwefel term's stationary point: t = r^2 with tan r = -r/2
    x, f, _ = oracle.nelder_mead("schwefel", np.full(4, 405.0), -500, 500, ftol=1e-15)
    assert np.allclose(x, xs, atol=1e-4)
    assert abs(f - oracle.cost("schwefel", np.full(4, xs))) < 1e-10
    # a simplex of 1% of the box stays in the basin of 0 (5% reaches the next one)
    x, f, _ = oracle.nelder_mead("rastrigin", [0.3, -0.2, 0.1], -5.12, 5.12, step_frac=0.01, ftol=1e-15)
    assert f < 1e-9 and np.abs(x).max() < 1e-5
    # n = 1 (a line search); its two vertices straddle 0 with equal f before they are close in x
    x, f, _ = oracle.nelder_mead("rastrigin", [0.3], -5.12, 5.12, step_frac=0.01, ftol=1e-15)
    assert f < 1e-9 and abs(x[0]) < 1e-5


def test_box_is_respected_and_f_never_rises():
    rng = np.random.default_rng(3)
    for cost, lo, hi in [("schwefel", -500.0, 500.0), ("rastrigin", -5.12, 5.12), ("rosenbrock", -2.0, 2.0)]:
        for _ in range(5):
            n = int(rng.integers(1, 7))
            x0 = rng.uniform(lo, hi, n)
            x, f, it = oracle.nelder_mead(cost, x0, lo, hi, max_iter=300)
            assert np.all(x >= lo) and np.all(x <= hi) and it <= 300
            assert f <= oracle.cost(cost, x0) and f == oracle.cost(cost, x)


def test_zero_iterations_return_the_best_initial_vertex():
    lo, hi = np.full(3, -500.0), np.full(3, 500.0)
    x0 = np.array([100.0, -200.0, 300.0])
    S = _simplex(x0, lo, hi, 0.05)
    F = [oracle.cost("schwefel", v) for v in S]
    x, f, it = oracle.nelder_mead("schwefel", x0, lo, hi, step_frac=0.05, max_iter=0)
    assert it == 0 and f == min(F) and np.array_equal(x, S[int(np.argmin(F))])


def test_rotated_with_identity_equals_unrotated():
    rng = np.random.default_rng(5)
    n = 5
    lo, hi = np.full(n, -5.12), np.full(n, 5.12)
    x0 = rng.uniform(-1.0, 1.0, n)
    a = oracle.nelder_mead("rot_rastrigin", x0, lo, hi, Q=np.eye(n), max_iter=400)
    b = oracle.nelder_mead("rastrigin", x0, lo, hi, max_iter=400)
    assert a[1] == b[1] and np.array_equal(a[0], b[0]) and a[2] == b[2]

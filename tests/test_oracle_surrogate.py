"""Pins of the FP64 surrogate oracle (MLP, Adam) and of the oracle's delayed
acceptance, against closed forms, finite differences and the Boltzmann law."""
import math

import numpy as np
import pytest

import oracle
from oracle import surrogate as S


def test_gelu_closed_forms():
    assert S.gelu(0.0) == 0.0
    # GELU(1) = Phi(1), the standard normal CDF at 1
    assert abs(float(S.gelu(1.0)) - 0.8413447460685429) < 1e-15
    z = np.linspace(-6, 6, 101)
    # z Phi(z) - (-z) Phi(-z) = z (Phi(z) + Phi(-z) = 1)
    assert np.allclose(S.gelu(z) - S.gelu(-z), z, atol=1e-14, rtol=0)
    assert abs(float(S.gelu_grad(0.0)) - 0.5) < 1e-15
    h = 1e-6
    fd = (S.gelu(z + h) - S.gelu(z - h)) / (2 * h)
    assert np.allclose(S.gelu_grad(z), fd, atol=1e-8, rtol=0)


def test_mlp_gradient_matches_central_differences():
    n, B = 5, 7
    rng = np.random.default_rng(3)
    p = S.init_params(n, seed=1)
    p[S.n_params(n) - 1] = 0.3  # non-zero b3
    X = rng.uniform(-1, 1, (B, n))
    t = rng.standard_normal(B)
    loss, g = S.loss_and_grad(p, X, t, n)
    # coordinates from every block: W1, b1, W2, b2, w3, b3
    W1n = S.H1 * n
    starts = [0, W1n, W1n + S.H1, W1n + S.H1 + S.H2 * S.H1, W1n + S.H1 + S.H2 * S.H1 + S.H2,
              S.n_params(n) - 1]
    idx = sorted(set(min(s + int(k), S.n_params(n) - 1) for s in starts for k in rng.integers(0, 5, 4)))
    h = 1e-5
    for i in idx:
        e = np.zeros_like(p)
        e[i] = h
        fd = (S.loss_and_grad(p + e, X, t, n)[0] - S.loss_and_grad(p - e, X, t, n)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1e-3, abs(g[i])), (i, fd, g[i])


def test_mlp_with_zero_hidden_weights_is_constant():
    n = 4
    p = S.init_params(n, seed=2)
    W1, b1, W2, b2, w3, b3 = S.unpack(p, n)
    W2[:] = 0.0
    b2[:] = np.linspace(-2, 2, S.H2)
    b3[:] = -0.7
    X = np.random.default_rng(0).uniform(-3, 3, (9, n))
    y, _ = S.forward(p, X, n)
    expect = float(w3 @ S.gelu(b2)) - 0.7
    assert np.allclose(y, expect, atol=1e-12, rtol=0)


def test_adam_first_step_and_convergence():
    rng = np.random.default_rng(4)
    p0 = rng.standard_normal(10)
    g = rng.standard_normal(10)
    p1, m, v = S.adam_step(p0, g, np.zeros(10), np.zeros(10), 1, lr=0.01)
    # bias correction makes the first step lr g / (|g| + eps)
    assert np.allclose(p1, p0 - 0.01 * g / (np.abs(g) + 1e-8), atol=1e-15, rtol=0)
    # minimises a convex quadratic
    target = rng.standard_normal(10)
    p, m, v = p0.copy(), np.zeros(10), np.zeros(10)
    for k in range(1, 3001):
        p, m, v = S.adam_step(p, p - target, m, v, k, lr=0.01)
    assert np.abs(p - target).max() < 1e-3


# ------------------------------------------------------------------ delayed acceptance
@pytest.mark.parametrize("cost,n", [("schwefel", 4), ("rastrigin", 6), ("ackley", 3), ("rot_rastrigin", 5)])
def test_da_with_constant_surrogate_is_plain_metropolis(cost, n):
    from paper_2408_00018_gb300 import inputs
    lo, hi = inputs.box(cost, n)
    Q = inputs.rotation(n, 1) if cost.startswith("rot") else None
    p = oracle.Problem(cost, n, lo, hi, chains=16, L=150, T0=20.0, rho=0.9, seed=8, Q=Q, mode=1)
    for c in range(16):
        F, x, acc, bits = p.chain_level(0, c, trace=True)
        F2, x2, b2, a2, ev = p.da_chain_level(0, c, 1.5, np.full(150, 1.5))
        assert np.array_equal(bits, b2) and F == F2 and np.array_equal(x, x2) and a2 == acc and ev == 150


def test_da_with_perfect_surrogate_accepts_every_evaluated_move():
    from paper_2408_00018_gb300 import inputs
    lo, hi = inputs.box("rastrigin", 3)
    p = oracle.Problem("rastrigin", 3, lo, hi, chains=32, L=300, T0=5.0, rho=0.9, seed=9, mode=1)
    total_ev = 0
    for c in range(32):
        F, x, bits, acc, ev = p.da_chain_level_fn(0, c, 1.0, 0.0)
        assert acc == ev  # stage 2's ratio is exp(0): every survivor of stage 1 is accepted
        total_ev += ev
    assert total_ev < 32 * 300  # stage 1 rejected some moves without a true evaluation


def test_da_with_wrong_surrogate_still_samples_boltzmann():
    # Stage 2 corrects any surrogate: with f~ = 0.5 f + 3 sin(x) the level-0 states
    # at fixed T must still follow exp(-f/T) (detailed balance of the two stages).
    T = 10.0
    C, L = 20000, 200
    p = oracle.Problem("rastrigin", 1, -5.12, 5.12, chains=C, L=L, T0=T, rho=0.9, seed=5, mode=1)
    xs = np.empty(C)
    ev_total = 0
    for c in range(C):
        _, x, _, _, ev = p.da_chain_level_fn(0, c, 0.5, 3.0)
        xs[c] = x[0]
        ev_total += ev
    f = lambda t: t * t - 10 * np.cos(2 * np.pi * t) + 10
    edges = np.linspace(-5.12, 5.12, 41)
    obs, _ = np.histogram(xs, edges)
    t = np.linspace(-5.12, 5.12, 20001)
    w = np.exp(-(f(t) - f(t).min()) / T)
    dens = w / np.trapezoid(w, t)
    cdf = np.concatenate([[0], np.cumsum((dens[1:] + dens[:-1]) / 2 * np.diff(t))])
    exp_ = np.diff(np.interp(edges, t, cdf)) * C
    chi2 = float(((obs - exp_) ** 2 / exp_).sum())
    assert chi2 < 80.0, chi2
    assert ev_total < C * L


def test_propose_step_is_the_chains_own_move():
    """propose_step gives the move (d, x'_d) the chain itself makes at step s: applying
    it wherever the traced chain accepted reproduces the chain's final state exactly
    (the temperature scaling of the step and the counters are the chain's)."""
    from paper_2408_00018_gb300 import inputs
    n, L = 5, 300
    lo, hi = inputs.box("schwefel", n)
    p = oracle.Problem("schwefel", n, lo, hi, chains=4, L=L, T0=50.0, rho=0.7, seed=9, mode=1)
    for level, c in ((0, 1), (3, 2)):
        x0 = p.init_point(c)
        _, x_end, _, bits = p.chain_level(level, c, x0, trace=True)
        acc = np.unpackbits(bits.view(np.uint8), bitorder="little")[:L].astype(bool)
        x = x0.copy()
        for s in range(L):
            d, xp = p.propose_step(level, c, s, x)
            if acc[s]:
                x[d] = xp
        assert np.array_equal(x, x_end)


def test_da_trace_equals_steps_and_plant_changes_decisions():
    """The traced delayed-acceptance replay returns the same bits and differences as
    the untraced one, tau = -T ln u3 where stage 1 passed (NaN elsewhere), and the
    planted stage-2 sign error (a hook for the GPU parity tests' own tests) changes
    the decisions of a chain with a non-constant surrogate."""
    from paper_2408_00018_gb300 import inputs
    n, L = 6, 200
    lo, hi = inputs.box("rot_schwefel", n)
    Q = inputs.rotation(n, 1)
    p = oracle.Problem("rot_schwefel", n, lo, hi, chains=3, L=L, T0=5.0, rho=0.8, seed=2, Q=Q, mode=1)
    rng = np.random.default_rng(0)
    ftp = rng.standard_normal(L) * 3.0
    x0 = p.init_point(0)
    F1, x1, b1, a1, e1, dF1 = p.da_chain_level_steps(0, 0, 0.5, ftp, x0)
    F2, x2, b2, a2, e2, dF2, tau = p.da_chain_level_trace(0, 0, 0.5, ftp, x0)
    assert F1 == F2 and np.array_equal(x1, x2) and np.array_equal(b1, b2) and (a1, e1) == (a2, e2)
    assert np.array_equal(np.isnan(dF1), np.isnan(dF2)) and np.array_equal(dF1[~np.isnan(dF1)], dF2[~np.isnan(dF2)])
    assert np.array_equal(np.isnan(tau), np.isnan(dF2))
    key = oracle.stream_key(2, 0)
    for s in np.nonzero(~np.isnan(tau))[0][:20]:
        w = oracle.philox([s, 0, 0, 0], key)
        assert abs(tau[s] + 5.0 * np.log(oracle.uniform(w[3]))) <= 1e-14 * abs(tau[s])
    _, _, b3, _, _, _, _ = p.da_chain_level_trace(0, 0, 0.5, ftp, x0, plant=1)
    assert not np.array_equal(b3, b2)

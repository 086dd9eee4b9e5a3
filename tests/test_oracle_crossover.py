"""Pins of the oracle's stochastic crossover (a reading of the SOS scheme cited in
Sec. 2.2: at an exchange each chain restarts from a chain drawn with Boltzmann
weights exp(-(F_j - F_min) / T) instead of from the minimum)."""
import numpy as np
from scipy import stats

import oracle


def _problem(**kw):
    args = dict(chains=64, L=40, T0=20.0, rho=0.8, seed=5, crossover=True)
    args.update(kw)
    return oracle.Problem("schwefel", 4, -500.0, 500.0, **args)


def test_draw_follows_the_boltzmann_weights():
    """20000 chains over 5 distinct values: the counts of each value's chains match
    exp(-(F - F_min) / T) normalised (chi-square), at two temperatures."""
    C = 20000
    F = np.repeat([0.0, 0.5, 1.0, 2.0, 4.0], C // 5)
    for level, T0 in ((0, 1.0), (3, 2.0)):
        p = _problem(chains=C, T0=T0, rho=0.5)
        T = oracle.temperature(T0, 0.5, level)
        src = p.crossover_sources(level, F)
        counts = np.bincount((src // (C // 5)).astype(int), minlength=5)
        w = np.exp(-(np.array([0.0, 0.5, 1.0, 2.0, 4.0]) - 0.0) / T)
        expect = C * w / w.sum()
        keep = expect > 5
        assert stats.chisquare(counts[keep], expect[keep] * counts[keep].sum() / expect[keep].sum()).pvalue > 1e-3


def test_draw_is_the_first_crossing_of_the_running_sum():
    """Brute force on a few chains: src[c] is the first j whose running sum of weights
    exceeds u_c times the total, u_c from word 0 of Philox (0, level, c, 0), tag 5."""
    rng = np.random.default_rng(1)
    C, level, T0, rho, seed = 37, 2, 3.0, 0.9, 11
    F = rng.normal(0.0, 2.0, C)
    F[5] = np.inf
    p = _problem(chains=C, T0=T0, rho=rho, seed=seed)
    src = p.crossover_sources(level, F)
    T = oracle.temperature(T0, rho, level)
    Fmin = F[np.isfinite(F)].min()
    S = np.cumsum([np.exp(-(f - Fmin) / T) if np.isfinite(f) else 0.0 for f in F])
    key = oracle.stream_key(seed, 5)
    for c in range(C):
        t = oracle.uniform(oracle.philox([0, level, c, 0], key)[0]) * S[-1]
        assert src[c] == int(np.nonzero(S > t)[0][0])
        assert src[c] != 5  # a non-finite value is never drawn


def test_zero_temperature_limit_is_the_minimum():
    """At a temperature far below every difference of F, each chain draws the minimum,
    and the run equals the synchronous run (every exchange from the minimum) bit for bit."""
    a = _problem(T0=1e-300, rho=0.5, crossover=True).run(4, trace_levels=4)
    b = _problem(T0=1e-300, rho=0.5, crossover=False).run(4, trace_levels=4)
    assert np.array_equal(a["argmin"], b["argmin"]) and np.array_equal(a["bits"], b["bits"])
    assert a["f_inc"] == b["f_inc"]
    assert (a["xo_src"][:3] == a["argmin"][:3, None]).all()


def test_infinite_temperature_draws_uniformly():
    C = 30000
    F = np.linspace(0.0, 10.0, C)
    src = _problem(chains=C, T0=1e300, rho=0.5).crossover_sources(0, F)
    assert stats.kstest(src / C, "uniform").pvalue > 1e-3


def test_run_bookkeeping_and_periodic_exchange():
    r = _problem(chains=200).run(5, want_final=True)
    assert r["xo_src"].shape == (5, 200) and (r["xo_src"][:4] >= 0).all() and (r["xo_src"][4] == -1).all()
    assert r["f_inc"] == r["f_level"].min()
    # with exchange_every = 2 the draw follows only levels 1 and 3 (exchanges before levels 2 and 4)
    q = _problem(chains=100, exchange_every=2).run(5)
    assert (q["xo_src"][[0, 2, 4]] == -1).all() and (q["xo_src"][[1, 3]] >= 0).all()

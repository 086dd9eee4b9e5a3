"""Delayed acceptance with the learned surrogate on the GPU, against the oracle.

The GPU records the surrogate's value at every chain's start state and at
every proposal; the oracle replays the two-stage acceptance with exactly those
values (a table surrogate) from the same FP32 start states.  Stage 1 then
decides identically; stage 2 may differ only at near-ties of the true
difference, as for the plain rotated path.  Further tests show what the
trained network gains: it predicts the true differences better than the
untrained one, and it saves true evaluations against plain Metropolis.
"""
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


def _bits_to_bool(bits, L):
    return np.unpackbits(np.ascontiguousarray(bits).view(np.uint8), axis=-1, bitorder="little")[..., :L].astype(bool)


def _create(sa, cost, n, C, L, K, T0, rho, seed, Q, trace_levels=0, surrogate=1, cost_repeat=1):
    lo, hi = inputs.box(cost, n)
    sch = sa.Schedule(T0=T0, rho=rho, levels=K, sigma_frac=0.1, precision="fp32", trace_levels=trace_levels,
                      surrogate=surrogate, cost_repeat=cost_repeat)
    return sa.create(cost, lo, hi, n, C, L, sch, seed=seed, Q=Q)


@pytest.mark.parametrize("cost,n,C,box", [("rot_schwefel", 64, 256, "uniform"), ("rot_rastrigin", 40, 130, "uniform"),
                                          ("rot_schwefel", 24, 70, "per-coordinate")])
def test_da_decisions_match_oracle_replay(sa, cost, n, C, box):
    L, K, T0, rho, seed = 150, 3, 30.0, 0.6, 4
    Q = inputs.rotation(n, 2)
    lo, hi = inputs.box(cost, n)
    if box != "uniform":
        lo, hi = lo * np.linspace(0.4, 1.0, n), hi * np.linspace(1.0, 0.6, n)
    sch = sa.Schedule(T0=T0, rho=rho, levels=K, sigma_frac=0.1, precision="fp32", trace_levels=K, surrogate=1)
    h = sa.create(cost, lo, hi, n, C, L, sch, seed=seed, Q=Q)
    p = oracle.Problem(cost, n, lo, hi, chains=C, L=L, T0=T0, rho=rho, seed=seed, Q=Q, mode=1)
    start = lambda c: p.init_point(c).astype(np.float32).astype(np.float64)
    total_full = total = 0
    for level in range(K):
        h.run(1)
        X, F = h.trace_states(level)
        bits = _bits_to_bool(h.trace(level), L)
        ft0, ftp = h.da_trace(level)
        for c in range(C):
            Fo, xo, ob, acc, ev = p.da_chain_level(level, c, float(ft0[c]), ftp[:, c].astype(np.float64), start(c))
            ob = _bits_to_bool(ob, L)
            total += 1
            total_full += int(np.array_equal(ob, bits[c]))
            fx = oracle.cost(cost, X[c], Q)
            assert abs(F[c] - fx) <= 1e-9 * max(1.0, abs(fx)), (level, c)
        pstar = int(h.level_log()["argmin"][level])
        assert pstar == int(np.argmin(F))
        x_restart = X[pstar].copy()
        start = lambda c, xr=x_restart: xr
    assert total_full >= 0.9 * total, (total_full, total)
    _, f, st = h.best()
    assert 0 < st["true_evals"] <= st["steps"] and st["accepts"] <= st["true_evals"]


def test_trained_surrogate_predicts_true_differences(sa):
    """At level 0 the network is untrained; after a few levels of online training
    its predicted differences f~(x') - f~(x) correlate with the true ones."""
    cost, n, C, L, K = "rot_schwefel", 32, 1024, 100, 6
    Q = inputs.rotation(n, 3)
    h = _create(sa, cost, n, C, L, K, 40.0, 0.8, 1, Q, trace_levels=K)
    lo, hi = inputs.box(cost, n)
    p = oracle.Problem(cost, n, lo, hi, chains=C, L=L, T0=40.0, rho=0.8, seed=1, Q=Q, mode=1)
    corr = {}
    start = lambda c: p.init_point(c).astype(np.float32).astype(np.float64)
    for level in range(K):
        h.run(1)
        X, F = h.trace_states(level)
        if level in (0, K - 2, K - 1):
            ft0, ftp = h.da_trace(level)
            a, b = [], []
            for c in range(0, C, 8):
                _, _, ob, _, _, dF = p.da_chain_level_steps(level, c, float(ft0[c]), ftp[:, c].astype(np.float64),
                                                           start(c))
                # surrogate differences along the replayed path
                bits = _bits_to_bool(ob, L)
                cur = float(ft0[c])
                for s in range(L):
                    if not np.isnan(dF[s]):
                        a.append(dF[s])
                        b.append(float(ftp[s, c]) - cur)
                    if bits[s]:
                        cur = float(ftp[s, c])
            corr[level] = float(np.corrcoef(a, b)[0, 1])
        pstar = int(h.level_log()["argmin"][level])
        start = lambda c, xr=X[pstar].copy(): xr
    trained = 0.5 * (corr[K - 2] + corr[K - 1])
    assert trained > 0.3 and min(corr[K - 2], corr[K - 1]) > corr[0] + 0.25, corr


def test_surrogate_saves_true_evaluations_against_plain(sa):
    """Same problem and schedule, in a regime where most moves are rejected (the
    surrogate can only spare evaluations of moves it rejects): delayed acceptance
    evaluates f for fewer proposals than plain Metropolis, and reaches a
    comparable best value."""
    cost, n, C, L, K = "rot_schwefel", 32, 2048, 200, 10
    Q = inputs.rotation(n, 5)
    plain = _create(sa, cost, n, C, L, K, 5.0, 0.8, 3, Q, surrogate=0)
    da = _create(sa, cost, n, C, L, K, 5.0, 0.8, 3, Q, surrogate=1)
    plain.run()
    da.run()
    _, fp, sp = plain.best()
    _, fd, sd = da.best()
    assert sp["true_evals"] == sp["steps"]
    print("true evaluations: plain", sp["true_evals"], "delayed acceptance", sd["true_evals"],
          "accepts", sp["accepts"], sd["accepts"], "best", fp, fd)
    assert sd["true_evals"] < 0.8 * sd["steps"], (sd["true_evals"], sd["steps"])
    assert abs(fd - fp) <= 0.05 * abs(fp) + 1.0, (fd, fp)


def test_surrogate_rejects_bad_arguments(sa):
    n = 16
    lo, hi = inputs.box("schwefel", n)
    with pytest.raises(sa.SAError):  # separable cost
        sa.create("schwefel", lo, hi, n, 64, 10, sa.Schedule(precision="fp32", surrogate=1))
    Q = inputs.rotation(n, 0)
    with pytest.raises(sa.SAError):  # FP64
        sa.create("rot_schwefel", lo, hi, n, 64, 10, sa.Schedule(precision="fp64", surrogate=1), Q=Q)
    h = sa.create("rot_schwefel", lo, hi, n, 64, 10, sa.Schedule(precision="fp32", surrogate=1, levels=2), Q=Q)
    h.run(1)
    with pytest.raises(sa.SAError):  # no checkpoints for surrogate handles
        h.checkpoint()

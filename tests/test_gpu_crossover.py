"""GPU parity of the stochastic crossover (Boltzmann selection at each exchange)
with the oracle: FP64 bit for bit, FP32 and rotated chain by chain from the
oracle's draw on the GPU's own final values."""
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


@pytest.mark.parametrize("cost,n,C,m,proposal", [("schwefel", 5, 300, 1, "gaussian"), ("rastrigin", 7, 1100, 1, "uniform"),
                                                 ("ackley", 4, 257, 2, "gaussian"), ("shekel", 4, 130, 1, "uniform")])
def test_fp64_bit_parity(sa, cost, n, C, m, proposal):
    """Every accept bit of every level, the argmins and the incumbent equal the oracle's
    run with the crossover: the draws (over 1100 chains: two scan blocks) are the oracle's."""
    L, K, T0, rho, seed = 50, 5, 20.0, 0.7, 12
    tab = inputs.table("shekel", n, 10) if cost == "shekel" else None
    lo, hi = (np.zeros(n), np.full(n, 10.0)) if tab is not None else inputs.box(cost, n)
    sch = sa.Schedule(T0=T0, rho=rho, levels=K, precision="fp64", trace_levels=K, crossover=1, exchange_every=m,
                      proposal=proposal)
    with sa.create(cost, lo, hi, n, C, L, sch, seed=seed, table=tab) as h:
        h.run()
        bits = [h.trace(l) for l in range(K)]
        x, f, _ = h.best()
        log = h.level_log()
    ref = oracle.Problem(cost, n, lo, hi, chains=C, L=L, T0=T0, rho=rho, seed=seed, mode=0, table=tab, crossover=True,
                         exchange_every=m, proposal=proposal).run(K, trace_levels=K)
    for l in range(K):
        assert np.array_equal(bits[l], ref["bits"][l]), l
    assert np.array_equal(log["argmin"], ref["argmin"])
    assert abs(f - ref["f_inc"]) <= 1e-12 * max(1.0, abs(ref["f_inc"]))
    assert np.allclose(x, ref["x_inc"], rtol=0, atol=1e-12 * (hi - lo).max())


def _level1_from_oracle_draw(p, X0, F0, bits1, L, tol_fn):
    """Level 1 of every chain against the oracle started from the state the oracle
    draws from the GPU's level-0 values: a chain whose draw differed would disagree
    from its first steps on, not only at a near-tie."""
    src = p.crossover_sources(0, F0)
    gb = _bits_to_bool(bits1, L)
    full = 0
    for c in range(len(F0)):
        Fo, xo, ob, dF, tau = p.chain_steps(1, c, X0[src[c]])
        diff = np.nonzero(_bits_to_bool(ob, L) != gb[c])[0]
        if diff.size == 0:
            full += 1
        else:
            s = diff[0]
            assert abs(dF[s] - tau[s]) <= tol_fn(dF[s], tau[s], xo), (c, s, dF[s], tau[s])
    return full


@pytest.mark.parametrize("cost,warp", [("schwefel", "0"), ("schwefel", "1"), ("rastrigin", "1"), ("ackley", "0")])
def test_fp32_level1_starts_from_the_oracle_draw(sa, cost, warp, monkeypatch):
    monkeypatch.setenv("SA_WARP_MODE", warp)
    n, C, L, T0, rho, seed = 12, 600, 120, 10.0, 0.8, 4
    lo, hi = inputs.box(cost, n)
    sch = sa.Schedule(T0=T0, rho=rho, levels=2, precision="fp32", trace_levels=2, crossover=1)
    with sa.create(cost, lo, hi, n, C, L, sch, seed=seed) as h:
        h.run(1)
        X0, F0 = h.trace_states(0)  # the final states of level 0 (readable until level 1 starts)
        h.run(1)
        bits1 = h.trace(1)
    # every chain's value is exact (FP64 of its FP32 state), not only the candidates'
    for c in range(0, C, 7):
        assert abs(F0[c] - oracle.cost(cost, X0[c])) <= 1e-9 * max(1.0, abs(F0[c]))
    assert np.isfinite(F0).all()
    p = oracle.Problem(cost, n, lo, hi, chains=C, L=L, T0=T0, rho=rho, seed=seed, mode=1, crossover=True)
    scale = {"schwefel": 12.2 / n, "rastrigin": 73.0, "ackley": 2.0}[cost] * 1e-3 * 0.1 * (hi[0] - lo[0])
    full = _level1_from_oracle_draw(p, X0, F0, bits1, L,
                                    lambda dF, tau, xo: 1e-3 * (abs(dF) + abs(tau)) + scale)
    assert full >= 0.9 * C, full


@pytest.mark.parametrize("cost,n", [("rot_rastrigin", 32), ("rot_schwefel", 24)])
def test_rotated_level1_starts_from_the_oracle_draw(sa, cost, n):
    C, L, T0, rho, seed = 200, 150, 20.0, 0.7, 9
    lo, hi = inputs.box(cost, n)
    Q = inputs.rotation(n, 6)
    sch = sa.Schedule(T0=T0, rho=rho, levels=2, precision="fp32", trace_levels=2, crossover=1)
    with sa.create(cost, lo, hi, n, C, L, sch, seed=seed, Q=Q) as h:
        h.run(1)
        X0, F0 = h.trace_states(0)
        h.run(1)
        bits1 = h.trace(1)
    p = oracle.Problem(cost, n, lo, hi, chains=C, L=L, T0=T0, rho=rho, seed=seed, Q=Q, mode=1, crossover=True)
    sigma = 0.1 * (hi[0] - lo[0]) * np.sqrt(rho)

    def tol(dF, tau, xo):
        G = float(np.abs(oracle.grad(cost, xo, Q)).max()) + 1.0
        return 1e-4 * (abs(dF) + abs(tau)) + 1e-4 * sigma * G

    full = _level1_from_oracle_draw(p, X0, F0, bits1, L, tol)
    assert full >= 0.9 * C, full


def test_batch_draws_within_each_problem(sa):
    probs = [dict(cost="schwefel", n=3, chains=150, lo=np.full(3, -500.0), hi=np.full(3, 500.0)),
             dict(cost="griewank", n=6, chains=90, lo=np.full(6, -600.0), hi=np.full(6, 600.0))]
    L, K, T0, rho, seed = 40, 4, 15.0, 0.8, 3
    sch = sa.Schedule(T0=T0, rho=rho, levels=K, precision="fp64", trace_levels=K, crossover=1)
    with sa.create_batch(probs, L, sch, seed=seed) as h:
        h.run()
        bits = [h.trace(l) for l in range(K)]
        for p, pr in enumerate(probs):
            ref = oracle.Problem(pr["cost"], pr["n"], pr["lo"], pr["hi"], chains=pr["chains"], L=L, T0=T0, rho=rho,
                                 seed=seed, problem=p, mode=0, crossover=True).run(K, trace_levels=K)
            for l in range(K):
                assert np.array_equal(bits[l][p], ref["bits"][l]), (p, l)
            assert np.array_equal(h.level_log(p)["argmin"], ref["argmin"])


def test_rejects_what_the_crossover_does_not_support(sa):
    lo, hi = inputs.box("schwefel", 4)
    with pytest.raises(RuntimeError):
        sa.create("schwefel", lo, hi, 4, 64, 10, sa.Schedule(levels=3, precision="fp32", crossover=1, independent=1))
    with pytest.raises(RuntimeError):
        sa.create("rot_schwefel", lo, hi, 4, 64, 10, sa.Schedule(levels=3, precision="fp32", crossover=1, surrogate=1),
                  Q=np.eye(4))
    h = sa.create("schwefel", lo, hi, 4, 64, 10, sa.Schedule(levels=3, precision="fp32", crossover=1))
    with pytest.raises(RuntimeError):
        h.set_chain_offset(64)
    h.destroy()

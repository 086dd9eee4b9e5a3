"""Asynchronous chains (Sec. 2.2.1: no exchange between levels, every chain
continues from its own state) against the oracle's asynchronous run."""
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


def _bits(b, L):
    return np.unpackbits(np.ascontiguousarray(b).view(np.uint8), axis=-1, bitorder="little")[..., :L].astype(bool)


def test_fp64_asynchronous_run_is_the_oracles(sa):
    n, C, L, K = 2, 300, 60, 5
    lo, hi = inputs.box("schwefel", n)
    sch = sa.Schedule(T0=100.0, rho=0.9, levels=K, precision="fp64", trace_levels=2, independent=1)
    h = sa.create("schwefel", lo, hi, n, C, L, sch, seed=7)
    h.run()
    _, f, st = h.best()
    log = h.level_log()
    ref = oracle.Problem("schwefel", n, lo, hi, chains=C, L=L, T0=100.0, rho=0.9, seed=7, mode=0,
                         independent=True).run(K, trace_levels=2)
    for level in range(2):
        assert np.array_equal(h.trace(level), ref["bits"][level]), level
    # argmins exactly; values to the FP64 resolution (CUDA's and libm's sin may differ by an ulp)
    assert np.array_equal(log["argmin"], ref["argmin"])
    assert np.allclose(log["f_level"], ref["f_level"], rtol=1e-12, atol=0)
    assert abs(f - ref["f_inc"]) <= 1e-12 * abs(ref["f_inc"]) and st["accepts"] == int(ref["accepts"].sum())
    # the synchronous run differs from level 1 on
    sync = oracle.Problem("schwefel", n, lo, hi, chains=C, L=L, T0=100.0, rho=0.9, seed=7, mode=0).run(K)
    assert not np.array_equal(sync["f_level"][1:], ref["f_level"][1:])


@pytest.mark.parametrize("cost,n,warp", [("schwefel", 16, "0"), ("rastrigin", 40, "1"), ("rot_rastrigin", 24, None)])
def test_fp32_asynchronous_level1_from_each_chains_own_state(sa, cost, n, warp, monkeypatch):
    if warp is not None:
        monkeypatch.setenv("SA_WARP_MODE", warp)
    C, L, T0, rho, seed = 400, 150, 30.0, 0.7, 3
    lo, hi = inputs.box(cost, n)
    Q = inputs.rotation(n, 1) if cost.startswith("rot") else None
    sch = sa.Schedule(T0=T0, rho=rho, levels=2, precision="fp32", trace_levels=2, independent=1)
    h = sa.create(cost, lo, hi, n, C, L, sch, seed=seed, Q=Q)
    if warp is not None:
        assert h.describe()[0]["kind"] == ("fp32_warp" if warp == "1" else "fp32_thread")
    h.run(1)
    X0, _ = h.trace_states(0)
    h.run(1)
    X1, F1 = h.trace_states(1)
    gb = _bits(h.trace(1), L)
    p = oracle.Problem(cost, n, lo, hi, chains=C, L=L, T0=T0, rho=rho, seed=seed, Q=Q, mode=1)
    full = 0
    for c in range(C):
        Fo, xo, ob, dF, tau = p.chain_steps(1, c, X0[c])  # the chain's own level-0 end state
        diff = np.nonzero(_bits(ob, L) != gb[c])[0]
        if diff.size == 0:
            full += 1
        else:
            s = diff[0]
            assert abs(dF[s] - tau[s]) <= 1e-3 * (abs(dF[s]) + abs(tau[s])) + 0.05, (c, s, dF[s], tau[s])
        fx = oracle.cost(cost, X1[c], Q)
        assert abs(F1[c] - fx) <= 1e-9 * max(1.0, abs(fx))
    assert full >= 0.9 * C, full
    assert int(h.level_log()["argmin"][1]) == int(np.argmin(F1))
    with pytest.raises(sa.SAError):
        h.checkpoint()


@pytest.mark.parametrize("m", [2, 3])
def test_fp64_periodic_exchange_is_the_oracles(sa, m):
    n, C, L, K = 2, 257, 50, 6
    lo, hi = inputs.box("schwefel", n)
    sch = sa.Schedule(T0=80.0, rho=0.85, levels=K, precision="fp64", exchange_every=m)
    h = sa.create("schwefel", lo, hi, n, C, L, sch, seed=5)
    h.run()
    log = h.level_log()
    ref = oracle.Problem("schwefel", n, lo, hi, chains=C, L=L, T0=80.0, rho=0.85, seed=5, mode=0,
                         exchange_every=m).run(K)
    assert np.array_equal(log["argmin"], ref["argmin"])
    assert np.allclose(log["f_level"], ref["f_level"], rtol=1e-12, atol=0)
    assert abs(h.best()[1] - ref["f_inc"]) <= 1e-12 * abs(ref["f_inc"])

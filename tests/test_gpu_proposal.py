"""GPU parity of the uniform redraw of the selected coordinate (Sec. 2.1 Step 2)
with the oracle, on every sweep, and the paper's Schwefel accuracy table
reproduced with it.
"""
import numpy as np
import pytest

import oracle
from paper_2408_00018_gb300 import inputs
from tests.conftest import read_golden

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


@pytest.mark.parametrize("cost,n,table", [("schwefel", 5, None), ("rastrigin", 9, None), ("ackley", 4, None),
                                          ("rosenbrock", 6, None), ("six_hump_camel", 2, None),
                                          ("shekel", 4, "shekel")])
def test_fp64_bit_parity(sa, cost, n, table):
    C, L, K, T0, rho, seed = 300, 64, 4, 20.0, 0.7, 8
    if cost == "six_hump_camel":
        lo, hi = np.array([-3.0, -2.0]), np.array([3.0, 2.0])  # a box that differs per coordinate
    elif table:
        lo, hi = np.zeros(n), np.full(n, 10.0)
    else:
        lo, hi = inputs.box(cost, n)
    tab = inputs.table(table, n, 10) if table else None
    sch = sa.Schedule(T0=T0, rho=rho, levels=K, precision="fp64", trace_levels=2, proposal="uniform")
    with sa.create(cost, lo, hi, n, C, L, sch, seed=seed, table=tab) as h:
        h.run()
        bits = [h.trace(0), h.trace(1)]
        x, f, _ = h.best()
        log = h.level_log()
    ref = oracle.Problem(cost, n, lo, hi, chains=C, L=L, T0=T0, rho=rho, seed=seed, mode=0, table=tab,
                         proposal="uniform").run(K, trace_levels=2)
    for lev in range(2):
        assert np.array_equal(bits[lev], ref["bits"][lev]), lev
    assert np.array_equal(log["argmin"], ref["argmin"])
    assert abs(f - ref["f_inc"]) <= 1e-12 * max(1.0, abs(ref["f_inc"]))


_LIP = {"schwefel": 12.2, "rastrigin": 73.0, "ackley": 2.0, "rosenbrock": 1.0e5}


@pytest.mark.parametrize("cost", ["schwefel", "rastrigin", "ackley", "rosenbrock"])
@pytest.mark.parametrize("warp", ["0", "1"])
def test_fp32_decisions_differ_only_at_near_ties(sa, cost, warp, monkeypatch):
    """FP32 chain-per-thread and chain-per-warp layouts: a decision differs from the
    oracle's only where the oracle's margin |dF - tau| is within the FP32 error of
    the move (the FP32 redraw of a coordinate differs from the FP64 one by an ulp)."""
    if warp == "1" and cost == "ackley":
        pytest.skip("Ackley runs the chain-per-thread layout only")
    monkeypatch.setenv("SA_WARP_MODE", warp)
    n, C, L, T0, seed = 16, 500, 200, 20.0, 31
    lo, hi = inputs.box(cost, n)
    sch = sa.Schedule(T0=T0, rho=0.9, levels=1, precision="fp32", trace_levels=1, proposal="uniform")
    with sa.create(cost, lo, hi, n, C, L, sch, seed=seed) as h:
        h.run()
        X, Fg = h.trace_states(0)
        gb = _bits_to_bool(h.trace(0), L)
        argmin = int(h.level_log()["argmin"][0])
    p = oracle.Problem(cost, n, lo, hi, chains=C, L=L, T0=T0, rho=0.9, seed=seed, mode=1, proposal="uniform")
    ulp_move = 2.0 ** -22 * max(abs(lo[0]), abs(hi[0])) * _LIP[cost]
    full = 0
    for c in range(C):
        Fo, xo, ob, dF, tau = p.chain_steps(0, c)
        diff = np.nonzero(_bits_to_bool(ob, L) != gb[c])[0]
        if diff.size == 0:
            full += 1
        else:
            s = diff[0]
            assert abs(dF[s] - tau[s]) <= 1e-3 * (abs(dF[s]) + abs(tau[s])) + 1e3 * ulp_move, (c, s, dF[s], tau[s])
        assert abs(Fg[c] - oracle.cost(cost, X[c])) <= 1e-9 * max(1.0, abs(Fg[c]))
    assert full >= 0.9 * C, full
    assert argmin == int(np.argmin(Fg))


@pytest.mark.parametrize("cost,n", [("rot_rastrigin", 48, ), ("rot_schwefel", 40)])
def test_rotated_level0_matches_oracle(sa, cost, n):
    C, L, T0, seed = 128, 200, 20.0, 6
    lo, hi = inputs.box(cost, n)
    Q = inputs.rotation(n, 2)
    sch = sa.Schedule(T0=T0, rho=0.5, levels=1, precision="fp32", trace_levels=1, proposal="uniform")
    with sa.create(cost, lo, hi, n, C, L, sch, seed=seed, Q=Q) as h:
        h.run()
        X, F = h.trace_states(0)
        gb = _bits_to_bool(h.trace(0), L)
        argmin = int(h.level_log()["argmin"][0])
    p = oracle.Problem(cost, n, lo, hi, chains=C, L=L, T0=T0, rho=0.5, seed=seed, Q=Q, mode=1, proposal="uniform")
    full = 0
    for c in range(C):
        Fo, xo, ob, dF, tau = p.chain_steps(0, c, p.init_point(c).astype(np.float32).astype(np.float64))
        diff = np.nonzero(_bits_to_bool(ob, L) != gb[c])[0]
        if diff.size == 0:
            full += 1
        else:
            s = diff[0]
            G = float(np.abs(oracle.grad(cost, xo, Q)).max()) + 1.0
            assert abs(dF[s] - tau[s]) <= 1e-4 * (abs(dF[s]) + abs(tau[s])) + 1e-5 * (hi[0] - lo[0]) * G, (c, s)
        assert abs(F[c] - oracle.cost(cost, X[c], Q)) <= 1e-9 * max(1.0, abs(F[c]))
    assert full >= 0.9 * C, full
    assert argmin == int(np.argmin(F))


def test_surrogate_refuses_uniform_moves(sa):
    lo, hi = inputs.box("rot_schwefel", 8)
    with pytest.raises(RuntimeError):
        sa.create("rot_schwefel", lo, hi, 8, 128, 10, sa.Schedule(levels=2, precision="fp32", surrogate=1,
                                                                    proposal="uniform"), Q=inputs.rotation(8, 1))


def test_paper_schwefel_accuracy_table(sa):
    """The paper's configuration (T0 = 1000, T_min = 0.01: 1146 levels; N = 100;
    rho = 0.99; 16384 chains; box [-512, 512]^n; FP32): the synchronous run (V2)
    ends within 10x the paper's printed mean V2 error for every n of its table,
    and the asynchronous run (V1) is never better than V2 from n = 16 on, as the
    paper finds."""
    fs = inputs.SCHWEFEL_F_STAR
    for row in read_golden("table1_schwefel_accuracy.txt"):
        n = int(row[0])
        v1_paper, v2_paper = float(row[3]), float(row[5])
        lo, hi = np.full(n, -512.0), np.full(n, 512.0)
        err = {}
        for indep in (0, 1):
            sch = sa.Schedule(T0=1000.0, rho=0.99, levels=0, T_min=0.01, precision="fp32", independent=indep,
                              proposal="uniform")
            with sa.create("schwefel", lo, hi, n, 16384, 100, sch, seed=0) as h:
                h.run()
                x, f, st = h.best()
            assert st["levels_done"] == 1146 and st["steps"] == 16384 * 100 * 1146
            err[indep] = abs(f - fs)
        assert err[0] <= 10.0 * v2_paper, (n, err[0], v2_paper)
        if n >= 16:
            assert err[1] >= err[0], (n, err)

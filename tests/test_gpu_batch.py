"""GPU parity of the batched multi-problem solver (sa_create_batch) against the oracle.

Each problem p of a batch draws from Philox counter word 3 = p, so it must
reproduce the oracle run of that problem with problem index p: FP64 decisions
bit for bit; FP32 decisions equal except at near-ties.  Autotuning changes
launch shapes only, never results.
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


def _problems(spec):
    out = []
    for cost, n, C in spec:
        lo, hi = inputs.box(cost, n)
        out.append({"cost": cost, "n": n, "chains": C, "lo": lo, "hi": hi})
    return out


def test_fp64_batch_bit_parity_per_problem(sa):
    spec = [("schwefel", 2, 100), ("rastrigin", 5, 257), ("ackley", 17, 64), ("rosenbrock", 40, 33),
            ("schwefel", 70, 130), ("rastrigin", 3, 1)]
    probs = _problems(spec)
    L, K, T0, rho, seed = 50, 4, 50.0, 0.8, 17
    sch = sa.Schedule(T0=T0, rho=rho, levels=K, precision="fp64", trace_levels=1)
    with sa.create_batch(probs, L, sch, seed=seed) as h:
        h.run()
        bits = h.trace(0)
        for p, pr in enumerate(probs):
            x, f, st = h.best(p)
            log = h.level_log(p)
            ref = oracle.Problem(pr["cost"], pr["n"], pr["lo"], pr["hi"], chains=pr["chains"], L=L, T0=T0, rho=rho,
                                 seed=seed, problem=p, mode=0).run(K, trace_levels=1)
            assert np.array_equal(bits[p], ref["bits"][0]), p
            assert np.array_equal(log["argmin"], ref["argmin"]), p
            assert abs(f - ref["f_inc"]) <= 1e-12 * max(1.0, abs(ref["f_inc"])), p
            assert st["steps"] == pr["chains"] * L * K


@pytest.mark.parametrize("one_launch", [True, False])
def test_fp32_batch_per_problem_against_oracle(sa, one_launch, monkeypatch):
    spec = [("schwefel", 3, 96), ("rastrigin", 20, 130), ("ackley", 40, 64), ("rosenbrock", 100, 70),
            ("schwefel", 200, 64), ("rastrigin", 300, 40), ("schwefel", 600, 33)]
    probs = _problems(spec)
    L, T0, seed = 120, 20.0, 23
    sch = sa.Schedule(T0=T0, rho=0.9, levels=1, precision="fp32", trace_levels=1)
    monkeypatch.setenv("SA_BATCH_LEVEL", "1" if one_launch else "0")
    with sa.create_batch(probs, L, sch, seed=seed) as h:
        groups = h.describe()
        if one_launch:  # one launch per level for the whole batch
            assert len(groups) == 1 and groups[0]["kind"] == "fp32_batch_level"
        else:
            assert len(groups) >= 5  # problems are split by dimension
        h.run()
        bits = h.trace(0)
        states = h.trace_states(0)
        for p, pr in enumerate(probs):
            X, Fg = states[p]
            gb = _bits_to_bool(bits[p], L)
            op = oracle.Problem(pr["cost"], pr["n"], pr["lo"], pr["hi"], chains=pr["chains"], L=L, T0=T0, rho=0.9,
                                seed=seed, problem=p, mode=1)
            full = 0
            for c in range(0, pr["chains"], max(1, pr["chains"] // 16)):
                Fo, xo, ob, dF, tau = op.chain_steps(0, c)
                diff = np.nonzero(_bits_to_bool(ob, L) != gb[c])[0]
                if diff.size == 0:
                    full += 1
                    assert abs(Fg[c] - oracle.cost(pr["cost"], X[c])) <= 1e-9 * max(1.0, abs(Fg[c]))
                else:
                    s = diff[0]
                    assert abs(dF[s] - tau[s]) <= 1e-3 * (abs(dF[s]) + abs(tau[s])) + 0.05, (p, c, s)
            assert full >= 1, p
            x, f, st = h.best(p)
            assert f == Fg.min() or np.isclose(f, np.nanmin(Fg), rtol=0, atol=0), p


def test_autotune_changes_launch_shapes_not_results(sa):
    probs = [{"cost": c, "n": n, "chains": C, "lo": inputs.box(c, n)[0], "hi": inputs.box(c, n)[1]}
             for c, n, C in [("schwefel", 30, 300), ("rastrigin", 120, 500), ("ackley", 60, 200), ("rosenbrock", 250, 150)]]
    L, K = 64, 3
    sch = sa.Schedule(T0=30.0, rho=0.8, levels=K, precision="fp32", trace_levels=K)
    res = []
    for tune in (False, True):
        with sa.create_batch(probs, L, sch, seed=5) as h:
            if tune:
                ms = h.autotune()
                assert ms > 0
            h.run()
            res.append(([h.trace(l) for l in range(K)], [h.best(p)[1] for p in range(len(probs))],
                        [h.level_log(p)["argmin"] for p in range(len(probs))]))
    (b0, f0, a0), (b1, f1, a1) = res
    for l in range(K):
        for p in range(len(probs)):
            assert np.array_equal(b0[l][p], b1[l][p])
    assert f0 == f1 and all(np.array_equal(x, y) for x, y in zip(a0, a1))


def test_batch_of_the_generated_workload_runs(sa):
    """A reduced draw of the 512-problem workload (same generator, fewer chains
    and levels): every problem completes and stays inside its box."""
    probs = inputs.batch_problems(count=64, seed=0, chain_range=(32, 256))
    sch = sa.Schedule(T0=100.0, rho=0.95, levels=3, precision="fp32")
    with sa.create_batch(probs, 50, sch, seed=0) as h:
        h.autotune()
        h.run()
        for p, pr in enumerate(probs):
            x, f, st = h.best(p)
            assert np.isfinite(f) and (x >= pr["lo"]).all() and (x <= pr["hi"]).all()
            assert abs(oracle.cost(pr["cost"], x) - f) <= 1e-9 * max(1.0, abs(f))


def test_one_launch_level_equals_dimension_groups(sa, monkeypatch):
    """The batched level kernel (one launch per level: every tile of every
    problem, each problem's level ended by its last tile) gives the same accept
    bits, argmins, results and visited states as one launch per dimension group
    with the separate argmin: partial tiles, every cost, every tile layout
    (Ackley above n = 128: chains fed by producer warps, 29 to 53 chains a tile)."""
    spec = [("schwefel", 3, 300), ("rastrigin", 20, 257), ("ackley", 40, 100), ("ackley", 300, 70),
            ("rosenbrock", 100, 129), ("schwefel", 200, 65), ("rastrigin", 300, 40), ("schwefel", 520, 33),
            ("rosenbrock", 400, 31), ("ackley", 511, 61), ("ackley", 130, 200)]
    probs = _problems(spec)
    L, K = 97, 4
    sch = sa.Schedule(T0=25.0, rho=0.8, levels=K, precision="fp32", trace_levels=K)
    res = []
    for one in ("1", "0"):
        monkeypatch.setenv("SA_BATCH_LEVEL", one)
        with sa.create_batch(probs, L, sch, seed=7) as h:
            h.run()
            res.append(([h.trace(l) for l in range(K)], [h.best(p)[:2] for p in range(len(probs))],
                        [h.level_log(p) for p in range(len(probs))], h.describe()))
    (b1, best1, log1, d1), (b0, best0, log0, d0) = res
    assert len(d1) == 1 and len(d0) > 1
    for l in range(K):
        for p in range(len(probs)):
            assert np.array_equal(b1[l][p], b0[l][p]), (l, p)
    for p in range(len(probs)):
        assert best1[p][1] == best0[p][1] and np.array_equal(best1[p][0], best0[p][0]), p
        assert np.array_equal(log1[p]["argmin"], log0[p]["argmin"])
        assert np.array_equal(log1[p]["f_inc"], log0[p]["f_inc"])


def test_generated_draw_at_its_chain_counts_against_oracle(sa):
    """64 problems of the batched workload's generator at their own chain counts
    (256 .. 16384), one launch per level: per problem, sampled chains of a traced
    level against the FP64 oracle (identical decisions except where the oracle's
    own margin is within the FP32 error), and the FP64 batch of the same draw
    decision for decision."""
    probs = inputs.batch_problems(count=64, seed=0)
    L, T0, seed = 200, 20.0, 0
    sch = sa.Schedule(T0=T0, rho=0.9, levels=1, precision="fp32", trace_levels=1)
    with sa.create_batch(probs, L, sch, seed=seed) as h:
        assert h.describe()[0]["kind"] == "fp32_batch_level"
        h.run()
        bits = h.trace(0)
        for p, pr in enumerate(probs):
            gb = _bits_to_bool(bits[p], L)
            op = oracle.Problem(pr["cost"], pr["n"], pr["lo"], pr["hi"], chains=pr["chains"], L=L, T0=T0, rho=0.9,
                                seed=seed, problem=p, mode=1)
            for c in (0, pr["chains"] // 2, pr["chains"] - 1):
                _, _, ob, dF, tau = op.chain_steps(0, c)
                diff = np.nonzero(_bits_to_bool(ob, L) != gb[c])[0]
                if diff.size:
                    s = diff[0]
                    assert abs(dF[s] - tau[s]) <= 1e-3 * (abs(dF[s]) + abs(tau[s])) + 0.05, (p, c, s)
            x, f, _ = h.best(p)
            assert abs(oracle.cost(pr["cost"], x) - f) <= 1e-9 * max(1.0, abs(f))
    # FP64: every accept bit of the sampled chains equals the oracle's (full evaluation, same order)
    L64 = 40
    sch64 = sa.Schedule(T0=T0, rho=0.9, levels=1, precision="fp64", trace_levels=1)
    with sa.create_batch(probs, L64, sch64, seed=seed) as h:
        h.run()
        bits = h.trace(0)
        for p, pr in enumerate(probs):
            gb = _bits_to_bool(bits[p], L64)
            op = oracle.Problem(pr["cost"], pr["n"], pr["lo"], pr["hi"], chains=pr["chains"], L=L64, T0=T0,
                                rho=0.9, seed=seed, problem=p, mode=0)
            for c in (0, pr["chains"] - 1):
                _, _, _, ob = op.chain_level(0, c, trace=True)
                assert np.array_equal(_bits_to_bool(ob, L64), gb[c]), (p, c)

"""GPU parity of the rotated costs f(x) = F(Q x) against the FP64 oracle.

The CUDA path keeps x in FP32 and y = Q x as an FP32 pair, decides in FP32
with an error bound and re-takes in FP64 every decision inside the bound, so
each decision is the FP64 decision on its own (FP32) state.  The oracle is
started from the same FP32 states; a decision may then differ only where the
oracle's own margin |dF - tau| is within the difference of the proposals
(FP32 against FP64 arithmetic of the Gaussian step).  Final values are the
FP64 cost of the final FP32 state, the argmin is exact over them.
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


def _create(sa, cost, n, C, L, K, T0, rho, seed, Q, trace_levels=0):
    lo, hi = inputs.box(cost, n)
    sch = sa.Schedule(T0=T0, rho=rho, levels=K, sigma_frac=0.1, precision="fp32", trace_levels=trace_levels)
    return sa.create(cost, lo, hi, n, C, L, sch, seed=seed, Q=Q)


def _check_level(p, level, X, Fg, bits, L, starts, chains):
    """Chain-by-chain comparison of one traced level with the oracle started from `starts`."""
    sigma = 0.1 * (p.hi[0] - p.lo[0]) * np.sqrt(oracle.temperature(p.T0, p.rho, level) / p.T0)
    gb = _bits_to_bool(bits, L)
    full = 0
    for c in chains:
        Fo, xo, ob, dF, tau = p.chain_steps(level, c, starts(c))
        diff = np.nonzero(_bits_to_bool(ob, L) != gb[c])[0]
        if diff.size == 0:
            full += 1
        else:
            s = diff[0]
            G = float(np.abs(oracle.grad(p.cost, xo, p.Q)).max()) + 1.0
            tol = 1e-4 * (abs(dF[s]) + abs(tau[s])) + 1e-4 * sigma * G
            assert abs(dF[s] - tau[s]) <= tol, (level, c, s, dF[s], tau[s], tol)
        # the reported value is the FP64 cost of the reported FP32 state
        fx = oracle.cost(p.cost, X[c], p.Q)
        assert abs(Fg[c] - fx) <= 1e-9 * max(1.0, abs(fx)), (level, c, Fg[c], fx)
    return full


@pytest.mark.parametrize("cost,n,C,T0", [("rot_rastrigin", 64, 256, 30.0), ("rot_rastrigin", 100, 130, 10.0),
                                         ("rot_schwefel", 128, 256, 30.0), ("rot_schwefel", 37, 70, 50.0)])
def test_rot_two_levels_match_oracle(sa, cost, n, C, T0):
    L, seed = 300, 5
    Q = inputs.rotation(n, 3)
    h = _create(sa, cost, n, C, L, 2, T0, 0.5, seed, Q, trace_levels=2)
    lo, hi = inputs.box(cost, n)
    p = oracle.Problem(cost, n, lo, hi, chains=C, L=L, T0=T0, rho=0.5, seed=seed, Q=Q, mode=1)
    h.run(1)
    X0, F0 = h.trace_states(0)
    full0 = _check_level(p, 0, X0, F0, h.trace(0), L,
                         lambda c: p.init_point(c).astype(np.float32).astype(np.float64), range(C))
    log = h.level_log()
    pstar = int(log["argmin"][0])
    assert pstar == int(np.argmin(F0))
    assert log["f_level"][0] == F0[pstar]
    h.run(1)
    X1, F1 = h.trace_states(1)
    full1 = _check_level(p, 1, X1, F1, h.trace(1), L, lambda c: X0[pstar], range(C))
    assert int(h.level_log()["argmin"][1]) == int(np.argmin(F1))
    assert full0 >= 0.9 * C and full1 >= 0.9 * C, (full0, full1)
    _, f, st = h.best()
    assert f == min(F0.min(), F1.min())
    assert st["steps"] == 2 * C * L and 0 <= st["rechecks"] <= 0.01 * st["steps"]


def test_rot_candidate_argmin_equals_full_argmin(sa):
    """Traced levels re-evaluate every chain in FP64, untraced ones only the
    candidates inside the error band: both must pick the same chains."""
    n, C, L, K = 256, 4096, 200, 4
    Q = inputs.rotation(n, 1)
    a = _create(sa, "rot_rastrigin", n, C, L, K, 50.0, 0.7, 2, Q, trace_levels=K)
    b = _create(sa, "rot_rastrigin", n, C, L, K, 50.0, 0.7, 2, Q, trace_levels=0)
    a.run()
    b.run()
    la, lb = a.level_log(), b.level_log()
    assert np.array_equal(la["argmin"], lb["argmin"])
    assert np.array_equal(la["f_level"], lb["f_level"])
    assert a.best()[1] == b.best()[1]


def test_rot_checkpoint_resume_bit_identical(sa):
    n, C, L = 48, 512, 100
    Q = inputs.rotation(n, 4)
    h = _create(sa, "rot_schwefel", n, C, L, 4, 40.0, 0.8, 9, Q)
    h.run(2)
    ck = h.checkpoint()
    h.run(2)
    x1, f1, _ = h.best()
    log1 = h.level_log()
    g = _create(sa, "rot_schwefel", n, C, L, 4, 40.0, 0.8, 9, Q)
    g.restore(ck)
    g.run(2)
    x2, f2, _ = g.best()
    assert f1 == f2 and np.array_equal(x1, x2)
    assert np.array_equal(log1["argmin"], g.level_log()["argmin"])


def test_rot_in_a_batch_uses_its_problem_index(sa):
    """A rotated problem inside a batch draws Philox word 3 = its index."""
    L, T0 = 200, 20.0
    nr, Cr = 40, 96
    Q = inputs.rotation(nr, 6)
    lo_s, hi_s = inputs.box("schwefel", 8)
    lo_r, hi_r = inputs.box("rot_rastrigin", nr)
    probs = [dict(cost="schwefel", n=8, chains=300, lo=lo_s, hi=hi_s),
             dict(cost="rot_rastrigin", n=nr, chains=Cr, lo=lo_r, hi=hi_r, Q=Q)]
    sch = sa.Schedule(T0=T0, rho=0.5, levels=1, precision="fp32", trace_levels=1)
    h = sa.create_batch(probs, L, sch, seed=11)
    h.run()
    X, F = h.trace_states(0)[1]
    bits = h.trace(0)[1]
    p = oracle.Problem("rot_rastrigin", nr, lo_r, hi_r, chains=Cr, L=L, T0=T0, rho=0.5, seed=11, problem=1, Q=Q,
                       mode=1)
    full = _check_level(p, 0, X, F, bits, L, lambda c: p.init_point(c).astype(np.float32).astype(np.float64),
                        range(Cr))
    assert full >= 0.9 * Cr
    assert any(g["kind"] == "rot_warp" for g in h.describe())


def test_rot_rastrigin_n1024_full_size_level0_sampled(sa):
    """Rotated Rastrigin n=1024, 65536 chains, L=500 (the mixed-precision workload):
    level 0 at full size, checked chain by chain on a sample, argmin over all chains."""
    cfg = inputs.ROT_RASTRIGIN_N1024
    n, C, L = cfg["n"], cfg["chains"], cfg["L"]
    Q = inputs.rotation(n, cfg["q_seed"])
    h = _create(sa, "rot_rastrigin", n, C, L, 1, cfg["T0"], cfg["rho"], cfg["seed"], Q, trace_levels=1)
    h.run()
    X, F = h.trace_states(0)
    lo, hi = inputs.box("rot_rastrigin", n)
    p = oracle.Problem("rot_rastrigin", n, lo, hi, chains=C, L=L, T0=cfg["T0"], rho=cfg["rho"], seed=cfg["seed"],
                       Q=Q, mode=1)
    sample = sorted(set([0, 1, 3, 4, C // 2, C - 1] + list(np.random.default_rng(1).integers(0, C, 24))))
    full = _check_level(p, 0, X, F, h.trace(0), L,
                        lambda c: p.init_point(c).astype(np.float32).astype(np.float64), sample)
    assert full >= 0.8 * len(sample)
    assert int(h.level_log()["argmin"][0]) == int(np.argmin(F))
    st = h.best()[2]
    assert st["rechecks"] <= 0.01 * st["steps"]


def test_rot_rejects_bad_arguments(sa):
    n = 8
    lo, hi = inputs.box("rot_rastrigin", n)
    Q = inputs.rotation(n, 0)
    with pytest.raises(sa.SAError):  # no Q
        sa.create("rot_rastrigin", lo, hi, n, 64, 10, sa.Schedule(precision="fp32"))
    with pytest.raises(sa.SAError):  # FP64 sweep has no rotated form
        sa.create("rot_rastrigin", lo, hi, n, 64, 10, sa.Schedule(precision="fp64"), Q=Q)
    Qn = Q.copy()
    Qn[2, 3] = np.nan
    with pytest.raises(sa.SAError):
        sa.create("rot_rastrigin", lo, hi, n, 64, 10, sa.Schedule(precision="fp32"), Q=Qn)


def _level0_vs_oracle(sa, cost, n, C, L, T0, seed, Q, lo, hi, boundary="reflect"):
    sch = sa.Schedule(T0=T0, rho=0.5, levels=1, sigma_frac=0.1, precision="fp32", trace_levels=1, boundary=boundary)
    h = sa.create(cost, lo, hi, n, C, L, sch, seed=seed, Q=Q)
    h.run()
    X, F = h.trace_states(0)
    p = oracle.Problem(cost, n, lo, hi, chains=C, L=L, T0=T0, rho=0.5, seed=seed, Q=Q, mode=1, boundary=boundary)
    full = _check_level(p, 0, X, F, h.trace(0), L, lambda c: p.init_point(c).astype(np.float32).astype(np.float64),
                        range(C))
    assert int(h.level_log()["argmin"][0]) == int(np.argmin(F))
    assert (X >= lo).all() and (X <= hi).all()
    return full


@pytest.mark.parametrize("cost", ["rot_rastrigin", "rot_schwefel"])
def test_rot_per_coordinate_box(sa, cost):
    """A box with a different interval per coordinate (the proposal scale and the
    reflection follow the coordinate's own interval)."""
    n, C, L = 20, 96, 150
    base_lo, base_hi = inputs.box(cost, n)
    lo = base_lo * np.linspace(0.3, 1.0, n)
    hi = base_hi * np.linspace(1.0, 0.5, n)
    full = _level0_vs_oracle(sa, cost, n, C, L, 20.0, 3, inputs.rotation(n, 5), lo, hi)
    assert full >= 0.9 * C


@pytest.mark.parametrize("cost", ["rot_rastrigin", "rot_schwefel"])
def test_rot_degenerate_shapes(sa, cost):
    # n = 1 (Q = [-1]), a single chain with a single step, and the clip-only boundary
    lo1, hi1 = inputs.box(cost, 1)
    assert _level0_vs_oracle(sa, cost, 1, 33, 50, 10.0, 1, -np.eye(1), lo1, hi1) >= 0.9 * 33
    lo, hi = inputs.box(cost, 7)
    assert _level0_vs_oracle(sa, cost, 7, 1, 1, 10.0, 2, inputs.rotation(7, 1), lo, hi) == 1
    assert _level0_vs_oracle(sa, cost, 7, 70, 120, 50.0, 4, inputs.rotation(7, 2), lo, hi, boundary="clip") >= 63

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
from oracle import surrogate as S
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


def _bf16(a):
    import torch
    return torch.tensor(np.asarray(a, np.float32)).to(torch.bfloat16).to(torch.float64).numpy()


def _net_values(net, X, n, scale=1.0):
    """The surrogate's values at the rows of X by the FP64 oracle network, with the
    GPU's rounding of its operands: inputs (x - mid) / half formed in FP32 and
    rounded to BF16, weights W1, W2 rounded to BF16.  Returns (y, f~) with
    f~ = mu + sigma y.  scale != 1 plants a wrong input scaling (tests of this check)."""
    p, (mu, sig), mid, ih = net
    Xs = ((np.asarray(X, np.float32) - mid) * ih).astype(np.float32) * np.float32(scale)
    q = np.array(p, np.float64)
    W1, b1, W2, b2, w3, b3 = S.unpack(q, n)
    W1[:] = _bf16(W1)
    W2[:] = _bf16(W2)
    y, _ = S.forward(q, _bf16(Xs), n)
    return y, mu + sig * y


def _surrogate_mismatch(net, X, ft_gpu, n, scale=1.0):
    """Largest |network output of the GPU's f~ - the oracle network's output| over the
    rows, in units of the BF16 bound of the forward test (1e-2 (max |y| + 1))."""
    mu, sig = net[1]
    y, _ = _net_values(net, X, n, scale)
    y_gpu = (np.asarray(ft_gpu, np.float64) - mu) / sig
    return float(np.abs(y_gpu - y).max() / (1e-2 * (np.abs(y).max() + 1.0)))


def _check_da_level(p, level, bits, ft0, ftp, L, starts, chains, plant=0):
    """Chain-by-chain replay of one traced delayed-acceptance level by the oracle,
    from the GPU's start states and with the GPU's surrogate values.  Returns
    (chains identical bit for bit, violations).  At the first differing step of a
    chain: stage 1 (deterministic given the recorded f~) must have passed in the
    oracle too, and the oracle's stage-2 margin |(dF - dFs) - tau| must lie within
    the difference of the two proposals (FP32 against FP64 arithmetic of the
    Gaussian step), the tolerance of the plain rotated path."""
    T = oracle.temperature(p.T0, p.rho, level)
    sigma = 0.1 * float(np.max(p.hi - p.lo)) * np.sqrt(T / p.T0)
    gb = _bits_to_bool(bits, L)
    full, bad = 0, []
    for c in chains:
        _, xo, ob, _, _, dF, tau = p.da_chain_level_trace(level, c, float(ft0[c]), ftp[:, c].astype(np.float64),
                                                         starts(c), plant=plant)
        ob = _bits_to_bool(ob, L)
        diff = np.nonzero(ob != gb[c])[0]
        if diff.size == 0:
            full += 1
            continue
        s = int(diff[0])
        if np.isnan(dF[s]):  # the oracle's stage 1 rejected where the GPU went on to stage 2
            bad.append(("stage1", level, c, s))
            continue
        prev = np.nonzero(gb[c][:s])[0]  # accepted steps before s (identical on both sides)
        ft_cur = float(ftp[prev[-1], c]) if prev.size else float(ft0[c])
        dFs = float(ftp[s, c]) - ft_cur
        G = float(np.abs(oracle.grad(p.cost, xo, p.Q)).max()) + 1.0
        tol = 1e-4 * (abs(dF[s] - dFs) + abs(tau[s])) + 1e-4 * sigma * G
        if abs((dF[s] - dFs) - tau[s]) > tol:
            bad.append(("stage2", level, c, s, float(dF[s] - dFs), float(tau[s]), tol))
    return full, bad


@pytest.mark.parametrize("cost,n,C,box", [("rot_schwefel", 64, 256, "uniform"), ("rot_rastrigin", 40, 130, "uniform"),
                                          ("rot_schwefel", 24, 70, "per-coordinate")])
def test_da_decisions_match_oracle_replay(sa, cost, n, C, box):
    """Every chain of three traced levels against the oracle's replay (see
    _check_da_level), and the surrogate values the sweep used against the FP64
    oracle network with the level's parameters: at every start state and at the
    proposals of the first steps.  Planted mistakes in the oracle -- a stage-2
    sign error, an input scaled by the full instead of the half width of the box
    -- must each be caught."""
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
    planted_caught = 0
    for level in range(K):
        h.run(1)
        X, F = h.trace_states(level)
        bits = h.trace(level)
        ft0, ftp = h.da_trace(level)
        full, bad = _check_da_level(p, level, bits, ft0, ftp, L, start, range(C))
        assert not bad, bad[:5]
        total_full += full
        total += C
        # a stage-2 sign error planted in the oracle is caught on some chain of the level
        _, bad_planted = _check_da_level(p, level, bits, ft0, ftp, L, start, range(C), plant=1)
        planted_caught += int(len(bad_planted) > 0)
        for c in range(C):
            fx = oracle.cost(cost, X[c], Q)
            assert abs(F[c] - fx) <= 1e-9 * max(1.0, abs(fx)), (level, c)
        # the surrogate values the sweep used: at the level's start states ...
        net = h.da_network()
        S0 = np.array([start(c) for c in range(C)])
        assert _surrogate_mismatch(net, S0, ft0, n) <= 1.0
        # ... and at every chain's proposal of steps 0 and 1 (the chain's state there is
        # its start state, or after step 0's move when that was accepted)
        gb = _bits_to_bool(bits, L)
        for s in (0, 1):
            Xp = np.empty((C, n))
            for c in range(C):
                x = start(c).copy()
                if s == 1 and gb[c, 0]:
                    d0, xp0 = p.propose_step(level, c, 0, x)
                    x[d0] = xp0
                d, xp = p.propose_step(level, c, s, x)
                x[d] = xp
                Xp[c] = x
            assert _surrogate_mismatch(net, Xp, ftp[s], n) <= 1.0, (level, s)
        # a planted wrong input scaling (the full width of the box instead of the half) is caught
        assert _surrogate_mismatch(net, S0, ft0, n, scale=0.5) > 1.0
        pstar = int(h.level_log()["argmin"][level])
        assert pstar == int(np.argmin(F))
        x_restart = X[pstar].copy()
        start = lambda c, xr=x_restart: xr
    assert total_full >= 0.9 * total, (total_full, total)
    assert planted_caught == K
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

"""GPU parity: the CUDA library (through its C ABI) against the FP64 CPU oracle.

FP64 path: accept/reject decisions bit for bit, the same argmin at every
level, the same incumbent to 1e-9 relative.  FP32 path: a decision may differ
from the oracle only at a near-tie (the oracle's margin |dF - tau| within the
FP32 error of the kernel's dF and tau), the argmin is exact over the FP64
re-evaluated candidates, and converged runs reach the closed-form minimum.
"""
import math

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


# ------------------------------------------------------------------ kernels on their own
def test_philox_matches_oracle_and_known_answers(sa):
    import torch
    from tests.conftest import read_golden
    for row in read_golden("philox4x32_10_kat.txt"):
        v = [int(t, 16) for t in row]
        out = torch.zeros(4, dtype=torch.int32, device="cuda")
        sa.philox_fill(v[0:4], v[4:6], out)
        got = [int(x) & 0xFFFFFFFF for x in out.cpu().tolist()]
        assert got == v[6:10]
    ctr, key = [0xFFFFFF00, 7, 123456, 5], [0xDEADBEEF, 0x01234567]
    count = 100000
    out = torch.zeros(4 * count, dtype=torch.int32, device="cuda")
    sa.philox_fill(ctr, key, out)
    g = out.cpu().numpy().view(np.uint32).reshape(count, 4)
    for i in list(range(0, 300)) + list(range(count - 50, count)) + [255, 256, 257]:
        ref = oracle.philox([(ctr[0] + i) & 0xFFFFFFFF, ctr[1], ctr[2], ctr[3]], key)
        assert (g[i] == ref).all(), i


@pytest.mark.parametrize("count", [1, 5, 2047, 2048, 2049, 100003, 1 << 20])
def test_argmin_lowest_index_and_nan(sa, count):
    import torch
    rng = np.random.default_rng(count)
    F = np.round(rng.standard_normal(count) * 3, 1)  # many exact ties
    if count > 10:
        F[rng.integers(0, count, count // 10)] = np.nan
    if count > 1:
        F[count - 1] = F[~np.isnan(F)].min()  # a tie at the far end
    d = torch.tensor(F, device="cuda")
    idx, val = sa.argmin_f64(d)
    finite = np.where(np.isnan(F), np.inf, F)
    exp = int(np.argmin(finite))
    assert int(idx.item()) == exp and float(val.item()) == F[exp]


# ------------------------------------------------------------------ FP64 path
def _run_gpu(sa, cost, n, C, L, K, T0, rho, seed, precision, trace_levels=0, lo=None, hi=None, boundary="reflect",
             sigma_frac=0.1):
    if lo is None:
        lo, hi = inputs.box(cost, n)
    sch = sa.Schedule(T0=T0, rho=rho, levels=K, sigma_frac=sigma_frac, precision=precision,
                      trace_levels=trace_levels, boundary=boundary)
    h = sa.create(cost, lo, hi, n, C, L, sch, seed=seed)
    h.run()
    x, f, st = h.best()
    out = {"x": x, "f": f, "st": st, "log": h.level_log(), "h": h}
    out["bits"] = [h.trace(l) for l in range(min(trace_levels, K))]
    return out


def test_config_schwefel_n2_fp64_bit_parity(sa):
    """Schwefel n=2, box [-500,500]^2, 1024 chains, L=100, 50 levels, T0=100, rho=0.9, FP64, seed 0."""
    cfg = inputs.SCHWEFEL_N2_FP64
    n, C, L, K = cfg["n"], cfg["chains"], cfg["L"], cfg["levels"]
    lo, hi = inputs.box("schwefel", n)
    g = _run_gpu(sa, "schwefel", n, C, L, K, cfg["T0"], cfg["rho"], cfg["seed"], "fp64", trace_levels=2)
    ref = oracle.Problem("schwefel", n, lo, hi, chains=C, L=L, T0=cfg["T0"], rho=cfg["rho"], seed=cfg["seed"],
                         mode=0).run(K, trace_levels=2)
    # every decision of the first two levels (2 * 1024 * 100 steps), bit for bit
    for l in range(2):
        assert np.array_equal(g["bits"][l], ref["bits"][l]), f"level {l}"
    assert np.array_equal(g["log"]["argmin"], ref["argmin"])
    assert np.allclose(g["log"]["f_level"], ref["f_level"], rtol=1e-12, atol=0)
    assert abs(g["f"] - ref["f_inc"]) <= 1e-9 * abs(ref["f_inc"])
    assert np.allclose(g["x"], ref["x_inc"], rtol=1e-9, atol=0)
    assert g["st"]["steps"] == C * L * K
    assert g["st"]["accepts"] == int(ref["accepts"].sum())
    # and the closed-form minimum (Sec. 4.1) to 1e-6 relative
    assert abs(g["f"] - inputs.SCHWEFEL_F_STAR) <= 1e-6 * abs(inputs.SCHWEFEL_F_STAR)


@pytest.mark.parametrize("cost", ["schwefel", "rastrigin", "ackley", "rosenbrock"])
@pytest.mark.parametrize("C,L", [(300, 64), (257, 50)])
def test_fp64_costs_ragged_shapes(sa, cost, C, L):
    n, K = 5, 4
    lo, hi = inputs.box(cost, n)
    g = _run_gpu(sa, cost, n, C, L, K, 50.0, 0.8, 3, "fp64", trace_levels=1)
    ref = oracle.Problem(cost, n, lo, hi, chains=C, L=L, T0=50.0, rho=0.8, seed=3, mode=0).run(K, trace_levels=1)
    assert np.array_equal(g["bits"][0], ref["bits"][0])
    assert np.array_equal(g["log"]["argmin"], ref["argmin"])
    assert abs(g["f"] - ref["f_inc"]) <= 1e-12 * max(1.0, abs(ref["f_inc"]))


def test_fp64_clip_boundary_and_tiny_box(sa):
    n, C, L, K = 3, 100, 40, 3
    lo, hi = np.array([-1.0, 0.0, 5.0]), np.array([2.0, 1e-9, 5.0])  # includes a degenerate interval
    g = _run_gpu(sa, "rastrigin", n, C, L, K, 10.0, 0.5, 4, "fp64", trace_levels=1, lo=lo, hi=hi, boundary="clip",
                 sigma_frac=2.0)
    ref = oracle.Problem("rastrigin", n, lo, hi, chains=C, L=L, T0=10.0, rho=0.5, seed=4, mode=0, boundary="clip",
                         sigma_frac=2.0).run(K, trace_levels=1)
    assert np.array_equal(g["bits"][0], ref["bits"][0])
    assert np.array_equal(g["log"]["argmin"], ref["argmin"])
    assert (g["x"] >= lo).all() and (g["x"] <= hi).all()


def test_single_chain_single_step(sa):
    g = _run_gpu(sa, "schwefel", 1, 1, 1, 1, 100.0, 0.9, 5, "fp64", trace_levels=1)
    ref = oracle.Problem("schwefel", 1, -500, 500, chains=1, L=1, T0=100, rho=0.9, seed=5, mode=0).run(1, trace_levels=1)
    assert np.array_equal(g["bits"][0], ref["bits"][0]) and g["f"] == pytest.approx(ref["f_inc"], rel=1e-12)


def test_checkpoint_resume_bit_identical(sa):
    for prec in ("fp64", "fp32"):
        n, C, L, K = 8, 500, 80, 6
        lo, hi = inputs.box("schwefel", n)
        sch = sa.Schedule(T0=100.0, rho=0.9, levels=K, precision=prec)
        with sa.create("schwefel", lo, hi, n, C, L, sch, seed=11) as full:
            full.run()
            xf, ff, _ = full.best()
            logf = full.level_log()
        with sa.create("schwefel", lo, hi, n, C, L, sch, seed=11) as a:
            a.run(3)
            blob = a.checkpoint()
        with sa.create("schwefel", lo, hi, n, C, L, sch, seed=11) as b:
            b.restore(blob)
            b.run()
            xb, fb, st = b.best()
            logb = b.level_log()
        assert fb == ff and np.array_equal(xb, xf), prec
        assert np.array_equal(logb["argmin"], logf["argmin"]) and st["levels_done"] == K


# ------------------------------------------------------------------ FP32 path
# Lipschitz-type scale of one coordinate's term over the box, used to size the
# tolerance of state differences between FP32 and FP64 trajectories.
_LIP = {"schwefel": 12.2, "rastrigin": 73.0, "ackley": 2.0, "rosenbrock": 1.0e5}


def _fp32_vs_oracle(sa, cost, n, C, L, T0, seed, min_match=0.9):
    lo, hi = inputs.box(cost, n)
    g = _run_gpu(sa, cost, n, C, L, 1, T0, 0.9, seed, "fp32", trace_levels=1)
    X, Fg = g["h"].trace_states(0)
    gb = _bits_to_bool(g["bits"][0], L)
    p = oracle.Problem(cost, n, lo, hi, chains=C, L=L, T0=T0, rho=0.9, seed=seed, mode=1)
    sigma = 0.1 * (hi[0] - lo[0])
    full = 0
    for c in range(C):
        Fo, xo, ob, dF, tau = p.chain_steps(0, c)
        obb = _bits_to_bool(ob, L)
        diff = np.nonzero(obb != gb[c])[0]
        if diff.size == 0:
            full += 1
            tolF = 1e-3 * sigma * _LIP[cost] / (n if cost == "schwefel" else 1) + 1e-6 * abs(Fo)
            assert abs(Fg[c] - Fo) <= tolF, (c, Fg[c], Fo)
            assert abs(Fg[c] - oracle.cost(cost, X[c])) <= 1e-9 * max(1.0, abs(Fo))
        else:
            s = diff[0]
            margin = abs(dF[s] - tau[s])
            tol = 1e-3 * (abs(dF[s]) + abs(tau[s])) + 1e-3 * sigma * _LIP[cost] / (n if cost == "schwefel" else 1)
            assert margin <= tol, (c, s, dF[s], tau[s])
    assert full >= min_match * C, (full, C)
    # argmin of the level over every chain's FP64 value, lowest index
    assert g["log"]["argmin"][0] == int(np.argmin(Fg))
    return g


@pytest.mark.parametrize("cost", ["schwefel", "rastrigin", "ackley", "rosenbrock"])
def test_fp32_decisions_differ_only_at_near_ties(sa, cost):
    _fp32_vs_oracle(sa, cost, 16, 700, 200, 50.0, 21)


def test_fp32_candidate_argmin_equals_full_argmin(sa):
    """A traced run re-evaluates every chain in FP64; an untraced one only the
    candidates within the FP32 error band.  Both must choose the same chains."""
    n, C, L, K = 256, 20000, 400, 4
    lo, hi = inputs.box("schwefel", n)
    a = _run_gpu(sa, "schwefel", n, C, L, K, 100.0, 0.95, 0, "fp32", trace_levels=K)
    b = _run_gpu(sa, "schwefel", n, C, L, K, 100.0, 0.95, 0, "fp32", trace_levels=0)
    assert np.array_equal(a["log"]["argmin"], b["log"]["argmin"])
    assert np.array_equal(a["log"]["f_level"], b["log"]["f_level"])


def test_schwefel_n256_full_size_level0_sampled(sa):
    """The n=256 workload at full size (262144 chains, L=1000): level 0 checked
    chain by chain on a sample against the oracle, and the argmin over all chains."""
    cfg = inputs.SCHWEFEL_N256_FP32
    n, C, L = cfg["n"], cfg["chains"], cfg["L"]
    lo, hi = inputs.box("schwefel", n)
    g = _run_gpu(sa, "schwefel", n, C, L, 1, cfg["T0"], cfg["rho"], cfg["seed"], "fp32", trace_levels=1)
    X, Fg = g["h"].trace_states(0)
    gb = _bits_to_bool(g["bits"][0], L)
    p = oracle.Problem("schwefel", n, lo, hi, chains=C, L=L, T0=cfg["T0"], rho=cfg["rho"], seed=cfg["seed"], mode=1)
    sample = sorted(set([0, 1, 63, 64, C // 2, C - 1] + list(np.random.default_rng(0).integers(0, C, 40))))
    full = 0
    for c in sample:
        Fo, xo, ob, dF, tau = p.chain_steps(0, c)
        obb = _bits_to_bool(ob, L)
        diff = np.nonzero(obb != gb[c])[0]
        if diff.size == 0:
            full += 1
            assert abs(Fg[c] - Fo) <= 0.05, (c, Fg[c], Fo)
        else:
            s = diff[0]
            assert abs(dF[s] - tau[s]) <= 1e-3 * (abs(dF[s]) + abs(tau[s])) + 0.05, (c, s)
    assert full >= 0.5 * len(sample)
    assert g["log"]["argmin"][0] == int(np.argmin(Fg))
    assert abs(Fg[g["log"]["argmin"][0]] - oracle.cost("schwefel", X[g["log"]["argmin"][0]])) < 1e-9


@pytest.mark.parametrize("cost", ["schwefel", "rastrigin", "ackley", "rosenbrock"])
@pytest.mark.parametrize("n", [3, 20, 100])
def test_fp32_speculative_groups_are_exact(sa, cost, n, monkeypatch):
    """Evaluating several steps of a chain together and committing them in order
    gives exactly the one-step-at-a-time chain: the chain-per-thread layout with
    U = 1, 2, 4 steps per group and with the randomness of 16 steps drawn as one
    batch, and the group layouts of 2, 4, 8 and 32 lanes per chain, with and
    without the cached terms, all give the same accept bits, argmins and result."""
    C, L, K = 300, 97, 3   # L not a multiple of 4 or 32: partial groups at the end
    results = []
    # (group layout, steps per group of the chain-per-thread layout, randomness batch, lanes, cached terms)
    shapes = [("0", "1", "1", "4", "0"), ("0", "2", "1", "4", "0"), ("0", "4", "1", "4", "0"), ("0", "2", "16", "4", "0"),
              ("0", "1", "16", "4", "0")]
    if cost != "ackley":
        shapes += [("1", "1", "1", ln, ch) for ln, ch in (("2", "0"), ("4", "0"), ("4", "1"), ("8", "0"), ("8", "1"),
                                                         ("32", "1"))]
    for wm, u, r, ln, ch in shapes:
        monkeypatch.setenv("SA_WARP_MODE", wm)
        monkeypatch.setenv("SA_UNROLL", u)
        monkeypatch.setenv("SA_RAND_BATCH", r)
        monkeypatch.setenv("SA_CHAIN_LANES", ln)
        monkeypatch.setenv("SA_TERM_CACHE", ch)
        g = _run_gpu(sa, cost, n, C, L, K, 30.0, 0.8, 13, "fp32", trace_levels=K)
        results.append((g["bits"], g["log"]["argmin"], g["f"], g["x"]))
        g["h"].destroy()
    for b, a, f, x in results[1:]:
        for l in range(K):
            assert np.array_equal(b[l], results[0][0][l])
        assert np.array_equal(a, results[0][1]) and f == results[0][2] and np.array_equal(x, results[0][3])


def test_fp32_nonuniform_box_matches_uniform_path(sa):
    """A box whose bounds differ per coordinate takes the table path; with all
    coordinates equal except an irrelevant last digit it must agree with the
    uniform path where the boxes coincide."""
    n, C, L, K = 40, 256, 64, 3
    lo, hi = np.full(n, -5.12), np.full(n, 5.12)
    a = _run_gpu(sa, "rastrigin", n, C, L, K, 10.0, 0.8, 2, "fp32", trace_levels=1, lo=lo, hi=hi)
    lo2 = lo.copy()
    lo2[-1] = np.nextafter(lo2[-1], -10)  # forces the per-coordinate path; same FP32 box after rounding up
    b = _run_gpu(sa, "rastrigin", n, C, L, K, 10.0, 0.8, 2, "fp32", trace_levels=1, lo=lo2, hi=hi)
    assert np.array_equal(a["bits"][0], b["bits"][0])

"""GPU parity of the hybrid-SA polish (box-projected gradient descent) with the oracle's."""
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


@pytest.mark.parametrize("cost,n,spread", [("schwefel", 7, 30.0), ("rastrigin", 40, 0.3), ("ackley", 5, 0.5),
                                           ("rosenbrock", 4, 0.3), ("schwefel", 300, 10.0)])
def test_polish_matches_oracle_from_seeded_starts(sa, cost, n, spread):
    rng = np.random.default_rng(n)
    lo, hi = inputs.box(cost, n)
    centre = {"schwefel": 420.97, "rastrigin": 0.0, "ackley": 0.0, "rosenbrock": 1.0}[cost]
    k = 9
    x0 = np.clip(centre + spread * rng.standard_normal((k, n)), lo, hi)
    x0[-1] = lo + 0.25 * (hi - lo)  # a start far from the minimum
    xg, fg, itg = sa.polish(cost, x0, lo, hi, max_iter=1000, tol=1e-10)
    for j in range(k):
        xo, fo, ito = oracle.pgd(cost, x0[j], lo, hi, max_iter=1000, tol=1e-10)
        # same algorithm; the sums differ only by rounding order, so the two reach the same local
        # minimum: values agree to the FP64 resolution of f there
        assert abs(fg[j] - fo) <= 1e-9 * max(1.0, abs(fo)), (j, fg[j], fo, itg[j], ito)
        assert abs(oracle.cost(cost, xg[j]) - fg[j]) <= 1e-12 * max(1.0, abs(fg[j]))
        assert (xg[j] >= lo).all() and (xg[j] <= hi).all()


def test_hybrid_run_polishes_the_best_final_states(sa):
    """Schwefel n=32 stopped early (few levels): the polish of the 64 best final
    states lowers the incumbent, and the polished point is a KKT point of the box problem."""
    n, C, L, K = 32, 4096, 200, 6
    lo, hi = inputs.box("schwefel", n)
    res = {}
    for k in (0, 64):
        sch = sa.Schedule(T0=100.0, rho=0.8, levels=K, precision="fp32", polish_k=k)
        with sa.create("schwefel", lo, hi, n, C, L, sch, seed=3) as h:
            h.run()
            res[k] = h.best()
    x0, f0, _ = res[0]
    x1, f1, _ = res[64]
    assert f1 < f0
    assert abs(oracle.cost("schwefel", x1) - f1) <= 1e-12 * abs(f1)
    g = oracle.grad("schwefel", x1)
    pg = np.clip(x1 - g, lo, hi) - x1
    assert np.abs(pg).max() < 1e-6


@pytest.mark.parametrize("cost,n,spread", [("rot_schwefel", 16, 40.0), ("rot_rastrigin", 24, 0.4), ("rot_schwefel", 128, 20.0)])
def test_rotated_polish_matches_oracle(sa, cost, n, spread):
    rng = np.random.default_rng(n + 1)
    lo, hi = inputs.box(cost, n)
    Q = inputs.rotation(n, 4)
    k = 6
    x0 = np.clip(spread * rng.standard_normal((k, n)) + (0.0 if "rastrigin" in cost else 100.0), lo, hi)
    xg, fg, itg = sa.polish(cost, x0, lo, hi, max_iter=1000, tol=1e-10, Q=Q)
    for j in range(k):
        xo, fo, ito = oracle.pgd(cost, x0[j], lo, hi, Q=Q, max_iter=1000, tol=1e-10)
        assert abs(fg[j] - fo) <= 1e-9 * max(1.0, abs(fo)), (j, fg[j], fo, itg[j], ito)
        assert abs(oracle.cost(cost, xg[j], Q) - fg[j]) <= 1e-12 * max(1.0, abs(fg[j]))
        assert fg[j] <= oracle.cost(cost, x0[j], Q) + 1e-12


def test_hybrid_run_polishes_rotated_schwefel(sa):
    """Rotated Schwefel with the polish of the 16 best final states (the hybrid of
    the rotated workload at a small size): the incumbent improves and is a KKT point."""
    n, C, L, K = 24, 2048, 200, 4
    lo, hi = inputs.box("rot_schwefel", n)
    Q = inputs.rotation(n, 8)
    res = {}
    for k in (0, 16):
        sch = sa.Schedule(T0=100.0, rho=0.8, levels=K, precision="fp32", polish_k=k)
        with sa.create("rot_schwefel", lo, hi, n, C, L, sch, seed=2, Q=Q) as h:
            h.run()
            res[k] = h.best()
    f0, f1, x1 = res[0][1], res[16][1], res[16][0]
    assert f1 < f0
    assert abs(oracle.cost("rot_schwefel", x1, Q) - f1) <= 1e-12 * abs(f1)
    g = oracle.grad("rot_schwefel", x1, Q)
    assert np.abs(np.clip(x1 - g, lo, hi) - x1).max() < 1e-6

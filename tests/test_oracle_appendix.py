"""Pins of the oracle's Appendix test functions (Tests 2-12 and 15-19) and of the
suite's tables.

Each function is pinned by what the paper prints (its minima and minimisers,
`tests/golden/appendix_minima.txt`), by exhaustive search (a grid over the
whole box for the two-variable tests; a per-coordinate search for the separable
Michalewicz), and by closed forms at special points, chosen so that a dropped
term, a wrong sign, coefficient or index changes one of them.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2408_00018_gb300 import inputs
from tests.conftest import read_golden

BOX = {p["cost"]: (p["lo"][:2], p["hi"][:2]) for p in inputs.appendix_suite() if p["n"] == 2}


def _table(cost, n, m):
    return inputs.table(cost, n, None if m == "-" else int(m)) if cost in inputs.TABLE_COSTS else None


def _point(text, n):
    if "*" in text:
        v, k = text.split("*")
        return np.full(int(k), float(v))
    return np.array([{"pi": math.pi, "-pi": -math.pi}.get(t, None) or float(t) for t in text.split(",")])


def _rows():
    return [r for r in read_golden("appendix_minima.txt") if r[6] != "none"]


@pytest.mark.parametrize("row", _rows(), ids=lambda r: f"{r[0]}:{r[6][:20]}")
def test_printed_minima(row):
    """Polished from the printed minimiser (a simplex of 1e-7 of the box), f equals
    the printed f* to one unit of its last printed digit (the paper rounds some
    values and truncates others: Test 11's n = 5 minimum is -0.96499992)."""
    name, cost, n, m, fs, dec, xs = row
    n, fs, dec = int(n), float(fs), int(dec)
    x = _point(xs, n)
    assert x.size == n
    tab = _table(cost, n, m)
    lo, hi = x - 1.0, x + 1.0
    xp, fp, _ = oracle.nelder_mead(cost, x, lo, hi, step_frac=1e-7, ftol=1e-15, xtol=1e-13, table=tab)
    assert abs(fp - fs) <= 10.0 ** -dec + 1e-12, (name, fp, fs)
    assert np.abs(xp - x).max() < 0.01  # the printed point is the minimiser found


def test_shekel_and_langerman_tables_are_the_printed_ones():
    """Langerman's A and c are the first five rows of the foxholes table (both printed);
    every Shekel row is a lattice point of [0, 10]^4 with c_i in (0, 1)."""
    A, c = np.array(inputs.FOXHOLES_A), np.array(inputs.FOXHOLES_C)
    assert A.shape == (30, 10) and c.shape == (30,)
    assert np.array_equal(A[:5], np.array(inputs.LANGERMAN_A)) and np.array_equal(c[:5], inputs.LANGERMAN_C)
    S = np.array(inputs.SHEKEL_A, float)
    assert S.shape == (10, 4) and (S >= 0).all() and (S <= 10).all()
    assert all(0 < v < 1 for v in inputs.SHEKEL_C)
    t = inputs.table("shekel", 4, 7)
    assert t.shape == (7, 5) and np.array_equal(t[:, 4], inputs.SHEKEL_C[:7])


GRID_2D = [("branin", 0.397887, 6), ("dekkers_aarts", -24776.518, 3), ("easom", -1.0, 6),
           ("goldstein_price", 3.0, 6), ("himmelblau", 0.0, 6), ("six_hump_camel", -1.0316, 4),
           ("shubert", -186.7309, 4), ("cosine_mixture", -0.2, 6), ("levy_montalvo", 0.0, 6),
           ("langerman", -1.080938, 6), ("foxholes", -12.1190, 4)]


@pytest.mark.parametrize("cost,fs,dec", GRID_2D)
def test_two_variable_global_minimum_by_exhaustive_search(cost, fs, dec):
    """The lowest value on a 241 x 241 grid over the whole box, polished from the 12
    best grid points, is the printed global minimum, and no grid point lies below it."""
    lo, hi = BOX[cost]
    tab = inputs.table(cost, 2) if cost in inputs.TABLE_COSTS else None
    g0, g1 = np.linspace(lo[0], hi[0], 241), np.linspace(lo[1], hi[1], 241)
    F = np.array([[oracle.cost(cost, np.array([a, b]), table=tab) for b in g1] for a in g0])
    assert F.min() >= fs - 10.0 ** -dec - 1e-9
    best = np.argsort(F, axis=None)[:12]
    step = 0.5 * (hi - lo).min() / 240 / (hi - lo).max()
    polished = []
    for k in best:
        i, j = divmod(int(k), 241)
        _, f, _ = oracle.nelder_mead(cost, np.array([g0[i], g1[j]]), lo, hi, step_frac=step, ftol=1e-15,
                                     xtol=1e-13, table=tab)
        polished.append(f)
    assert abs(min(polished) - fs) <= 10.0 ** -dec + 1e-12, (min(polished), fs)


@pytest.mark.parametrize("n,fs", [(2, -1.8013), (5, -4.6877), (10, -9.6602)])
def test_michalewicz_by_per_coordinate_search(n, fs):
    """Michalewicz is a sum of one-variable terms, so its minimum is the sum of each
    term's minimum on [0, pi]: a fine grid per coordinate, then polish."""
    g = np.linspace(0.0, math.pi, 20001)
    x = np.zeros(n)
    for i in range(n):
        e = np.zeros(n)
        vals = []
        for t in g:
            e[i] = t
            vals.append(oracle.cost("michalewicz", e))
        x[i] = g[int(np.argmin(vals))]
    _, f, _ = oracle.nelder_mead("michalewicz", x, 0.0, math.pi, step_frac=1e-6, ftol=1e-15, xtol=1e-13)
    assert abs(f - fs) <= 1e-4, (f, fs)


def test_closed_forms():
    pi = math.pi
    # Branin: (pi, 2.275), (-pi, 12.275), (3 pi, 2.475) and, inside [-20, 20]^2, (5 pi, 12.875)
    # zero the square, so f = 10 / (8 pi) there
    for x in ([pi, 2.275], [-pi, 12.275], [3 * pi, 2.475], [5 * pi, 12.875]):
        assert abs(oracle.cost("branin", np.array(x)) - 10.0 / (8.0 * pi)) < 1e-13
    # Goldstein-Price: 3 at (0, -1); the textbook local minima 30, 84, 840
    for x, v in (([0, -1], 3.0), ([-0.6, -0.4], 30.0), ([1.8, 0.2], 84.0), ([1.2, 0.8], 840.0)):
        assert abs(oracle.cost("goldstein_price", np.array(x, float)) - v) < 1e-9 * v
    # Griewank at x_i = pi sqrt(i): every cosine is -1, so f = 1 + pi^2 n (n + 1) / 8000 - (-1)^n
    for n in (3, 4, 100):
        x = pi * np.sqrt(np.arange(1, n + 1))
        assert abs(oracle.cost("griewank", x) - (1 + pi * pi * n * (n + 1) / 8000 - (-1) ** n)) < 1e-11
    # Salomon: 0.1 on the unit sphere, 2.05 on the sphere of radius 1/2
    assert abs(oracle.cost("salomon", np.eye(10)[3]) - 0.1) < 1e-15
    assert abs(oracle.cost("salomon", np.full(4, 0.25)) - 2.05) < 1e-15
    # exponential at (1, 1, 1, 1): -exp(-2); cosine mixture at the corners: 1.1 n
    assert abs(oracle.cost("exponential", np.ones(4)) + math.exp(-2.0)) < 1e-16
    assert abs(oracle.cost("cosine_mixture", np.array([1.0, -1.0, 1.0])) - 3.3) < 1e-14
    # Levy-Montalvo at x = 1 (y = 3/2): (pi/n) (10 + 11/4 (n - 1) + 1/4)
    for n in (1, 2, 7):
        assert abs(oracle.cost("levy_montalvo", np.ones(n)) - pi / n * (10 + 2.75 * (n - 1) + 0.25)) < 1e-13
    # Easom at (pi, pi): -1; Himmelblau at (3, 2): 0; Dekkers-Aarts at 0: 0
    assert oracle.cost("easom", np.array([pi, pi])) == -1.0
    assert oracle.cost("himmelblau", np.array([3.0, 2.0])) == 0.0
    assert oracle.cost("dekkers_aarts", np.zeros(2)) == 0.0


def test_symmetries():
    rng = np.random.default_rng(7)
    for _ in range(20):
        a, b, c, d = rng.uniform(-3, 3, 4)
        # Shubert is a product of one-variable factors: f(a,b) f(c,d) = f(a,d) f(c,b)
        s = lambda u, v: oracle.cost("shubert", np.array([u, v]))  # noqa: E731
        assert abs(s(a, b) * s(c, d) - s(a, d) * s(c, b)) <= 1e-9 * (1 + abs(s(a, b) * s(c, d)))
        # six-hump camel: f(x) = f(-x); Dekkers-Aarts: even in each coordinate
        assert abs(oracle.cost("six_hump_camel", np.array([a, b])) - oracle.cost("six_hump_camel", np.array([-a, -b]))) < 1e-12
        assert oracle.cost("dekkers_aarts", np.array([a, b])) == oracle.cost("dekkers_aarts", np.array([-a, b]))
        # Shekel with one row is -1 / (|x - a|^2 + c)
        x = rng.uniform(0, 10, 4)
        row = np.array([[1.0, 2.0, 3.0, 4.0, 0.3]])
        assert abs(oracle.cost("shekel", x, table=row) + 1.0 / (np.sum((x - row[0, :4]) ** 2) + 0.3)) < 1e-15


def test_run_and_argument_rules():
    """The oracle's runs accept the Appendix costs with the full recompute (mode 0) and
    refuse a local difference (mode 1), a missing table and a two-variable test at n != 2."""
    p = oracle.Problem("shekel", 4, 0.0, 10.0, chains=64, L=50, T0=1.0, rho=0.8, seed=3,
                       table=inputs.table("shekel", 4, 10))
    r = p.run(4)
    assert np.isfinite(r["f_inc"]) and r["f_inc"] <= r["f_level"].min() + 0.0
    assert abs(oracle.cost("shekel", r["x_inc"], table=inputs.table("shekel", 4, 10)) - r["f_inc"]) < 1e-15
    with pytest.raises(ValueError):
        oracle.Problem("shekel", 4, 0.0, 10.0, chains=8, L=5, mode=1, table=inputs.table("shekel", 4, 5)).run(1)
    with pytest.raises(ValueError):
        oracle.Problem("foxholes", 2, -5.0, 15.0, chains=8, L=5).run(1)
    with pytest.raises(ValueError):
        oracle.Problem("branin", 3, -20.0, 20.0, chains=8, L=5).run(1)
    with pytest.raises(ValueError):
        oracle.pgd("branin", np.zeros(2), -20.0, 20.0)  # no gradient for the Appendix's extra tests


def test_suite_has_the_41_problems():
    s = inputs.appendix_suite()
    assert len(s) == 41 and len({p["name"] for p in s}) == 41
    assert sum(p["cost"] == "schwefel" for p in s) == 7 and max(p["n"] for p in s) == 512
    for p in s:
        assert p["lo"].shape == (p["n"],) and (p["lo"] < p["hi"]).all()
        assert (p["table"] is not None) == (p["cost"] in inputs.TABLE_COSTS)

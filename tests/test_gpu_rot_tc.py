"""The rotated costs' level-0 transform on the tensor cores (sa_rotate_rows):
Y = X Q^T from exact BF16 slices of X and Q, summed into double-float pairs.

Each element is compared with the FP64 product, per element, against the bound
the split fixes: the dropped slice pairs (order >= 8: at most 5.02 n 2^(E + F - 48))
and the slices' remainders (2 n 2^(E + F - 48)), with 2^E > max |x| of the row
and 2^F > max |q| of the coordinate, plus the rounding of the pairs' sums
(2^-42 sum_j |x_j q_j|) and of the FP64 reference itself (n 2^-53 sum_j |x_j q_j|).
A sample of rows is also checked against the oracle's own y = Q x.  The scales
of the test's rows and coordinates keep 2^(E + F) above 2^-72, the range where
the pairs' FP32 parts hold the result (smaller products are flushed).
"""
import numpy as np
import pytest

import oracle
from paper_2408_00018_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2408_00018_gb300 import sa
    return sa, torch


def _bound(X, Q):
    n = X.shape[1]
    E = np.frexp(np.abs(X).max(axis=1))[1].astype(np.float64)    # 2^E > max |x| of the row
    F = np.frexp(np.abs(Q).max(axis=1))[1].astype(np.float64)    # 2^F > max |q| of the coordinate
    E[np.abs(X).max(axis=1) == 0] = 0
    S = np.abs(X) @ np.abs(Q).T
    return 7.2 * n * np.ldexp(1.0, (E[:, None] + F[None, :] - 48).astype(int)) + (2.0 ** -42 + n * 2.0 ** -53) * S


def _states(rng, rows, n):
    X = rng.uniform(-5.12, 5.12, (rows, n)).astype(np.float32)
    X[1] = 0.0                                          # a zero row
    X[2] = (rng.standard_normal(n) * 1e-6).astype(np.float32)
    X[2, 3] = 5.0                                       # one large element, the rest tiny
    X[3] = (rng.standard_normal(n) * 1e-12).astype(np.float32)  # all small (2^(E+F) stays above 2^-72)
    X[4] = np.where(np.arange(n) % 2 == 0, 5.12, -5.12).astype(np.float32)
    X[5] = np.ldexp(1.0, rng.integers(-20, 3, n)).astype(np.float32) * rng.choice([-1, 1], n)
    return X


@pytest.mark.parametrize("n,rows,qkind", [(64, 256, "rotation"), (128, 384, "rotation"), (1024, 256, "rotation"),
                                          (256, 128, "scaled")])
def test_rotate_rows_within_split_bound(env, n, rows, qkind):
    sa, torch = env
    rng = np.random.default_rng(n + rows)
    X = _states(rng, rows, n)
    if qkind == "rotation":
        Q = inputs.rotation(n, 1)
    else:  # rows of very different magnitude and a row of zeros
        Q = rng.standard_normal((n, n)) * np.ldexp(1.0, rng.integers(-20, 10, n))[:, None]
        Q[7] = 0.0
    Y, st = sa.rotate_rows(torch.tensor(X, device="cuda"), torch.tensor(Q, device="cuda"))
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    Yd = Y.double().cpu().numpy()
    y = Yd[..., 0] + Yd[..., 1]
    ref = X.astype(np.float64) @ Q.T
    err = np.abs(y - ref)
    tol = _bound(X, Q)
    assert (err <= tol).all(), float((err / tol).max())
    # far inside one FP32 product's rounding: the pairs carry the split's ~45 bits
    scale = np.abs(X).max(axis=1)[:, None] * np.abs(Q).max(axis=1)[None, :] * n + 1e-300
    assert float((err / scale).max()) < 2.0 ** -40
    # hi is the FP32 rounding of the pair (|lo| <= half an ulp of hi)
    assert (np.abs(Yd[..., 1]) <= np.abs(np.spacing(Yd[..., 0].astype(np.float32))).astype(np.float64)).all()
    for r in (0, 2, 4, 5):  # the oracle's y = Q x, row by row
        yo = oracle.rotate(Q, X[r].astype(np.float64))
        assert (np.abs(y[r] - yo) <= tol[r]).all(), r


def test_rotate_rows_rejects_other_shapes(env):
    sa, torch = env
    X = torch.zeros((128, 100), dtype=torch.float32, device="cuda")
    Q = torch.zeros((100, 100), dtype=torch.float64, device="cuda")
    with pytest.raises(sa.SAError):
        sa.rotate_rows(X, Q)
    X = torch.zeros((100, 128), dtype=torch.float32, device="cuda")
    Q = torch.zeros((128, 128), dtype=torch.float64, device="cuda")
    with pytest.raises(sa.SAError):
        sa.rotate_rows(X, Q)


def test_rotated_level0_with_tensor_core_transform(env, monkeypatch):
    """A rotated run whose level 0 starts from the tensor-core transform against the
    same run started from the FP64 GEMM: the start pairs differ by the split's few
    units of 2^-45, so the accept bits agree except at near-ties of the decisions,
    and every reported value is the FP64 cost of its state."""
    sa, torch = env
    n, C, L = 128, 256, 200
    Q = inputs.rotation(n, 4)
    lo, hi = inputs.box("rot_rastrigin", n)
    sch = sa.Schedule(T0=30.0, rho=0.8, levels=1, sigma_frac=0.1, precision="fp32", trace_levels=1)
    res = []
    for tc in ("1", "0"):
        monkeypatch.setenv("SA_ROT_TC", tc)
        with sa.create("rot_rastrigin", lo, hi, n, C, L, sch, seed=9, Q=Q) as h:
            h.run()
            X, F = h.trace_states(0)
            res.append((h.trace(0).copy(), X, F, h.best()[1]))
    (b1, X1, F1, f1), (b0, X0, F0, f0) = res
    same = sum(np.array_equal(b1[c], b0[c]) for c in range(C))
    assert same >= 0.97 * C, same
    for X, F in ((X1, F1), (X0, F0)):
        for c in range(0, C, 7):
            fx = oracle.cost("rot_rastrigin", X[c], Q)
            assert abs(F[c] - fx) <= 1e-9 * max(1.0, abs(fx)), c

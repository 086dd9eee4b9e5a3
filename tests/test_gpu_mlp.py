"""GPU surrogate network (tensor-core forward/backward, Adam) against the FP64 oracle.

The oracle runs on the same FP32 parameters and inputs rounded to BF16 where
the GPU rounds them (weights and inputs of the matrix products); the GPU also
rounds the hidden activations to BF16, so values agree to a few 1e-3 relative.
"""
import numpy as np
import pytest

from oracle import surrogate as S

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


def _bf16(a):
    import torch
    return torch.tensor(np.asarray(a, np.float32)).to(torch.bfloat16).to(torch.float64).numpy()


def _bf16_params(p, n):
    q = np.array(p, np.float64)
    W1, b1, W2, b2, w3, b3 = S.unpack(q, n)
    W1[:] = _bf16(W1)
    W2[:] = _bf16(W2)
    return q


@pytest.mark.parametrize("n,B", [(128, 256), (37, 200), (5, 1)])
def test_forward_matches_oracle(env, n, B):
    sa, torch = env
    P = sa.mlp_param_count(n)
    assert P == S.n_params(n)
    p = torch.empty(P, dtype=torch.float32, device="cuda")
    sa.mlp_init(p, n, seed=3)
    rng = np.random.default_rng(n)
    X = rng.uniform(-1, 1, (B, n)).astype(np.float32)
    y = sa.mlp_forward(p, n, torch.tensor(X, device="cuda")).cpu().numpy()
    pr = _bf16_params(p.cpu().numpy(), n)
    yr, _ = S.forward(pr, _bf16(X), n)
    scale = np.abs(yr).max() + 1.0
    assert np.abs(y - yr).max() <= 1e-2 * scale, np.abs(y - yr).max()
    # the initial weights are He-normal: sample moments of W1 and W2
    W1, b1, W2, b2, w3, b3 = S.unpack(p.cpu().numpy().astype(np.float64), n)
    assert abs(W1.std() * np.sqrt(n / 2.0) - 1.0) < 0.05 and abs(W2.std() * np.sqrt(512 / 2.0) - 1.0) < 0.01
    assert not b1.any() and not b2.any() and b3[0] == 0.0


@pytest.mark.parametrize("n,B", [(128, 512), (20, 300), (128, 4096)])
def test_loss_and_gradient_match_oracle(env, n, B):
    sa, torch = env
    P = sa.mlp_param_count(n)
    p = torch.empty(P, dtype=torch.float32, device="cuda")
    sa.mlp_init(p, n, seed=5)
    # non-zero biases so every gradient block is exercised
    pn = p.cpu().numpy()
    o = S.unpack(pn, n)
    rng = np.random.default_rng(7)
    o[1][:] = rng.standard_normal(512) * 0.1
    o[3][:] = rng.standard_normal(512) * 0.1
    o[5][:] = 0.2
    p.copy_(torch.tensor(pn))
    X = rng.uniform(-1, 1, (B, n)).astype(np.float32)
    t = rng.standard_normal(B).astype(np.float32)
    loss, g = sa.mlp_loss_grad(p, n, torch.tensor(X, device="cuda"), torch.tensor(t, device="cuda"))
    lr_, gr = S.loss_and_grad(_bf16_params(pn, n), _bf16(X), t.astype(np.float64), n)
    assert abs(float(loss) - lr_) <= 1e-2 * lr_
    g = g.cpu().numpy().astype(np.float64)
    off = 0
    for name, size in [("W1", 512 * n), ("b1", 512), ("W2", 512 * 512), ("b2", 512), ("w3", 512), ("b3", 1)]:
        a, b = g[off:off + size], gr[off:off + size]
        if name == "b3":
            # the mean residual: a cancelling sum, judged against the residuals' RMS
            assert abs(a[0] - b[0]) <= 3e-2 * np.sqrt(2.0 * lr_), (a, b, lr_)
        else:
            rel = np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30)
            assert rel < 3e-2, (name, rel)
        off += size
    assert off == P


def test_adam_step_matches_oracle(env):
    sa, torch = env
    rng = np.random.default_rng(11)
    cnt = 10007
    p0 = rng.standard_normal(cnt).astype(np.float32)
    g = rng.standard_normal(cnt).astype(np.float32)
    m0 = (rng.standard_normal(cnt) * 0.1).astype(np.float32)
    v0 = (rng.random(cnt) * 0.1).astype(np.float32)
    p, gg, m, v = (torch.tensor(a, device="cuda") for a in (p0, g, m0, v0))
    sa.mlp_adam(p, gg, m, v, step=7, lr=3e-3)
    # the kernel's hyper-parameters are FP32 values: give the oracle the same ones
    f32 = lambda a: float(np.float32(a))
    pr, mr, vr = S.adam_step(p0.astype(np.float64), g.astype(np.float64), m0.astype(np.float64), v0.astype(np.float64),
                             7, lr=f32(3e-3), beta1=f32(0.9), beta2=f32(0.999), eps=f32(1e-8))
    assert np.allclose(p.cpu().numpy(), pr, atol=1e-6, rtol=0)
    assert np.allclose(m.cpu().numpy(), mr, atol=1e-8, rtol=1e-6)
    assert np.allclose(v.cpu().numpy(), vr, atol=1e-9, rtol=1e-6)


def test_training_on_gpu_fits_a_known_function(env):
    """A few hundred Adam steps on the GPU fit f(x) = sum x^2 - cos(3 x_0) on [-1,1]^8."""
    sa, torch = env
    n, B = 8, 1024
    P = sa.mlp_param_count(n)
    p = torch.empty(P, dtype=torch.float32, device="cuda")
    sa.mlp_init(p, n, seed=1)
    m = torch.zeros_like(p)
    v = torch.zeros_like(p)
    gen = torch.Generator(device="cuda").manual_seed(0)
    f = lambda X: (X * X).sum(1) - torch.cos(3 * X[:, 0])
    Xv = torch.rand(4096, n, device="cuda", generator=gen) * 2 - 1
    tv = f(Xv)
    mu, sd = float(tv.mean()), float(tv.std())
    err0 = float(((sa.mlp_forward(p, n, Xv) * sd + mu - tv) ** 2).mean())
    for k in range(1, 401):
        X = torch.rand(B, n, device="cuda", generator=gen) * 2 - 1
        loss, g = sa.mlp_loss_grad(p, n, X, (f(X) - mu) / sd)
        sa.mlp_adam(p, g, m, v, k, lr=1e-3)
    err = float(((sa.mlp_forward(p, n, Xv) * sd + mu - tv) ** 2).mean())
    assert err < 0.02 * float(tv.var()) and err < 0.05 * err0, (err0, err, float(tv.var()))


@pytest.mark.parametrize("n,B", [(128, 128 * 152 * 2 + 77), (64, 5000), (100, 1000), (37, 1), (200, 300)])
def test_fused_forward_equals_two_gemm_path(env, n, B, monkeypatch):
    """The one-kernel forward pass (inputs padded to 64 or 128 columns) against the two
    GEMMs with fused epilogues: the same FP32 accumulators, the same BF16 rounding of
    the hidden layer and the same order of the head's sums, so equal bit for bit; at
    2 x 152 + 1 tiles every CTA of the persistent kernel runs more than one tile.
    n = 200 (248 padded columns) takes the two-GEMM path either way."""
    sa, torch = env
    P = sa.mlp_param_count(n)
    p = torch.empty(P, dtype=torch.float32, device="cuda")
    sa.mlp_init(p, n, seed=11)
    pn = p.cpu().numpy()
    o = S.unpack(pn, n)
    rng = np.random.default_rng(n + B)
    o[1][:] = rng.standard_normal(512) * 0.3
    o[3][:] = rng.standard_normal(512) * 0.3
    o[4][:] = rng.standard_normal(512)
    o[5][:] = -0.7
    p.copy_(torch.tensor(pn))
    X = torch.tensor(rng.uniform(-1, 1, (B, n)).astype(np.float32), device="cuda")
    y_fused = sa.mlp_forward(p, n, X).cpu().numpy()
    monkeypatch.setenv("SA_MLP_FUSED", "0")
    y_two = sa.mlp_forward(p, n, X).cpu().numpy()
    assert np.all(np.isfinite(y_fused))
    assert np.array_equal(y_fused, y_two), np.abs(y_fused - y_two).max()
    # and both against the FP64 oracle on a sample of rows
    rows = rng.choice(B, size=min(B, 64), replace=False)
    yr, _ = S.forward(_bf16_params(pn, n), _bf16(X.cpu().numpy()[rows]), n)
    assert np.abs(y_fused[rows] - yr).max() <= 1e-2 * (np.abs(yr).max() + 1.0)

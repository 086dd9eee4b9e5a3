"""TEST INFRASTRUCTURE ONLY: FP64 reference of the learned surrogate and of
two-stage delayed acceptance.  Only tests, the smoke check and the benchmark's
CPU-baseline leg may import this module; it shares no code with the CUDA path.

The surrogate is a multilayer perceptron f~(x) = w3 . g(W2 g(W1 x + b1) + b2) + b3
with g the erf form of GELU, g(z) = z/2 (1 + erf(z / sqrt 2)), fitted by the
mean squared error to standardised (x, f) pairs with Adam (Kingma & Ba, ICLR
2015).  Delayed acceptance (Christen & Fox, J. Comput. Graph. Stat. 2005) uses
f~ as a first Metropolis stage: a move passes stage 1 with probability
min(1, exp(-(f~(x') - f~(x)) / T)); only then is the true f evaluated and the
move accepted with probability min(1, exp(-[(f(x') - f(x)) - (f~(x') - f~(x))] / T)).
For a symmetric proposal the two stages together satisfy detailed balance
for exp(-f/T), whatever f~ is.  The paper itself has no surrogate.

Parameter vector layout (also the CUDA path's): W1 [H1 x n] row-major, b1 [H1],
W2 [H2 x H1] row-major, b2 [H2], w3 [H2], b3 [1].
"""
from __future__ import annotations

import math

import numpy as np

H1 = 512
H2 = 512
_SQRT2 = math.sqrt(2.0)
_INV_SQRT_2PI = 1.0 / math.sqrt(2.0 * math.pi)
_erf = np.vectorize(math.erf, otypes=[np.float64])


def n_params(n: int) -> int:
    return H1 * n + H1 + H2 * H1 + H2 + H2 + 1


def unpack(p: np.ndarray, n: int):
    """Views (W1, b1, W2, b2, w3, b3) into the flat parameter vector."""
    o = 0
    W1 = p[o:o + H1 * n].reshape(H1, n); o += H1 * n
    b1 = p[o:o + H1]; o += H1
    W2 = p[o:o + H2 * H1].reshape(H2, H1); o += H2 * H1
    b2 = p[o:o + H2]; o += H2
    w3 = p[o:o + H2]; o += H2
    b3 = p[o:o + 1]; o += 1
    assert o == p.size
    return W1, b1, W2, b2, w3, b3


def gelu(z):
    """GELU, erf form: z Phi(z) with Phi the standard normal CDF."""
    z = np.asarray(z, np.float64)
    return 0.5 * z * (1.0 + _erf(z / _SQRT2))


def gelu_grad(z):
    """d/dz of z Phi(z) = Phi(z) + z phi(z)."""
    z = np.asarray(z, np.float64)
    return 0.5 * (1.0 + _erf(z / _SQRT2)) + z * _INV_SQRT_2PI * np.exp(-0.5 * z * z)


def forward(p, X, n):
    """Rows of X (B x n) -> surrogate values (B,), with the intermediates."""
    W1, b1, W2, b2, w3, b3 = unpack(np.asarray(p, np.float64), n)
    X = np.asarray(X, np.float64)
    Z1 = X @ W1.T + b1
    A1 = gelu(Z1)
    Z2 = A1 @ W2.T + b2
    A2 = gelu(Z2)
    y = A2 @ w3 + b3[0]
    return y, (X, Z1, A1, Z2, A2)


def loss_and_grad(p, X, t, n):
    """L = (1 / 2B) sum (f~(x_b) - t_b)^2 and dL/dp by the chain rule, layer by layer."""
    W1, b1, W2, b2, w3, b3 = unpack(np.asarray(p, np.float64), n)
    y, (X, Z1, A1, Z2, A2) = forward(p, X, n)
    B = X.shape[0]
    r = y - np.asarray(t, np.float64)
    loss = 0.5 * float(r @ r) / B
    dy = r / B
    dw3 = A2.T @ dy
    db3 = np.array([dy.sum()])
    dZ2 = np.outer(dy, w3) * gelu_grad(Z2)
    dW2 = dZ2.T @ A1
    db2 = dZ2.sum(axis=0)
    dZ1 = (dZ2 @ W2) * gelu_grad(Z1)
    dW1 = dZ1.T @ X
    db1 = dZ1.sum(axis=0)
    g = np.concatenate([dW1.ravel(), db1, dW2.ravel(), db2, dw3, db3])
    return loss, g


def adam_step(p, g, m, v, t, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update at step t >= 1 (bias-corrected moments); returns (p, m, v)."""
    m = beta1 * m + (1.0 - beta1) * g
    v = beta2 * v + (1.0 - beta2) * g * g
    mh = m / (1.0 - beta1 ** t)
    vh = v / (1.0 - beta2 ** t)
    return p - lr * mh / (np.sqrt(vh) + eps), m, v


def init_params(n, seed=0):
    """He-style normal initialisation of the weights, zero biases (seeded)."""
    rng = np.random.default_rng([seed, n, 7])
    p = np.zeros(n_params(n))
    W1, b1, W2, b2, w3, b3 = unpack(p, n)
    W1[:] = rng.standard_normal(W1.shape) * math.sqrt(2.0 / n)
    W2[:] = rng.standard_normal(W2.shape) * math.sqrt(2.0 / H1)
    w3[:] = rng.standard_normal(w3.shape) * math.sqrt(1.0 / H2)
    return p


def da_decide(dFs, dF_true_fn, u_da, u3, T):
    """Two-stage decision for one proposal.  dFs = f~(x') - f~(x); dF_true_fn()
    evaluates f(x') - f(x) only when stage 1 passes.  Returns (accepted, evaluated)."""
    if not (dFs <= 0.0 or u_da < math.exp(-dFs / T)):
        return False, False
    r = dF_true_fn() - dFs
    return (r <= 0.0 or u3 < math.exp(-r / T)), True

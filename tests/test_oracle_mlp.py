"""Pins for the FP64 surrogate-network reference: analytic gradients against
central finite differences (with exact FP64 weights, so the BF16 rounding of
the kernels' operands does not blur the comparison), a hand-computed tiny
network, and the BF16 rounding rule against known bit patterns."""
import numpy as np

from oracle import mlp


def _setup(d=5, w=7, n=11, seed=3):
    r = np.random.default_rng(seed)
    p = r.standard_normal(mlp.n_params(d, w)) * 0.4
    x = r.standard_normal((n, d))
    t = r.standard_normal(n)
    norm = (r.standard_normal(d) * 0.1, 1.0 + r.random(d), 0.3, 1.7)
    return p, x, t, d, w, norm


def test_gradient_matches_finite_differences():
    p, x, t, d, w, norm = _setup()
    loss, g = mlp.loss_and_grad(p, x, t, d, w, norm, bf16=False)
    h = 1e-6
    fd = np.empty_like(p)
    for k in range(p.size):
        e = np.zeros_like(p)
        e[k] = h
        lp, _ = mlp.loss_and_grad(p + e, x, t, d, w, norm, bf16=False)
        lm, _ = mlp.loss_and_grad(p - e, x, t, d, w, norm, bf16=False)
        fd[k] = (lp - lm) / (2 * h)
    np.testing.assert_allclose(g, fd, rtol=1e-6, atol=1e-9)


def test_tiny_network_by_hand():
    """d = 1, w = 1: y = w3 tanh(W2 tanh(W1 xn + b1) + b2) + b3 (identity norm)."""
    W1, b1, W2, b2, w3, b3 = 0.5, -0.25, 2.0, 0.125, -1.5, 0.75
    p = np.array([W1, b1, W2, b2, w3, b3])
    x = np.array([[0.8]])
    norm = (np.zeros(1), np.ones(1), 0.0, 1.0)
    y, _ = mlp.forward(p, x, 1, 1, norm, bf16=False)
    h1 = np.tanh(W1 * 0.8 + b1)
    want = w3 * np.tanh(W2 * h1 + b2) + b3
    assert y[0] == want


def test_bf16_rounding():
    vals = np.array([1.0, 1.0 + 2**-8, 1.0 + 2**-9, 1.0 + 3 * 2**-9, -2.5], dtype=np.float32)
    got = mlp.bf16_round(vals)
    # BF16 spacing at 1 is 2^-7: 1 + 2^-8 is a tie (to even: 1), 1 + 3 2^-9 rounds up
    np.testing.assert_array_equal(got, [1.0, 1.0, 1.0, 1.0 + 2**-7, -2.5])

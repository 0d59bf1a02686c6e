"""Pins of the warm-start network reference (oracle/mlp.py).

The gradient is checked against central finite differences of the loss; the
forward pass against a closed form on a one-unit case; Adam against its first
step, which moves every parameter by lr * sign(g) (bias correction makes
m_hat = g and v_hat = g^2).  bfloat16 rounding against bit patterns.
"""
import numpy as np
import pytest

from oracle import mlp


def _case(n_in=5, hidden=6, N=7, seed=0):
    rng = np.random.default_rng(seed)
    p = rng.standard_normal(mlp.n_params(n_in, hidden)) * 0.5
    X = rng.standard_normal((N, n_in))
    T = rng.standard_normal((N, 2))
    w = rng.uniform(0.5, 2.0, N)
    return p, X, T, w, hidden


def test_gradient_matches_finite_differences():
    p, X, T, w, H = _case()
    L, g = mlp.loss_grad(p, X, T, w, H)
    h = 1e-6
    fd = np.empty_like(p)
    for k in range(p.size):
        e = np.zeros_like(p)
        e[k] = h
        fd[k] = (mlp.loss_grad(p + e, X, T, w, H)[0] - mlp.loss_grad(p - e, X, T, w, H)[0]) / (2 * h)
    assert np.abs(g - fd).max() < 1e-7 * max(1.0, np.abs(fd).max())


def test_loss_matches_forward():
    p, X, T, w, H = _case(seed=3)
    y = mlp.forward(p, X, H)
    L, _ = mlp.loss_grad(p, X, T, w, H)
    assert L == pytest.approx((w * ((y - T) ** 2).sum(1)).sum() / w.sum(), rel=1e-14)


def test_one_unit_closed_form():
    # n_in = 1, hidden = 1: y_c = W3_c tanh(W2 tanh(W1 x + b1) + b2) + b3_c
    p = np.array([0.7, -0.2, 1.3, 0.4, 2.0, -1.0, 0.25, 0.5])
    x = 0.9
    a1 = np.tanh(0.7 * x - 0.2)
    a2 = np.tanh(1.3 * a1 + 0.4)
    y = mlp.forward(p, np.array([[x]]), 1)[0]
    assert y == pytest.approx([2.0 * a2 + 0.25, -1.0 * a2 + 0.5], rel=1e-15)


def test_first_adam_step_is_signed_lr():
    rng = np.random.default_rng(1)
    p = rng.standard_normal(20)
    g = rng.standard_normal(20)
    p1, m, v = mlp.adam_step(p, g, np.zeros(20), np.zeros(20), 1, lr=1e-2, eps=0.0)
    assert np.allclose(p1, p - 1e-2 * np.sign(g), rtol=0, atol=1e-15)


def test_round_bf16():
    a = np.array([1.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -9, -3.1415926, 1e-3], dtype=np.float32)
    r = mlp.round_bf16(a)
    assert r[0] == 1.0
    assert r[1] == 1.0                     # halfway between 1 and 1 + 2^-7: ties to even
    assert r[2] == np.float32(1.0 + 2 ** -7)
    assert (r.view(np.uint32) & 0xFFFF == 0).all()
    assert np.abs(r - a).max() <= np.abs(a).max() * 2 ** -8


def test_bf16_forward_reduces_to_exact_when_rounding_is_the_identity():
    """Inputs that bfloat16 represents and a first layer whose activations it
    represents (W1 = 0, b1 = atanh(v) with v bfloat16 values): the rounded
    network is the exact one, whatever the other layers."""
    rng = np.random.default_rng(7)
    n_in, H, N = 5, 8, 9
    p = rng.standard_normal(mlp.n_params(n_in, H)) * 0.5
    W1, b1 = mlp.unpack(p, n_in, H)[:2]
    v = mlp.round_bf16(rng.uniform(-0.9, 0.9, H).astype(np.float32)).astype(np.float64)
    W1[:] = 0.0
    b1[:] = np.arctanh(v)
    X = mlp.round_bf16(rng.standard_normal((N, n_in)).astype(np.float32)).astype(np.float64)
    a1 = mlp.hidden1(p, X, H, bf16=True)
    assert np.abs(a1 - v).max() < 1e-15
    assert np.array_equal(mlp.round_bf16(a1.astype(np.float32)), np.broadcast_to(v.astype(np.float32), (N, H)))
    y, yb = mlp.forward(p, X, H), mlp.forward(p, X, H, bf16=True)
    assert np.abs(y - yb).max() < 1e-14 * np.abs(y).max()


def test_bf16_forward_and_gradient_within_rounding_bounds():
    """The rounded network differs from the exact one by the bfloat16
    rounding (relative 2^-9 per rounded value): the outputs by at most
    |W3| |W2| (2^-9 |a1| + |W1| 2^-9 |x|) entrywise (tanh' <= 1), the
    gradient by a few 2^-8 of its scale; a transposed operand or a dropped
    term is an O(1) change."""
    n_in, H, N = 6, 16, 40
    rng = np.random.default_rng(11)
    p = rng.standard_normal(mlp.n_params(n_in, H)) * 0.4
    X = rng.standard_normal((N, n_in))
    T = rng.standard_normal((N, 2))
    w = rng.uniform(0.5, 2.0, N)
    W1, b1, W2, b2, W3, b3 = mlp.unpack(p, n_in, H)
    a1 = np.tanh(X @ W1.T + b1)
    bound = (2.0 ** -9 * np.abs(a1) + 2.0 ** -9 * np.abs(X) @ np.abs(W1).T) @ np.abs(W2).T @ np.abs(W3).T
    dy = np.abs(mlp.forward(p, X, H, bf16=True) - mlp.forward(p, X, H))
    assert (dy <= 1.01 * bound + 1e-15).all()
    assert dy.max() > 0.0
    L, g = mlp.loss_grad(p, X, T, w, H)
    Lb, gb = mlp.loss_grad(p, X, T, w, H, bf16=True)
    assert abs(Lb - L) <= 1e-2 * L
    sizes = [H * n_in, H, H * H, H, 2 * H, 2]
    o = 0
    for k in sizes:  # every parameter block: the rounded gradient tracks the exact one
        ge, gr = g[o:o + k], gb[o:o + k]
        assert np.abs(gr - ge).max() <= 2e-2 * np.abs(ge).max(), o
        o += k

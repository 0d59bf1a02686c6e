"""Reference of the warm-start network (test infrastructure; see the package
docstring for who may import it).

The warm start has no counterpart in the paper: it is a per-node multilayer
perceptron written here from its definition, in numpy float64:

    a1 = tanh(W1 x + b1),  a2 = tanh(W2 a1 + b2),  y = W3 a2 + b3,

parameters one flat vector [W1 (row-major), b1, W2, b2, W3, b3], loss
L = sum_i w_i |y_i - t_i|^2 / sum_i w_i, its gradient by the chain rule, and
one bias-corrected Adam step (Kingma & Ba 2015, Algorithm 1).  Pinned in
tests/test_oracle_mlp.py against central finite differences and against
closed forms on tiny cases.

With bf16=True the same network is evaluated with the bfloat16 roundings of
a tensor-core implementation, whose matrix products take bfloat16 operands
and accumulate in float32 (the roundings are the definition; every other
step is exact):

    forward   xr = bf(x); a1r = bf(tanh(W1 xr + b1)); a2 = tanh(W2 a1r + b2);
              y = W3 a2 + b3
    gradient  with e = y - t and the unnormalised d3 = 2 w e (the loss and
              every sum below are divided by sum_i w_i at the end):
              gW3 = bf(d3)^T bf(a2), gb3 = sum d3;
              d2 = (d3 W3) (1 - a2^2), gW2 = bf(d2)^T a1r, gb2 = sum bf(d2);
              d1 = (bf(d2) W2) (1 - a1r^2), gW1 = bf(d1)^T xr, gb1 = sum bf(d1)

bf = round to the nearest bfloat16 (ties to even) of the float32 value.
"""
import numpy as np


def unpack(p, n_in, hidden):
    """Views (W1, b1, W2, b2, W3, b3) of the flat parameter vector p."""
    p = np.asarray(p, dtype=np.float64)
    sizes = [(hidden, n_in), (hidden,), (hidden, hidden), (hidden,), (2, hidden), (2,)]
    out, o = [], 0
    for s in sizes:
        k = int(np.prod(s))
        out.append(p[o:o + k].reshape(s))
        o += k
    if o != p.size:
        raise ValueError("parameter vector has the wrong length")
    return out


def n_params(n_in, hidden):
    return hidden * n_in + hidden + hidden * hidden + hidden + 2 * hidden + 2


def _bf(a):
    return round_bf16(np.asarray(a, dtype=np.float64).astype(np.float32)).astype(np.float64)


def forward(p, X, hidden, bf16=False):
    """y (N x 2) for inputs X (N x n_in); bf16: with the bfloat16 roundings
    of the module docstring."""
    X = np.asarray(X, dtype=np.float64)
    W1, b1, W2, b2, W3, b3 = unpack(p, X.shape[1], hidden)
    if bf16:
        X = _bf(X)
    a1 = np.tanh(X @ W1.T + b1)
    if bf16:
        a1 = _bf(a1)
    a2 = np.tanh(a1 @ W2.T + b2)
    return a2 @ W3.T + b3


def hidden1(p, X, hidden, bf16=False):
    """The first hidden layer a1 (N x hidden), before any rounding of it."""
    X = np.asarray(X, dtype=np.float64)
    W1, b1 = unpack(p, X.shape[1], hidden)[:2]
    if bf16:
        X = _bf(X)
    return np.tanh(X @ W1.T + b1)


def loss_grad(p, X, T, w, hidden, bf16=False):
    """(L, dL/dp) of L = sum_i w_i |y_i - t_i|^2 / sum_i w_i; bf16: the
    gradient with the bfloat16 roundings of the module docstring."""
    X = np.asarray(X, dtype=np.float64)
    T = np.asarray(T, dtype=np.float64)
    w = np.asarray(w, dtype=np.float64)
    W1, b1, W2, b2, W3, b3 = unpack(p, X.shape[1], hidden)
    bf = _bf if bf16 else (lambda a: a)
    X = bf(X)
    a1 = bf(np.tanh(X @ W1.T + b1))
    a2 = np.tanh(a1 @ W2.T + b2)
    y = a2 @ W3.T + b3
    ws = w.sum()
    e = y - T
    L = float((w * (e * e).sum(1)).sum() / ws)
    d3 = 2.0 * w[:, None] * e               # dL/dy times sum_i w_i
    gW3, gb3 = bf(d3).T @ bf(a2), d3.sum(0)
    d2 = bf((d3 @ W3) * (1.0 - a2 * a2))    # dL/dz2 times sum_i w_i
    gW2, gb2 = d2.T @ a1, d2.sum(0)
    d1 = bf((d2 @ W2) * (1.0 - a1 * a1))    # dL/dz1 times sum_i w_i
    gW1, gb1 = d1.T @ X, d1.sum(0)
    g = np.concatenate([gW1.ravel(), gb1, gW2.ravel(), gb2, gW3.ravel(), gb3]) / ws
    return L, g


def adam_step(p, g, m, v, t, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam step at step number t (1-based); returns (p, m, v)."""
    m = beta1 * m + (1.0 - beta1) * g
    v = beta2 * v + (1.0 - beta2) * g * g
    mh = m / (1.0 - beta1 ** t)
    vh = v / (1.0 - beta2 ** t)
    return p - lr * mh / (np.sqrt(vh) + eps), m, v


def round_bf16(a):
    """Round float32 values to the nearest bfloat16 (ties to even), returned
    as float32: the weights the network kernels read."""
    a = np.ascontiguousarray(a, dtype=np.float32)
    u = a.view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return (r.astype(np.uint32)).view(np.float32)

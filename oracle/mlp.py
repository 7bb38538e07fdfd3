"""FP64 numpy oracle for the cost model's multi-layer perceptron (test infrastructure only).

The network has no counterpart in the paper: it is the learned cost model that picks the
TOCAB block count, the per-subgraph load-balancing variant and the push/pull direction
(Sec. 3.1 block size trade-off, Sec. 3.2 load balancing choice; Sec. 4.3 shows the block
size is a measured trade-off).  Architecture, written out plainly:

    h1 = relu(x @ W1 + b1)          x: [N, 16]
    h2 = relu(h1 @ W2 + b2)         hidden width 64
    z  = h2 @ W3 + b3               z: [N, sum(heads)]
    loss = mean_n sum_k CE(softmax(z[n, head_k]), y[n, k])

Parameters are a dict {W1 [16,64], b1 [64], W2 [64,64], b2 [64], W3 [64,H], b3 [H]}.
``heads`` lists the class count of each head, e.g. (7, 3, 2).
"""
from __future__ import annotations

import numpy as np


def _split(heads):
    offs = np.cumsum([0] + list(heads))
    return [(int(offs[k]), int(offs[k + 1])) for k in range(len(heads))]


def mlp_forward(params, x):
    x = np.asarray(x, np.float64)
    a1 = x @ params["W1"] + params["b1"]
    h1 = np.maximum(a1, 0.0)
    a2 = h1 @ params["W2"] + params["b2"]
    h2 = np.maximum(a2, 0.0)
    z = h2 @ params["W3"] + params["b3"]
    return z, {"x": x, "a1": a1, "h1": h1, "a2": a2, "h2": h2}


def _log_softmax(z):
    m = z.max(axis=1, keepdims=True)
    return z - m - np.log(np.exp(z - m).sum(axis=1, keepdims=True))


def mlp_loss(params, x, y, heads):
    """Mean over samples of the summed cross-entropy of every head."""
    z, _ = mlp_forward(params, x)
    y = np.asarray(y, np.int64)
    N = z.shape[0]
    total = 0.0
    for k, (lo, hi) in enumerate(_split(heads)):
        ls = _log_softmax(z[:, lo:hi])
        total += -ls[np.arange(N), y[:, k]].sum()
    return total / N


def mlp_backward(params, x, y, heads):
    """Gradients of ``mlp_loss`` with respect to every parameter (chain rule, FP64)."""
    z, c = mlp_forward(params, x)
    y = np.asarray(y, np.int64)
    N = z.shape[0]
    dz = np.zeros_like(z)
    for k, (lo, hi) in enumerate(_split(heads)):
        p = np.exp(_log_softmax(z[:, lo:hi]))
        p[np.arange(N), y[:, k]] -= 1.0
        dz[:, lo:hi] = p / N
    g = {}
    g["W3"] = c["h2"].T @ dz
    g["b3"] = dz.sum(axis=0)
    dh2 = dz @ params["W3"].T
    da2 = dh2 * (c["a2"] > 0)
    g["W2"] = c["h1"].T @ da2
    g["b2"] = da2.sum(axis=0)
    dh1 = da2 @ params["W2"].T
    da1 = dh1 * (c["a1"] > 0)
    g["W1"] = c["x"].T @ da1
    g["b1"] = da1.sum(axis=0)
    return g


def adam_step(params, grads, m, v, t, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (Kingma & Ba 2015, Algorithm 1), returns new (params, m, v)."""
    out_p, out_m, out_v = {}, {}, {}
    for k in params:
        out_m[k] = beta1 * m[k] + (1 - beta1) * grads[k]
        out_v[k] = beta2 * v[k] + (1 - beta2) * grads[k] ** 2
        mhat = out_m[k] / (1 - beta1 ** t)
        vhat = out_v[k] / (1 - beta2 ** t)
        out_p[k] = params[k] - lr * mhat / (np.sqrt(vhat) + eps)
    return out_p, out_m, out_v

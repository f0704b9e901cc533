"""FP64 oracle of the neural regression of Sec. 2: the NN+ search space (eq. (e:nnp)),
Algorithm 1 (BaseAlg: mini-batch Adam, output ReLU off for the first half of the
epochs, closed-form refit of the last layer at epoch floor(E/2), best parameters kept
on the full sample) inside Algorithm 2 (backward learning over the pricing dates,
each date warm-started from the next one).

TEST INFRASTRUCTURE ONLY (see the package docstring). Plain numpy in binary64.

Parameters of an h = 2 hidden-layer network of width u on d inputs:
  W1 [u, d], b1 [u], W2 [u, u], b2 [u], w3 [u], b3 (scalar), mu (scalar)
zeta(z) = w3 . relu(W2 relu(W1 z + b1) + b2) + b3 and the NN+ output is
zeta(z)^+ + mu (pos = 1) or zeta(z) + mu (pos = 0).
"""
from __future__ import annotations

from typing import Dict, List, Sequence

import numpy as np

NAMES = ("W1", "b1", "W2", "b2", "w3", "b3", "mu")


def standardize(X: np.ndarray):
    """Per-feature mean 0 / variance 1 over the samples (X is [M, d])."""
    mu = X.mean(axis=0)
    sd = X.std(axis=0)
    sd = np.where(sd > 0, sd, 1.0)
    return (X - mu) / sd, mu, sd


def forward(p: Dict[str, np.ndarray], Z: np.ndarray, pos: int):
    a1 = Z @ p["W1"].T + p["b1"]
    h1 = np.maximum(a1, 0.0)
    a2 = h1 @ p["W2"].T + p["b2"]
    h2 = np.maximum(a2, 0.0)
    out = h2 @ p["w3"] + p["b3"]
    pred = (np.maximum(out, 0.0) if pos else out) + p["mu"]
    return pred, (h1, h2, out)


def loss(p, Z, y, pos) -> float:
    pred, _ = forward(p, Z, pos)
    return float(np.mean((pred - y) ** 2))


def grads(p, Z, y, pos):
    """Gradient of mean((pred - y)^2) with respect to every parameter (backpropagation)."""
    B = Z.shape[0]
    pred, (h1, h2, out) = forward(p, Z, pos)
    dpred = 2.0 * (pred - y) / B
    dout = dpred * ((out > 0).astype(np.float64) if pos else 1.0)
    g = {"mu": np.array(dpred.sum()), "b3": np.array(dout.sum()), "w3": h2.T @ dout}
    dh2 = np.outer(dout, p["w3"]) * (h2 > 0)
    g["W2"] = dh2.T @ h1
    g["b2"] = dh2.sum(axis=0)
    dh1 = (dh2 @ p["W2"]) * (h1 > 0)
    g["W1"] = dh1.T @ Z
    g["b1"] = dh1.sum(axis=0)
    return g


class Adam:
    """Kingma & Ba: m <- b1 m + (1-b1) g, v <- b2 v + (1-b2) g^2,
    theta <- theta - lr (m / (1-b1^t)) / (sqrt(v / (1-b2^t)) + eps)."""

    def __init__(self, p, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
        self.lr, self.b1, self.b2, self.eps = lr, beta1, beta2, eps
        self.m = {k: np.zeros_like(v, dtype=np.float64) for k, v in p.items()}
        self.v = {k: np.zeros_like(v, dtype=np.float64) for k, v in p.items()}
        self.t = 0

    def step(self, p, g):
        self.t += 1
        for k in NAMES:
            self.m[k] = self.b1 * self.m[k] + (1 - self.b1) * g[k]
            self.v[k] = self.b2 * self.v[k] + (1 - self.b2) * g[k] ** 2
            mh = self.m[k] / (1 - self.b1 ** self.t)
            vh = self.v[k] / (1 - self.b2 ** self.t)
            p[k] = p[k] - self.lr * mh / (np.sqrt(vh) + self.eps)


def refit_last_layer(p, Z, y):
    """Closed-form least squares of (w3, b3) on the last hidden layer with mu fixed and
    no output ReLU (the tuning step of Algorithm 1 at epoch floor(E/2))."""
    _, (h1, h2, out) = forward(p, Z, 0)
    A = np.concatenate([h2, np.ones((h2.shape[0], 1))], axis=1)
    sol, *_ = np.linalg.lstsq(A, y - p["mu"], rcond=None)
    p["w3"] = sol[:-1].copy()
    p["b3"] = np.array(sol[-1])


def batches(M: int, n_batches: int) -> List[slice]:
    """Contiguous path ranges (the memory-contiguous batch layout of Sec. 3.2)."""
    edges = [(b * M) // n_batches for b in range(n_batches + 1)]
    return [slice(edges[b], edges[b + 1]) for b in range(n_batches)]


def base_alg(p0, Z, y, n_batches=32, epochs=8, lr=1e-3, trace=None):
    """Algorithm 1 (BaseAlg) at one date; returns the best parameters and their loss."""
    p = {k: np.array(v, dtype=np.float64, copy=True) for k, v in p0.items()}
    opt = Adam(p, lr=lr)
    pos = 0
    best, best_p = np.inf, None
    for epoch in range(1, epochs + 1):
        for sl in batches(Z.shape[0], n_batches):
            opt.step(p, grads(p, Z[sl], y[sl], pos))
        if epoch == epochs // 2:
            refit_last_layer(p, Z, y)
            pos = 1
        full = loss(p, Z, y, 1)
        if trace is not None:
            trace.append(full)
        if full < best:
            best = full
            best_p = {k: v.copy() for k, v in p.items()}
    return best_p, best


def backward_alg(p_init, features: Sequence[np.ndarray], targets: Sequence[np.ndarray],
                 dates: Sequence[int], **kw):
    """Algorithm 2: dates in decreasing order, each BaseAlg warm-started from the
    parameters of the date after it. features[i] is [d, M] (raw state), targets[i] [M].
    Returns {date: (params, best loss, predictions [M])}."""
    out = {}
    p = p_init
    for i in sorted(dates, reverse=True):
        Z, _, _ = standardize(np.asarray(features[i], dtype=np.float64).T)
        y = np.asarray(targets[i], dtype=np.float64)
        p, best = base_alg(p, Z, y, **kw)
        out[i] = (p, best, forward(p, Z, 1)[0])
    return out


def bf16(x):
    """Round to bfloat16 (8-bit significand), round-to-nearest-even, returned as float64."""
    u = np.ascontiguousarray(np.asarray(x, dtype=np.float32)).view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def grads_bf16(p, Z, y, pos):
    """The gradient of `grads`, with the operands of the four matrix products rounded to
    bfloat16 where a tensor-core implementation feeds them (inputs, W1, W2, the first
    hidden layer, dH2 and dH1); every sum and every other operation in binary64."""
    B = Z.shape[0]
    Zb, W1b, W2b = bf16(Z), bf16(p["W1"]), bf16(p["W2"])
    a1 = Zb @ W1b.T + p["b1"]
    h1 = np.maximum(a1, 0.0)
    h1b = bf16(h1)
    a2 = h1b @ W2b.T + p["b2"]
    h2 = np.maximum(a2, 0.0)
    out = h2 @ p["w3"] + p["b3"]
    pred = (np.maximum(out, 0.0) if pos else out) + p["mu"]
    dpred = 2.0 * (pred - y) / B
    dout = dpred * ((out > 0).astype(np.float64) if pos else 1.0)
    g = {"mu": np.array(dpred.sum()), "b3": np.array(dout.sum()), "w3": h2.T @ dout}
    dh2b = bf16(np.outer(dout, p["w3"]) * (h2 > 0))
    g["W2"] = dh2b.T @ h1b
    g["b2"] = dh2b.sum(axis=0)
    dh1b = bf16((dh2b @ W2b) * (h1 > 0))
    g["W1"] = dh1b.T @ Zb
    g["b1"] = dh1b.sum(axis=0)
    return g

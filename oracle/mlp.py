"""Learned reflection filters: FP64 forward/backward of the direction -> filter network and
its Adam update.  TEST INFRASTRUCTURE ONLY (part of the oracle): only tests/, the smoke test
and the benchmark's CPU baseline use it; it shares no code with the CUDA path.

The paper fits one reflection filter g_i >= 0 per measured direction (Sec. III, Eq. 3 with
G >= 0; Algorithm 1).  The learned part replaces the table lookup by a small network that
maps a direction to a filter, so that directions between the measured grid get filters too:

    x   = (sin az, cos az, sin el, cos el, ear)          ear = -1 (left), +1 (right)
    h1  = relu(W1 x + b1)          W1: 256 x 5
    h2  = relu(W2 h1 + b2)         W2: 256 x 256
    h3  = relu(W3 h2 + b3)         W3: 256 x 256
    g   = softplus(W4 h3 + b4)     W4: Lg x 256     (softplus keeps every tap >= 0, as G >= 0)

trained by least squares on the reflection rows that the factorization (Algorithm 1)
produces: L = 1/(2B) sum_b ||g_b - G_b||^2 over a batch of B rows.  Updates use Adam
(Kingma & Ba, "Adam: A method for stochastic optimization", 2015, Algorithm 1), with the
bias corrections written out.

Parameters travel as one flat vector in the order W1, b1, W2, b2, W3, b3, W4, b4, each
weight matrix row-major [out][in] (the layout the CUDA library uses too; it is an
interface, not shared code).  Library primitives used as steps: numpy matrix products.
"""
from __future__ import annotations

import numpy as np

N_IN = 5
HIDDEN = 256
N_HIDDEN_LAYERS = 3


def layer_sizes(refl_len: int):
    return [N_IN] + [HIDDEN] * N_HIDDEN_LAYERS + [refl_len]


def param_count(refl_len: int) -> int:
    s = layer_sizes(refl_len)
    return sum(s[i + 1] * s[i] + s[i + 1] for i in range(len(s) - 1))


def unpack(params, refl_len: int):
    """Flat vector -> [(W, b)] per layer (views, FP64)."""
    p = np.asarray(params, dtype=np.float64)
    s = layer_sizes(refl_len)
    out, o = [], 0
    for i in range(len(s) - 1):
        W = p[o:o + s[i + 1] * s[i]].reshape(s[i + 1], s[i])
        o += s[i + 1] * s[i]
        b = p[o:o + s[i + 1]]
        o += s[i + 1]
        out.append((W, b))
    assert o == p.size
    return out


def features(az, el, ear) -> np.ndarray:
    """Network input per row: (sin az, cos az, sin el, cos el, ear); angles in radians."""
    az = np.asarray(az, dtype=np.float64)
    el = np.asarray(el, dtype=np.float64)
    ear = np.asarray(ear, dtype=np.float64)
    return np.stack([np.sin(az), np.cos(az), np.sin(el), np.cos(el), ear], axis=1)


def relu(z):
    return np.maximum(z, 0.0)


def softplus(z):
    """log(1 + e^z), evaluated without overflow as max(z, 0) + log1p(e^-|z|)."""
    z = np.asarray(z, dtype=np.float64)
    return np.maximum(z, 0.0) + np.log1p(np.exp(-np.abs(z)))


def sigmoid(z):
    z = np.asarray(z, dtype=np.float64)
    e = np.exp(-np.abs(z))
    return np.where(z >= 0, 1.0 / (1.0 + e), e / (1.0 + e))


def forward(params, X, refl_len: int):
    """Returns (g, cache) for inputs X [B][5]; cache holds every layer's input and
    pre-activation."""
    layers = unpack(params, refl_len)
    h = np.asarray(X, dtype=np.float64)
    cache = []
    for i, (W, b) in enumerate(layers):
        z = h @ W.T + b
        cache.append((h, z))
        h = softplus(z) if i == len(layers) - 1 else relu(z)
    return h, cache


def loss(params, X, T, refl_len: int) -> float:
    g, _ = forward(params, X, refl_len)
    d = g - np.asarray(T, dtype=np.float64)
    return 0.5 * float(np.sum(d * d)) / max(len(d), 1)


def backward(params, cache, dG, refl_len: int) -> np.ndarray:
    """Gradient of sum(dG * g) w.r.t. the flat parameter vector (chain rule, layer by layer
    from the output: softplus' = sigmoid, relu' = [z > 0])."""
    layers = unpack(params, refl_len)
    grads = []
    d = np.asarray(dG, dtype=np.float64)
    for i in range(len(layers) - 1, -1, -1):
        W, _ = layers[i]
        h_in, z = cache[i]
        dz = d * (sigmoid(z) if i == len(layers) - 1 else (z > 0))
        grads.append((dz.T @ h_in, dz.sum(axis=0)))
        d = dz @ W
    grads.reverse()
    return np.concatenate([np.concatenate([gW.ravel(), gb]) for gW, gb in grads])


def loss_and_grad(params, X, T, refl_len: int):
    """L = 1/(2B) sum ||g - T||^2 and dL/dparams."""
    g, cache = forward(params, X, refl_len)
    B = max(len(g), 1)
    d = (g - np.asarray(T, dtype=np.float64)) / B
    return 0.5 * float(np.sum((g - T) ** 2)) / B, backward(params, cache, d, refl_len)


def adam_step(p, g, m, v, t: int, lr: float, beta1: float = 0.9, beta2: float = 0.999,
              eps: float = 1e-8):
    """One Adam update (step t >= 1): returns new (p, m, v)."""
    p, g = np.asarray(p, np.float64), np.asarray(g, np.float64)
    m = beta1 * np.asarray(m, np.float64) + (1.0 - beta1) * g
    v = beta2 * np.asarray(v, np.float64) + (1.0 - beta2) * g * g
    m_hat = m / (1.0 - beta1 ** t)
    v_hat = v / (1.0 - beta2 ** t)
    return p - lr * m_hat / (np.sqrt(v_hat) + eps), m, v


def numeric_grad(params, X, T, refl_len: int, idx, h: float = 1e-6) -> np.ndarray:
    """Central finite differences of loss() at the parameter indices idx."""
    p = np.array(params, dtype=np.float64)
    out = np.empty(len(idx))
    for n, i in enumerate(idx):
        old = p[i]
        p[i] = old + h
        lp = loss(p, X, T, refl_len)
        p[i] = old - h
        lm = loss(p, X, T, refl_len)
        p[i] = old
        out[n] = (lp - lm) / (2 * h)
    return out

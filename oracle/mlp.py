"""FP64 emission-surrogate MLP (test infrastructure only; the paper has no counterpart).

Inputs x: 7 standardised features of (F, T, phi_w, R); layers 7 -> 128 -> 128 -> 128 -> 2 with
GELU(z) = z/2 (1 + erf(z/sqrt 2)) on the hidden layers;
outputs (log10 J [A/m^2], eps_N = P_N/J [eV]) standardised by (y - ym)/ys.
Loss: mean over the batch of the sum over the two outputs of (y_hat - y)^2 / 2.
"""
import math

import numpy as np
import scipy.special as ss

SIZES = (7, 128, 128, 128, 2)


def gelu(z):
    return 0.5 * z * (1.0 + ss.erf(z / math.sqrt(2.0)))


def gelu_grad(z):
    return 0.5 * (1.0 + ss.erf(z / math.sqrt(2.0))) + z * np.exp(-0.5 * z * z) / math.sqrt(2.0 * math.pi)


def init_params(rng):
    params = []
    for a, b in zip(SIZES[:-1], SIZES[1:]):
        params.append((rng.normal(0.0, math.sqrt(2.0 / a), size=(b, a)), np.zeros(b)))
    return params


def forward(params, x):
    """x: (N, 4) standardised inputs; returns output (N, 2) and the cache for backward."""
    h = np.asarray(x, dtype=np.float64)
    cache = []
    for li, (W, b) in enumerate(params):
        z = h @ W.T + b
        cache.append((h, z))
        h = gelu(z) if li < len(params) - 1 else z
    return h, cache


def loss_and_grad(params, x, y):
    out, cache = forward(params, x)
    n = len(x)
    d = (out - y) / n
    loss = 0.5 * np.sum((out - y) ** 2) / n
    grads = [None] * len(params)
    for li in range(len(params) - 1, -1, -1):
        h, z = cache[li]
        if li < len(params) - 1:
            d = d * gelu_grad(z)
        W, _ = params[li]
        grads[li] = (d.T @ h, d.sum(axis=0))
        d = d @ W
    return loss, grads


def adam_update(params, grads, state, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam step (Kingma & Ba); state = dict(t, m, v)."""
    state["t"] += 1
    t = state["t"]
    out = []
    for i, ((W, b), (gW, gb)) in enumerate(zip(params, grads)):
        new = []
        for j, (p, g) in enumerate(((W, gW), (b, gb))):
            key = (i, j)
            m = beta1 * state["m"].get(key, 0.0) + (1 - beta1) * g
            v = beta2 * state["v"].get(key, 0.0) + (1 - beta2) * g * g
            state["m"][key], state["v"][key] = m, v
            mh = m / (1 - beta1 ** t)
            vh = v / (1 - beta2 ** t)
            new.append(p - lr * mh / (np.sqrt(vh) + eps))
        out.append(tuple(new))
    return out

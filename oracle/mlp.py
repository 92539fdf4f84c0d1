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


def bf16(a):
    """Round to bfloat16 (8-bit significand, round to nearest even) through float32, returned as
    float64: the storage format of the tensor-core operands."""
    u = np.asarray(a, dtype=np.float32).view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def bf16_tie_distance(a):
    """Distance from a to the nearest bfloat16 rounding boundary (midpoint of two neighbouring
    bfloat16 values): a perturbation smaller than this leaves bf16(a) unchanged."""
    a = np.abs(np.asarray(a, dtype=np.float64))
    r = bf16(a)
    e = np.floor(np.log2(np.maximum(r, 1e-300)))
    ulp = 2.0 ** (e - 7)                         # spacing above r; below a power of two it halves
    lo_mid, hi_mid = r - 0.5 * ulp * np.where(r == 2.0 ** e, 0.5, 1.0), r + 0.5 * ulp
    return np.where(a > 0, np.minimum(np.abs(a - lo_mid), np.abs(hi_mid - a)), 0.0)


def near_bf16_tie(a, rel=1e-5):
    """True where a lies within rel |a| of a bfloat16 rounding boundary (the midpoint of two
    neighbouring bfloat16 values): there a float32 evaluation of a may round the other way."""
    a = np.asarray(a, dtype=np.float64)
    lo = bf16(a * (1 - rel))
    hi = bf16(a * (1 + rel))
    return lo != hi


def init_params(rng):
    params = []
    for a, b in zip(SIZES[:-1], SIZES[1:]):
        params.append((rng.normal(0.0, math.sqrt(2.0 / a), size=(b, a)), np.zeros(b)))
    return params


# Layers whose products run on BF16 operands in the mixed-precision form: the two hidden
# 128 x 128 layers (indices 1 and 2).  Their inputs (the activations of layers 0 and 1) and, in
# the backward pass, the gradients they multiply are rounded to BF16.
BF16_LAYERS = (1, 2)


def forward(params, x, bf16_operands=False):
    """x: (N, 7) standardised inputs; returns output (N, 2) and the cache for backward.
    bf16_operands: the activations that feed the BF16 layers are rounded to BF16 (the weights of
    those layers are passed already rounded); every sum is still taken in float64."""
    h = np.asarray(x, dtype=np.float64)
    cache = []
    for li, (W, b) in enumerate(params):
        if bf16_operands and li in BF16_LAYERS:
            h = bf16(h)
        z = h @ W.T + b
        cache.append((h, z))
        h = gelu(z) if li < len(params) - 1 else z
    return h, cache


def loss_and_grad(params, x, y, bf16_operands=False):
    """Loss and gradients.  bf16_operands: as in forward, and the back-propagated gradient that
    enters a BF16 layer's two products (its weight gradient and the gradient of its input) is
    rounded to BF16, while its bias gradient sums the unrounded values."""
    out, cache = forward(params, x, bf16_operands)
    n = len(x)
    d = (out - y) / n
    loss = 0.5 * np.sum((out - y) ** 2) / n
    grads = [None] * len(params)
    for li in range(len(params) - 1, -1, -1):
        h, z = cache[li]
        if li < len(params) - 1:
            d = d * gelu_grad(z)
        W, _ = params[li]
        dm = bf16(d) if bf16_operands and li in BF16_LAYERS else d
        grads[li] = (dm.T @ h, d.sum(axis=0))
        d = dm @ W
    return loss, grads


def bf16_ambiguous_rows(params, x, rel=4e-6, absz=2e-7):
    """Rows with an activation, rounded to BF16 for a BF16 layer, closer to a rounding boundary
    than rel |a| + absz (|z| + 1) (a float32 evaluation of gelu(z) may then land on the other side
    and round to the neighbouring BF16 value)."""
    _, cache = forward(params, x, True)
    rows = np.zeros(len(x), dtype=bool)
    for li in BF16_LAYERS:
        z = cache[li - 1][1]
        a = gelu(z)
        rows |= (bf16_tie_distance(a) < rel * np.abs(a) + absz * (np.abs(z) + 1.0)).any(axis=1)
    return rows

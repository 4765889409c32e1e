"""Oracle for the learned fit start (test infrastructure only).

A multilayer perceptron maps the 64-bin normalised histogram of a toy
dataset to a starting point of its fit.  The paper has no learned component;
this follows the learned-start configuration: 64 inputs, hidden layers of 128
units with GELU (erf form), 6 outputs, BF16 weights with FP32 accumulation.

The oracle computes in float64 with exactly the roundings that belong to the
method: every GEMM operand (weights, incoming activations, and in the
backward pass the propagated gradients) rounded to BF16 (round to nearest
even); products and sums exact (float64); GELU and its derivative in float64.
With rounding=False every rounding is skipped (used to pin the backward
formulas against finite differences).  Loss: mean squared error over batch and outputs.
Adam (Kingma & Ba 2015) on float32 master weights.

Parameter layout (flat float32): for each layer W[n_in x n_out] row-major,
then b[n_out].
"""
from __future__ import annotations

import math

import numpy as np
from scipy.special import erf


def bf16(x):
    """Round float32 values to bfloat16 precision, nearest even (returns float64)."""
    a = np.ascontiguousarray(x, dtype=np.float32)
    u = a.view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def layer_shapes(n_in=64, n_hidden=128, n_layers=3, n_out=6):
    dims = [n_in] + [n_hidden] * n_layers + [n_out]
    return [(dims[i], dims[i + 1]) for i in range(len(dims) - 1)]


def unpack(params, shapes):
    out, o = [], 0
    for (i, j) in shapes:
        W = params[o:o + i * j].reshape(i, j)
        o += i * j
        b = params[o:o + j]
        o += j
        out.append((W, b))
    return out


def gelu(z):
    return 0.5 * z * (1.0 + erf(z / math.sqrt(2.0)))


def gelu_grad(z):
    return 0.5 * (1.0 + erf(z / math.sqrt(2.0))) + z * np.exp(-0.5 * z * z) / math.sqrt(2.0 * math.pi)


def _r(x, rounding):
    return bf16(np.asarray(x, dtype=np.float32)) if rounding else np.asarray(x, dtype=np.float64)


def forward(params, x, shapes, rounding=True):
    """Returns the output and the per-layer (input activation, pre-activation)."""
    layers = unpack(np.asarray(params, dtype=np.float64 if not rounding else np.float32), shapes)
    a = np.asarray(x, dtype=np.float64)
    cache = []
    for li, (W, b) in enumerate(layers):
        z = _r(a, rounding) @ _r(W, rounding) + np.asarray(b, dtype=np.float64)
        cache.append((a, z))
        a = gelu(z) if li < len(layers) - 1 else z
    return a, cache


def loss_and_grad(params, x, y, shapes, rounding=True):
    """MSE loss and its gradient in the flat parameters (float64)."""
    out, cache = forward(params, x, shapes, rounding)
    B, n_out = out.shape
    loss = float(np.mean((out - y) ** 2))
    d = 2.0 * (out - y) / (B * n_out)
    layers = unpack(np.asarray(params, dtype=np.float64 if not rounding else np.float32), shapes)
    grads = [None] * len(layers)
    for li in range(len(layers) - 1, -1, -1):
        W, b = layers[li]
        a_in, z = cache[li]
        dz = d if li == len(layers) - 1 else d * gelu_grad(z)
        dW = _r(a_in, rounding).T @ _r(dz, rounding)
        db = dz.sum(axis=0)
        grads[li] = (dW, db)
        d = _r(dz, rounding) @ _r(W, rounding).T
    flat = np.concatenate([np.concatenate([g[0].ravel(), g[1]]) for g in grads])
    return loss, flat


def adam(params, grad, m, v, t, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam step on float32 master weights (returns new params, m, v)."""
    m = b1 * m + (1 - b1) * grad
    v = b2 * v + (1 - b2) * grad * grad
    mh = m / (1 - b1 ** t)
    vh = v / (1 - b2 ** t)
    p = params.astype(np.float64) - lr * mh / (np.sqrt(vh) + eps)
    return p.astype(np.float32), m, v

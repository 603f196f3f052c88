"""FP64 CPU oracle for the warm-start MLP -- TEST INFRASTRUCTURE ONLY.

Plain numpy: y = W3 g(W2 g(W1 x + b1) + b2) + b3 with g(z) = z Phi(z) (GELU,
Phi the standard normal CDF), loss = mean((y - t)^2), and the gradients by
the chain rule, g'(z) = Phi(z) + z phi(z).  Used to check the GPU kernels'
forward pass and gradients; it shares nothing with them.
"""
from __future__ import annotations

import math

import numpy as np

_erf = np.vectorize(math.erf)


def gelu(z):
    return z * 0.5 * (1.0 + _erf(z / math.sqrt(2.0)))


def gelu_grad(z):
    cdf = 0.5 * (1.0 + _erf(z / math.sqrt(2.0)))
    pdf = np.exp(-0.5 * z * z) / math.sqrt(2.0 * math.pi)
    return cdf + z * pdf


def forward(params, X):
    """params: [(W1, b1), (W2, b2), (W3, b3)], W_l of shape [out, in]."""
    acts, pres = [X], []
    h = X
    for li, (W, b) in enumerate(params):
        z = h @ W.T + b
        if li < len(params) - 1:
            pres.append(z)
            h = gelu(z)
            acts.append(h)
        else:
            h = z
    return h, acts, pres


def loss_and_grads(params, X, T):
    Y, acts, pres = forward(params, X)
    loss = float(np.mean((Y - T) ** 2))
    d = 2.0 * (Y - T) / Y.size
    grads = [None] * len(params)
    for li in range(len(params) - 1, -1, -1):
        W, _ = params[li]
        grads[li] = (d.T @ acts[li], d.sum(axis=0))
        if li > 0:
            d = (d @ W) * gelu_grad(pres[li - 1])
    return loss, Y, grads


def round_bf16(x):
    """Round-to-nearest-even to bfloat16 (returned as float64)."""
    f = np.asarray(x, dtype=np.float32).copy()
    u = f.view(np.uint32)
    lsb = (u >> 16) & 1
    u = (u + 0x7FFF + lsb) & 0xFFFF0000
    return u.view(np.float32).astype(np.float64)

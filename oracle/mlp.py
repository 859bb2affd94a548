"""FP64 oracle of the BF16 surrogate MLP (test infrastructure).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).  Plain numpy in float64:
the same network as the CUDA kernels (ReLU hidden layers, linear output,
mean squared error), with the values that the GPU stores in BF16 (hidden
activations, back-propagated gradients) rounded to BF16 by round-to-nearest-
even, so that the GPU's FP32-accumulated results differ from it only by
accumulation order (at most one BF16 ulp per stored value).  With
``rounding=False`` it is the exact fp64 network, which the tests check against
central finite differences.
"""
from __future__ import annotations

import numpy as np


def bf16_round(x):
    """Round float64 values to the nearest BF16 value (ties to even)."""
    x = np.asarray(x, np.float64)
    m, e = np.frexp(x)  # x = m 2^e, 0.5 <= |m| < 1
    return np.ldexp(np.rint(m * 256.0), e - 8)


def _r(x, rounding):
    return bf16_round(x) if rounding else np.asarray(x, np.float64)


def forward(P, x, rounding=True):
    """P: dict of float64 arrays W1 [n1,k], b1, W2 [n2,n1], b2, W3, b3, w4 [n3], b4.
    Returns (y [M], acts) with acts = (h0, h1, h2, h3)."""
    h0 = np.asarray(x, np.float64)
    h1 = _r(np.maximum(h0 @ P["W1"].T + P["b1"], 0.0), rounding)
    h2 = _r(np.maximum(h1 @ P["W2"].T + P["b2"], 0.0), rounding)
    h3 = _r(np.maximum(h2 @ P["W3"].T + P["b3"], 0.0), rounding)
    y = h3 @ P["w4"] + P["b4"]
    return y, (h0, h1, h2, h3)


def loss_and_grad(P, x, t, rounding=True):
    """Mean squared error and its gradient (dict like P), by back-propagation
    through the same BF16 rounding points as the GPU."""
    y, (h0, h1, h2, h3) = forward(P, x, rounding)
    M = y.shape[0]
    e = y - np.asarray(t, np.float64)
    loss = float(np.mean(e * e))
    dy = 2.0 * e / M
    G = {"w4": h3.T @ dy, "b4": np.array(dy.sum())}
    dz3 = _r(np.outer(dy, P["w4"]) * (h3 > 0), rounding)
    G["W3"] = dz3.T @ h2
    G["b3"] = dz3.sum(0)
    dz2 = _r((dz3 @ P["W3"]) * (h2 > 0), rounding)
    G["W2"] = dz2.T @ h1
    G["b2"] = dz2.sum(0)
    dz1 = _r((dz2 @ P["W2"]) * (h1 > 0), rounding)
    G["W1"] = dz1.T @ h0
    G["b1"] = dz1.sum(0)
    return loss, G, y

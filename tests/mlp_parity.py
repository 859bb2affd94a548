"""Element-wise parity checks of the BF16 network's passes (test helpers).

Each stored BF16 value of the GPU is RN_bf16(f(v)) where v is an FP32 sum
(tensor-core products, FP32 accumulation) of exact products of BF16 values
and f is ReLU or the identity.  Given the GPU's own inputs to that sum, its
exact value E (float64) differs from the FP32 sum by at most
B = c (K + 2) u sum|terms| (K terms and a bias, u = 2^-24, c a safety factor
for the tensor cores' accumulation order).  Round-to-nearest and ReLU are
monotone, so the stored value must lie in [RN(f(E - B)), RN(f(E + B))]: it
equals RN(f(E)) exactly unless E lies within B of a rounding midpoint, where
the two neighbours are both allowed.  FP32 sums that are not rounded to BF16
(weight and bias gradients over M rows, outputs) must lie within
c (n + 2) u sum|terms| of the exact value, n the number of terms added.
"""
from __future__ import annotations

import numpy as np

from oracle.mlp import bf16_round

U = 2.0 ** -24
SAFETY = 4.0


def stored_bounds(E, S_abs, K, relu):
    B = SAFETY * (K + 2) * U * S_abs
    lo, hi = E - B, E + B
    if relu:
        lo, hi = np.maximum(lo, 0.0), np.maximum(hi, 0.0)
    return bf16_round(lo), bf16_round(hi)


def check_stored(name, gpu, E, S_abs, K, relu, mask=None):
    """Stored BF16 values gpu against exact pre-rounding values E (float64,
    same shape) whose sums of |terms| are S_abs.  Returns the fraction of
    entries where two values were allowed."""
    lo, hi = stored_bounds(E, S_abs, K, relu)
    if mask is not None:
        lo, hi = np.where(mask, lo, 0.0), np.where(mask, hi, 0.0)
    bad = (gpu < lo) | (gpu > hi)
    assert not bad.any(), (f"{name}: {int(bad.sum())} of {bad.size} stored values outside their rounding "
                           f"interval, e.g. {gpu[bad][:3]} vs {E[bad][:3]}")
    return float(np.mean(lo != hi))


def check_sum(name, gpu, E, S_abs, n):
    """FP32 sums gpu of n terms against their exact values E."""
    B = SAFETY * (n + 2) * U * S_abs + 1e-30
    err = np.abs(np.asarray(gpu, np.float64) - E)
    bad = err > B
    assert not bad.any(), (f"{name}: {int(bad.sum())} of {bad.size} entries beyond the accumulation bound, "
                           f"worst {float(np.max(err / B)):.3g} x the bound")


def dense(H, W, b=None):
    """E = H W^T (+ b) in float64 and the sums of |terms| per entry."""
    E = H @ W.T
    S = np.abs(H) @ np.abs(W).T
    if b is not None:
        E = E + b
        S = S + np.abs(b)
    return E, S


def check_forward(P, x, st):
    """The stored activations H1, H2, H3 and the outputs y of a forward pass
    against the network's definition on the GPU's own inputs to each layer.
    Returns the fractions of entries where two roundings were allowed."""
    amb = {}
    E, S = dense(x, P["W1"], P["b1"])
    amb["H1"] = check_stored("H1", st["H1"], E, S, x.shape[1], True)
    E, S = dense(st["H1"], P["W2"], P["b2"])
    amb["H2"] = check_stored("H2", st["H2"], E, S, 256, True)
    E, S = dense(st["H2"], P["W3"], P["b3"])
    amb["H3"] = check_stored("H3", st["H3"], E, S, 256, True)
    H3 = st["H3"]
    y_e = H3 @ P["w4"] + P["b4"]
    check_sum("y", st["y"], y_e, np.abs(H3) @ np.abs(P["w4"]) + abs(float(P["b4"])), 256)
    return amb


def head_gradient(P, y, t, H3, dy_gpu=None):
    """The head's FP32 arithmetic emulated exactly: dy = (2 (y - t)) (1 / M)
    and D3 = dy w4 (FP32 product) rounded to BF16 where H3 > 0.  If the GPU's
    stored dy is given it must equal dy bit for bit.  Returns (dy, D3)."""
    f32 = np.float32
    M = len(y)
    e = np.asarray(y).astype(f32) - np.asarray(t).astype(f32)
    dy = (f32(2.0) * e) * f32(1.0 / M)
    if dy_gpu is not None:
        bad = np.asarray(dy_gpu, f32) != dy
        assert not bad.any(), f"dy: {int(bad.sum())} of {M} entries differ from the head's arithmetic"
    d3 = bf16_round((dy[:, None] * P["w4"].astype(f32)[None, :]).astype(np.float64))
    return dy, np.where(H3 > 0, d3, 0.0)


def check_passes(P, x, t, st, grads, loss):
    """Every stored value and every gradient of one backward pass against the
    network's definition evaluated on the GPU's own stored inputs.
    P: parameters (float64, as params()); x [M,16], t [M]; st: stored
    tensors as float64 numpy (H1, H2, H3, D3, D2, D1, y); grads: as grads()."""
    M = x.shape[0]
    amb = check_forward(P, x, st)
    H3 = st["H3"]
    # the head's FP32 arithmetic on the GPU's y, emulated exactly: the stored
    # dy bit for bit, and D3 (rebuilt on chip from dy and the mask of H3) as
    # the input of D2
    dy, d3 = head_gradient(P, st["y"], t, H3, st.get("dy"))
    E, S = d3 @ P["W3"], np.abs(d3) @ np.abs(P["W3"])
    amb["D2"] = check_stored("D2", st["D2"], E, S, 256, False, mask=st["H2"] > 0)
    E, S = st["D2"] @ P["W2"], np.abs(st["D2"]) @ np.abs(P["W2"])
    amb["D1"] = check_stored("D1", st["D1"], E, S, 256, False, mask=st["H1"] > 0)
    # gradients: FP32 sums over the M rows
    dy64 = dy.astype(np.float64)
    check_sum("grad w4", grads["w4"], H3.T @ dy64, np.abs(H3).T @ np.abs(dy64), M)
    check_sum("grad b4", grads["b4"], dy64.sum(), np.abs(dy64).sum(), M)
    for l, (D, Hp) in {3: (d3, st["H2"]), 2: (st["D2"], st["H1"]), 1: (st["D1"], x)}.items():
        check_sum(f"grad W{l}", grads[f"W{l}"], D.T @ Hp, np.abs(D).T @ np.abs(Hp), M)
        check_sum(f"grad b{l}", grads[f"b{l}"], D.sum(0), np.abs(D).sum(0), M)
    ee = (st["y"].astype(np.float32) - t.astype(np.float32)).astype(np.float64)
    check_sum("loss", loss, float(np.sum(ee * ee) / M), float(np.sum(ee * ee) / M), 2 * M)
    return amb

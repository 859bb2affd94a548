"""The element-wise checks of the network's passes (tests/mlp_parity.py) on
the CPU: passes computed with FP32 sums (numpy) satisfy them, and a single
planted mistake fails them - a weight-gradient entry off by 10 %, one stored
activation one BF16 ulp off where the rounding is not ambiguous, one stored
dy one FP32 ulp off."""
import numpy as np
import pytest

from oracle.mlp import bf16_round
from tests import mlp_parity as mp


def simulated_passes(M, seed):
    rng = np.random.default_rng(seed)
    f32 = np.float32
    bf = lambda a: bf16_round(np.asarray(a, np.float64))  # noqa: E731
    x = np.zeros((M, 16))
    x[:, :13] = bf(rng.normal(0, 0.7, (M, 13)))
    P = {"W1": bf(rng.normal(0, 0.3, (256, 16))), "b1": rng.normal(0, 0.1, 256).astype(f32).astype(np.float64),
         "W2": bf(rng.normal(0, 0.06, (256, 256))), "b2": rng.normal(0, 0.1, 256).astype(f32).astype(np.float64),
         "W3": bf(rng.normal(0, 0.06, (256, 256))), "b3": rng.normal(0, 0.1, 256).astype(f32).astype(np.float64),
         "w4": bf(rng.normal(0, 0.06, 256)), "b4": np.array(0.05)}
    P["W1"][:, 13:] = 0.0
    t = rng.normal(size=M).astype(f32).astype(np.float64)

    def layer(H, W, b):
        z = (H.astype(f32) @ W.astype(f32).T) + b.astype(f32)
        return bf(np.maximum(z, 0))

    H1 = layer(x, P["W1"], P["b1"])
    H2 = layer(H1, P["W2"], P["b2"])
    H3 = layer(H2, P["W3"], P["b3"])
    y = (H3.astype(f32) @ P["w4"].astype(f32) + f32(P["b4"])).astype(np.float64)
    e = y.astype(f32) - t.astype(f32)
    dy = (f32(2.0) * e) * f32(1.0 / M)
    D3 = np.where(H3 > 0, bf((dy[:, None] * P["w4"].astype(f32)[None, :]).astype(np.float64)), 0.0)
    D2 = np.where(H2 > 0, bf(D3.astype(f32) @ P["W3"].astype(f32)), 0.0)
    D1 = np.where(H1 > 0, bf(D2.astype(f32) @ P["W2"].astype(f32)), 0.0)
    g = lambda A, B: (A.astype(f32).T @ B.astype(f32)).astype(np.float64)  # noqa: E731
    grads = {"W3": g(D3, H2), "W2": g(D2, H1), "W1": g(D1, x), "b3": D3.astype(f32).sum(0).astype(np.float64),
             "b2": D2.astype(f32).sum(0).astype(np.float64), "b1": D1.astype(f32).sum(0).astype(np.float64),
             "w4": (H3.astype(f32).T @ dy).astype(np.float64), "b4": np.array(float(dy.sum()))}
    loss = float(np.sum(e.astype(f32) * e.astype(f32) / f32(M)))
    st = {"H1": H1, "H2": H2, "H3": H3, "D3": D3, "D2": D2, "D1": D1, "y": y, "dy": dy.astype(np.float64)}
    return P, x, t, st, grads, loss


@pytest.mark.parametrize("M", [64, 1000])
def test_fp32_passes_satisfy_the_checks(M):
    amb = mp.check_passes(*simulated_passes(M, M))
    # two neighbouring values are allowed only near rounding midpoints; every
    # other stored value must be exactly RN(f(E))
    assert all(v < 0.5 for v in amb.values()), amb


def test_a_gradient_entry_off_by_ten_percent_fails():
    P, x, t, st, grads, loss = simulated_passes(1000, 3)
    for k in ("W3", "W2", "W1", "w4"):
        g = {kk: np.array(v, copy=True) for kk, v in grads.items()}
        D, Hp = {"W3": (st["D3"], st["H2"]), "W2": (st["D2"], st["H1"]), "W1": (st["D1"], x),
                 "w4": (None, None)}[k]
        if k == "w4":
            i = int(np.argmax(np.abs(g[k])))
        else:
            ratio = np.abs(D.T @ Hp) / (np.abs(D).T @ np.abs(Hp) + 1e-300)
            i = int(np.argmax(ratio))  # a typical well-conditioned entry
        g[k].reshape(-1)[i] *= 1.1
        with pytest.raises(AssertionError):
            mp.check_passes(P, x, t, st, g, loss)


def test_a_stored_value_one_ulp_off_fails():
    P, x, t, st, grads, loss = simulated_passes(500, 4)
    E, S = mp.dense(st["H1"], P["W2"], P["b2"])
    lo, hi = mp.stored_bounds(E, S, 256, True)
    cand = np.argwhere((lo == hi) & (st["H2"] > 0))
    m, j = cand[len(cand) // 2]
    bad = {k: np.array(v, copy=True) for k, v in st.items()}
    v = bad["H2"][m, j]
    bad["H2"][m, j] = bf16_round(v * (1 + 2.0 ** -7))  # the next BF16 value up
    assert bad["H2"][m, j] != v
    with pytest.raises(AssertionError):
        mp.check_passes(P, x, t, bad, grads, loss)
    bad = {k: np.array(v, copy=True) for k, v in st.items()}
    i = int(np.argmax(np.abs(bad["dy"])))
    bad["dy"][i] = float(np.nextafter(np.float32(bad["dy"][i]), np.float32(np.inf)))
    with pytest.raises(AssertionError):
        mp.check_passes(P, x, t, bad, grads, loss)

"""Pins of the fp64 MLP oracle: BF16 rounding against a library conversion,
back-propagation against central finite differences of the loss."""
import numpy as np
import pytest

from oracle import mlp


def test_bf16_round_matches_library_conversion():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(0)
    x = np.concatenate([rng.normal(size=4000), rng.normal(size=2000) * 1e-6, rng.normal(size=2000) * 1e6]).astype(np.float32)
    # exact halfway cases between neighbouring BF16 values (ties to even)
    ties = np.array([1 + 2.0 ** -8, 1 + 3 * 2.0 ** -8, -(1 + 5 * 2.0 ** -8), 3 * (1 + 2.0 ** -8)], np.float32)
    x = np.concatenate([x, ties, [0.0, -0.0]]).astype(np.float32)
    want = torch.from_numpy(x).to(torch.bfloat16).float().numpy().astype(np.float64)
    assert np.array_equal(mlp.bf16_round(x.astype(np.float64)), want)


def small_net(rng, k=5, n1=7, n2=6, n3=4):
    return {"W1": rng.normal(size=(n1, k)), "b1": rng.normal(size=n1) * 0.1, "W2": rng.normal(size=(n2, n1)),
            "b2": rng.normal(size=n2) * 0.1, "W3": rng.normal(size=(n3, n2)), "b3": rng.normal(size=n3) * 0.1,
            "w4": rng.normal(size=n3), "b4": np.array(0.3)}


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_backprop_matches_finite_differences(seed):
    rng = np.random.default_rng(seed)
    P = small_net(rng)
    x = rng.normal(size=(9, 5))
    t = rng.normal(size=9)
    loss, G, _ = mlp.loss_and_grad(P, x, t, rounding=False)
    h = 1e-6
    for k, v in P.items():
        v = np.asarray(v, np.float64)
        flat = v.reshape(-1)
        for i in range(flat.size):
            Pp = {kk: np.array(vv, np.float64, copy=True) for kk, vv in P.items()}
            Pm = {kk: np.array(vv, np.float64, copy=True) for kk, vv in P.items()}
            Pp[k].reshape(-1)[i] += h
            Pm[k].reshape(-1)[i] -= h
            lp, _, _ = mlp.loss_and_grad(Pp, x, t, rounding=False)
            lm, _, _ = mlp.loss_and_grad(Pm, x, t, rounding=False)
            fd = (lp - lm) / (2 * h)
            assert abs(fd - np.asarray(G[k]).reshape(-1)[i]) <= 1e-6 * max(1.0, abs(fd)), (k, i)


def test_rounded_gradient_close_to_exact():
    rng = np.random.default_rng(5)
    P = small_net(rng, k=8, n1=32, n2=32, n3=32)
    x = rng.normal(size=(64, 8))
    t = rng.normal(size=64)
    _, G0, _ = mlp.loss_and_grad(P, x, t, rounding=False)
    _, G1, _ = mlp.loss_and_grad(P, x, t, rounding=True)
    for k in G0:
        a, b = np.asarray(G0[k]).ravel(), np.asarray(G1[k]).ravel()
        assert np.linalg.norm(a - b) <= 0.05 * np.linalg.norm(a) + 1e-12, k

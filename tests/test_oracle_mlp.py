"""Pins of the MLP oracle (learned adaptation indicator): finite-difference gradient, closed-form
softmax cross-entropy, BF16 rounding against torch's conversion, feature identities (no GPU)."""
import numpy as np
import pytest

import oracle as O
from oracle import mlp
from paper_2306_06744_gb300 import workloads as W


def _params(n_in, seed, scale=0.3):
    n = mlp.layout(n_in)["total"]
    return (W.random_uniform(n, seed) - 0.5) * 2 * scale


def test_gradient_matches_finite_differences():
    n_in, B = 7, 5
    P = _params(n_in, 1)
    X = (W.random_uniform(B * n_in, 2).reshape(B, n_in) - 0.5) * 4
    y = np.array([-1, 0, 1, 1, -1])
    cw = [2.0, 0.5, 3.0]
    loss, g = mlp.loss_and_grad(P, X, y, cw)
    rng = np.random.default_rng(3)
    for idx in rng.choice(P.size, 40, replace=False):
        e = np.zeros_like(P)
        e[idx] = 1e-6
        lp, _ = mlp.loss_and_grad(P + e, X, y, cw)
        lm, _ = mlp.loss_and_grad(P - e, X, y, cw)
        assert abs((lp - lm) / 2e-6 - g[idx]) < 1e-7 * max(1.0, abs(g[idx])), idx


def test_softmax_cross_entropy_closed_form():
    n_in = 4
    L = mlp.layout(n_in)
    P = np.zeros(L["total"])
    o, _ = L["b4"]
    P[o:o + 3] = [0.3, -1.2, 2.0]
    X = np.ones((3, n_in))
    y = np.array([-1, 0, 1])
    cw = np.array([1.0, 2.0, 0.5])
    loss, g = mlp.loss_and_grad(P, X, y, cw)
    sm = np.exp(P[o:o + 3]) / np.exp(P[o:o + 3]).sum()
    w = cw[y + 1]
    want = -(w * np.log(sm[y + 1])).sum() / w.sum()
    assert abs(loss - want) < 1e-14
    gb4 = sum(w[k] * (sm - np.eye(3)[y[k] + 1]) for k in range(3)) / w.sum()
    assert np.allclose(g[o:o + 3], gb4, atol=1e-14)


def test_bf16_rounding_matches_torch():
    torch = pytest.importorskip("torch")
    x = (W.random_uniform(5000, 4) - 0.5) * 1e3
    x[:10] = [0.0, 1.0, -1.0, 1.00390625, 1.005859375, 3.1415926, 1e-30, -7.5e7, 65504.0, 2.0 ** -20]
    want = torch.tensor(x, dtype=torch.float32).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(mlp.bf16(x), want)


@pytest.mark.parametrize("dim,p", [(2, 2), (3, 2), (3, 3)])
def test_features_identities(dim, p):
    # constant state -> zero deviations; level feature in [0, 1]; p=2: sample points are the nodes
    o = O.operators(p)
    N, nv = (p + 1) ** dim, dim + 2
    M = 4
    u = np.zeros((M, nv, N))
    u[:, 0] = 1.3
    u[:, 1] = 0.2
    u[:, -1] = 3.0
    f = mlp.features(u, [4, 5, 6, 7], dim, p, 1.4, 4, 7, o["x"])
    assert f.shape == (M, 2 * 3 ** dim + 1)
    assert np.abs(f[:, :-1]).max() < 1e-12
    assert np.allclose(f[:, -1], [0, 1 / 3, 2 / 3, 1])
    if p == 2:
        rnd = W.random_uniform(M * N, 5).reshape(M, N)
        u[:, 0] = 1.0 + 0.1 * rnd
        f = mlp.features(u, [4] * M, dim, p, 1.4, 4, 7, o["x"])
        rm = u[:, 0].mean(axis=1, keepdims=True)
        assert np.allclose(f[:, :N], 100 * (u[:, 0] - rm) / rm, atol=1e-11)

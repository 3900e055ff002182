"""GPU kernels of the learned adaptation indicator against the FP64 numpy oracle (oracle/mlp.py).

Tolerances follow the arithmetic: both sides round inputs, weights and activations to BF16 and
the GPU accumulates in FP32 (the oracle in FP64); an FP32 rounding difference can move a
pre-activation across a BF16 rounding boundary, which changes that activation by one BF16 ulp
(2^-8 relative).  Logits agree within 1e-2 of their scale, gradients within 2e-2 relative L2.
Features: within one BF16 ulp.
"""
import numpy as np
import pytest

import oracle as O
from oracle import mlp
from paper_2306_06744_gb300 import fr, learned
from paper_2306_06744_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _rand_params(n_in, seed, scale=0.25):
    n = fr.mlp_param_count(n_in)
    return ((W.random_uniform(n, seed) - 0.5) * 2 * scale).astype(np.float32)


def _rand_X(n, n_in, seed):
    import torch
    X = (W.random_uniform(n * n_in, seed).reshape(n, n_in) - 0.5) * 6
    Xt = torch.tensor(X, dtype=torch.float32).to(torch.bfloat16)
    return Xt.cuda(), Xt.to(torch.float64).numpy()


def test_param_count_matches_oracle_layout():
    for n_in in (19, 55, 7):
        assert fr.mlp_param_count(n_in) == mlp.layout(n_in)["total"]


@pytest.mark.parametrize("n_in,n", [(55, 1000), (19, 257)])
def test_forward_parity(n_in, n):
    import torch
    P = _rand_params(n_in, 1)
    Xd, Xh = _rand_X(n, n_in, 2)
    logits, flags = fr.mlp_forward(torch.from_numpy(P).cuda(), Xd)
    want, _ = mlp.forward(P, Xh, bf16_round=True)
    got = logits.cpu().numpy()
    scale = np.abs(want).max()
    assert np.abs(got - want).max() < 1e-2 * scale
    am = np.argmax(want, axis=1) - 1
    clear = np.sort(want, axis=1)[:, -1] - np.sort(want, axis=1)[:, -2] > 1e-2 * scale
    assert np.array_equal(flags.cpu().numpy()[clear], am[clear])


@pytest.mark.parametrize("n_in,B", [(55, 512), (19, 300)])
def test_gradient_parity(n_in, B):
    import torch
    P = _rand_params(n_in, 3)
    Xd, Xh = _rand_X(B, n_in, 4)
    y = (np.floor(W.random_uniform(B, 5) * 3) - 1).astype(np.int8)
    cw = [1.5, 0.5, 2.0]
    loss, g = fr.mlp_grad(torch.from_numpy(P).cuda(), Xd, torch.from_numpy(y).cuda(), cw)
    wl, wg = mlp.loss_and_grad(P, Xh, y, cw, bf16_round=True)
    assert abs(loss - wl) < 1e-3 * abs(wl)
    g = g.cpu().numpy()
    assert np.linalg.norm(g - wg) < 2e-2 * np.linalg.norm(wg)


def test_training_learns_a_separable_rule():
    import torch
    n_in, n = 19, 16384
    Xd, Xh = _rand_X(n, n_in, 6)
    s = Xh[:, 0] + 0.5 * Xh[:, 1]
    y = np.where(s > 1.0, 1, np.where(s < -1.0, -1, 0)).astype(np.int8)
    params, hist = learned.train(Xd, torch.from_numpy(y).cuda(), epochs=8, batch=1024, lr=3e-3)
    acc, _ = learned.accuracy(params, Xd, torch.from_numpy(y).cuda())
    assert hist[-1] < 0.5 * hist[0]
    assert acc > 0.9


@pytest.mark.parametrize("name,p,Dbase,Dmax", [("vortex2d_p3", 3, 4, 6), ("vortex2d_p2_small", 1, 3, 5),
                                               ("vortex3d_p2_tube", 3, 2, 4), ("vortex3d_p2_tube", 4, 2, 3)])
def test_features_parity(name, p, Dbase, Dmax):
    cfg = W.config(name)
    cfg.update(p=p, Dbase=Dbase, Dmax=Dmax)
    g = fr.Mesh(cfg)
    g.step(2)
    X = g.features().to(__import__("torch").float64).cpu().numpy()
    dim = cfg["dim"]
    depths = O.morton_decode(dim, Dmax, g.leaves())[:, 0]
    want = mlp.bf16(mlp.features(g.state(), depths, dim, p, cfg["gamma"], Dbase, Dmax,
                                 O.operators(p)["x"]))
    assert X.shape == want.shape == (g.M, 2 * 3 ** dim + 1)
    # one BF16 ulp, plus an absolute floor for far-field elements where density and pressure are
    # nearly constant: a feature is 100 (q_i - mean q) / mean q of O(1..3) values, interpolated on
    # the GPU in double-word arithmetic (2^-47 relative per value) over up to 125 terms with
    # weights below 1.5, i.e. at most 100 * 2 * 125 * 1.5 * 3 * 2^-47 ~ 8e-10 of absolute noise
    floor = 100 * 2 * 125 * 1.5 * 3 * 2.0 ** -47
    assert np.all(np.abs(X - want) <= 2.0 ** -7 * np.abs(want) + floor)


def test_features_parity_and_indicator_modes():
    cfg = W.config("vortex3d_p2_tube")
    cfg.update(Dbase=2, Dmax=4, indicator=3)
    g = fr.Mesh(cfg)
    g.step(3)
    X = g.features().to(__import__("torch").float64).cpu().numpy()
    u = g.state()
    depths = O.morton_decode(3, cfg["Dmax"], g.leaves())[:, 0]
    want = mlp.bf16(mlp.features(u, depths, 3, cfg["p"], cfg["gamma"], cfg["Dbase"], cfg["Dmax"],
                                 O.operators(cfg["p"])["x"]))
    assert X.shape == want.shape == (g.M, 55)
    assert np.all(np.abs(X - want) <= 2.0 ** -7 * np.abs(want) + 100 * 2 * 125 * 1.5 * 3 * 2.0 ** -47)
    # without weights the learned indicator falls back to the density gradient
    g0 = fr.Mesh(dict(cfg, indicator=0))
    g0.step(3)
    fl3, _ = g.flags()
    fl0, _ = g0.flags()
    assert np.array_equal(fl3, fl0)
    # with weights, adaptation uses the MLP's argmax on the features
    import torch
    P = _rand_params(55, 9)
    g.set_learned_indicator(P)
    _, flags = fr.mlp_forward(torch.from_numpy(P).cuda(), g.features())
    keys0 = g.leaves()
    want_keys = fr.tree_adapt(3, cfg["Dbase"], cfg["Dmax"], keys0, flags.cpu().numpy())
    g.adapt()
    assert np.array_equal(g.leaves(), want_keys)


def test_forward_wait_timeout_is_reported_and_device_stays_usable():
    # the inference kernel's completion waits are bounded; with the bound set below an MMA's
    # latency the waits give up, the blocks drain what they issued (default bound) and free their
    # tensor memory, and the call reports FR_ETIMEOUT; with the default bound restored the next
    # call on the same device matches the oracle
    import torch
    n_in, n = 55, 20000
    P = _rand_params(n_in, 5)
    Xd, Xh = _rand_X(n, n_in, 6)
    Pd = torch.from_numpy(P).cuda()
    fr.tc_set_wait_limit(1)
    try:
        with pytest.raises(fr.FRError) as e:
            fr.mlp_forward(Pd, Xd)
        assert e.value.code == fr.FR_ETIMEOUT
    finally:
        fr.tc_set_wait_limit(0)
    logits, _ = fr.mlp_forward(Pd, Xd)
    want, _ = mlp.forward(P, Xh, bf16_round=True)
    assert np.abs(logits.cpu().numpy() - want).max() < 1e-2 * np.abs(want).max()

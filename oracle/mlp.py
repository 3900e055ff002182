"""Plain FP64 numpy oracle of the learned adaptation indicator (an extension of the paper, whose
adaptation criterion is analytic, Sec. 5.2).  TEST INFRASTRUCTURE ONLY.

Network: IN -> 64 -> 64 -> 64 -> 3 logits, GELU (exact erf form) after each hidden layer, weighted
softmax cross-entropy.  Parameters in one flat array
[W1 (64 x IN) | b1 | W2 (64 x 64) | b2 | W3 | b3 | W4 (3 x 64) | b4].  The GPU stores inputs,
weights and activations in BF16 and accumulates in FP32; `bf16=True` makes this oracle round the
same quantities to BF16 (round to nearest even) while keeping every sum in FP64.
"""
from __future__ import annotations

import numpy as np
from scipy.special import erf

H = 64


def layout(n_in):
    sizes = [("W1", H * n_in), ("b1", H), ("W2", H * H), ("b2", H), ("W3", H * H), ("b3", H),
             ("W4", 3 * H), ("b4", 3)]
    off, out = 0, {}
    for name, sz in sizes:
        out[name] = (off, sz)
        off += sz
    out["total"] = off
    return out


def unpack(params, n_in):
    L = layout(n_in)
    g = {k: params[v[0]:v[0] + v[1]] for k, v in L.items() if k != "total"}
    return (g["W1"].reshape(H, n_in), g["b1"], g["W2"].reshape(H, H), g["b2"],
            g["W3"].reshape(H, H), g["b3"], g["W4"].reshape(3, H), g["b4"])


def bf16(x):
    """Round float32 values to bfloat16 (nearest, ties to even), returned as float64."""
    a = np.ascontiguousarray(np.asarray(x, dtype=np.float32))
    u = a.view(np.uint32).astype(np.uint64)
    lsb = (u >> np.uint64(16)) & np.uint64(1)
    r = ((u + np.uint64(0x7FFF) + lsb) >> np.uint64(16)) << np.uint64(16)
    return (r & np.uint64(0xFFFFFFFF)).astype(np.uint32).view(np.float32).astype(np.float64)


def gelu(z):
    return 0.5 * z * (1.0 + erf(z / np.sqrt(2.0)))


def gelu_d(z):
    return 0.5 * (1.0 + erf(z / np.sqrt(2.0))) + z * np.exp(-0.5 * z * z) / np.sqrt(2.0 * np.pi)


def forward(params, X, bf16_round=False):
    """Logits [n][3] and the cache for backward."""
    n_in = X.shape[1]
    P = bf16(params) if bf16_round else np.asarray(params, dtype=np.float64)
    W1, b1, W2, b2, W3, b3, W4, b4 = unpack(P, n_in)
    r = bf16 if bf16_round else (lambda v: v)
    a0 = np.asarray(X, dtype=np.float64)
    z1 = a0 @ W1.T + b1
    a1 = r(gelu(z1))
    z2 = a1 @ W2.T + b2
    a2 = r(gelu(z2))
    z3 = a2 @ W3.T + b3
    a3 = r(gelu(z3))
    z4 = a3 @ W4.T + b4
    return z4, (P, a0, z1, a1, z2, a2, z3, a3)


def loss_and_grad(params, X, y, class_w, bf16_round=False):
    """Weighted mean softmax cross-entropy over the batch and its gradient (flat)."""
    n_in = X.shape[1]
    z4, (P, a0, z1, a1, z2, a2, z3, a3) = forward(params, X, bf16_round)
    W1, b1, W2, b2, W3, b3, W4, b4 = unpack(P, n_in)
    cls = np.asarray(y, dtype=np.int64) + 1
    w = np.asarray(class_w, dtype=np.float64)[cls]
    wsum = w.sum()
    zmax = z4.max(axis=1, keepdims=True)
    e = np.exp(z4 - zmax)
    p = e / e.sum(axis=1, keepdims=True)
    n = X.shape[0]
    loss = float(-(w * np.log(p[np.arange(n), cls])).sum() / wsum)
    d4 = p.copy()
    d4[np.arange(n), cls] -= 1.0
    d4 *= (w / wsum)[:, None]
    d3 = (d4 @ W4) * gelu_d(z3)
    d2 = (d3 @ W3) * gelu_d(z2)
    d1 = (d2 @ W2) * gelu_d(z1)
    grads = [d1.T @ a0, d1.sum(0), d2.T @ a1, d2.sum(0), d3.T @ a2, d3.sum(0), d4.T @ a3, d4.sum(0)]
    return loss, np.concatenate([g.ravel() for g in grads])


def features(u, depths, dim, p, gamma, Dbase, Dmax, x_nodes):
    """Features of every element: density and pressure at the 3^dim order-3 Gauss points
    (Lagrange interpolation from the element's p+1 points per axis at `x_nodes`), as 100 x the
    relative deviation from their element means, then (D - Dbase) / max(1, Dmax - Dbase)."""
    n = p + 1
    g3 = np.array([-np.sqrt(0.6), 0.0, np.sqrt(0.6)])
    I = np.ones((3, n))
    for t in range(3):
        for j in range(n):
            for k in range(n):
                if k != j:
                    I[t, j] *= (g3[t] - x_nodes[k]) / (x_nodes[j] - x_nodes[k])
    M, nv, N = u.shape
    S = 3 ** dim
    if dim == 2:
        T = np.einsum("ai,bj->baji", I, I).reshape(S, N)  # sample t = s0 + 3 s1, point i0 + n i1
    else:
        T = np.einsum("ai,bj,ck->cbakji", I, I, I).reshape(S, N)
    q = np.einsum("tn,evn->evt", T, u)
    rho = q[:, 0]
    m2 = (q[:, 1:1 + dim] ** 2).sum(axis=1)
    pr = (gamma - 1.0) * (q[:, -1] - 0.5 * m2 / rho)
    rm = rho.mean(axis=1, keepdims=True)
    pm = pr.mean(axis=1, keepdims=True)
    lev = (np.asarray(depths, dtype=np.float64) - Dbase) / max(1, Dmax - Dbase)
    return np.concatenate([100.0 * (rho - rm) / rm, 100.0 * (pr - pm) / pm, lev[:, None]], axis=1)

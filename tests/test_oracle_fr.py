"""Pins of the oracle's FR numerics: textbook operator identities, the DG lift identity, the
SSP-RK3 stability polynomial, transfer identities, the vortex as a steady Euler solution,
freestream preservation and discrete conservation on nonconforming trees, the entropy-wave
residual against a weak-form nodal DG residual written here, p+1 convergence, and the paper's
printed uniform-mesh L2 error (no GPU)."""
import math
import os

import numpy as np
import pytest

import oracle as O
from paper_2306_06744_gb300 import workloads as W


def _gl_closed_form(n):
    if n == 2:
        return [-1 / math.sqrt(3), 1 / math.sqrt(3)]
    if n == 3:
        return [-math.sqrt(3 / 5), 0.0, math.sqrt(3 / 5)]
    if n == 4:
        a = math.sqrt(3 / 7 - 2 / 7 * math.sqrt(6 / 5))
        b = math.sqrt(3 / 7 + 2 / 7 * math.sqrt(6 / 5))
        return [-b, -a, a, b]
    if n == 5:
        a = math.sqrt(5 - 2 * math.sqrt(10 / 7)) / 3
        b = math.sqrt(5 + 2 * math.sqrt(10 / 7)) / 3
        return [-b, -a, 0.0, a, b]


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_operators(p):
    n = p + 1
    o = O.operators(p)
    assert np.allclose(o["x"], _gl_closed_form(n), atol=1e-15, rtol=0)
    xr, wr = np.polynomial.legendre.leggauss(n)
    assert np.allclose(o["w"], wr, atol=1e-14, rtol=0)
    assert abs(o["w"].sum() - 2.0) < 1e-14
    # differentiation matrix: exact on monomials of degree <= p, rows sum to zero
    for k in range(n):
        fx = o["x"] ** k
        dfx = k * o["x"] ** (k - 1) if k else np.zeros(n)
        assert np.allclose(o["D"] @ fx, dfx, atol=1e-13)
    # boundary interpolation reproduces polynomials of degree <= p
    for k in range(n):
        assert abs(o["lm"] @ o["x"] ** k - (-1.0) ** k) < 1e-13
        assert abs(o["lp"] @ o["x"] ** k - 1.0) < 1e-13
    # correction function: g_L(-1) = 1, g_L(1) = 0 (Sec. 2.1)
    assert abs(O.correction_gL(p, -1.0) - 1.0) < 1e-15
    assert abs(O.correction_gL(p, 1.0)) < 1e-15
    # DG lift identity (Huynh): the Radau correction recovers nodal DG,
    # g_L'(x_i) = -l_i(-1)/w_i and g_R'(x_i) = l_i(1)/w_i
    assert np.allclose(o["gL"], -o["lm"] / o["w"], atol=1e-12)
    assert np.allclose(o["gR"], o["lp"] / o["w"], atol=1e-12)


def test_rk3_stability_polynomial():
    for z in (-0.3, -1.0, 0.5, -2.4):
        got = O.rk3_scalar(z, 1.0, 1.0)
        assert abs(got - (1 + z + z * z / 2 + z ** 3 / 6)) < 1e-15


def _poly_field(dim, p, xs, coeff_seed):
    """A random polynomial of degree <= p per axis, sampled at the tensor points xs (1D)."""
    c = W.random_uniform((p + 1) ** dim, coeff_seed) - 0.5
    n = p + 1
    pts = np.array(np.meshgrid(*([xs] * dim), indexing="ij")).reshape(dim, -1)[::-1]
    # meshgrid 'ij' then reverse -> pts[a] varies with x fastest in the flattened index

    def f(X):
        val = 0.0
        for idx in range(n ** dim):
            t, term = idx, c[idx]
            for a in range(dim):
                term *= X[a] ** (t % n)
                t //= n
            val += term
        return val

    return f


@pytest.mark.parametrize("dim,p", [(2, 1), (2, 2), (2, 3), (3, 2), (3, 3)])
def test_transfer_identities(dim, p):
    o = O.operators(p)
    n = p + 1
    N = n ** dim
    xs = o["x"]
    idx = np.arange(N)
    coords = [xs[(idx // n ** a) % n] for a in range(dim)]
    f = _poly_field(dim, p, xs, 5 + dim * 10 + p)
    parent = np.array([[f([coords[a][i] for a in range(dim)]) for i in range(N)]] * 2)
    parent[1] *= 2.0
    kids = []
    for c in range(1 << dim):
        k = O.prolong(dim, p, parent, c)
        # refinement reproduces the degree-p polynomial exactly at the child points
        want = [f([(coords[a][i] + 2 * ((c >> a) & 1) - 1) / 2 for a in range(dim)]) for i in range(N)]
        assert np.allclose(k[0], want, atol=1e-13)
        kids.append(k)
    kids = np.array(kids)
    back = O.restrict(dim, p, kids)
    # restriction after refinement is the identity
    assert np.allclose(back, parent, atol=1e-13)
    # restriction conserves the integral sum_i w_i |J| u_i for arbitrary child data
    W1 = np.ones(N)
    for a in range(dim):
        W1 = W1 * o["w"][(idx // n ** a) % n]
    rnd = (W.random_uniform(kids.size, 99).reshape(kids.shape) - 0.5)
    pr = O.restrict(dim, p, rnd)
    lhs = (pr * W1).sum(axis=-1)
    rhs = (rnd * W1).sum(axis=-1).sum(axis=0) / 2 ** dim
    assert np.allclose(lhs, rhs, atol=1e-14)


def test_vortex_is_steady_euler_solution():
    # In the frame moving with the freestream the isentropic vortex is a steady Euler solution:
    # isentropic (p = rho^gamma for rho_inf = p_inf = 1) and in radial balance dp/dr = rho v_t^2 / r.
    cfg = W.config("vortex2d_p2_small")
    cfg["uinf"] = (0.0, 0.0, 0.0)
    g = cfg["gamma"]
    r = np.linspace(0.2, 3.0, 15)
    h = 1e-5
    pts = np.array([[5.0 + rr, 5.0, 0.0] for rr in r])
    ptsp = np.array([[5.0 + rr + h, 5.0, 0.0] for rr in r])
    ptsm = np.array([[5.0 + rr - h, 5.0, 0.0] for rr in r])

    def pres(q):
        return (g - 1) * (q[:, 3] - 0.5 * (q[:, 1] ** 2 + q[:, 2] ** 2) / q[:, 0])

    q, qp, qm = O.exact(cfg, 0.0, pts), O.exact(cfg, 0.0, ptsp), O.exact(cfg, 0.0, ptsm)
    rho, p = q[:, 0], pres(q)
    assert np.allclose(p, rho ** g, rtol=1e-13)
    vt = q[:, 2] / rho  # on the +x ray the tangential velocity is v
    dpdr = (pres(qp) - pres(qm)) / (2 * h)
    assert np.allclose(dpdr, rho * vt ** 2 / r, rtol=1e-6)
    # centre value, far field, and advection by the freestream
    cfg2 = W.config("vortex2d_p2_small")
    qc = O.exact(cfg2, 0.0, np.array([[5.0, 5.0, 0.0]]))
    dT = -(g - 1) * 25 / (8 * g * math.pi ** 2) * math.e
    assert abs(qc[0, 0] - (1 + dT) ** (1 / (g - 1))) < 1e-14
    qf = O.exact(cfg2, 0.0, np.array([[0.0, 0.0, 0.0]]))
    assert abs(qf[0, 0] - 1.0) < 1e-9
    x0 = np.array([[5.3, 4.1, 0.0]])
    q0 = O.exact(cfg2, 0.0, x0)
    q1 = O.exact(cfg2, 1.7, x0 + np.array([[1.7, 1.7, 0.0]]))
    assert np.allclose(q0, q1, atol=1e-13)


def _random_nonconforming_mesh(dim, p, Dbase, Dmax, seed, psplit):
    cfg = W.config("vortex2d_p2_small" if dim == 2 else "vortex3d_p2_tube")
    cfg.update(dim=dim, p=p, Dbase=Dbase, Dmax=Dmax, init_passes=0, indicator=2, dt=1e-3)
    m = O.OracleMesh(cfg)
    for k in range(50):  # first seed of the sequence whose tree has hanging faces
        boxes = W.random_tree_boxes(dim, Dbase, Dmax, seed=seed + 1000 * k, p_split=psplit)
        keys = O.balance(dim, Dmax, np.sort(O.morton_encode(dim, Dmax, boxes)))
        if (O.conn(dim, Dmax, keys)[1] == 2).any():
            break
    return cfg, m, keys


def _depths(dim, Dmax, keys):
    return O.morton_decode(dim, Dmax, keys)[:, 0]


@pytest.mark.parametrize("dim,p,Dbase,Dmax,seed", [(2, 1, 2, 5, 1), (2, 2, 2, 5, 2), (2, 3, 2, 5, 3),
                                                   (3, 1, 1, 3, 4), (3, 2, 1, 3, 5)])
def test_freestream_preservation(dim, p, Dbase, Dmax, seed):
    cfg, m, keys = _random_nonconforming_mesh(dim, p, Dbase, Dmax, seed, 0.35)
    _, ft, _ = O.conn(dim, Dmax, keys)
    assert (ft == 1).any() and (ft == 2).any(), "mesh must have hanging faces"
    M, nv, N = keys.shape[0], dim + 2, (p + 1) ** dim
    q = np.array([1.3, 1.3 * 0.7, -1.3 * 0.4, 0.0, 0.0][:nv])
    if dim == 3:
        q[3] = 1.3 * 0.25
    q[-1] = 2.0 / (cfg["gamma"] - 1) + 0.5 * (q[1:1 + dim] ** 2).sum() / q[0]
    u = np.broadcast_to(q[None, :, None], (M, nv, N)).copy()
    m.set_state(keys, u)
    R = m.rhs()
    assert np.abs(R).max() < 1e-12


@pytest.mark.parametrize("dim,p,Dbase,Dmax,seed", [(2, 2, 2, 5, 6), (2, 3, 2, 6, 7), (3, 2, 1, 3, 8),
                                                   (3, 3, 1, 3, 9)])
def test_discrete_conservation(dim, p, Dbase, Dmax, seed):
    # sum_e sum_i w_i |J_e| R_{e,i} = 0 on a nonconforming periodic mesh with a random state:
    # the mortar back-projection is an L2 projection (Sec. 4.3)
    cfg, m, keys = _random_nonconforming_mesh(dim, p, Dbase, Dmax, seed, 0.35)
    M, nv, N, n = keys.shape[0], dim + 2, (p + 1) ** dim, p + 1
    rnd = W.random_uniform(M * nv * N, seed + 40).reshape(M, nv, N) - 0.5
    u = np.zeros((M, nv, N))
    u[:, 0] = 1.0 + 0.2 * rnd[:, 0]
    for b in range(dim):
        u[:, 1 + b] = 0.3 * rnd[:, 1 + b]
    u[:, -1] = 2.5 + 0.2 * rnd[:, -1]
    m.set_state(keys, u)
    R = m.rhs()
    o = O.operators(p)
    idx = np.arange(N)
    Wt = np.ones(N)
    for a in range(dim):
        Wt = Wt * o["w"][(idx // n ** a) % n]
    h = cfg["L"] / 2.0 ** _depths(dim, Dmax, keys)
    J = (h / 2) ** dim
    tot = np.einsum("evi,i,e->v", R, Wt, J)
    scale = np.einsum("evi,i,e->v", np.abs(R), Wt, J)
    assert np.all(np.abs(tot) < 1e-13 * scale.max() + 1e-14), (tot, scale)


def test_3d_tube_reduces_to_2d():
    # a z-uniform 3D mesh carrying the vortex tube must reproduce the 2D residual in every layer
    c2 = W.config("vortex2d_p2_small")
    c2.update(Dbase=3, Dmax=3, init_passes=0, indicator=2)
    c3 = dict(c2, dim=3)
    m2, m3 = O.OracleMesh(c2), O.OracleMesh(c3)
    R2, R3 = m2.rhs(), m3.rhs()
    k3 = m3.leaves()
    b3 = O.morton_decode(3, 3, k3)
    k2 = m2.leaves()
    b2 = O.morton_decode(2, 3, k2)
    pos2 = {(x, y): i for i, (_, x, y, _) in enumerate(b2)}
    n, N2 = 3, 9
    for e in range(0, len(k3), 7):
        _, x, y, z = b3[e]
        e2 = pos2[(x, y)]
        for iz in range(n):
            layer = R3[e, :, iz * N2:(iz + 1) * N2]
            assert np.allclose(layer[[0, 1, 2, 4]], R2[e2], atol=1e-12)
            assert np.abs(layer[3]).max() < 1e-12


def _uniform_error(p, D, t_end, dt, L=20.0):
    cfg = W.config("vortex2d_p2_small")
    cfg.update(p=p, L=L, Dbase=D, Dmax=D, init_passes=0, indicator=2, dt=dt,
               vort=np.array([[L / 2, L / 2, 5.0, 1.0]]))
    m = O.OracleMesh(cfg)
    m.step(int(round(t_end / dt)))
    return m.norms()["l2_rho"]


@pytest.mark.parametrize("p", [1, 2, 3])
def test_convergence_order(p):
    # order ~ p+1 on uniform meshes for the advected vortex (Sec. 5.2, Table of uniform meshes)
    dt = 0.01 if p < 3 else 0.005
    e1 = _uniform_error(p, 4, 0.5, dt)
    e2 = _uniform_error(p, 5, 0.5, dt)
    order = math.log(e1 / e2) / math.log(2.0)
    assert order > p + 0.5, (e1, e2, order)


def test_adaptive_matches_uniform_error():
    # Sec. 5.2: adaptive and uniform meshes with the same finest spacing give L2 density errors
    # that differ only trivially.  Analytic-centre criterion with the paper's radii 5 and 6.
    L = 20.0

    def run(Dbase, Dmax, passes, ind):
        cfg = W.config("vortex2d_p2_small")
        cfg.update(p=2, L=L, Dbase=Dbase, Dmax=Dmax, init_passes=passes, indicator=ind, dt=0.01,
                   th_refine=5.0, th_coarsen=6.0, adapt_every=10,
                   vort=np.array([[L / 2, L / 2, 5.0, 1.0]]))
        m = O.OracleMesh(cfg)
        m.run(50)
        return m.norms()["l2_rho"], m.M

    eu, Mu = run(5, 5, 0, 2)
    ea, Ma = run(3, 5, -1, 1)
    assert Ma < Mu / 2
    assert abs(ea - eu) < 0.01 * eu, (ea, eu)


@pytest.mark.parametrize("dim,Dmax,p", [(2, 3, 1), (2, 3, 2), (2, 3, 3), (2, 3, 4), (3, 2, 1), (3, 2, 2),
                                        (3, 2, 3)])
def test_entropy_wave_residual_is_weak_form_nodal_dg(dim, Dmax, p):
    # With constant velocity v and pressure, the Euler equations carry the density as a linear
    # advection wave (mass flux rho*v), and FR with the Radau (DG) correction functions is nodal
    # DG (Huynh).  So on a uniform periodic mesh the oracle's density residual must equal the
    # weak-form nodal DG residual written out here from its own definition:
    #   w_i (h/2) drho_i/dt = sum_j w_j D_ji f_j - l_i(+1) F*(+1) + l_i(-1) F*(-1)
    # per line of nodes (diagonal GL mass matrix; the quadrature is exact for these degree-2p
    # integrands), with the Rusanov flux on the face traces, lambda = max(|v_n| + c) of the two traces,
    # point by point.
    cfg = W.config("vortex2d_p2_small" if dim == 2 else "vortex3d_p2_tube")
    cfg.update(dim=dim, p=p, Dbase=Dmax, Dmax=Dmax, init_passes=0, indicator=2, dt=1e-3)
    L, g = cfg["L"], cfg["gamma"]
    nc, n = 2 ** Dmax, p + 1
    h = L / nc
    m = O.OracleMesh(cfg)
    cells = np.array(np.meshgrid(*([np.arange(nc)] * dim), indexing="ij")).reshape(dim, -1).T
    boxes = np.zeros((cells.shape[0], 4), dtype=np.int32)
    boxes[:, 0] = Dmax
    boxes[:, 1:1 + dim] = cells
    keys = np.sort(O.morton_encode(dim, Dmax, boxes))
    B = O.morton_decode(dim, Dmax, keys)
    M, N = keys.shape[0], n ** dim
    # GL nodes and weights (library routine), Lagrange basis by its barycentric weights
    x, w = np.polynomial.legendre.leggauss(n)
    bw = np.array([1.0 / np.prod([x[i] - x[k] for k in range(n) if k != i]) for i in range(n)])
    Dm = np.zeros((n, n))
    for i in range(n):
        for j in range(n):
            if i != j:
                Dm[i, j] = bw[j] / bw[i] / (x[i] - x[j])
        Dm[i, i] = -Dm[i].sum()
    lm = np.array([np.prod([(-1.0 - x[k]) / (x[i] - x[k]) for k in range(n) if k != i]) for i in range(n)])
    lp = np.array([np.prod([(1.0 - x[k]) / (x[i] - x[k]) for k in range(n) if k != i]) for i in range(n)])
    v = np.array([0.7, -0.45, 0.3][:dim])
    pr = 1.3
    # state at the solution points (point index ix + n*iy + n^2*iz)
    idx = np.arange(N)
    loc = [(idx // n ** a) % n for a in range(dim)]
    X = [(B[:, 1 + a][:, None] + 0.5 * (x[loc[a]][None, :] + 1.0)) * h for a in range(dim)]
    rho = 1.0 + 0.25 * np.sin(2 * np.pi * X[0] / L + 0.3) * np.cos(4 * np.pi * X[1] / L)
    if dim == 3:
        rho = rho + 0.1 * np.sin(2 * np.pi * X[2] / L)
    u = np.zeros((M, dim + 2, N))
    u[:, 0] = rho
    for a in range(dim):
        u[:, 1 + a] = rho * v[a]
    u[:, -1] = pr / (g - 1) + 0.5 * rho * (v @ v)
    m.set_state(keys, u)
    R = m.rhs()[:, 0, :]
    # the same density on a structured array: cell axes (z, y, x) then node axes (z, y, x)
    G = np.zeros((nc,) * dim + (n,) * dim)
    for e in range(M):
        G[tuple(B[e, 1:1 + dim][::-1])] = rho[e].reshape((n,) * dim)
    Rg = np.zeros_like(G)
    for a in range(dim):
        ca, na = dim - 1 - a, 2 * dim - 1 - a  # cell and node axes of direction a
        vals = np.moveaxis(G, na, -1)
        tm, tp = vals @ lm, vals @ lp  # own traces at -1 and +1
        nb_m, nb_p = np.roll(tp, 1, axis=ca), np.roll(tm, -1, axis=ca)  # neighbours' traces

        def rus(rl, rr):
            lam = np.maximum(abs(v[a]) + np.sqrt(g * pr / rl), abs(v[a]) + np.sqrt(g * pr / rr))
            return 0.5 * v[a] * (rl + rr) - 0.5 * lam * (rr - rl)

        Fm, Fp = rus(nb_m, tm), rus(tp, nb_p)
        vol = np.einsum("j,ji,...j->...i", w, Dm, v[a] * vals)
        du = (2.0 / h) * (vol - lp * Fp[..., None] + lm * Fm[..., None]) / w
        Rg += np.moveaxis(du, -1, na)
    Rdg = np.array([Rg[tuple(B[e, 1:1 + dim][::-1])].reshape(N) for e in range(M)])
    assert np.abs(Rdg).max() > 1e-2
    assert np.abs(R - Rdg).max() < 1e-12 * np.abs(Rdg).max(), np.abs(R - Rdg).max()


def _paper_uniform_l2():
    path = os.path.join(os.path.dirname(__file__), "golden", "paper_uniform_l2.txt")
    rows = {}
    with open(path) as fh:
        for line in fh:
            if line.strip() and not line.startswith("#"):
                p, dx, l2, _ = line.split()
                rows[(int(p), float(dx))] = float(l2)
    return rows


def paper_uniform_cfg(p, D, dt):
    """The paper's grid-refinement runs (Sec. 5.2): the vortex on a uniform periodic mesh of
    [-12.5, 12.5]^2 (here [0, 25]^2 with the centre in the middle), advected by u = (1, 1) for one
    period, t = 25; its Mach number 0.5 read as p_inf = rho_inf |u|^2 / (gamma Ma^2) with
    |u| = sqrt(2) (the paper leaves the freestream pressure implicit; this reading reproduces its
    tables, p_inf = 1 does not).  dx = 25 / 2^D."""
    L, g = 25.0, 1.4
    cfg = W.config("vortex2d_p2_small")
    cfg.update(p=p, L=L, Dbase=D, Dmax=D, init_passes=0, indicator=2, dt=dt, adapt_every=10 ** 9,
               rho_inf=1.0, p_inf=1.0 * 2.0 / (g * 0.5 ** 2), vort=np.array([[L / 2, L / 2, 5.0, 1.0]]))
    return cfg


# coarsest row of the table; the time steps are larger than the paper's 0.001, with time errors
# far below the spatial ones (p = 1: dt = 0.004, 0.008 and 0.0125 agree to 0.02%).  p = 2 takes
# about 90 s on the oracle and runs by default; p = 3 (about 230 s) with FR_SLOW_PINS=1.
@pytest.mark.parametrize("p,dt,tol", [(1, 0.0125, 0.02), (2, 0.00625, 0.02),
                                      pytest.param(3, 0.005, 0.02, marks=pytest.mark.skipif(
                                          not os.environ.get("FR_SLOW_PINS"), reason="FR_SLOW_PINS"))])
def test_paper_uniform_l2_error(p, dt, tol):
    expect = _paper_uniform_l2()[(p, 0.390625)]
    m = O.OracleMesh(paper_uniform_cfg(p, 6, dt))
    m.run(int(round(25.0 / dt)))
    assert abs(m.info()["t"] - 25.0) < 1e-9
    l2 = m.norms()["l2_rho"]
    assert abs(l2 - expect) < tol * expect, (l2, expect)


def paper_topdown_start(m, cfg):
    """Top-down initial adaptive mesh for the paper's runs on a mesh object `m` with the oracle's
    (or the CUDA binding's) calls: uniform at Dmax with the closed-form state, Dmax - Dbase
    adaptations by the mesh's own criterion (which coarsen away from the vortex), then the
    closed-form state at the leaves and t = 0.  2D."""
    L, p, Dmax, n = cfg["L"], cfg["p"], cfg["Dmax"], cfg["p"] + 1
    x = O.operators(p)["x"]

    def exact_state(keys):
        B = O.morton_decode(2, Dmax, keys)
        h = L / 2.0 ** B[:, 0]
        idx = np.arange(n * n)
        X = B[:, 1:2] * (L / 2 ** Dmax) + 0.5 * (x[idx % n][None, :] + 1) * h[:, None]
        Y = B[:, 2:3] * (L / 2 ** Dmax) + 0.5 * (x[idx // n][None, :] + 1) * h[:, None]
        q = O.exact(cfg, 0.0, np.stack([X.ravel(), Y.ravel(), np.zeros(X.size)], 1))
        return np.ascontiguousarray(q.reshape(len(keys), n * n, 4).transpose(0, 2, 1))

    nc = 2 ** Dmax
    boxes = np.array([(Dmax, i, j, 0) for i in range(nc) for j in range(nc)], dtype=np.int32)
    keys = np.sort(O.morton_encode(2, Dmax, boxes))
    m.set_state(keys, exact_state(keys))
    for _ in range(Dmax - cfg["Dbase"]):
        m.adapt()
    keys = np.ascontiguousarray(m.leaves())
    m.set_state(keys, exact_state(keys))
    m.set_time(0.0)


@pytest.mark.skipif(not os.environ.get("FR_SLOW_PINS"), reason="FR_SLOW_PINS (5, 10, 16 minutes)")
@pytest.mark.parametrize("p,expect,count", [(1, 4.64e-2, 961), (2, 1.18e-3, 952), (3, 2.68e-5, 952)])
def test_paper_large_domain_adaptive_row(p, expect, count):
    # The paper's adaptive table for the large domain (Sec. 5.2; 100 wide: its element counts,
    # 65536 at dx = 25/64, fix the width the text misprints; one period t = 100), Dmax 8 rows:
    # printed L2 and element count.  Its initial mesh is read top-down (paper_topdown_start).
    # (Bottom-up from Dmin, as the library builds its initial mesh, leaves this mesh uniform at
    # Dmin: its 12.5-wide elements never hold more points inside radius 5 than beyond 6, and the
    # error comes out 2.8x larger; on the small domain both readings give the same run.)
    L = 100.0
    cfg = paper_uniform_cfg(p, 8, 0.001)
    cfg.update(L=L, Dbase=3, init_passes=0, indicator=1, th_refine=5.0, th_coarsen=6.0,
               adapt_every=10, vort=np.array([[L / 2, L / 2, 5.0, 1.0]]))
    m = O.OracleMesh(cfg)
    paper_topdown_start(m, cfg)
    for _ in range(10000):
        m.step(10)
        m.adapt()
    assert abs(m.info()["t"] - 100.0) < 1e-9
    assert abs(m.norms()["l2_rho"] - expect) < 0.02 * expect
    assert m.M == count


def _solution_points(dim, p, Dmax, L, keys):
    """Physical coordinates [M][N][3] of each leaf's Gauss-Legendre solution points (nodes from
    numpy's Gauss-Legendre rule, x fastest in the point index) and the leaf widths h."""
    n, N = p + 1, (p + 1) ** dim
    xi, _ = np.polynomial.legendre.leggauss(n)
    bx = O.morton_decode(dim, Dmax, keys)
    h = L / 2.0 ** bx[:, 0]
    cell = L / 2.0 ** Dmax
    idx = np.arange(N)
    X = np.zeros((keys.shape[0], N, 3))
    for a in range(dim):
        ia = (idx // n ** a) % n
        X[:, :, a] = bx[:, 1 + a, None] * cell + (xi[ia][None, :] + 1) / 2 * h[:, None]
    return X, h


@pytest.mark.parametrize("dim,p,Dbase,Dmax,seed", [(2, 1, 2, 5, 1), (2, 2, 2, 5, 2), (2, 3, 2, 5, 3),
                                                   (2, 4, 2, 5, 4), (3, 1, 1, 3, 4), (3, 2, 1, 3, 5),
                                                   (3, 3, 1, 3, 9)])
def test_density_gradient_indicator(dim, p, Dbase, Dmax, seed):
    # eta = h * max over the solution points of |grad rho| (the density-gradient reading of the
    # indicator, Sec. 5.2), on a nonconforming tree:
    # * rho linear along each axis and along an oblique direction b: the degree-p interpolant is
    #   exact, so eta = h |b| in every element (a dropped 2/h, a missing square root or a wrong
    #   axis fails);
    # * for p >= 2, rho = c (x_a - x0)^2 + beta x_b: the gradient varies over the element, so eta
    #   = h * max_i sqrt((2c (x_a,i - x0))^2 + beta^2) pins the set the maximum runs over;
    # * flags: 1 above the refine threshold, -1 below the coarsen threshold, from the expected eta.
    # Tolerance: eta is formed from O(1) densities by an n-term sum with |D_ij| <= n^2, so its
    # rounding error is ~n^3 * 3 * 2^-53 absolute in reference coordinates against a gradient of
    # h|b|/2 >= 0.05 there: 1e-12 relative.
    cfg, _, keys = _random_nonconforming_mesh(dim, p, Dbase, Dmax, seed, 0.35)
    M, nv, N = keys.shape[0], dim + 2, (p + 1) ** dim
    X, h = _solution_points(dim, p, Dmax, cfg["L"], keys)
    bnorm = 0.37
    th_r, th_c = 0.99 * bnorm * h.max(), 1.01 * bnorm * h.min()
    assert th_r > th_c
    cfg = dict(cfg, indicator=0, th_refine=th_r, th_coarsen=th_c)
    m = O.OracleMesh(cfg)
    cases = []
    for a in range(dim):
        cases.append((2.0 + bnorm * X[:, :, a], h * bnorm))
    b = np.array([0.21, -0.33, 0.12 if dim == 3 else 0.0])
    cases.append((2.0 + X @ b, h * np.linalg.norm(b)))
    if p >= 2:
        x0, c, beta = 0.3 * cfg["L"], 0.05, 0.11
        for a in range(dim):
            o = (a + 1) % dim
            g = np.sqrt((2 * c * (X[:, :, a] - x0)) ** 2 + beta ** 2)
            cases.append((2.0 + c * (X[:, :, a] - x0) ** 2 + beta * X[:, :, o], h * g.max(axis=1)))
    for k, (rho, want) in enumerate(cases):
        u = np.zeros((M, nv, N))
        u[:, 0] = rho
        u[:, -1] = 1.0 / (cfg["gamma"] - 1.0)
        m.set_state(keys, u)
        flags, eta = m.flags()
        assert np.max(np.abs(eta - want) / want) < 1e-12
        expect = np.where(want > th_r, 1, np.where(want < th_c, -1, 0))
        assert np.array_equal(flags, expect)
        if k == 0:  # the thresholds sit just inside the coarsest and finest h: all three flags occur
            assert set(expect.tolist()) == {-1, 0, 1} or len(set(h.tolist())) == 2

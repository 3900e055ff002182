"""Precision forms of the time-step kernels against the FP64 oracle, through the C ABI.

precision 4 (double-word: two floats on the FP32 pipes, ~48-bit significand) must meet the same
bars as FP64: residual within 1e-12 relative L2, 100 steps with adaptation within 1e-10.  Its
arithmetic error is ~2^-48 per operation (3.6e-15), so these bars hold with margin.
precision 1 (FP32 operators, fluxes and traces, FP64 Runge-Kutta combination) is an approximate
form: the derivative sums O(|f|) terms to an O(h|grad f|) result, so FP32 rounding (6e-8 per
operation) is amplified by that cancellation times |Dt| (together O(10^2..10^3) on these meshes);
its residual error is bounded by 1e-4 relative L2 (measured 1.4e-5 on the 2D p=2 case) and its
freestream residual by 1e-4 absolute.
"""
import numpy as np
import pytest

import oracle as O
from paper_2306_06744_gb300 import fr
from paper_2306_06744_gb300 import workloads as W
from tests.test_gpu_fr import _random_tree, _smooth_state, rel_l2

pytestmark = pytest.mark.gpu


def _cfg(name, **kw):
    c = W.config(name)
    c.update(kw)
    return c


@pytest.mark.parametrize("prec,tol", [(4, 1e-12), (1, 1e-4)])
@pytest.mark.parametrize("dim,p,Dbase,Dmax,seed", [(2, 2, 3, 7, 2), (2, 3, 3, 7, 3), (3, 2, 1, 4, 6),
                                                   (3, 3, 1, 4, 7)])
def test_rhs_precision_forms(prec, tol, dim, p, Dbase, Dmax, seed):
    cfg = _cfg("vortex2d_p2_small" if dim == 2 else "vortex3d_p2_tube", dim=dim, p=p, Dbase=Dbase,
               Dmax=Dmax, init_passes=0, indicator=2, dt=1e-3)
    keys = _random_tree(dim, Dbase, Dmax, seed)
    u = _smooth_state(cfg, keys, seed)
    o = O.OracleMesh(cfg)
    o.set_state(keys, u)
    g = fr.Mesh(dict(cfg, precision=prec))
    g.set_state(keys, u)
    err = rel_l2(g.rhs(), o.rhs())
    assert err < tol, err


@pytest.mark.parametrize("prec,tol", [(4, 1e-12), (1, 1e-4), (2, 1e-4), (3, 1e-4)])
def test_freestream_precision_forms(prec, tol):
    cfg = _cfg("vortex3d_p2_tube", p=3, Dbase=1, Dmax=4, init_passes=0, indicator=2, dt=1e-3,
               precision=prec)
    keys = _random_tree(3, 1, 4, 77)
    M, nv, N = len(keys), 5, 64
    q = np.array([1.2, 0.5, -0.3, 0.2, 0.0])
    q[-1] = 2.5 + 0.5 * (q[1:4] ** 2).sum() / q[0]
    g = fr.Mesh(cfg)
    g.set_state(keys, np.broadcast_to(q[None, :, None], (M, nv, N)).copy())
    assert np.abs(g.rhs()).max() < tol


def test_double_word_100_steps_with_adaptation():
    cfg = _cfg("vortex2d_p2_small")
    g = fr.Mesh(dict(cfg, precision=4))
    o = O.OracleMesh(cfg)
    assert np.array_equal(g.leaves(), o.leaves())
    for cycle in range(10):
        g.step(10)
        o.step(10)
        assert rel_l2(g.state(), o.state()) < 1e-10
        fo, eo = o.flags()
        g.adapt(fo)
        o.adapt(fo)
        assert np.array_equal(g.leaves(), o.leaves()), cycle
    assert rel_l2(g.state(), o.state()) < 1e-10
    ng, no = g.norms(), o.norms()
    assert abs(ng["l2_rho"] - no["l2_rho"]) < 1e-8 * no["l2_rho"]


def test_fp32_mixed_form_error_is_bounded():
    # the mixed form drifts from FP64 by FP32 rounding only: after 50 steps of the small vortex
    # the state differs by < 1e-6 relative L2 and the vortex L2 error by < 1%
    cfg = _cfg("vortex2d_p2_small")
    g64 = fr.Mesh(cfg)
    g32 = fr.Mesh(dict(cfg, precision=1))
    g64.step(50)
    g32.step(50)
    assert rel_l2(g32.state(), g64.state()) < 1e-6
    e64, e32 = g64.norms()["l2_rho"], g32.norms()["l2_rho"]
    assert abs(e32 - e64) < 0.01 * e64
    # conservation of the mixed form holds to FP32 rounding of the fluxes
    i64, i32 = np.array(g64.norms()["integral"]), np.array(g32.norms()["integral"])
    assert np.allclose(i32, i64, rtol=1e-6)

"""Error paths of the library on the GPU, with failures made on the host: an adaptation whose
device allocation fails (the binding's allocator returns NULL) must leave the mesh as it was, and
the mesh must keep stepping exactly like the oracle.  No GPU fault is involved."""
import numpy as np
import pytest

import oracle as O
from paper_2306_06744_gb300 import fr
from paper_2306_06744_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def rel_l2(a, b):
    return float(np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(b.ravel()), 1e-300))


def test_failed_adaptation_leaves_mesh_usable():
    cfg = W.config("vortex2d_p2_small")
    g = fr.Mesh(cfg)
    o = O.OracleMesh(cfg)
    g.step(3)
    o.step(3)
    keys0, u0 = g.leaves().copy(), g.state().copy()
    nbr0, ft0, sl0 = (a.copy() for a in g.conn())
    # refine every leaf, so the adaptation needs blocks larger than any the mesh holds, and fail
    # the k-th allocation of the call for k = 0, 1, ... until one adaptation goes through
    flags = np.ones(g.M, dtype=np.int8)
    failed = 0
    for k in range(200):
        g._alloc.fail_in = k
        try:
            g.adapt(flags)
        except fr.FRError as e:
            assert e.code == fr.FR_ENOMEM
            failed += 1
            # nothing of the mesh changed: keys, state and connectivity as before the call
            assert np.array_equal(g.leaves(), keys0)
            assert np.array_equal(g.state(), u0)
            nbr, ft, sl = g.conn()
            assert np.array_equal(nbr, nbr0) and np.array_equal(ft, ft0) and np.array_equal(sl, sl0)
            continue
        finally:
            g._alloc.fail_in = None
        break
    assert failed >= 1, "no allocation of the adaptation was failed: the test pins nothing"
    # the adaptation that went through, and the steps after it, match the oracle
    o.adapt(flags)
    assert np.array_equal(g.leaves(), o.leaves())
    g.step(5)
    o.step(5)
    assert rel_l2(g.state(), o.state()) < 1e-10

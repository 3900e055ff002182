"""GPU parity of the tree kernels against the oracle, through the C ABI (bit-exact)."""
import numpy as np
import pytest

import oracle as O
from paper_2306_06744_gb300 import fr
from paper_2306_06744_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _tree(dim, Dbase, Dmax, seed, p, max_leaves=200000):
    boxes = W.random_tree_boxes(dim, Dbase, Dmax, seed=seed, p_split=p, max_leaves=max_leaves)
    return boxes, np.sort(O.morton_encode(dim, Dmax, boxes))


@pytest.mark.parametrize("dim,Dmax", [(2, 6), (2, 20), (3, 5), (3, 10), (3, 19)])
def test_encode(dim, Dmax):
    boxes = W.random_tree_boxes(dim, 2, Dmax, seed=3 + Dmax, p_split=0.3, max_leaves=50000)
    assert np.array_equal(fr.morton_encode(dim, Dmax, boxes), O.morton_encode(dim, Dmax, boxes))


def test_encode_rejects_misaligned_box():
    with pytest.raises(fr.FRError) as e:
        fr.morton_encode(2, 4, np.array([[2, 1, 0, 0]]))
    assert e.value.code == fr.FR_EINVAL


@pytest.mark.parametrize("n", [0, 1, 2, 2047, 2048, 2049, 6000, 100003, 1 << 20])
def test_sort(n):
    rng = np.random.default_rng(n)
    keys = rng.integers(0, 1 << 34, size=n, dtype=np.uint64)
    keys[: n // 3] = keys[n // 3: 2 * (n // 3)]  # duplicates
    got = fr.keys_sort(3, 10, keys)
    assert np.array_equal(got, np.sort(keys))


@pytest.mark.parametrize("dim,Dbase,Dmax,seed,p", [(2, 2, 6, 1, 0.4), (2, 3, 9, 2, 0.3),
                                                    (3, 2, 5, 3, 0.3), (3, 1, 7, 4, 0.25)])
def test_linearise(dim, Dbase, Dmax, seed, p):
    boxes, keys = _tree(dim, Dbase, Dmax, seed, p)
    extra = []
    for b in boxes[::2]:
        d = b[0]
        while d > 0:
            d -= 1
            w = 1 << (Dmax - d)
            extra.append([d, b[1] // w * w, b[2] // w * w, b[3] // w * w if dim == 3 else 0])
    allk = np.concatenate([keys, keys[::3], O.morton_encode(dim, Dmax, np.array(extra))])
    np.random.default_rng(seed).shuffle(allk)
    assert np.array_equal(fr.keys_linearise(dim, Dmax, allk), O.linearise(dim, Dmax, allk))


@pytest.mark.parametrize("dim,Dbase,Dmax,seed,p", [(2, 1, 6, 11, 0.4), (2, 2, 9, 12, 0.3),
                                                    (2, 3, 12, 13, 0.25), (3, 1, 5, 14, 0.35),
                                                    (3, 2, 7, 15, 0.25)])
def test_balance(dim, Dbase, Dmax, seed, p):
    _, keys = _tree(dim, Dbase, Dmax, seed, p)
    want = O.balance(dim, Dmax, keys)
    assert len(want) > len(keys)  # the case must need balancing
    assert np.array_equal(fr.tree_balance(dim, Dmax, keys), want)


@pytest.mark.parametrize("dim,Dbase,Dmax,seed", [(2, 3, 8, 21), (2, 4, 10, 22), (3, 2, 6, 23)])
def test_adapt_map_conn(dim, Dbase, Dmax, seed):
    _, keys = _tree(dim, Dbase, Dmax, seed, 0.25)
    keys = O.balance(dim, Dmax, keys)
    flags = W.random_flags(len(keys), seed, p_refine=0.1, p_coarsen=0.8)
    want = O.adapt_keys(dim, Dbase, Dmax, keys, flags)
    got = fr.tree_adapt(dim, Dbase, Dmax, keys, flags)
    assert np.array_equal(got, want)
    s_o, t_o = O.map_trees(dim, Dmax, keys, want)
    s_g, t_g = fr.tree_map(dim, Dmax, keys, got)
    assert np.array_equal(s_g, s_o) and np.array_equal(t_g, t_o)
    assert set(np.unique(t_o)) == {0, 1, 2}
    for a, b in zip(fr.tree_conn(dim, Dmax, got), O.conn(dim, Dmax, want)):
        assert np.array_equal(a, b)


@pytest.mark.parametrize("dim", [2, 3])
def test_degenerate_trees(dim):
    # the root alone (its own neighbour through every periodic face) and the 2^dim leaves of
    # depth 1: balance, connectivity, fusing every leaf back into the root and refining the root
    Dmax = 4
    root = O.morton_encode(dim, Dmax, np.array([[0, 0, 0, 0]]))
    kids = np.sort(O.morton_encode(dim, Dmax, np.array(
        [[1, (c & 1) * 8, ((c >> 1) & 1) * 8, ((c >> 2) & 1) * 8 if dim == 3 else 0] for c in range(1 << dim)])))
    for keys in (root, kids):
        assert np.array_equal(fr.tree_balance(dim, Dmax, keys), O.balance(dim, Dmax, keys))
        for a, b in zip(fr.tree_conn(dim, Dmax, keys), O.conn(dim, Dmax, keys)):
            assert np.array_equal(a, b)
    for keys, flag, Dbase in ((kids, -1, 0), (root, 1, 0), (kids, -1, 1), (kids, 1, 1)):
        flags = np.full(len(keys), flag, dtype=np.int8)
        want = O.adapt_keys(dim, Dbase, Dmax, keys, flags)
        got = fr.tree_adapt(dim, Dbase, Dmax, keys, flags)
        assert np.array_equal(got, want)
        s_o, t_o = O.map_trees(dim, Dmax, keys, want)
        s_g, t_g = fr.tree_map(dim, Dmax, keys, got)
        assert np.array_equal(s_g, s_o) and np.array_equal(t_g, t_o)


def test_conn_rejects_unbalanced():
    dim, Dmax = 2, 5
    boxes = [(1, 16, 0, 0), (1, 0, 16, 0), (1, 16, 16, 0)]
    q = [(1, 0, 0, 0)]
    for _ in range(3):
        c = q.pop(0)
        h = 1 << (Dmax - c[0] - 1)
        kids = [(c[0] + 1, c[1] + (k & 1) * h, c[2] + (k >> 1) * h, 0) for k in range(4)]
        q.append(kids[0])
        boxes += kids[1:]
    boxes += q
    keys = np.sort(O.morton_encode(dim, Dmax, np.array(boxes)))
    with pytest.raises(fr.FRError) as e:
        fr.tree_conn(dim, Dmax, keys)
    assert e.value.code == fr.FR_EINVAL
    # and balancing it first makes it valid
    bal = fr.tree_balance(dim, Dmax, keys)
    for a, b in zip(fr.tree_conn(dim, Dmax, bal), O.conn(dim, Dmax, O.balance(dim, Dmax, keys))):
        assert np.array_equal(a, b)


def test_balance_of_a_deep_strip_beside_a_coarse_leaf():
    # one quadrant refined to depth 14 along its right edge, beside a depth-1 leaf: the first
    # balance pass must split that leaf all the way down along 8192 finest cells, far more octants
    # than the room of the pass's single search (max(2^16, 2n)), so the pass is counted, scanned
    # and generated again at exact positions
    Dmax, X0 = 14, 8192
    boxes = [(1, 8192, 0, 0), (1, 0, 8192, 0), (1, 8192, 8192, 0)]
    stack = [(1, 0, 0)]
    while stack:
        d, x, y = stack.pop()
        w = 1 << (Dmax - d)
        if x + w == X0 and d < Dmax:
            for c in range(4):
                stack.append((d + 1, x + (c & 1) * (w // 2), y + (c >> 1) * (w // 2)))
        else:
            boxes.append((d, x, y, 0))
    keys = np.sort(O.morton_encode(2, Dmax, np.array(boxes)))
    want = O.balance(2, Dmax, keys)
    assert len(keys) == 24577 and len(want) == 37000
    assert np.array_equal(fr.tree_balance(2, Dmax, keys), want)


def test_large_balance_sampled():
    # a 2D tree of ~10^6 leaves at Dmax 14: compare the whole result (the oracle finishes it)
    _, keys = _tree(2, 6, 14, 99, 0.22, max_leaves=1200000)
    got = fr.tree_balance(2, 14, keys)
    want = O.balance(2, 14, keys)
    assert np.array_equal(got, want)


@pytest.mark.parametrize("dim,Dmin,Dmax,n,kind", [(2, 2, 8, 500, "uniform"), (2, 3, 12, 3000, "surface"),
                                                  (3, 1, 6, 800, "uniform"), (3, 4, 9, 20000, "surface"),
                                                  (3, 2, 5, 0, "uniform"), (2, 0, 10, 1, "uniform")])
def test_tree_complete(dim, Dmin, Dmax, n, kind):
    L = 2.5
    if kind == "uniform":
        pts = W.random_uniform(n * dim, 5 + n).reshape(n, dim) * L
    else:
        pts = W.torus_points(n, 9, dim, L)
    got = fr.tree_complete(dim, Dmin, Dmax, L, pts)
    want = O.tree_complete(dim, Dmin, Dmax, L, pts)
    assert np.array_equal(got, want)
    if 0 < n <= 3000:
        # the completed tree balances and connects like any other tree
        bal = fr.tree_balance(dim, Dmax, got)
        assert np.array_equal(bal, O.balance(dim, Dmax, want))

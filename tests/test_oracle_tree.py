"""Pins of the oracle's tree routines against hand-derived keys, the paper's worked example and
brute-force pairwise geometry on tiny trees (no GPU)."""
import os

import numpy as np
import pytest

import oracle as O
from paper_2306_06744_gb300 import workloads as W
from tests import brute

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _load(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            line = line.split("#")[0].strip()
            if line:
                rows.append(line.split())
    return rows


def test_keys_by_hand():
    for r in _load("morton_keys_by_hand.txt"):
        dim, Dmax, d, x, y, z, key = map(int, r)
        k = O.morton_encode(dim, Dmax, np.array([[d, x, y, z]]))
        assert int(k[0]) == key, r
        b = O.morton_decode(dim, Dmax, k)
        assert list(b[0]) == [d, x, y, z]


@pytest.mark.parametrize("dim,Dmax", [(2, 6), (3, 4), (2, 12), (3, 10)])
def test_encode_decode_roundtrip_and_order(dim, Dmax):
    boxes = W.random_tree_boxes(dim, min(2, Dmax), Dmax, seed=7, p_split=0.35, max_leaves=3000)
    keys = O.morton_encode(dim, Dmax, boxes)
    assert np.array_equal(O.morton_decode(dim, Dmax, keys), boxes)
    # pre-order: a parent sorts before its first child and the difference is exactly 1 (Sec. 3.2)
    for b in boxes[:200]:
        if b[0] == 0:
            continue
        w = 1 << (Dmax - b[0] + 1)
        par = [b[0] - 1, b[1] // w * w, b[2] // w * w, b[3] // w * w if dim == 3 else 0]
        kp = int(O.morton_encode(dim, Dmax, np.array([par]))[0])
        kc = int(O.morton_encode(dim, Dmax, np.array([[par[0] + 1] + par[1:]]))[0])
        assert kc - kp == 1
        assert kp < int(O.morton_encode(dim, Dmax, np.array([b]))[0])


def test_sibling_raw_ids_consecutive():
    # Sec. 4.1: the 2^dim siblings are stored consecutively, raw Morton IDs increasing by one
    dim, Dmax = 3, 3
    mb = 2
    par = [1, 4, 0, 4]
    kids = brute.children(dim, Dmax, tuple(par))
    keys = O.morton_encode(dim, Dmax, np.array(kids))
    raw = (keys >> np.uint64(mb)) >> np.uint64(dim * (Dmax - 2))
    assert list(np.diff(raw.astype(np.int64))) == [1] * 7
    assert list(np.argsort(keys)) == list(range(8))


def _tree(dim, Dbase, Dmax, seed, p):
    boxes = W.random_tree_boxes(dim, Dbase, Dmax, seed=seed, p_split=p)
    keys = np.sort(O.morton_encode(dim, Dmax, boxes))
    return boxes, keys


@pytest.mark.parametrize("dim,Dbase,Dmax,seed,p", [(2, 1, 4, 1, 0.4), (2, 2, 5, 2, 0.3),
                                                    (3, 1, 3, 3, 0.3), (2, 1, 5, 4, 0.5)])
def test_linearise_brute(dim, Dbase, Dmax, seed, p):
    boxes, keys = _tree(dim, Dbase, Dmax, seed, p)
    # add duplicates and every ancestor of a few leaves: linearisation must remove them
    extra = []
    for b in boxes[::3]:
        d = b[0]
        while d > 0:
            d -= 1
            w = 1 << (Dmax - d)
            extra.append([d, b[1] // w * w, b[2] // w * w, b[3] // w * w if dim == 3 else 0])
    allb = np.concatenate([boxes, boxes[::2], np.array(extra, dtype=np.int32).reshape(-1, 4)])
    k = O.morton_encode(dim, Dmax, allb)
    rng = np.random.default_rng(seed)
    rng.shuffle(k)
    lin = O.linearise(dim, Dmax, k)
    want = brute.linearise(Dmax, [tuple(b) for b in allb])
    got = sorted(tuple(b) for b in O.morton_decode(dim, Dmax, lin))
    assert got == want
    assert np.all(np.diff(lin.astype(np.float64)) > 0)


@pytest.mark.parametrize("dim,Dbase,Dmax,seed,p", [(2, 1, 4, 11, 0.4), (2, 1, 5, 12, 0.35),
                                                    (2, 2, 5, 13, 0.25), (3, 1, 3, 14, 0.35),
                                                    (3, 1, 4, 15, 0.3), (2, 1, 6, 16, 0.3)])
def test_balance_brute(dim, Dbase, Dmax, seed, p):
    boxes, keys = _tree(dim, Dbase, Dmax, seed, p)
    if len(boxes) > 700:
        pytest.skip("tree too large for the O(M^2) brute force")
    bal = O.balance(dim, Dmax, keys)
    got = sorted(tuple(b) for b in O.morton_decode(dim, Dmax, bal))
    want = brute.balance(dim, Dmax, [tuple(b) for b in boxes])
    assert got == want
    assert brute.is_balanced(dim, Dmax, got)
    assert brute.volume(dim, Dmax, got) == (1 << Dmax) ** dim
    # idempotent, and a refinement of the input
    assert np.array_equal(O.balance(dim, Dmax, bal), bal)
    for b in got:
        assert any(brute.contains(Dmax, a, b) for a in map(tuple, boxes))


def test_balance_periodic_wrap():
    # a single fine corner leaf at the origin forces refinement on the opposite (wrapped) corner
    dim, Dmax = 2, 4
    boxes = [(1, 8, 0, 0), (1, 0, 8, 0), (1, 8, 8, 0)]
    cell = (1, 0, 0, 0)
    q = [cell]
    for lev in range(3):  # refine the corner at the origin down to depth 4
        c = q.pop(0)
        kids = brute.children(dim, Dmax, c)
        q.append(kids[0])
        boxes += kids[1:]
    boxes += q
    keys = np.sort(O.morton_encode(dim, Dmax, np.array(boxes)))
    bal = sorted(tuple(b) for b in O.morton_decode(dim, Dmax, O.balance(dim, Dmax, keys)))
    assert bal == brute.balance(dim, Dmax, boxes)
    # the far corner (touching the origin through the periodic wrap) must now be at depth >= 3
    far = [b for b in bal if brute.contains(Dmax, b, (4, 15, 15, 0))][0]
    assert far[0] >= 3


@pytest.mark.parametrize("dim,Dbase,Dmax,seed,p", [(2, 1, 4, 21, 0.4), (2, 2, 5, 22, 0.3),
                                                    (3, 1, 3, 23, 0.3), (3, 1, 4, 24, 0.12)])
def test_conn_brute(dim, Dbase, Dmax, seed, p):
    boxes, keys = _tree(dim, Dbase, Dmax, seed, p)
    if len(boxes) > 700:
        pytest.skip("tree too large for the O(M^2) brute force")
    keys = O.balance(dim, Dmax, keys)
    bx = [tuple(b) for b in O.morton_decode(dim, Dmax, keys)]
    nbr, ft, sl = O.conn(dim, Dmax, keys)
    for e in range(len(bx)):
        for f in range(2 * dim):
            nb = brute.face_neighbours(dim, Dmax, bx, e, f)
            axis = f // 2
            if len(nb) == 1 and bx[nb[0]][0] == bx[e][0]:
                assert ft[e, f] == 0 and nbr[e, f] == nb[0] and sl[e, f] == -1
            elif len(nb) == 1 and bx[nb[0]][0] == bx[e][0] - 1:
                assert ft[e, f] == 1 and nbr[e, f] == nb[0]
                bits = brute.child_bits(dim, Dmax, bx[e])
                infc = [bits[b] for b in range(dim) if b != axis]
                assert sl[e, f] == sum(v << i for i, v in enumerate(infc))
            else:
                assert len(nb) == (1 << (dim - 1))
                assert all(bx[j][0] == bx[e][0] + 1 for j in nb)
                assert ft[e, f] == 2 and nbr[e, f] == min(nb)
                # the contributors see e as their coarse neighbour through the matching face
                for j in nb:
                    assert ft[j, f ^ 1] == 1 and nbr[j, f ^ 1] == e


def test_face_slots_paper_example():
    # 2D, Dmax 2: a coarse leaf at depth 1 on the left, the four children of the right-bottom
    # depth-1 box as leaves; Sec. 3.3 example (golden fixture).
    dim, Dmax = 2, 2
    boxes = [(1, 0, 0, 0), (1, 0, 2, 0), (1, 2, 2, 0)] + brute.children(dim, Dmax, (1, 2, 0, 0))
    keys = np.sort(O.morton_encode(dim, Dmax, np.array(boxes)))
    bx = [tuple(b) for b in O.morton_decode(dim, Dmax, keys)]
    nbr, ft, sl = O.conn(dim, Dmax, keys)
    for r in _load("face_slots_2d.txt"):
        c, f, slot = map(int, r)
        kid = brute.children(dim, Dmax, (1, 2, 0, 0))[c]
        e = bx.index(kid)
        assert ft[e, f] == 1, (c, f)
        assert sl[e, f] == slot, (c, f)


@pytest.mark.parametrize("dim,Dbase,Dmax,seed", [(2, 2, 5, 31), (3, 1, 4, 32), (2, 2, 6, 33)])
def test_adapt_and_map(dim, Dbase, Dmax, seed):
    boxes, keys = _tree(dim, Dbase, Dmax, seed, 0.25)
    keys = O.balance(dim, Dmax, keys)
    M = keys.shape[0]
    flags = W.random_flags(M, seed + 100, p_refine=0.15, p_coarsen=0.6)
    ob = [tuple(b) for b in O.morton_decode(dim, Dmax, keys)]
    # flag about half of the complete sibling groups entirely for coarsening
    coin = W.random_uniform(M, seed + 200)
    pos = {b: i for i, b in enumerate(ob)}
    for i, b in enumerate(ob):
        if b[0] == 0 or coin[i] > 0.5:
            continue
        w = 1 << (Dmax - b[0] + 1)
        par = (b[0] - 1, b[1] // w * w, b[2] // w * w, b[3] // w * w)
        kids = brute.children(dim, Dmax, par)
        if kids[0] == b and all(k in pos for k in kids):
            for k in kids:
                flags[pos[k]] = -1
    new = O.adapt_keys(dim, Dbase, Dmax, keys, flags)
    nb = [tuple(b) for b in O.morton_decode(dim, Dmax, new)]
    assert brute.volume(dim, Dmax, nb) == (1 << Dmax) ** dim
    if len(nb) <= 700:
        assert brute.is_balanced(dim, Dmax, nb)
    nset = set(nb)
    for i, b in enumerate(ob):
        if flags[i] == 1 and b[0] < Dmax:
            # refined: no new leaf contains b any more, and b is covered by its children or finer
            assert b not in nset
            assert not any(brute.contains(Dmax, a, b) for a in nb)
    # leaves change by at most one level
    src, tag = O.map_trees(dim, Dmax, keys, new)
    for j, b in enumerate(nb):
        a = ob[src[j]]
        if tag[j] == 0:
            assert a == b
        elif tag[j] == 1:
            assert brute.contains(Dmax, a, b) and b[0] == a[0] + 1
        else:
            assert tag[j] == 2 and brute.contains(Dmax, b, a) and a[0] == b[0] + 1
            kids = brute.children(dim, Dmax, b)
            assert ob[src[j]: src[j] + (1 << dim)] == kids
            # coarsening only where all siblings were flagged -1 and above Dbase
            assert all(flags[src[j] + c] == -1 for c in range(1 << dim))
            assert b[0] >= Dbase


def _point_cells(dim, Dmax, L, pts):
    side = 1 << Dmax
    cells = set()
    for p in pts:
        c = [min(side - 1, max(0, int(np.floor(p[a] / L * side)))) for a in range(dim)]
        cells.add((Dmax, c[0], c[1], c[2] if dim == 3 else 0))
    return cells


@pytest.mark.parametrize("dim,Dmin,Dmax,npts,seed", [(2, 2, 6, 40, 1), (2, 0, 7, 25, 2), (3, 1, 4, 30, 3),
                                                     (3, 2, 5, 12, 4)])
def test_tree_complete_properties(dim, Dmin, Dmax, npts, seed):
    # Sec. 3.1: the completed tree covers the domain, keeps every point cell as a leaf, stays at or
    # below Dmin, and is the coarsest such tree (no leaf could be merged into its parent)
    L = 3.0
    pts = (W.random_uniform(npts * dim, seed).reshape(npts, dim)) * L
    keys = O.tree_complete(dim, Dmin, Dmax, L, pts)
    boxes = [tuple(b) for b in O.morton_decode(dim, Dmax, keys)]
    assert np.all(np.diff(keys.astype(np.float64)) > 0)
    assert brute.volume(dim, Dmax, boxes) == (1 << Dmax) ** dim
    cells = _point_cells(dim, Dmax, L, pts)
    bset = set(boxes)
    assert cells <= bset
    assert all(b[0] >= Dmin for b in boxes)
    for b in boxes:
        if b in cells:
            continue
        w = 1 << (Dmax - b[0] + 1)
        par = (b[0] - 1, b[1] // w * w, b[2] // w * w, b[3] // w * w if dim == 3 else 0)
        assert par[0] < Dmin or any(brute.contains(Dmax, par, c) for c in cells), b


def test_tree_complete_closed_forms():
    # no points: the uniform grid at Dmin; one point: each of the Dmax-Dmin splits adds 2^dim-1
    for dim in (2, 3):
        assert len(O.tree_complete(dim, 2, 5, 1.0, np.zeros((0, dim)))) == (1 << (dim * 2))
        one = O.tree_complete(dim, 2, 5, 1.0, np.full((1, dim), 0.3))
        assert len(one) == (1 << (dim * 2)) + ((1 << dim) - 1) * (5 - 2)


def test_vectorised_draws_match_splitmix64():
    # the seeded input generator shared by tests and benchmark: vectorised draws = the scalar
    # SplitMix64 sequence, including a seed near 2^64 (wrap-around)
    for seed in (0, 7, 2 ** 64 - 3):
        r = W.SplitMix64(seed)
        want = np.array([r.uniform() for _ in range(257)])
        assert np.array_equal(W.random_uniform(257, seed), want)
    p = W.torus_points(1000, 3)
    assert p.shape == (1000, 3) and p.min() > 0.0 and p.max() < 1.0


@pytest.mark.parametrize("dim,Dbase,Dmax,seed,ps", [(2, 2, 5, 31, 0.25), (2, 2, 6, 33, 0.25), (2, 1, 5, 41, 0.3),
                                                    (3, 1, 3, 42, 0.25), (3, 1, 4, 43, 0.12)])
def test_adapt_keys_is_balance_of_brute_edit(dim, Dbase, Dmax, seed, ps):
    # Sec. 4.1 (edit, then 2:1 balance): the oracle's adaptation equals the brute-force edit by its
    # definition (refine flagged leaves, fuse complete all -1 sibling groups above Dbase) followed
    # by the brute-force balance closure; some fused parents must survive the balance, so an edit
    # that ignored the coarsening flags would fail here
    boxes, keys = _tree(dim, Dbase, Dmax, seed, ps)
    keys = O.balance(dim, Dmax, keys)
    M = keys.shape[0]
    ob = [tuple(b) for b in O.morton_decode(dim, Dmax, keys)]
    flags = W.random_flags(M, seed + 100, p_refine=0.1, p_coarsen=0.4)
    coin = W.random_uniform(M, seed + 200)
    pos = {b: i for i, b in enumerate(ob)}
    for i, b in enumerate(ob):
        if b[0] <= Dbase or coin[i] > 0.6:
            continue
        kids = brute.children(dim, Dmax, brute.parent(Dmax, b))
        if kids[0] == b and all(k in pos for k in kids):
            for k in kids:
                flags[pos[k]] = -1
    new = [tuple(b) for b in O.morton_decode(dim, Dmax, O.adapt_keys(dim, Dbase, Dmax, keys, flags))]
    edited, fused = brute.edit(dim, Dmax, Dbase, ob, flags)
    assert sorted(new) == brute.balance(dim, Dmax, edited)
    assert any(f in set(new) for f in fused), "no fused parent survived: the case pins nothing"

"""Brute-force geometry on tiny trees, used to pin the oracle's tree routines.

Boxes are (depth, x, y, z) with anchors in units of the finest cell (2^-Dmax of the domain).
Everything here is pairwise geometry with periodic wrap-around: no Morton keys, no search.
"""
import itertools


def width(Dmax, d):
    return 1 << (Dmax - d)


def contains(Dmax, A, B):
    """Box A contains box B."""
    if A[0] > B[0]:
        return False
    w = width(Dmax, A[0])
    return all(A[1 + a] <= B[1 + a] < A[1 + a] + w for a in range(3))


def _intervals_touch(a0, a1, b0, b1, n):
    """Closed periodic intervals [a0,a1] and [b0,b1] on a circle of length n intersect."""
    for s in (-n, 0, n):
        if a0 <= b1 + s and b0 + s <= a1:
            return True
    return False


def _intervals_overlap(a0, a1, b0, b1, n):
    """Open periodic intervals overlap with positive length."""
    for s in (-n, 0, n):
        if a0 < b1 + s and b0 + s < a1:
            return True
    return False


def touching(dim, Dmax, A, B):
    """Closed boxes intersect (periodic) and are different boxes."""
    if A == B:
        return False
    n = 1 << Dmax
    wa, wb = width(Dmax, A[0]), width(Dmax, B[0])
    return all(_intervals_touch(A[1 + a], A[1 + a] + wa, B[1 + a], B[1 + a] + wb, n)
               for a in range(dim))


def is_balanced(dim, Dmax, boxes):
    for A, B in itertools.combinations(boxes, 2):
        if touching(dim, Dmax, A, B) and abs(A[0] - B[0]) > 1:
            return False
    return True


def children(dim, Dmax, A):
    d = A[0] + 1
    h = width(Dmax, d)
    out = []
    for c in range(1 << dim):
        out.append((d, A[1] + (c & 1) * h, A[2] + ((c >> 1) & 1) * h,
                    A[3] + ((c >> 2) & 1) * h if dim == 3 else 0))
    return out


def balance(dim, Dmax, boxes):
    """Split any leaf touching a leaf two or more levels finer, until nothing changes (O(M^2))."""
    cur = sorted(set(map(tuple, boxes)))
    while True:
        split = set()
        for A in cur:
            for B in cur:
                if B[0] >= A[0] + 2 and touching(dim, Dmax, A, B):
                    split.add(A)
                    break
        if not split:
            return cur
        nxt = [b for b in cur if b not in split]
        for A in split:
            nxt.extend(children(dim, Dmax, A))
        cur = sorted(set(nxt))


def linearise(Dmax, boxes):
    s = set(map(tuple, boxes))
    return sorted(A for A in s if not any(B != A and contains(Dmax, A, B) for B in s))


def volume(dim, Dmax, boxes):
    return sum(width(Dmax, b[0]) ** dim for b in boxes)


def face_neighbours(dim, Dmax, boxes, e, f):
    """Leaves sharing a (dim-1)-face region of positive measure with face f of leaf e."""
    n = 1 << Dmax
    E = boxes[e]
    axis, side = f // 2, f % 2
    we = width(Dmax, E[0])
    plane = (E[1 + axis] + (we if side else 0)) % n
    out = []
    for j, B in enumerate(boxes):
        wb = width(Dmax, B[0])
        # B's opposite face lies on the plane
        bplane = (B[1 + axis] + (0 if side else wb)) % n
        if bplane != plane:
            continue
        if all(_intervals_overlap(E[1 + b], E[1 + b] + we, B[1 + b], B[1 + b] + wb, n)
               for b in range(dim) if b != axis):
            out.append(j)
    return out


def child_bits(dim, Dmax, B):
    w = width(Dmax, B[0])
    return [(B[1 + a] // w) & 1 for a in range(dim)]


def parent(Dmax, A):
    w = width(Dmax, A[0] - 1)
    return (A[0] - 1, A[1] // w * w, A[2] // w * w, A[3] // w * w)


def edit(dim, Dmax, Dbase, boxes, flags):
    """The refine/coarsen edit by its definition (Sec. 4.1), with refinement clamped at Dmax and
    coarsening at Dbase: a leaf flagged 1 below Dmax becomes its 2^dim children; a complete group
    of 2^dim sibling leaves, every one flagged -1 and deeper than Dbase, becomes its parent; every
    other leaf stays.  Returns the edited leaves (sorted) and the parents that fused."""
    boxes = [tuple(b) for b in boxes]
    pos = {b: i for i, b in enumerate(boxes)}
    out, fused = set(), set()
    for i, b in enumerate(boxes):
        if flags[i] == 1 and b[0] < Dmax:
            out.update(children(dim, Dmax, b))
            continue
        if flags[i] == -1 and b[0] > Dbase:
            par = parent(Dmax, b)
            if all(k in pos and flags[pos[k]] == -1 for k in children(dim, Dmax, par)):
                out.add(par)
                fused.add(par)
                continue
        out.add(b)
    return sorted(out), sorted(fused)

"""Seeded synthetic inputs shared by the GPU library's callers and by the oracle's tests.

This module holds no arithmetic of the method: it only describes the vortex workloads as plain
parameter dictionaries and draws seeded random numbers (vortex centres and strengths, random
refinement patterns given as boxes, random flags, random perturbations).  Both the GPU path and
the CPU oracle receive the same dictionaries and arrays and do all method arithmetic themselves.

Random numbers come from splitmix64 (Steele, Lea & Flood, "Fast splittable pseudorandom number
generators", OOPSLA 2014), written out from its published definition.
"""
from __future__ import annotations

import numpy as np

_MASK = (1 << 64) - 1


class SplitMix64:
    """splitmix64: state += golden gamma; two xor-shift-multiply rounds; final xor-shift."""

    def __init__(self, seed: int):
        self.state = seed & _MASK

    def next_u64(self) -> int:
        self.state = (self.state + 0x9E3779B97F4A7C15) & _MASK
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK
        return z ^ (z >> 31)

    def uniform(self) -> float:
        """Uniform double in [0, 1) from the top 53 bits."""
        return (self.next_u64() >> 11) * (1.0 / 9007199254740992.0)


def vortex_centres(seed: int, count: int, L: float, min_sep: float = 0.0,
                   beta_range=(5.0, 5.0), core: float = 1.0, max_tries: int = 100000):
    """Seeded vortex list [count][4] = (xc, yc, beta, core radius), centres uniform in [0,L)^2.

    With ``min_sep`` > 0 the centres are drawn by rejection so that every pair, including the
    nearest periodic images, is at least ``min_sep`` apart.
    """
    rng = SplitMix64(seed)
    out = []
    tries = 0
    while len(out) < count:
        tries += 1
        if tries > max_tries:
            raise ValueError("could not place the vortices with the requested separation")
        x, y = rng.uniform() * L, rng.uniform() * L
        ok = True
        for (xo, yo, _, _) in out:
            dx = abs(x - xo)
            dy = abs(y - yo)
            dx = min(dx, L - dx)
            dy = min(dy, L - dy)
            if dx * dx + dy * dy < min_sep * min_sep:
                ok = False
                break
        if not ok:
            continue
        lo, hi = beta_range
        beta = lo + (hi - lo) * rng.uniform()
        out.append((x, y, beta, core))
    return np.array(out, dtype=np.float64).reshape(count, 4)


def _base(**kw):
    cfg = dict(dim=2, p=2, L=10.0, Dbase=4, Dmax=6, gamma=1.4,
               vort=np.array([[5.0, 5.0, 5.0, 1.0]]), uinf=(1.0, 1.0, 0.0),
               rho_inf=1.0, p_inf=1.0, cfl=0.3, dt=0.0, adapt_every=10, indicator=0,
               th_refine=0.05, th_coarsen=0.01, precision=0, init_passes=-1, steps=100)
    cfg.update(kw)
    return cfg


def config(name: str) -> dict:
    """The vortex workloads by name.

    vortex2d_p2_small : 2D, p=2, periodic [0,10]^2, base level 4, max level 6, one vortex at the
                        centre (beta 5, core 1), freestream u=v=1, rho=p=1, CFL 0.3, 100 steps,
                        adaptation every 10 steps, density-gradient indicator, FP64.
    vortex2d_p3       : 2D, p=3, periodic [0,40]^2, seeded centre (seed 1), base level 5, max 9,
                        1000 steps.
    vortex3d_p2_tube  : 3D tube (2D profile extruded along z), p=2, periodic [0,10]^3, base 4,
                        max 7, 500 steps.
    vortex3d_p3_multi : 3D, p=3, periodic [0,80]^3, four seeded tubes (seed 3, beta in [3,6],
                        pairwise separation >= 16), base 5, max 10.
    The 2D p=3 thresholds (1e-8, 2.5e-9) refine wherever the density varies by more than about the
    p=3 error level across an element; a single core-1 vortex then gives 19k-26k leaves.  The 3D
    thresholds put the initial meshes in the stated ranges: 177k leaves for the tube (50k-200k)
    and 2.95M for the four tubes (2M-4M).
    """
    if name == "vortex2d_p2_small":
        return _base()
    if name == "vortex2d_p3":
        return _base(p=3, L=40.0, Dbase=5, Dmax=9, vort=vortex_centres(1, 1, 40.0),
                     th_refine=1e-8, th_coarsen=2.5e-9, steps=1000)
    if name == "vortex3d_p2_tube":
        return _base(dim=3, p=2, L=10.0, Dbase=4, Dmax=7, vort=np.array([[5.0, 5.0, 5.0, 1.0]]),
                     th_refine=0.03, th_coarsen=0.0075, steps=500)
    if name == "vortex3d_p3_multi":
        return _base(dim=3, p=3, L=80.0, Dbase=5, Dmax=10,
                     vort=vortex_centres(3, 4, 80.0, min_sep=16.0, beta_range=(3.0, 6.0)),
                     th_refine=0.05, th_coarsen=0.0125, steps=100)
    raise KeyError(name)


CONFIG_NAMES = ("vortex2d_p2_small", "vortex2d_p3", "vortex3d_p2_tube", "vortex3d_p3_multi")


def random_tree_boxes(dim: int, Dbase: int, Dmax: int, seed: int, p_split: float = 0.3,
                      max_leaves: int = 200000) -> np.ndarray:
    """A random complete tree given as boxes [n][4] = (depth, x, y, z), anchors in finest units.

    Starts from the uniform grid at ``Dbase`` and visits boxes depth by depth; each box below
    ``Dmax`` is split into its 2^dim equal sub-boxes with probability ``p_split``.  Pure geometry:
    the caller encodes and orders the boxes.  The result is complete but not 2:1 balanced.
    """
    rng = SplitMix64(seed)
    side = 1 << Dbase
    w = 1 << (Dmax - Dbase)
    work = []
    for k in range(side ** dim):
        x = (k % side) * w
        y = ((k // side) % side) * w
        z = (k // (side * side)) * w if dim == 3 else 0
        work.append((Dbase, x, y, z))
    out = []
    while work:
        nxt = []
        for (d, x, y, z) in work:
            if d < Dmax and rng.uniform() < p_split and len(out) + len(nxt) + len(work) < max_leaves:
                h = 1 << (Dmax - d - 1)
                for c in range(1 << dim):
                    nxt.append((d + 1, x + (c & 1) * h, y + ((c >> 1) & 1) * h,
                                z + ((c >> 2) & 1) * h if dim == 3 else 0))
            else:
                out.append((d, x, y, z))
        work = nxt
    return np.array(out, dtype=np.int32).reshape(-1, 4)


def random_flags(n: int, seed: int, p_refine: float = 0.2, p_coarsen: float = 0.5) -> np.ndarray:
    """Seeded int8 flags in {-1, 0, 1}."""
    rng = SplitMix64(seed)
    out = np.zeros(n, dtype=np.int8)
    for i in range(n):
        r = rng.uniform()
        out[i] = 1 if r < p_refine else (-1 if r < p_refine + p_coarsen else 0)
    return out


def random_uniform(n: int, seed: int) -> np.ndarray:
    """n seeded uniforms in [0,1): the first n draws of SplitMix64(seed), vectorised (the k-th
    state is seed + k * gamma modulo 2^64)."""
    with np.errstate(over="ignore"):
        k = np.arange(1, n + 1, dtype=np.uint64)
        z = np.uint64(seed & _MASK) + k * np.uint64(0x9E3779B97F4A7C15)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        z = z ^ (z >> np.uint64(31))
    return (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def torus_points(n: int, seed: int, dim: int = 3, L: float = 1.0) -> np.ndarray:
    """n seeded points on a torus surface (3D: radii 0.28 and 0.1 about the centre of the box) or a
    circle (2D: radius 0.3), inside [0, L)^dim: a synthetic stand-in for a scanned surface."""
    u = random_uniform(2 * n, seed).reshape(n, 2) * 2 * np.pi
    if dim == 2:
        return np.stack([0.5 + 0.3 * np.cos(u[:, 0]), 0.5 + 0.3 * np.sin(u[:, 0])], 1) * L
    R, r = 0.28, 0.1
    x = (R + r * np.cos(u[:, 1])) * np.cos(u[:, 0])
    y = (R + r * np.cos(u[:, 1])) * np.sin(u[:, 0])
    z = r * np.sin(u[:, 1])
    return (np.stack([x, y, z], 1) + 0.5) * L

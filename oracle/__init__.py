"""ctypes binding of the CPU oracle (``oracle/fr_oracle.cpp``).

TEST INFRASTRUCTURE ONLY: imported by the test suite, the smoke check and the benchmark's
CPU-baseline leg.  The GPU library and its Python binding never import this package.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fr_oracle.cpp")
_LIB = os.path.join(_HERE, "libfr_oracle.so")


def build(force: bool = False) -> str:
    """Compile the oracle with the host C++ compiler (plain -O2, no FMA contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < max(
            os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "fr_oracle.h"))):
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-fPIC", "-shared",
                               "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


class OracleConfig(C.Structure):
    _fields_ = [("dim", C.c_int32), ("p", C.c_int32), ("L", C.c_double),
                ("Dbase", C.c_int32), ("Dmax", C.c_int32), ("gamma", C.c_double),
                ("nvort", C.c_int32), ("vort", C.POINTER(C.c_double)),
                ("uinf", C.c_double * 3), ("rho_inf", C.c_double), ("p_inf", C.c_double),
                ("cfl", C.c_double), ("dt", C.c_double), ("adapt_every", C.c_int32),
                ("indicator", C.c_int32), ("th_refine", C.c_double), ("th_coarsen", C.c_double),
                ("precision", C.c_int32), ("init_passes", C.c_int32)]


class OracleNorms(C.Structure):
    _fields_ = [("t", C.c_double), ("l2_rho", C.c_double), ("integral", C.c_double * 5),
                ("min_rho", C.c_double), ("min_p", C.c_double), ("M", C.c_int64)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        _lib.oracle_last_error.restype = C.c_char_p
        _lib.oracle_rk3_scalar.restype = C.c_double
        _lib.oracle_rk3_scalar.argtypes = [C.c_double, C.c_double, C.c_double]
        _lib.oracle_correction_gL.restype = C.c_double
        _lib.oracle_correction_gL.argtypes = [C.c_int, C.c_double]
        _lib.oracle_mesh_free.argtypes = [C.c_void_p]
    return _lib


def _ptr(a, ct):
    return a.ctypes.data_as(C.POINTER(ct))


def _check(rc):
    if rc != 0:
        raise RuntimeError("oracle error %d: %s" % (rc, lib().oracle_last_error().decode()))


def make_config(cfg: dict):
    vort = np.ascontiguousarray(np.asarray(cfg["vort"], dtype=np.float64).reshape(-1, 4))
    c = OracleConfig(dim=cfg["dim"], p=cfg["p"], L=cfg["L"], Dbase=cfg["Dbase"], Dmax=cfg["Dmax"],
                     gamma=cfg["gamma"], nvort=vort.shape[0], vort=_ptr(vort, C.c_double),
                     rho_inf=cfg["rho_inf"], p_inf=cfg["p_inf"], cfl=cfg["cfl"], dt=cfg["dt"],
                     adapt_every=cfg["adapt_every"], indicator=cfg["indicator"],
                     th_refine=cfg["th_refine"], th_coarsen=cfg["th_coarsen"],
                     precision=cfg.get("precision", 0), init_passes=cfg.get("init_passes", -1))
    for a in range(3):
        c.uinf[a] = cfg["uinf"][a]
    return c, vort  # keep vort alive with the struct


# ---- primitives ----

def morton_encode(dim, Dmax, boxes):
    boxes = np.ascontiguousarray(boxes, dtype=np.int32).reshape(-1, 4)
    keys = np.zeros(boxes.shape[0], dtype=np.uint64)
    _check(lib().oracle_morton_encode(dim, Dmax, C.c_int64(boxes.shape[0]), _ptr(boxes, C.c_int32),
                                      _ptr(keys, C.c_uint64)))
    return keys


def morton_decode(dim, Dmax, keys):
    keys = np.ascontiguousarray(keys, dtype=np.uint64)
    boxes = np.zeros((keys.shape[0], 4), dtype=np.int32)
    _check(lib().oracle_morton_decode(dim, Dmax, C.c_int64(keys.shape[0]), _ptr(keys, C.c_uint64),
                                      _ptr(boxes, C.c_int32)))
    return boxes


def _keys_call(fn, dim, Dmax, keys, cap_factor, *extra_front):
    keys = np.ascontiguousarray(keys, dtype=np.uint64)
    cap = max(16, keys.shape[0] * cap_factor)
    out = np.zeros(cap, dtype=np.uint64)
    nout = C.c_int64(0)
    _check(fn(*extra_front, _ptr(keys, C.c_uint64), C.c_int64(keys.shape[0]), _ptr(out, C.c_uint64),
              C.c_int64(cap), C.byref(nout)))
    return out[: nout.value].copy()


def linearise(dim, Dmax, keys):
    return _keys_call(lib().oracle_linearise, dim, Dmax, keys, 1, dim, Dmax)


def balance(dim, Dmax, keys):
    keys = np.ascontiguousarray(keys, dtype=np.uint64)
    cap = max(64, keys.shape[0] * (1 << dim) * 8)
    out = np.zeros(cap, dtype=np.uint64)
    nout = C.c_int64(0)
    _check(lib().oracle_balance(dim, Dmax, _ptr(keys, C.c_uint64), C.c_int64(keys.shape[0]),
                                _ptr(out, C.c_uint64), C.c_int64(cap), C.byref(nout)))
    return out[: nout.value].copy()


def tree_complete(dim, Dmin, Dmax, L, pts):
    pts = np.ascontiguousarray(pts, dtype=np.float64).reshape(-1, dim)
    cap = 1024
    while True:
        out = np.zeros(cap, dtype=np.uint64)
        nout = C.c_int64(0)
        rc = lib().oracle_tree_complete(dim, Dmin, Dmax, C.c_double(L), _ptr(pts, C.c_double),
                                        C.c_int64(pts.shape[0]), _ptr(out, C.c_uint64),
                                        C.c_int64(cap), C.byref(nout))
        if rc == -3 and nout.value > cap:
            cap = nout.value
            continue
        _check(rc)
        return out[: nout.value].copy()


def adapt_keys(dim, Dbase, Dmax, keys, flags):
    keys = np.ascontiguousarray(keys, dtype=np.uint64)
    flags = np.ascontiguousarray(flags, dtype=np.int8)
    cap = max(64, keys.shape[0] * (1 << dim) * 8)
    out = np.zeros(cap, dtype=np.uint64)
    nout = C.c_int64(0)
    _check(lib().oracle_adapt_keys(dim, Dbase, Dmax, _ptr(keys, C.c_uint64), _ptr(flags, C.c_int8),
                                   C.c_int64(keys.shape[0]), _ptr(out, C.c_uint64), C.c_int64(cap),
                                   C.byref(nout)))
    return out[: nout.value].copy()


def map_trees(dim, Dmax, old_keys, new_keys):
    o = np.ascontiguousarray(old_keys, dtype=np.uint64)
    n = np.ascontiguousarray(new_keys, dtype=np.uint64)
    src = np.zeros(n.shape[0], dtype=np.int32)
    tag = np.zeros(n.shape[0], dtype=np.int8)
    _check(lib().oracle_map(dim, Dmax, _ptr(o, C.c_uint64), C.c_int64(o.shape[0]),
                            _ptr(n, C.c_uint64), C.c_int64(n.shape[0]), _ptr(src, C.c_int32),
                            _ptr(tag, C.c_int8)))
    return src, tag


def conn(dim, Dmax, keys):
    keys = np.ascontiguousarray(keys, dtype=np.uint64)
    M = keys.shape[0]
    nbr = np.zeros(M * 2 * dim, dtype=np.int32)
    ftype = np.zeros(M * 2 * dim, dtype=np.int8)
    slot = np.zeros(M * 2 * dim, dtype=np.int8)
    _check(lib().oracle_conn(dim, Dmax, _ptr(keys, C.c_uint64), C.c_int64(M), _ptr(nbr, C.c_int32),
                             _ptr(ftype, C.c_int8), _ptr(slot, C.c_int8)))
    return nbr.reshape(M, 2 * dim), ftype.reshape(M, 2 * dim), slot.reshape(M, 2 * dim)


def operators(p):
    n = p + 1
    x, w, lm, lp, gL, gR = (np.zeros(n) for _ in range(6))
    D = np.zeros((n, n))
    _check(lib().oracle_operators(p, *(_ptr(a, C.c_double) for a in (x, w, D, lm, lp, gL, gR))))
    return dict(x=x, w=w, D=D, lm=lm, lp=lp, gL=gL, gR=gR)


def correction_gL(p, x):
    return lib().oracle_correction_gL(p, x)


def rk3_scalar(lam, u0, dt):
    return lib().oracle_rk3_scalar(lam, u0, dt)


def prolong(dim, p, parent, child):
    parent = np.ascontiguousarray(parent, dtype=np.float64)
    out = np.zeros_like(parent)
    nv = parent.shape[0]
    _check(lib().oracle_prolong(dim, p, nv, _ptr(parent, C.c_double), child, _ptr(out, C.c_double)))
    return out


def restrict(dim, p, children):
    children = np.ascontiguousarray(children, dtype=np.float64)
    nv = children.shape[1]
    out = np.zeros(children.shape[1:], dtype=np.float64)
    _check(lib().oracle_restrict(dim, p, nv, _ptr(children, C.c_double), _ptr(out, C.c_double)))
    return out


def exact(cfg: dict, t: float, xyz):
    c, _keep = make_config(cfg)
    xyz = np.ascontiguousarray(xyz, dtype=np.float64).reshape(-1, 3)
    nv = cfg["dim"] + 2
    q = np.zeros((xyz.shape[0], nv))
    _check(lib().oracle_exact(C.byref(c), C.c_double(t), C.c_int64(xyz.shape[0]),
                              _ptr(xyz, C.c_double), _ptr(q, C.c_double)))
    return q


class OracleMesh:
    """The oracle's mesh-level calls (same names as the GPU library, without prefix)."""

    def __init__(self, cfg: dict):
        self.cfg = dict(cfg)
        self.dim, self.p = cfg["dim"], cfg["p"]
        self.n = self.p + 1
        self.N = self.n ** self.dim
        self.nv = self.dim + 2
        c, self._vort = make_config(cfg)
        self._c = c
        h = C.c_void_p()
        _check(lib().oracle_mesh_init(C.byref(c), C.byref(h)))
        self.h = h

    def __del__(self):
        if getattr(self, "h", None) and self.h.value:
            lib().oracle_mesh_free(self.h)
            self.h = C.c_void_p()

    @property
    def M(self):
        m = C.c_int64(0)
        _check(lib().oracle_get_leaves(self.h, None, C.c_int64(0), C.byref(m)))
        return m.value

    def info(self):
        t, dt, M, st = C.c_double(), C.c_double(), C.c_int64(), C.c_int64()
        _check(lib().oracle_get_info(self.h, C.byref(t), C.byref(dt), C.byref(M), C.byref(st)))
        return dict(t=t.value, dt=dt.value, M=M.value, step=st.value)

    def step(self, nsteps=1):
        _check(lib().oracle_step(self.h, C.c_int(nsteps)))

    def run(self, nsteps):
        _check(lib().oracle_run(self.h, C.c_int(nsteps)))

    def adapt(self, flags=None):
        if flags is None:
            _check(lib().oracle_adapt(self.h, None))
        else:
            f = np.ascontiguousarray(flags, dtype=np.int8)
            assert f.shape[0] == self.M
            _check(lib().oracle_adapt(self.h, _ptr(f, C.c_int8)))

    def flags(self):
        M = self.M
        f = np.zeros(M, dtype=np.int8)
        eta = np.zeros(M)
        _check(lib().oracle_flags(self.h, _ptr(f, C.c_int8), _ptr(eta, C.c_double), C.c_int64(M)))
        return f, eta

    def rhs(self):
        M = self.M
        R = np.zeros((M, self.nv, self.N))
        _check(lib().oracle_rhs(self.h, _ptr(R, C.c_double), C.c_int64(R.size)))
        return R

    def norms(self):
        o = OracleNorms()
        _check(lib().oracle_norms(self.h, C.byref(o)))
        return dict(t=o.t, l2_rho=o.l2_rho, integral=list(o.integral)[: self.nv],
                    min_rho=o.min_rho, min_p=o.min_p, M=o.M)

    def leaves(self):
        M = self.M
        k = np.zeros(M, dtype=np.uint64)
        m = C.c_int64(0)
        _check(lib().oracle_get_leaves(self.h, _ptr(k, C.c_uint64), C.c_int64(M), C.byref(m)))
        return k

    def state(self):
        M = self.M
        u = np.zeros((M, self.nv, self.N))
        _check(lib().oracle_get_state(self.h, _ptr(u, C.c_double), C.c_int64(u.size)))
        return u

    def set_state(self, keys, u):
        keys = np.ascontiguousarray(keys, dtype=np.uint64)
        u = np.ascontiguousarray(u, dtype=np.float64)
        assert u.size == keys.shape[0] * self.nv * self.N
        _check(lib().oracle_set_state(self.h, _ptr(keys, C.c_uint64), C.c_int64(keys.shape[0]),
                                      _ptr(u, C.c_double)))

    def set_time(self, t):
        _check(lib().oracle_set_time(self.h, C.c_double(t)))

    def conn(self):
        M = self.M
        S = M * 2 * self.dim
        nbr = np.zeros(S, dtype=np.int32)
        ft = np.zeros(S, dtype=np.int8)
        sl = np.zeros(S, dtype=np.int8)
        _check(lib().oracle_get_conn(self.h, _ptr(nbr, C.c_int32), _ptr(ft, C.c_int8),
                                     _ptr(sl, C.c_int8), C.c_int64(S)))
        return nbr.reshape(M, -1), ft.reshape(M, -1), sl.reshape(M, -1)

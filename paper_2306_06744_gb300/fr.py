"""Python binding of the GB300 adaptive-FR library (``include/fr.h``), by ctypes.

Argument marshalling only: every step of the method runs in the library's CUDA kernels.  PyTorch
supplies device memory (its caching allocator is handed to the library as an ``fr_allocator``)
and the CUDA stream.  There is no CPU fallback: importing works anywhere, but every call raises
if the library or a CUDA device is missing.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

FR_EINVAL, FR_ENOMEM, FR_EOVERFLOW, FR_ETIMEOUT, FR_ECUDA = -1, -2, -3, -4, -5


class FRError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("fr error %d: %s" % (code, msg))
        self.code = code


class FRConfig(C.Structure):
    _fields_ = [("dim", C.c_int32), ("p", C.c_int32), ("L", C.c_double),
                ("Dbase", C.c_int32), ("Dmax", C.c_int32), ("gamma", C.c_double),
                ("nvort", C.c_int32), ("vort", C.POINTER(C.c_double)),
                ("uinf", C.c_double * 3), ("rho_inf", C.c_double), ("p_inf", C.c_double),
                ("cfl", C.c_double), ("dt", C.c_double), ("adapt_every", C.c_int32),
                ("indicator", C.c_int32), ("th_refine", C.c_double), ("th_coarsen", C.c_double),
                ("precision", C.c_int32), ("init_passes", C.c_int32)]


class FRNorms(C.Structure):
    _fields_ = [("t", C.c_double), ("l2_rho", C.c_double), ("integral", C.c_double * 5),
                ("min_rho", C.c_double), ("min_p", C.c_double), ("M", C.c_int64)]


class FRAdaptStats(C.Structure):
    _fields_ = [("M_old", C.c_int64), ("M_new", C.c_int64), ("n_refined", C.c_int64),
                ("n_coarsened", C.c_int64), ("balance_passes", C.c_int32),
                ("balance_exact_depth", C.c_int32),
                ("ms_tree", C.c_double), ("ms_transfer", C.c_double), ("ms_conn", C.c_double)]


class FRStepStats(C.Structure):
    _fields_ = [("steps", C.c_int64), ("dof_updates", C.c_int64), ("ms", C.c_double)]


class FRProfile(C.Structure):
    _fields_ = [("stage_launches", C.c_int64), ("face_launches", C.c_int64),
                ("stage_ms", C.c_double), ("face_ms", C.c_double), ("stage_points", C.c_int64),
                ("face_points", C.c_int64), ("kernel_launches", C.c_int64)]


class FRInfo(C.Structure):
    _fields_ = [("t", C.c_double), ("dt", C.c_double), ("M", C.c_int64), ("step", C.c_int64),
                ("dim", C.c_int32), ("p", C.c_int32), ("nv", C.c_int32), ("N", C.c_int32),
                ("n_conforming", C.c_int64), ("n_hanging", C.c_int64)]


ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p, C.c_void_p)


class FRAllocator(C.Structure):
    _fields_ = [("alloc", ALLOC_FN), ("free", FREE_FN), ("ctx", C.c_void_p)]


_lib = None
EXPORTS = ["fr_mesh_init", "fr_mesh_free", "fr_step", "fr_run", "fr_adapt", "fr_flags", "fr_rhs",
           "fr_norms", "fr_get_leaves", "fr_get_state", "fr_set_state", "fr_get_conn",
           "fr_set_exact", "fr_set_time", "fr_get_info", "fr_last_error", "fr_morton_encode",
           "fr_keys_sort", "fr_keys_linearise", "fr_tree_balance", "fr_tree_adapt", "fr_tree_map",
           "fr_tree_conn", "fr_profile_enable", "fr_profile_read", "fr_kernel_launches",
           "fr_keys_sort_noalloc", "fr_tree_complete", "fr_mlp_param_count", "fr_features",
           "fr_set_learned_indicator", "fr_mlp_forward", "fr_mlp_grad", "fr_mlp_train_step",
           "fr_tc_set_wait_limit"]
NOALLOC_SORT_MAX_KEYS = 1 << 18


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Loads (building first if needed) the CUDA library; raises if that is impossible."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if not os.path.exists(path):
        if not build_if_missing:
            raise RuntimeError("libfr_gb300.so is not built")
        _build.build()
    lib = C.CDLL(path)
    lib.fr_last_error.restype = C.c_char_p
    lib.fr_last_error.argtypes = [C.c_void_p]
    lib.fr_mesh_free.argtypes = [C.c_void_p]
    lib.fr_mesh_free.restype = None
    vp, i64 = C.c_void_p, C.c_int64
    lib.fr_mesh_init.argtypes = [C.POINTER(FRConfig), C.POINTER(FRAllocator), vp, C.POINTER(vp)]
    lib.fr_step.argtypes = [vp, C.c_int, C.POINTER(FRStepStats)]
    lib.fr_run.argtypes = [vp, C.c_int, C.POINTER(FRStepStats), C.POINTER(FRAdaptStats)]
    lib.fr_adapt.argtypes = [vp, vp, C.POINTER(FRAdaptStats)]
    lib.fr_flags.argtypes = [vp, vp, vp, i64]
    lib.fr_rhs.argtypes = [vp, vp, i64]
    lib.fr_norms.argtypes = [vp, C.POINTER(FRNorms)]
    lib.fr_get_leaves.argtypes = [vp, vp, i64, C.POINTER(i64)]
    lib.fr_get_state.argtypes = [vp, vp, i64]
    lib.fr_set_state.argtypes = [vp, vp, i64, vp]
    lib.fr_get_conn.argtypes = [vp, vp, vp, vp, i64]
    lib.fr_set_exact.argtypes = [vp, C.c_double]
    lib.fr_set_time.argtypes = [vp, C.c_double]
    lib.fr_get_info.argtypes = [vp, C.POINTER(FRInfo)]
    lib.fr_morton_encode.argtypes = [C.c_int, C.c_int, i64, vp, vp, vp]
    lib.fr_keys_sort.argtypes = [C.c_int, C.c_int, vp, i64, vp]
    lib.fr_keys_sort_noalloc.argtypes = [C.c_int, C.c_int, vp, i64, vp]
    lib.fr_keys_linearise.argtypes = [C.c_int, C.c_int, vp, i64, vp, i64, C.POINTER(i64), vp]
    lib.fr_tree_balance.argtypes = [C.c_int, C.c_int, vp, i64, vp, i64, C.POINTER(i64), vp]
    lib.fr_tree_adapt.argtypes = [C.c_int, C.c_int, C.c_int, vp, vp, i64, vp, i64, C.POINTER(i64), vp]
    lib.fr_tree_map.argtypes = [C.c_int, C.c_int, vp, i64, vp, i64, vp, vp, vp]
    lib.fr_tree_complete.argtypes = [C.c_int, C.c_int, C.c_int, C.c_double, vp, i64, vp, i64,
                                     C.POINTER(i64), vp]
    lib.fr_tree_conn.argtypes = [C.c_int, C.c_int, vp, i64, vp, vp, vp, vp]
    lib.fr_mlp_param_count.argtypes = [C.c_int]
    lib.fr_features.argtypes = [vp, vp, i64, C.POINTER(C.c_int32)]
    lib.fr_set_learned_indicator.argtypes = [vp, vp, i64]
    lib.fr_mlp_forward.argtypes = [C.c_int, vp, vp, i64, vp, vp, vp]
    lib.fr_mlp_grad.argtypes = [C.c_int, vp, vp, vp, i64, vp, vp, vp, vp]
    lib.fr_mlp_train_step.argtypes = [C.c_int, vp, vp, vp, i64, vp, vp, i64, vp, C.c_float, vp, vp]
    lib.fr_profile_enable.argtypes = [vp, C.c_int]
    lib.fr_profile_read.argtypes = [vp, C.POINTER(FRProfile)]
    lib.fr_tc_set_wait_limit.argtypes = [C.c_longlong]
    lib.fr_tc_set_wait_limit.restype = None
    lib.fr_kernel_launches.restype = C.c_int64
    lib.fr_kernel_launches.argtypes = []
    _lib = lib
    return lib


def _torch():
    import torch
    if not torch.cuda.is_available():
        raise RuntimeError("no CUDA device: the GB300 library has no CPU path")
    return torch


def _check(rc, mesh_handle=None):
    if rc != 0:
        msg = load().fr_last_error(mesh_handle)
        raise FRError(rc, msg.decode() if msg else "")


def _np_ptr(a):
    return C.c_void_p(a.ctypes.data)


def _stream_handle(stream):
    torch = _torch()
    if stream is None:
        stream = torch.cuda.current_stream()
    return C.c_void_p(stream.cuda_stream)


def _host_out(out, n, dtype):
    if out is None:
        return np.empty(n, dtype=dtype)
    if out.dtype != dtype or not out.flags["C_CONTIGUOUS"] or out.size < n:
        raise ValueError("out must be a contiguous %s array of at least %d entries" % (np.dtype(dtype), n))
    return out.reshape(-1)[:n]


def make_config(cfg: dict):
    vort = np.ascontiguousarray(np.asarray(cfg["vort"], dtype=np.float64).reshape(-1, 4))
    c = FRConfig(dim=cfg["dim"], p=cfg["p"], L=cfg["L"], Dbase=cfg["Dbase"], Dmax=cfg["Dmax"],
                 gamma=cfg["gamma"], nvort=vort.shape[0],
                 vort=vort.ctypes.data_as(C.POINTER(C.c_double)), rho_inf=cfg["rho_inf"],
                 p_inf=cfg["p_inf"], cfl=cfg["cfl"], dt=cfg["dt"], adapt_every=cfg["adapt_every"],
                 indicator=cfg["indicator"], th_refine=cfg["th_refine"],
                 th_coarsen=cfg["th_coarsen"], precision=cfg.get("precision", 0),
                 init_passes=cfg.get("init_passes", -1))
    for a in range(3):
        c.uinf[a] = cfg["uinf"][a]
    return c, vort


class _TorchAllocator:
    """Hands torch's CUDA caching allocator to the library.

    ``fail_in``: host-side failure injection for tests of the library's error paths: when set to
    k >= 0, the allocation after the next k returns NULL (the library then reports FR_ENOMEM),
    and the counter clears itself.  No GPU fault is involved."""

    def __init__(self, device):
        torch = _torch()
        self.device = device
        self.fail_in = None

        def _alloc(nbytes, stream, ctx):
            if self.fail_in is not None:
                if self.fail_in == 0:
                    self.fail_in = None
                    return None
                self.fail_in -= 1
            try:
                return torch.cuda.caching_allocator_alloc(int(nbytes), self.device, int(stream or 0))
            except Exception:  # the library reports FR_ENOMEM on NULL
                return None

        def _free(ptr, stream, ctx):
            if ptr:
                torch.cuda.caching_allocator_delete(int(ptr))

        self._a = ALLOC_FN(_alloc)
        self._f = FREE_FN(_free)
        self.struct = FRAllocator(self._a, self._f, None)


class Mesh:
    """One adaptive FR mesh on the current CUDA device (the library's fr_mesh)."""

    def __init__(self, cfg: dict, stream=None, torch_allocator: bool = True):
        torch = _torch()
        lib = load()
        self.cfg = dict(cfg)
        self.dim, self.p = cfg["dim"], cfg["p"]
        self.n = self.p + 1
        self.N = self.n ** self.dim
        self.nv = self.dim + 2
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self._alloc = _TorchAllocator(torch.cuda.current_device()) if torch_allocator else None
        c, self._vort = make_config(cfg)
        h = C.c_void_p()
        rc = lib.fr_mesh_init(C.byref(c), C.byref(self._alloc.struct) if self._alloc else None,
                              C.c_void_p(self.stream.cuda_stream), C.byref(h))
        _check(rc, None)
        self.h = h

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            load().fr_mesh_free(self.h)
            self.h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _ck(self, rc):
        _check(rc, self.h)

    # -- calls of include/fr.h --
    def info(self):
        o = FRInfo()
        self._ck(load().fr_get_info(self.h, C.byref(o)))
        return {k: getattr(o, k) for k, _ in FRInfo._fields_}

    @property
    def M(self):
        return self.info()["M"]

    def step(self, nsteps=1, stats=False):
        st = FRStepStats()
        self._ck(load().fr_step(self.h, nsteps, C.byref(st) if stats else None))
        return {k: getattr(st, k) for k, _ in FRStepStats._fields_} if stats else None

    def run(self, nsteps, stats=False):
        ss, ast = FRStepStats(), FRAdaptStats()
        self._ck(load().fr_run(self.h, nsteps, C.byref(ss) if stats else None,
                               C.byref(ast) if stats else None))
        if stats:
            return ({k: getattr(ss, k) for k, _ in FRStepStats._fields_},
                    {k: getattr(ast, k) for k, _ in FRAdaptStats._fields_})
        return None

    def adapt(self, flags=None, stats=False):
        """flags: None (configured indicator) or int8 values per leaf (host array or CUDA tensor)."""
        torch = _torch()
        st = FRAdaptStats()
        keep = None
        ptr = None
        if flags is not None:
            if isinstance(flags, torch.Tensor) and flags.is_cuda:
                keep = flags.to(torch.int8).contiguous()
            else:
                keep = torch.as_tensor(np.ascontiguousarray(flags, dtype=np.int8)).to(
                    "cuda", non_blocking=False)
            if keep.numel() != self.M:
                raise ValueError("flags must have one entry per leaf")
            ptr = C.c_void_p(keep.data_ptr())
            torch.cuda.current_stream().synchronize()
        self._ck(load().fr_adapt(self.h, ptr, C.byref(st) if stats else None))
        return {k: getattr(st, k) for k, _ in FRAdaptStats._fields_} if stats else None

    def flags(self):
        M = self.M
        f = np.zeros(M, dtype=np.int8)
        eta = np.zeros(M)
        self._ck(load().fr_flags(self.h, _np_ptr(f), _np_ptr(eta), M))
        return f, eta

    def rhs(self):
        M = self.M
        R = np.zeros((M, self.nv, self.N))
        self._ck(load().fr_rhs(self.h, _np_ptr(R), R.size))
        return R

    def norms(self):
        o = FRNorms()
        self._ck(load().fr_norms(self.h, C.byref(o)))
        return dict(t=o.t, l2_rho=o.l2_rho, integral=list(o.integral)[: self.nv],
                    min_rho=o.min_rho, min_p=o.min_p, M=o.M)

    def leaves(self, out=None):
        """Morton keys of the leaves (uint64[M]).  `out`: a contiguous uint64 host array of at least
        M entries to fill (e.g. a view of pinned memory); the result is then a view of it."""
        M = self.M
        k = _host_out(out, M, np.uint64)
        m = C.c_int64()
        self._ck(load().fr_get_leaves(self.h, _np_ptr(k), M, C.byref(m)))
        return k

    def state(self, out=None):
        """Conserved variables u[M][nv][N] (FP64).  `out`: a contiguous float64 host array of at
        least M*nv*N entries to fill; the result is then a view of it."""
        M = self.M
        u = _host_out(out, M * self.nv * self.N, np.float64)
        self._ck(load().fr_get_state(self.h, _np_ptr(u), u.size))
        return u.reshape(M, self.nv, self.N)

    def set_state(self, keys, u):
        keys = np.ascontiguousarray(keys, dtype=np.uint64)
        u = np.ascontiguousarray(u, dtype=np.float64)
        if u.size != keys.shape[0] * self.nv * self.N:
            raise ValueError("state size does not match the keys")
        self._ck(load().fr_set_state(self.h, _np_ptr(keys), keys.shape[0], _np_ptr(u)))

    def set_exact(self, t):
        self._ck(load().fr_set_exact(self.h, C.c_double(t)))

    def set_time(self, t):
        self._ck(load().fr_set_time(self.h, C.c_double(t)))

    def profile_enable(self, on=True, stride=1):
        """Per-kernel event timing of every `stride`-th stage (0/False stops)."""
        self._ck(load().fr_profile_enable(self.h, max(1, int(stride)) if on else 0))

    def profile_read(self):
        o = FRProfile()
        self._ck(load().fr_profile_read(self.h, C.byref(o)))
        return {k: getattr(o, k) for k, _ in FRProfile._fields_}

    def features(self):
        """BF16 features [M][in_dim] of the current state as a CUDA tensor (learned indicator)."""
        torch = _torch()
        n_in = C.c_int32()
        self._ck(load().fr_features(self.h, None, 0, C.byref(n_in)))
        X = torch.empty((self.M, n_in.value), dtype=torch.bfloat16, device="cuda")
        self._ck(load().fr_features(self.h, C.c_void_p(X.data_ptr()), X.numel(), None))
        return X

    def set_learned_indicator(self, params):
        """Installs MLP weights (FP32 host array) for indicator 3; None restores the fallback."""
        if params is None:
            self._ck(load().fr_set_learned_indicator(self.h, None, 0))
            return
        p = np.ascontiguousarray(params, dtype=np.float32)
        self._ck(load().fr_set_learned_indicator(self.h, _np_ptr(p), p.size))

    def conn(self):
        M = self.M
        S = M * 2 * self.dim
        nbr = np.zeros(S, dtype=np.int32)
        ft = np.zeros(S, dtype=np.int8)
        sl = np.zeros(S, dtype=np.int8)
        self._ck(load().fr_get_conn(self.h, _np_ptr(nbr), _np_ptr(ft), _np_ptr(sl), S))
        return nbr.reshape(M, -1), ft.reshape(M, -1), sl.reshape(M, -1)


def mlp_param_count(in_dim: int) -> int:
    n = load().fr_mlp_param_count(in_dim)
    if n < 0:
        _check(n)
    return n


def _class_w(cw, y):
    cw = np.asarray(cw, dtype=np.float64)
    yy = np.asarray(y.cpu().numpy() if hasattr(y, "cpu") else y, dtype=np.int64) + 1
    wsum = float(cw[yy].sum())
    return np.array([cw[0], cw[1], cw[2], 1.0 / wsum], dtype=np.float32)


def mlp_forward(params, X, stream=None):
    """Logits [n][3] (CUDA float tensor) of BF16 features X [n][in] with FP32 params (CUDA)."""
    torch = _torch()
    n, n_in = X.shape
    logits = torch.empty((n, 3), dtype=torch.float32, device="cuda")
    flags = torch.empty(n, dtype=torch.int8, device="cuda")
    _check(load().fr_mlp_forward(n_in, C.c_void_p(params.data_ptr()), C.c_void_p(X.data_ptr()), n,
                                 C.c_void_p(logits.data_ptr()), C.c_void_p(flags.data_ptr()),
                                 _stream_handle(stream)))
    return logits, flags


def tc_set_wait_limit(cycles: int) -> None:
    """Bound (clock cycles) of the tensor-core inference kernel's completion waits; <= 0: default."""
    load().fr_tc_set_wait_limit(int(cycles))


def mlp_grad(params, X, y, class_w, stream=None):
    torch = _torch()
    n, n_in = X.shape
    g = torch.empty_like(params)
    loss = torch.empty(1, dtype=torch.float32, device="cuda")
    cw = _class_w(class_w, y)
    _check(load().fr_mlp_grad(n_in, C.c_void_p(params.data_ptr()), C.c_void_p(X.data_ptr()),
                              C.c_void_p(y.data_ptr()), n, _np_ptr(cw), C.c_void_p(g.data_ptr()),
                              C.c_void_p(loss.data_ptr()), _stream_handle(stream)))
    return float(loss.item()), g


def mlp_train_step(params, m, v, step, X, y, class_w, lr, loss=None, stream=None):
    """One Adam step in place on `params` (CUDA FP32); X BF16 [B][in], y int8 in {-1,0,1}."""
    B, n_in = X.shape
    cw = _class_w(class_w, y)
    _check(load().fr_mlp_train_step(n_in, C.c_void_p(params.data_ptr()), C.c_void_p(m.data_ptr()),
                                    C.c_void_p(v.data_ptr()), step, C.c_void_p(X.data_ptr()),
                                    C.c_void_p(y.data_ptr()), B, _np_ptr(cw), C.c_float(lr),
                                    C.c_void_p(loss.data_ptr()) if loss is not None else None,
                                    _stream_handle(stream)))


def kernel_launches() -> int:
    return int(load().fr_kernel_launches())


# ---- tree primitives on device tensors ----

def _dev(a, dtype):
    torch = _torch()
    if isinstance(a, torch.Tensor):
        return a.to(device="cuda", dtype=dtype).contiguous()
    return torch.as_tensor(np.ascontiguousarray(a)).to(device="cuda", dtype=dtype).contiguous()


def _u64(t):
    torch = _torch()
    return t.view(torch.int64) if t.dtype != torch.int64 else t


def _to_np_u64(t):
    return t.cpu().numpy().view(np.uint64)


def morton_encode(dim, Dmax, boxes, stream=None):
    torch = _torch()
    b = _dev(np.asarray(boxes, dtype=np.int32).reshape(-1, 4), torch.int32)
    out = torch.empty(b.shape[0], dtype=torch.int64, device="cuda")
    _check(load().fr_morton_encode(dim, Dmax, b.shape[0], C.c_void_p(b.data_ptr()),
                                   C.c_void_p(out.data_ptr()), _stream_handle(stream)))
    return _to_np_u64(out)


def keys_sort(dim, Dmax, keys, stream=None):
    torch = _torch()
    k = _dev(np.asarray(keys, dtype=np.uint64).view(np.int64), torch.int64)
    _check(load().fr_keys_sort(dim, Dmax, C.c_void_p(k.data_ptr()), k.numel(), _stream_handle(stream)))
    return _to_np_u64(k)


def keys_sort_noalloc_(dim, Dmax, d_keys, stream=None):
    """Allocation-free sort of a CUDA int64 tensor in place (at most NOALLOC_SORT_MAX_KEYS keys):
    for callers that cannot allocate device memory during the call.  The tensor is the caller's."""
    _check(load().fr_keys_sort_noalloc(dim, Dmax, C.c_void_p(d_keys.data_ptr()), d_keys.numel(),
                                       _stream_handle(stream)))
    return d_keys


def keys_linearise(dim, Dmax, keys, stream=None):
    torch = _torch()
    k = _dev(np.asarray(keys, dtype=np.uint64).view(np.int64), torch.int64)
    out = torch.empty(max(1, k.numel()), dtype=torch.int64, device="cuda")
    n = C.c_int64()
    _check(load().fr_keys_linearise(dim, Dmax, C.c_void_p(k.data_ptr()), k.numel(),
                                    C.c_void_p(out.data_ptr()), out.numel(), C.byref(n),
                                    _stream_handle(stream)))
    return _to_np_u64(out[: n.value])


def _grow_call(fn, cap, *head, tail=()):
    torch = _torch()
    while True:
        out = torch.empty(cap, dtype=torch.int64, device="cuda")
        n = C.c_int64()
        rc = fn(*head, C.c_void_p(out.data_ptr()), cap, C.byref(n), *tail)
        if rc == FR_EOVERFLOW and n.value > cap:
            cap = n.value
            continue
        _check(rc)
        return _to_np_u64(out[: n.value])


def tree_balance(dim, Dmax, keys, stream=None):
    torch = _torch()
    k = _dev(np.asarray(keys, dtype=np.uint64).view(np.int64), torch.int64)
    return _grow_call(load().fr_tree_balance, max(16, 2 * k.numel()), dim, Dmax,
                      C.c_void_p(k.data_ptr()), k.numel(), tail=(_stream_handle(stream),))


def tree_adapt(dim, Dbase, Dmax, keys, flags, stream=None):
    torch = _torch()
    k = _dev(np.asarray(keys, dtype=np.uint64).view(np.int64), torch.int64)
    f = _dev(np.asarray(flags, dtype=np.int8), torch.int8)
    return _grow_call(load().fr_tree_adapt, max(16, 2 * k.numel()), dim, Dbase, Dmax,
                      C.c_void_p(k.data_ptr()), C.c_void_p(f.data_ptr()), k.numel(),
                      tail=(_stream_handle(stream),))


def tree_complete(dim, Dmin, Dmax, L, pts, stream=None):
    """Tree completion from points (host array or CUDA tensor [n][dim]); returns sorted keys."""
    torch = _torch()
    pt = _dev(np.asarray(pts, dtype=np.float64).reshape(-1, dim) if not isinstance(pts, torch.Tensor)
              else pts, torch.float64)
    return _grow_call(load().fr_tree_complete, max(16, 4 * pt.shape[0] + (1 << (dim * Dmin))),
                      dim, Dmin, Dmax, C.c_double(L), C.c_void_p(pt.data_ptr()), pt.shape[0],
                      tail=(_stream_handle(stream),))


def tree_map(dim, Dmax, old_keys, new_keys, stream=None):
    torch = _torch()
    o = _dev(np.asarray(old_keys, dtype=np.uint64).view(np.int64), torch.int64)
    n = _dev(np.asarray(new_keys, dtype=np.uint64).view(np.int64), torch.int64)
    src = torch.empty(n.numel(), dtype=torch.int32, device="cuda")
    tag = torch.empty(n.numel(), dtype=torch.int8, device="cuda")
    _check(load().fr_tree_map(dim, Dmax, C.c_void_p(o.data_ptr()), o.numel(),
                              C.c_void_p(n.data_ptr()), n.numel(), C.c_void_p(src.data_ptr()),
                              C.c_void_p(tag.data_ptr()), _stream_handle(stream)))
    return src.cpu().numpy(), tag.cpu().numpy()


def tree_conn(dim, Dmax, keys, stream=None):
    torch = _torch()
    k = _dev(np.asarray(keys, dtype=np.uint64).view(np.int64), torch.int64)
    M = k.numel()
    nbr = torch.empty(M * 2 * dim, dtype=torch.int32, device="cuda")
    ft = torch.empty(M * 2 * dim, dtype=torch.int8, device="cuda")
    sl = torch.empty(M * 2 * dim, dtype=torch.int8, device="cuda")
    _check(load().fr_tree_conn(dim, Dmax, C.c_void_p(k.data_ptr()), M, C.c_void_p(nbr.data_ptr()),
                               C.c_void_p(ft.data_ptr()), C.c_void_p(sl.data_ptr()),
                               _stream_handle(stream)))
    return (nbr.cpu().numpy().reshape(M, -1), ft.cpu().numpy().reshape(M, -1),
            sl.cpu().numpy().reshape(M, -1))

"""Thin Python binding of the kdfmm C ABI (``include/kdfmm.h``).

Argument marshalling only: every step of the force evaluation runs inside
``libkdfmm.so``.  PyTorch supplies device memory and streams.  If the library
is missing the import of this module's functions raises -- there is no CPU
fallback.

Functions carry the C names without the ``kdfmm_`` prefix:
``tree_create``, ``tree_destroy``, ``tree_build``, ``tree_moments``,
``fmm_accel``, ``fmm_accel_vjp``, ``total_momentum``, ``total_momentum_noalloc``,
``tree_stats``, ``tree_timing``,
``tree_export``, ``last_error``.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libkdfmm.so")

KDFMM_OK = 0
ERRORS = {-1: "INVALID_ARG", -2: "CUDA", -3: "OOM", -4: "TIMEOUT", -5: "CAPACITY",
          -6: "NONFINITE", -7: "INTERNAL"}
SOFT_PLUMMER, SOFT_M4 = 0, 1
FP64, MIXED = 0, 1
EXPANSION_PHANTOM, EXPANSION_STANDARD = 0, 1
WALK_LEAF, WALK_DUAL = 0, 1
MAX_LEAF = 32
STAT_NAMES = ("n", "ncells", "nleaves", "depth", "nfar", "nnear", "np2p", "nfallback", "nexact",
              "launches", "nheavy")
PHASES = ("build", "walk", "m2l", "p2p")


class KdfmmError(RuntimeError):
    def __init__(self, code: int, where: str, msg: str):
        super().__init__(f"{where}: {ERRORS.get(code, code)}: {msg}")
        self.code = code


class Params(ctypes.Structure):
    _fields_ = [("theta", ctypes.c_double), ("eps", ctypes.c_double), ("r_kern", ctypes.c_double),
                ("n_leaf", ctypes.c_int32), ("soft_kind", ctypes.c_int32),
                ("precision", ctypes.c_int32), ("expansion", ctypes.c_int32),
                ("walk", ctypes.c_int32), ("reserved", ctypes.c_int32)]


def make_params(theta=0.5, eps=0.01, r_kern=2.0, n_leaf=16, soft_kind=SOFT_PLUMMER,
                precision=MIXED, expansion=0, walk=0) -> Params:
    """expansion: 0 = Eq. 6 at full order (the paper's scheme), 1 = the standard
    p = 3 Cartesian series.  walk: 0 = the paper's leaf-only walk, 1 = the
    symmetric dual-tree walk."""
    return Params(float(theta), float(eps), float(r_kern), int(n_leaf), int(soft_kind),
                  int(precision), int(expansion), int(walk), 0)


_lib = None


def lib() -> ctypes.CDLL:
    """Loads libkdfmm.so; raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_2502_01496_gb300.build "
                           "(there is no CPU fallback)")
    L = ctypes.CDLL(LIB_PATH)
    P, i64, i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32
    L.kdfmm_tree_create.argtypes = [ctypes.POINTER(ctypes.c_void_p)]
    L.kdfmm_tree_destroy.argtypes = [P]
    L.kdfmm_tree_destroy.restype = None
    L.kdfmm_tree_build.argtypes = [P, P, P, P, i64, ctypes.POINTER(Params), P]
    L.kdfmm_tree_moments.argtypes = [P, P, P, P, P]
    L.kdfmm_fmm_accel.argtypes = [P, P, P, P]
    L.kdfmm_fmm_accel_vjp.argtypes = [P, P, P, P, P]
    L.kdfmm_total_momentum.argtypes = [P, P, i64, P, P]
    L.kdfmm_total_momentum_noalloc.argtypes = [P, P, i64, P, P]
    L.kdfmm_tree_stats.argtypes = [P, P]
    L.kdfmm_tree_export.argtypes = [P, P, P, P, P, P, P, P, P]
    L.kdfmm_forest_build.argtypes = [P, P, P, P, P, i32, P, P, P, ctypes.POINTER(Params), P]
    L.kdfmm_fmm_accel_batched.argtypes = [P, P, P, P, P, i32, P, P, P, ctypes.POINTER(Params),
                                          P, P, P]
    L.kdfmm_kick_drift.argtypes = [P, P, P, i64, ctypes.c_double, ctypes.c_double, P]
    L.kdfmm_tree_timing.argtypes = [P, ctypes.c_int, P]
    L.kdfmm_measure_peaks.argtypes = [P, P]
    L.kdfmm_tree_set_walk_budget.argtypes = [P, i32]
    L.kdfmm_tree_timing.restype = i32
    L.kdfmm_last_error.restype = ctypes.c_char_p
    L.kdfmm_last_error.argtypes = []
    for name in ("kdfmm_tree_create", "kdfmm_tree_build", "kdfmm_tree_moments", "kdfmm_fmm_accel",
                 "kdfmm_fmm_accel_vjp", "kdfmm_total_momentum", "kdfmm_total_momentum_noalloc",
                 "kdfmm_tree_stats", "kdfmm_tree_export", "kdfmm_forest_build",
                 "kdfmm_fmm_accel_batched", "kdfmm_kick_drift"):
        getattr(L, name).restype = i32
    _lib = L
    return L


def last_error() -> str:
    return lib().kdfmm_last_error().decode()


def _check(rc: int, where: str) -> None:
    if rc != KDFMM_OK:
        raise KdfmmError(rc, where, last_error())


def _ptr(t) -> ctypes.c_void_p | None:
    if t is None:
        return None
    if isinstance(t, int):
        return ctypes.c_void_p(t)
    return ctypes.c_void_p(t.data_ptr())


def _dev_f64(t, name: str, shape=None):
    import torch
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()):
        raise TypeError(f"{name} must be a contiguous float64 CUDA tensor")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} has shape {tuple(t.shape)}, expected {tuple(shape)}")
    return t


def _stream(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def tree_create() -> ctypes.c_void_p:
    h = ctypes.c_void_p()
    _check(lib().kdfmm_tree_create(ctypes.byref(h)), "tree_create")
    return h


def tree_destroy(tree) -> None:
    if tree:
        lib().kdfmm_tree_destroy(tree)


def tree_build(tree, x, m, h, params: Params, stream=None) -> None:
    n = x.shape[0]
    _dev_f64(x, "x", (n, 3))
    _dev_f64(m, "m", (n,))
    if h is not None:
        _dev_f64(h, "h", (n,))
    _check(lib().kdfmm_tree_build(tree, _ptr(x), _ptr(m), _ptr(h), n, ctypes.byref(params),
                                  _stream(stream)), "tree_build")


def _host_array(a, dtype, n, name):
    import numpy as np
    if a is None:
        return None, None
    arr = np.ascontiguousarray(a, dtype=dtype)
    if arr.shape != (n,):
        raise ValueError(f"{name} has shape {arr.shape}, expected ({n},)")
    return arr, arr.ctypes.data_as(ctypes.c_void_p)


def _systems(sys_offset, theta, eps, n_leaf):
    import numpy as np
    off = np.ascontiguousarray(sys_offset, dtype=np.int64)
    if off.ndim != 1 or off.size < 2:
        raise ValueError("sys_offset needs n_sys + 1 >= 2 entries")
    n_sys = off.size - 1
    keep = [off]
    ptrs = [off.ctypes.data_as(ctypes.c_void_p)]
    for a, dt, name in ((theta, np.float64, "theta"), (eps, np.float64, "eps"),
                        (n_leaf, np.int32, "n_leaf")):
        arr, ptr = _host_array(a, dt, n_sys, name)
        keep.append(arr)
        ptrs.append(ptr)
    return n_sys, ptrs, keep


def forest_build(tree, x, m, h, sys_offset, params: Params, theta=None, eps=None, n_leaf=None,
                 stream=None) -> None:
    """Builds one tree per system (particles sys_offset[k]:sys_offset[k+1])
    in the same launches; theta / eps / n_leaf per system or None for the
    value in params.  See include/kdfmm.h."""
    n = x.shape[0]
    _dev_f64(x, "x", (n, 3))
    _dev_f64(m, "m", (n,))
    if h is not None:
        _dev_f64(h, "h", (n,))
    n_sys, ptrs, keep = _systems(sys_offset, theta, eps, n_leaf)
    if int(keep[0][-1]) != n:
        raise ValueError(f"sys_offset ends at {int(keep[0][-1])}, x holds {n} particles")
    _check(lib().kdfmm_forest_build(tree, _ptr(x), _ptr(m), _ptr(h), ptrs[0], n_sys, ptrs[1],
                                    ptrs[2], ptrs[3], ctypes.byref(params), _stream(stream)),
           "forest_build")


def fmm_accel_batched(tree, x, m, h, sys_offset, params: Params, a, phi=None, theta=None,
                      eps=None, n_leaf=None, stream=None) -> None:
    """forest_build + fmm_accel in one call."""
    n = x.shape[0]
    _dev_f64(x, "x", (n, 3))
    _dev_f64(m, "m", (n,))
    if h is not None:
        _dev_f64(h, "h", (n,))
    _dev_f64(a, "a", (n, 3))
    if phi is not None:
        _dev_f64(phi, "phi", (n,))
    n_sys, ptrs, keep = _systems(sys_offset, theta, eps, n_leaf)
    if int(keep[0][-1]) != n:
        raise ValueError(f"sys_offset ends at {int(keep[0][-1])}, x holds {n} particles")
    _check(lib().kdfmm_fmm_accel_batched(tree, _ptr(x), _ptr(m), _ptr(h), ptrs[0], n_sys, ptrs[1],
                                         ptrs[2], ptrs[3], ctypes.byref(params), _ptr(a),
                                         _ptr(phi), _stream(stream)), "fmm_accel_batched")


def tree_moments(tree, x, m, h, stream=None) -> None:
    """New positions / masses / smoothing lengths of the same particles on the
    built tree (frozen topology and interaction lists); see include/kdfmm.h."""
    n = x.shape[0]
    _dev_f64(x, "x", (n, 3))
    _dev_f64(m, "m", (n,))
    if h is not None:
        _dev_f64(h, "h", (n,))
    _check(lib().kdfmm_tree_moments(tree, _ptr(x), _ptr(m), _ptr(h), _stream(stream)),
           "tree_moments")


def fmm_accel(tree, a, phi=None, stream=None) -> None:
    _dev_f64(a, "a")
    if phi is not None:
        _dev_f64(phi, "phi")
    _check(lib().kdfmm_fmm_accel(tree, _ptr(a), _ptr(phi), _stream(stream)), "fmm_accel")


def fmm_accel_vjp(tree, a_bar, x_bar, m_bar, stream=None) -> None:
    """x_bar (n,3), m_bar (n,) = (d a / d x)^T a_bar, (d a / d m)^T a_bar of the
    last evaluation, lists and topology held fixed."""
    n = a_bar.shape[0]
    _dev_f64(a_bar, "a_bar", (n, 3))
    _dev_f64(x_bar, "x_bar", (n, 3))
    _dev_f64(m_bar, "m_bar", (n,))
    _check(lib().kdfmm_fmm_accel_vjp(tree, _ptr(a_bar), _ptr(x_bar), _ptr(m_bar), _stream(stream)),
           "fmm_accel_vjp")


def total_momentum(m, v, out, stream=None) -> None:
    n = m.shape[0]
    _dev_f64(m, "m", (n,))
    _dev_f64(v, "v", (n, 3))
    _dev_f64(out, "out", (3,))
    _check(lib().kdfmm_total_momentum(_ptr(m), _ptr(v), n, _ptr(out), _stream(stream)),
           "total_momentum")


def total_momentum_noalloc(m, v, out, stream=None) -> None:
    """total_momentum without any device allocation (fixed library scratch);
    see include/kdfmm.h for who needs it and its limits."""
    n = m.shape[0]
    _dev_f64(m, "m", (n,))
    _dev_f64(v, "v", (n, 3))
    _dev_f64(out, "out", (3,))
    _check(lib().kdfmm_total_momentum_noalloc(_ptr(m), _ptr(v), n, _ptr(out), _stream(stream)),
           "total_momentum_noalloc")


def kick_drift(x, v, a, dt_kick: float, dt_drift: float, stream=None) -> None:
    """v += dt_kick a; x += dt_drift v (in place, leapfrog)."""
    n = x.shape[0]
    _dev_f64(x, "x", (n, 3))
    _dev_f64(v, "v", (n, 3))
    _dev_f64(a, "a", (n, 3))
    _check(lib().kdfmm_kick_drift(_ptr(x), _ptr(v), _ptr(a), n, float(dt_kick), float(dt_drift),
                                  _stream(stream)), "kick_drift")


def tree_stats(tree) -> dict:
    s = np.zeros(len(STAT_NAMES), dtype=np.int64)
    _check(lib().kdfmm_tree_stats(tree, s.ctypes.data_as(ctypes.c_void_p)), "tree_stats")
    return {k: int(v) for k, v in zip(STAT_NAMES, s)}


def tree_timing(tree, enable: bool = True, read: bool = True) -> dict | None:
    """Enables/disables phase timing; returns the last timed phase durations (ms)."""
    ms = np.zeros(len(PHASES), dtype=np.float32) if read else None
    _check(lib().kdfmm_tree_timing(tree, int(enable),
                                   None if ms is None else ms.ctypes.data_as(ctypes.c_void_p)),
           "tree_timing")
    return None if ms is None else {k: float(v) for k, v in zip(PHASES, ms)}


def tree_set_walk_budget(tree, budget: int) -> None:
    """Cells a walk thread visits before its leaf goes to the block-wide walk
    (0: the default); see kdfmm_tree_set_walk_budget."""
    _check(lib().kdfmm_tree_set_walk_budget(tree, int(budget)), "tree_set_walk_budget")


def measure_peaks(stream=None) -> dict:
    """Measured float32 / float64 FMA throughput of the current device and the
    derived float32 peak (see kdfmm_measure_peaks)."""
    out = np.zeros(5, dtype=np.float64)
    _check(lib().kdfmm_measure_peaks(out.ctypes.data_as(ctypes.c_void_p), _stream(stream)),
           "measure_peaks")
    return {"fp32_tflops": float(out[0]), "fp64_tflops": float(out[1]), "sms": int(out[2]),
            "sm_max_mhz": float(out[3]), "fp32_derived_tflops": float(out[4])}


@dataclass
class Export:
    perm: np.ndarray
    cell_ints: np.ndarray     # (ncells, 7): first count left right parent depth skip
    cell_reals: np.ndarray    # (ncells, 12): M com(3) s hmax Q(6)
    leaf_ids: np.ndarray
    far_off: np.ndarray | None
    far_idx: np.ndarray | None
    near_off: np.ndarray | None
    near_idx: np.ndarray | None


def tree_export(tree, lists: bool = True, dual: bool = False) -> Export:
    """Host copies of the tree and lists; with dual=True (the dual walk) the far
    lists are per cell (far_off has ncells + 1 entries)."""
    st = tree_stats(tree)
    n, nc, nl = st["n"], st["ncells"], st["nleaves"]
    perm = np.empty(n, dtype=np.int64)
    ci = np.empty((nc, 7), dtype=np.int64)
    cr = np.empty((nc, 12), dtype=np.float64)
    leaf = np.empty(nl, dtype=np.int32)
    fo = fi = no = ni = None
    if lists:
        fo = np.empty((nc if dual else nl) + 1, dtype=np.int64)
        no = np.empty(nl + 1, dtype=np.int64)
        fi = np.empty(max(st["nfar"], 1), dtype=np.int32)
        ni = np.empty(max(st["nnear"], 1), dtype=np.int32)
    p = lambda a: None if a is None else a.ctypes.data_as(ctypes.c_void_p)
    _check(lib().kdfmm_tree_export(tree, p(perm), p(ci), p(cr), p(leaf), p(fo), p(fi), p(no), p(ni)),
           "tree_export")
    if lists:
        fi, ni = fi[:st["nfar"]], ni[:st["nnear"]]
    return Export(perm, ci, cr, leaf, fo, fi, no, ni)


class KdFmm:
    """One particle set's tree on the current CUDA device.

    >>> f = KdFmm(theta=0.5, n_leaf=16, eps=0.01)
    >>> f.build(x, m)            # x (n,3), m (n,) float64 CUDA tensors
    >>> a, phi = f.accel()       # caller order, float64
    """

    def __init__(self, **params):
        self.params = make_params(**params)
        self.handle = tree_create()
        self.n = 0

    def __del__(self):
        h = getattr(self, "handle", None)
        if h:
            try:
                tree_destroy(h)
            except Exception:
                pass
            self.handle = None

    def build(self, x, m, h=None, stream=None):
        tree_build(self.handle, x, m, h, self.params, stream)
        self.n = x.shape[0]
        return self

    def build_forest(self, x, m, h, sys_offset, theta=None, eps=None, n_leaf=None, stream=None):
        """Independent systems in one handle (see forest_build)."""
        forest_build(self.handle, x, m, h, sys_offset, self.params, theta, eps, n_leaf, stream)
        self.n = x.shape[0]
        return self

    def accel(self, a=None, phi=None, want_phi=True, stream=None):
        import torch
        if a is None:
            a = torch.empty((self.n, 3), dtype=torch.float64, device="cuda")
        if phi is None and want_phi:
            phi = torch.empty(self.n, dtype=torch.float64, device="cuda")
        fmm_accel(self.handle, a, phi, stream)
        return a, phi

    def moments(self, x, m, h=None, stream=None):
        """Refresh the cell moments for moved particles; the next accel() reuses
        the topology and interaction lists of the last walk."""
        tree_moments(self.handle, x, m, h, stream)
        return self

    def vjp(self, a_bar, stream=None):
        """(x_bar, m_bar) of the last accel() for the cotangent a_bar (n, 3)."""
        import torch
        x_bar = torch.empty((self.n, 3), dtype=torch.float64, device="cuda")
        m_bar = torch.empty(self.n, dtype=torch.float64, device="cuda")
        fmm_accel_vjp(self.handle, a_bar, x_bar, m_bar, stream)
        return x_bar, m_bar

    def stats(self) -> dict:
        return tree_stats(self.handle)

    def export(self, lists: bool = True) -> Export:
        return tree_export(self.handle, lists, dual=self.params.walk == WALK_DUAL)

"""Plain FP64 CPU oracle of the kd-tree FMM force evaluation -- TEST INFRASTRUCTURE.

This package wraps ``kdfmm_oracle.c`` (plain C, single-threaded, FP64, compiled
with ``-ffp-contract=off``) through ``ctypes``.  It is the reference the GPU
library is checked against and it shares no code with that library.  Only the
test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py``
may import it; the product path never does.

Paper: Potashov & Yudin, arXiv 2502.01496.  Sec. 2 (kd-tree, Eqs. 4-8), Sec. 3
(Eq. 13 kernel-softened Green's function), Sec. 4 (leaf-only walk).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "kdfmm_oracle.c")
_LIB = os.path.join(_HERE, "libkdfmm_oracle.so")

SOFT_PLUMMER = 0
SOFT_M4 = 1
EXP_PHANTOM = 0    # Eq. 6 expanded to full order in the sink displacement
EXP_STANDARD = 1   # standard p = 3 Cartesian series (orders of sink and source add to <= 2)

_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle shared library in place (gcc, FP64, no contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        cmd = ["gcc", "-O2", "-std=c11", "-Wall", "-ffp-contract=off", "-fno-fast-math",
               "-fPIC", "-shared", "-o", _LIB + ".tmp", _SRC, "-lm"]
        # OpenMP only spreads orc_eval_threads' leaves over host cores; without
        # it that entry point runs on one thread
        if subprocess.run(cmd[:1] + ["-fopenmp"] + cmd[1:], capture_output=True).returncode != 0:
            subprocess.check_call(cmd)
        os.replace(_LIB + ".tmp", _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is not None:
        return _lib
    build()
    L = ctypes.CDLL(_LIB)
    P = ctypes.c_void_p
    i64, i32, f64 = ctypes.c_int64, ctypes.c_int32, ctypes.c_double
    L.orc_build.restype = P
    L.orc_build.argtypes = [i64, P, P, P, f64, i32, i32, f64, f64, i32]
    L.orc_free.argtypes = [P]
    for name in ("orc_ncells", "orc_nleaves", "orc_maxdepth", "orc_nfallback"):
        getattr(L, name).restype = i32
        getattr(L, name).argtypes = [P]
    L.orc_get_order.argtypes = [P, P]
    L.orc_get_cells.argtypes = [P, P, P]
    L.orc_walk.restype = P
    L.orc_walk.argtypes = [P]
    L.orc_lists_nfar.restype = i64
    L.orc_lists_nfar.argtypes = [P]
    L.orc_lists_nnear.restype = i64
    L.orc_lists_nnear.argtypes = [P]
    L.orc_ancestor_far.restype = i32
    L.orc_ancestor_far.argtypes = []
    L.orc_lists_get.argtypes = [P, P, P, P, P, P]
    L.orc_lists_free.argtypes = [P]
    L.orc_eval.restype = i32
    L.orc_eval.argtypes = [P, i32, P, P, P, P, P, P, P, P]
    L.orc_eval_threads.restype = i32
    L.orc_eval_threads.argtypes = [P, i32, P, P, P, i32]
    L.orc_max_threads.restype = i32
    L.orc_max_threads.argtypes = []
    L.orc_eval_lists.restype = i32
    L.orc_eval_lists.argtypes = [P, i32, P, P, P, P, P, P, P]
    L.orc_moments_frozen.restype = i32
    L.orc_moments_frozen.argtypes = [P, P, P, P]
    L.orc_direct.argtypes = [i64, P, P, P, i32, f64, i64, P, P, P]
    L.orc_monomials.restype = i32
    L.orc_monomials.argtypes = [P]
    L.orc_moments.argtypes = [i64, P, P, P, P, P, P]
    L.orc_dual_walk.restype = P
    L.orc_dual_walk.argtypes = [P]
    L.orc_dual_nfar.restype = i64
    L.orc_dual_nfar.argtypes = [P]
    L.orc_dual_nnear.restype = i64
    L.orc_dual_nnear.argtypes = [P]
    L.orc_dual_get.argtypes = [P, P, P, P, P]
    L.orc_dual_get.restype = None
    L.orc_dual_free.argtypes = [P]
    L.orc_dual_free.restype = None
    L.orc_eval_dual.restype = i32
    L.orc_eval_dual.argtypes = [P, P, P, P]
    L.orc_m2l.argtypes = [P, f64, P, i32, P, P]
    L.orc_l2p.argtypes = [P, P, P, P, P]
    L.orc_acc_node.argtypes = [P, f64, P, P]
    L.orc_pair.argtypes = [P, f64, f64, f64, i32, f64, P, P]
    L.orc_m4.argtypes = [f64, P, P, P]
    _lib = L
    return L


def _p(a: np.ndarray | None):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _f64(a, shape=None) -> np.ndarray:
    a = np.ascontiguousarray(a, dtype=np.float64)
    if shape is not None:
        a = a.reshape(shape)
    return a


@dataclass
class Cells:
    """Cell table in pre-order ids (root 0)."""
    first: np.ndarray
    count: np.ndarray
    left: np.ndarray
    right: np.ndarray
    parent: np.ndarray
    depth: np.ndarray
    skip: np.ndarray
    M: np.ndarray
    com: np.ndarray
    s: np.ndarray
    hmax: np.ndarray
    Q: np.ndarray          # (ncells, 6): xx xy xz yy yz zz

    @property
    def is_leaf(self) -> np.ndarray:
        return self.left < 0


@dataclass
class Lists:
    """Per-leaf interaction lists; leaves in ascending id, entries ascending."""
    leaf_ids: np.ndarray
    far_off: np.ndarray
    far_idx: np.ndarray
    near_off: np.ndarray
    near_idx: np.ndarray
    ancestor_far: int


@dataclass
class DualLists:
    """Symmetric dual-tree walk: far lists per cell, near lists per leaf."""
    far_off: np.ndarray
    far_idx: np.ndarray
    near_off: np.ndarray
    near_idx: np.ndarray


class Tree:
    """kd-tree built by the oracle (Sec. 2) for one particle set."""

    def __init__(self, x, m, h=None, *, theta=0.5, n_leaf=16, soft_kind=SOFT_PLUMMER,
                 eps=0.01, r_kern=2.0, expansion=EXP_PHANTOM):
        L = _load()
        self.x = _f64(x, (-1, 3))
        self.n = self.x.shape[0]
        self.m = _f64(m)
        self.h = None if h is None else _f64(h)
        self.theta, self.n_leaf, self.soft_kind = float(theta), int(n_leaf), int(soft_kind)
        self.eps, self.r_kern = float(eps), float(r_kern)
        self.expansion = int(expansion)
        self._t = L.orc_build(self.n, _p(self.x), _p(self.m), _p(self.h), self.theta,
                              self.n_leaf, self.soft_kind, self.eps, self.r_kern, self.expansion)
        if not self._t:
            raise ValueError("oracle build rejected the arguments")

    def __del__(self):
        t = getattr(self, "_t", None)
        if t and _lib is not None:
            _lib.orc_free(t)
            self._t = None

    @property
    def ncells(self) -> int:
        return _load().orc_ncells(self._t)

    @property
    def nleaves(self) -> int:
        return _load().orc_nleaves(self._t)

    @property
    def maxdepth(self) -> int:
        return _load().orc_maxdepth(self._t)

    @property
    def nfallback(self) -> int:
        return _load().orc_nfallback(self._t)

    def order(self) -> np.ndarray:
        o = np.empty(self.n, dtype=np.int64)
        _load().orc_get_order(self._t, _p(o))
        return o

    def cells(self) -> Cells:
        nc = self.ncells
        ints = np.empty((nc, 7), dtype=np.int64)
        reals = np.empty((nc, 12), dtype=np.float64)
        _load().orc_get_cells(self._t, _p(ints), _p(reals))
        return Cells(first=ints[:, 0].copy(), count=ints[:, 1].copy(), left=ints[:, 2].copy(),
                     right=ints[:, 3].copy(), parent=ints[:, 4].copy(), depth=ints[:, 5].copy(),
                     skip=ints[:, 6].copy(), M=reals[:, 0].copy(), com=reals[:, 1:4].copy(),
                     s=reals[:, 4].copy(), hmax=reals[:, 5].copy(), Q=reals[:, 6:12].copy())

    def walk(self) -> Lists:
        L = _load()
        h = L.orc_walk(self._t)
        try:
            nl = self.nleaves
            nf, nn = L.orc_lists_nfar(h), L.orc_lists_nnear(h)
            leaf_ids = np.empty(nl, dtype=np.int32)
            far_off = np.empty(nl + 1, dtype=np.int64)
            near_off = np.empty(nl + 1, dtype=np.int64)
            far_idx = np.empty(max(nf, 1), dtype=np.int32)
            near_idx = np.empty(max(nn, 1), dtype=np.int32)
            L.orc_lists_get(h, _p(leaf_ids), _p(far_off), _p(far_idx), _p(near_off), _p(near_idx))
            anc = L.orc_ancestor_far()
        finally:
            L.orc_lists_free(h)
        return Lists(leaf_ids, far_off, far_idx[:nf], near_off, near_idx[:nn], anc)

    def eval(self, leaves=None, parts: bool = False):
        """Force evaluation (Eq. 3) for the particles of ``leaves`` (all leaves
        when None).  Returns a (n,3) and phi (n,) in caller order; rows of
        particles outside the selection are NaN.  With ``parts`` also returns
        a_short, a_long, phi_short, phi_long and the stats (n_p2p, n_m2l)."""
        L = _load()
        a = np.full((self.n, 3), np.nan)
        phi = np.full(self.n, np.nan)
        extra = [np.full((self.n, 3), np.nan), np.full((self.n, 3), np.nan),
                 np.full(self.n, np.nan), np.full(self.n, np.nan)] if parts else [None] * 4
        stats = np.zeros(2, dtype=np.int64)
        if leaves is None:
            rc = L.orc_eval(self._t, -1, None, _p(a), _p(phi), *[_p(e) for e in extra], _p(stats))
        else:
            sel = np.ascontiguousarray(leaves, dtype=np.int32)
            rc = L.orc_eval(self._t, len(sel), _p(sel), _p(a), _p(phi),
                            *[_p(e) for e in extra], _p(stats))
        if rc != 0:
            raise ValueError(f"oracle eval failed ({rc})")
        if parts:
            return a, phi, dict(a_short=extra[0], a_long=extra[1], phi_short=extra[2],
                                phi_long=extra[3], n_p2p=int(stats[0]), n_m2l=int(stats[1]))
        return a, phi


    def eval_threads(self, leaves=None, nthreads: int = 0):
        """eval() with the leaves spread over host threads (OpenMP); the same
        a and phi bit for bit."""
        a = np.full((self.n, 3), np.nan)
        phi = np.full(self.n, np.nan)
        if leaves is None:
            rc = _load().orc_eval_threads(self._t, -1, None, _p(a), _p(phi), int(nthreads))
        else:
            sel = np.ascontiguousarray(leaves, dtype=np.int32)
            rc = _load().orc_eval_threads(self._t, len(sel), _p(sel), _p(a), _p(phi), int(nthreads))
        if rc != 0:
            raise ValueError(f"oracle eval_threads failed ({rc})")
        return a, phi

    def dual_walk(self) -> "DualLists":
        """Lists of the symmetric dual-tree walk: far list of every cell (ids in
        ascending order), near list of every leaf (leaves in ascending id)."""
        L = _load()
        h = L.orc_dual_walk(self._t)
        try:
            nc, nl = self.ncells, self.nleaves
            nf, nn = L.orc_dual_nfar(h), L.orc_dual_nnear(h)
            far_off = np.empty(nc + 1, dtype=np.int64)
            near_off = np.empty(nl + 1, dtype=np.int64)
            far_idx = np.empty(max(nf, 1), dtype=np.int32)
            near_idx = np.empty(max(nn, 1), dtype=np.int32)
            L.orc_dual_get(h, _p(far_off), _p(far_idx), _p(near_off), _p(near_idx))
            res = DualLists(far_off, far_idx[:nf], near_off, near_idx[:nn])
        finally:
            L.orc_dual_free(h)
        return res

    def eval_dual(self):
        """a, phi (caller order) from the symmetric dual-tree walk."""
        L = _load()
        h = L.orc_dual_walk(self._t)
        a = np.full((self.n, 3), np.nan)
        phi = np.full(self.n, np.nan)
        try:
            rc = L.orc_eval_dual(self._t, h, _p(a), _p(phi))
        finally:
            L.orc_dual_free(h)
        if rc != 0:
            raise ValueError(f"oracle eval_dual failed ({rc})")
        return a, phi

    def moments_frozen(self, x, m, h=None):
        """New positions / masses / smoothing lengths for the same particles,
        cells kept (frozen topology); see orc_moments_frozen."""
        x, m = _f64(x, (-1, 3)), _f64(m)
        h = None if h is None else _f64(h)
        assert x.shape[0] == self.n
        self.x, self.m, self.h = x, m, h
        _load().orc_moments_frozen(self._t, _p(x), _p(m), _p(h))

    def eval_lists(self, lists: "Lists"):
        """a, phi (caller order) of every leaf from the given interaction lists."""
        a = np.full((self.n, 3), np.nan)
        phi = np.full(self.n, np.nan)
        li = np.ascontiguousarray(lists.leaf_ids, dtype=np.int32)
        fo = np.ascontiguousarray(lists.far_off, dtype=np.int64)
        no = np.ascontiguousarray(lists.near_off, dtype=np.int64)
        fi = np.ascontiguousarray(lists.far_idx, dtype=np.int32)
        ni = np.ascontiguousarray(lists.near_idx, dtype=np.int32)
        rc = _load().orc_eval_lists(self._t, len(li), _p(li), _p(fo), _p(fi), _p(no), _p(ni),
                                    _p(a), _p(phi))
        if rc != 0:
            raise ValueError(f"oracle eval_lists failed ({rc})")
        return a, phi


def max_threads() -> int:
    """Host threads eval_threads uses by default."""
    return int(_load().orc_max_threads())


def direct(x, m, h=None, *, soft_kind=SOFT_PLUMMER, eps=0.01, targets=None):
    """O(N^2) direct summation with the same pair interaction (j != i).  Rows
    follow ``targets`` (all particles when None)."""
    L = _load()
    x = _f64(x, (-1, 3))
    m = _f64(m)
    h = None if h is None else _f64(h)
    n = x.shape[0]
    if targets is None:
        nt, tp = -1, None
        rows = n
    else:
        tgt = np.ascontiguousarray(targets, dtype=np.int64)
        nt, tp, rows = len(tgt), _p(tgt), len(tgt)
    a = np.empty((rows, 3))
    phi = np.empty(rows)
    L.orc_direct(n, _p(x), _p(m), _p(h), int(soft_kind), float(eps), nt, tp, _p(a), _p(phi))
    return a, phi


def monomials() -> np.ndarray:
    """Exponents (20, 3) of the Taylor coefficients used by the local expansion."""
    e = np.empty((20, 3), dtype=np.int32)
    _load().orc_monomials(_p(e))
    return e


def moments(x, m):
    """M, com, Q (xx xy xz yy yz zz), s of a particle set (Eq. 7, Sec. 2)."""
    x, m = _f64(x, (-1, 3)), _f64(m)
    M = np.zeros(1)
    com, Q, s = np.zeros(3), np.zeros(6), np.zeros(1)
    _load().orc_moments(x.shape[0], _p(x), _p(m), _p(M), _p(com), _p(Q), _p(s))
    return float(M[0]), com, Q, float(s[0])


def m2l(r, M, Q, expansion=EXP_PHANTOM):
    """Local-expansion Taylor coefficients of one source about r: potential (20,)
    and acceleration (3, 20) -- Eq. 6 and its derivatives (or the standard p = 3
    series with expansion=EXP_STANDARD)."""
    r, Q = _f64(r), _f64(Q)
    pot, acc = np.zeros(20), np.zeros(60)
    _load().orc_m2l(_p(r), float(M), _p(Q), int(expansion), _p(pot), _p(acc))
    return pot, acc.reshape(3, 20)


def l2p(pot, acc, x):
    """Eq. 8 (and the potential's third-order expansion) at displacement x."""
    pot, acc, x = _f64(pot), _f64(acc), _f64(x)
    a, phi = np.zeros(3), np.zeros(1)
    _load().orc_l2p(_p(pot), _p(acc), _p(x), _p(a), _p(phi))
    return a, float(phi[0])


def acc_node(r, M, Q):
    """Eq. 6 with plain doubles."""
    r, Q = _f64(r), _f64(Q)
    a = np.zeros(3)
    _load().orc_acc_node(_p(r), float(M), _p(Q), _p(a))
    return a


def pair(d, mj, hi=0.0, hj=0.0, *, soft_kind=SOFT_PLUMMER, eps=0.01):
    """Acceleration on i and potential from j, d = x_i - x_j."""
    d = _f64(d)
    a, phi = np.zeros(3), np.zeros(1)
    _load().orc_pair(_p(d), float(mj), float(hi), float(hj), int(soft_kind), float(eps), _p(a), _p(phi))
    return a, float(phi[0])


def m4(q):
    """M4 kernel pieces at q = r/h: w(q), enclosed fraction F(q), potential P(q)."""
    w, F, P = np.zeros(1), np.zeros(1), np.zeros(1)
    _load().orc_m4(float(q), _p(w), _p(F), _p(P))
    return float(w[0]), float(F[0]), float(P[0])

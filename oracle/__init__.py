"""Python access to the FP64 CPU oracle (``og_oracle.c``).

TEST INFRASTRUCTURE ONLY: the slow, obviously-correct reference that the CUDA
path is compared against.  Only the tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline / reference leg import this package.  The product
path never calls it and has no CPU fallback.

The PM long-range complement has its own numpy FP64 oracle in ``og_pm.py``
(``from oracle import og_pm``), the kick-drift-kick step one in
``og_kdk.py``, and the SPH density / smoothing-length iteration one in
``og_sph.py``.

``build()`` compiles the C file with gcc (``-O2 -ffp-contract=off``: no fused
multiply-add, so every FP64 decision formula is evaluated exactly as written).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "og_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None

_D = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
_I64 = np.ctypeslib.ndpointer(dtype=np.int64, flags="C_CONTIGUOUS")
_I32 = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")
_U64 = np.ctypeslib.ndpointer(dtype=np.uint64, flags="C_CONTIGUOUS")
_U32 = np.ctypeslib.ndpointer(dtype=np.uint32, flags="C_CONTIGUOUS")


def build(force: bool = False) -> str:
    """Compile the oracle shared library (if stale) and return its path."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
           "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            path = build()
            L = C.CDLL(path)
            L.orc_hilbert_cell.restype = C.c_uint64
            L.orc_hilbert_cell.argtypes = [C.c_uint32] * 3
            L.orc_hilbert_grid.restype = C.c_uint64
            L.orc_hilbert_grid.argtypes = [C.c_uint32] * 3 + [C.c_int]
            L.orc_keys.restype = C.c_int64
            L.orc_keys.argtypes = [_D, C.c_int64, C.c_double, _U64, C.c_void_p]
            L.orc_sort.restype = None
            L.orc_sort.argtypes = [_U64, C.c_int64, _U64, _I32]
            L.orc_kernel_f.restype = C.c_double
            L.orc_kernel_f.argtypes = [C.c_double, C.c_double]
            L.orc_kernel_K.restype = C.c_double
            L.orc_kernel_K.argtypes = [C.c_double, C.c_double]
            L.orc_direct.restype = None
            L.orc_direct.argtypes = [_D, _D, _D, C.c_int64, C.c_double, C.c_double, C.c_double,
                                     _I64, C.c_int64, _D, _I64]
            L.orc_tree_build.restype = C.c_void_p
            L.orc_tree_build.argtypes = [_D, _D, _D, C.c_int64, C.c_double, C.c_int]
            L.orc_tree_free.restype = None
            L.orc_tree_free.argtypes = [C.c_void_p]
            L.orc_tree_nnodes.restype = C.c_int64
            L.orc_tree_nnodes.argtypes = [C.c_void_p]
            L.orc_tree_nodes.restype = None
            L.orc_tree_nodes.argtypes = [C.c_void_p, _I32, _U32, _I64, _D, _D, _D, _I32, _I64, _I64, _I32]
            L.orc_tree_members.restype = None
            L.orc_tree_members.argtypes = [C.c_void_p, C.c_int64, _I64]
            L.orc_walk.restype = None
            L.orc_walk.argtypes = [C.c_void_p, C.c_double, C.c_double, C.c_double, _I64, C.c_int64, _D, _I64]
            L.orc_walk_cover_errors.restype = C.c_int64
            L.orc_walk_cover_errors.argtypes = [C.c_void_p, C.c_double, C.c_double, _I64, C.c_int64]
            L.orc_walk_lists.restype = None
            L.orc_walk_lists.argtypes = [C.c_void_p, C.c_double, C.c_double, _I64, C.c_int64, _I64,
                                         C.c_void_p, C.c_void_p]
            L.orc_adjoint.restype = None
            L.orc_adjoint.argtypes = [C.c_void_p, C.c_double, C.c_double, C.c_double, _D, C.c_void_p,
                                      C.c_int64, _D, _D, C.c_void_p, C.c_void_p]
            L.orc_fd.restype = None
            L.orc_fd.argtypes = [C.c_void_p, C.c_double, C.c_double, C.c_double, _D, _I64, C.c_int64,
                                 C.c_double, C.c_double, _D, _D, C.c_void_p]
            L.orc_loss.restype = C.c_double
            L.orc_loss.argtypes = [C.c_void_p, C.c_double, C.c_double, C.c_double, _D]
            _lib = L
    return _lib


def _pos(pos):
    return np.ascontiguousarray(pos, dtype=np.float64).reshape(-1, 3)


def softening_h(eps):
    """Spline support h = 2.8 eps (Plummer-equivalent softening convention)."""
    return 2.8 * np.asarray(eps, dtype=np.float64)


# ---------------------------------------------------------------- keys / sort

def hilbert_grid(q, bits: int) -> np.ndarray:
    """Hilbert index of integer cells q [m,3] on a 2^bits grid."""
    L = lib()
    q = np.asarray(q, dtype=np.uint32).reshape(-1, 3)
    return np.array([L.orc_hilbert_grid(int(a), int(b), int(c), bits) for a, b, c in q], dtype=np.uint64)


def keys(pos, box: float = 1.0):
    """(keys uint64 [n], n_bad, cells uint32 [n,3])."""
    L = lib()
    pos = _pos(pos)
    n = pos.shape[0]
    out = np.zeros(n, np.uint64)
    cells = np.zeros((n, 3), np.uint32)
    bad = L.orc_keys(pos.ravel(), n, box, out, cells.ctypes.data)
    return out, int(bad), cells


def sort(keys_in):
    """(keys_sorted, order int32) -- ascending key, ties by original index."""
    L = lib()
    k = np.ascontiguousarray(keys_in, dtype=np.uint64)
    ks = np.zeros_like(k)
    order = np.zeros(k.shape[0], np.int32)
    L.orc_sort(k, k.shape[0], ks, order)
    return ks, order


# ---------------------------------------------------------------- force law

def kernel_f(r: float, r_s: float) -> float:
    return lib().orc_kernel_f(float(r), float(r_s))


def kernel_K(r: float, h: float) -> float:
    return lib().orc_kernel_K(float(r), float(h))


def direct(pos, mass, h, box, r_s, rcut, targets=None):
    """Direct periodic short-range sum: (acc [nt,3], interactions [nt])."""
    L = lib()
    pos = _pos(pos)
    n = pos.shape[0]
    mass = np.ascontiguousarray(mass, dtype=np.float64)
    h = np.ascontiguousarray(np.broadcast_to(h, (n,)), dtype=np.float64)
    tg = np.arange(n, dtype=np.int64) if targets is None else np.ascontiguousarray(targets, dtype=np.int64)
    acc = np.zeros((tg.shape[0], 3))
    cnt = np.zeros(tg.shape[0], np.int64)
    L.orc_direct(pos.ravel(), mass, h, n, box, r_s, rcut, tg, tg.shape[0], acc.ravel(), cnt)
    return acc, cnt


# ---------------------------------------------------------------- tree / walk

class Tree:
    """Oracle octree (recursive octant subdivision of the integer cell grid)."""

    def __init__(self, pos, mass, h, box: float = 1.0, leaf_size: int = 16):
        self._L = lib()
        self.pos = _pos(pos)
        self.n = self.pos.shape[0]
        self.mass = np.ascontiguousarray(mass, dtype=np.float64)
        self.h = np.ascontiguousarray(np.broadcast_to(h, (self.n,)), dtype=np.float64)
        self.box = float(box)
        self.leaf_size = int(leaf_size)
        self._h = self._L.orc_tree_build(self.pos.ravel(), self.mass, self.h, self.n, self.box, self.leaf_size)

    def close(self):
        if getattr(self, "_h", None):
            self._L.orc_tree_free(self._h)
            self._h = None

    def __del__(self):
        self.close()

    @property
    def nnodes(self) -> int:
        return int(self._L.orc_tree_nnodes(self._h))

    def nodes(self) -> dict:
        m = self.nnodes
        out = dict(level=np.zeros(m, np.int32), cell=np.zeros((m, 3), np.uint32), count=np.zeros(m, np.int64),
                   mass=np.zeros(m), com=np.zeros((m, 3)), hmax=np.zeros(m), leaf=np.zeros(m, np.int32),
                   parent=np.zeros(m, np.int64), child0=np.zeros(m, np.int64), nchild=np.zeros(m, np.int32))
        self._L.orc_tree_nodes(self._h, out["level"], out["cell"].ravel(), out["count"], out["mass"],
                               out["com"].ravel(), out["hmax"], out["leaf"], out["parent"], out["child0"],
                               out["nchild"])
        return out

    def members(self, k: int) -> np.ndarray:
        if not hasattr(self, "_cnt"):
            self._cnt = self.nodes()["count"]
        out = np.zeros(int(self._cnt[k]), np.int64)
        self._L.orc_tree_members(self._h, int(k), out)
        return out

    def walk(self, r_s, rcut, theta, targets=None):
        tg = np.arange(self.n, dtype=np.int64) if targets is None else np.ascontiguousarray(targets, np.int64)
        acc = np.zeros((tg.shape[0], 3))
        cnt = np.zeros(tg.shape[0], np.int64)
        self._L.orc_walk(self._h, r_s, rcut, theta, tg, tg.shape[0], acc.ravel(), cnt)
        return acc, cnt

    def cover_errors(self, rcut, theta, targets=None) -> int:
        tg = np.arange(self.n, dtype=np.int64) if targets is None else np.ascontiguousarray(targets, np.int64)
        return int(self._L.orc_walk_cover_errors(self._h, rcut, theta, tg, tg.shape[0]))

    def lists(self, rcut, theta, targets):
        tg = np.ascontiguousarray(targets, np.int64)
        off = np.zeros(tg.shape[0] + 1, np.int64)
        self._L.orc_walk_lists(self._h, rcut, theta, tg, tg.shape[0], off, None, None)
        kind = np.zeros(max(int(off[-1]), 1), np.int32)
        ids = np.zeros(max(int(off[-1]), 1), np.int64)
        self._L.orc_walk_lists(self._h, rcut, theta, tg, tg.shape[0], off, kind.ctypes.data, ids.ctypes.data)
        return off, kind[: off[-1]], ids[: off[-1]]

    def adjoint(self, r_s, rcut, theta, w, samples=None, with_scale=False):
        """dL/dx [ns,3], dL/dm [ns] of L = sum_i w_i . a_i (frozen decisions).
        with_scale: also return the same sums over the absolute values of
        their terms (the scale of any evaluation's rounding error)."""
        w = np.ascontiguousarray(w, dtype=np.float64).reshape(-1, 3)
        if samples is None:
            ns = self.n
            sp = None
        else:
            samples = np.ascontiguousarray(samples, dtype=np.int64)
            ns = samples.shape[0]
            sp = samples.ctypes.data
        dpos = np.zeros((ns, 3))
        dmass = np.zeros(ns)
        dpa = np.zeros((ns, 3)) if with_scale else None
        dma = np.zeros(ns) if with_scale else None
        self._L.orc_adjoint(self._h, r_s, rcut, theta, w.ravel(), sp, ns, dpos.ravel(), dmass,
                            dpa.ctypes.data if with_scale else None, dma.ctypes.data if with_scale else None)
        return (dpos, dmass, dpa, dma) if with_scale else (dpos, dmass)

    def fd(self, r_s, rcut, theta, w, samples, hx=1e-6, hm_rel=1e-6, with_flags=False):
        """Central differences of the frozen-list loss.  with_flags: also the
        per-sample crossing flags (bit 0: a step moves an involved term across
        its softening length, bit 1: across rcut)."""
        w = np.ascontiguousarray(w, dtype=np.float64).reshape(-1, 3)
        samples = np.ascontiguousarray(samples, dtype=np.int64)
        ns = samples.shape[0]
        dpos = np.zeros((ns, 3))
        dmass = np.zeros(ns)
        flags = np.zeros(ns, np.int32)
        self._L.orc_fd(self._h, r_s, rcut, theta, w.ravel(), samples, ns, hx, hm_rel, dpos.ravel(), dmass,
                       flags.ctypes.data)
        return (dpos, dmass, flags) if with_flags else (dpos, dmass)

    def loss(self, r_s, rcut, theta, w) -> float:
        w = np.ascontiguousarray(w, dtype=np.float64).reshape(-1, 3)
        return float(self._L.orc_loss(self._h, r_s, rcut, theta, w.ravel()))

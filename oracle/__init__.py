"""CPU oracle for the lattice sum u = phi * f (test infrastructure).

This package is test infrastructure.  Only ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline / reference legs of ``bench.py`` may import it; the CUDA
library never does, and the two share no code.  It is plain and slow on
purpose: binary64 everywhere, exact phi near the origin, brute-force O(N_src*N_tgt)
sums with Neumaier compensation.

Contents (each follows the cited passage of the paper):
  phi_octant(R)       exact phi on 0 <= n <= m <= R           (eq. 1.8; see phi_exact)
  phi(d)              phi at integer offsets: table or eq. 3.1  (Sec. 3)
  phi_asym(d)         eq. 3.1 without its O(|m|^-6) remainder   (Sec. 3.1)
  lattice_sum(...)    u_i = sum_j phi(x_i - y_j) f_j            (eq. 1.7, eq. 2.1)
  near_sum(...)       the same restricted to same/adjacent leaves (eq. 2.2-2.4)
  uniform_tree(...)   root box and leaf level of the uniform quadtree (Sec. 6)
  apply_A(u_of)       the 5-point operator A of eq. 1.2 on a dict of values
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from .build import build_oracle
from .phi_exact import octant_index, phi_exact_fraction, phi_octant

DEFAULT_R = 256  # exact table radius; beyond it eq. 3.1 errs by < 0.15/|m|^6 < 6e-16

_lib = None


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build_oracle())
        i64, dp, i32p = ctypes.c_int64, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int32)
        i64p = ctypes.POINTER(ctypes.c_int64)
        lib.orc_phi_asym.restype = ctypes.c_double
        lib.orc_phi_asym.argtypes = [ctypes.c_double, ctypes.c_double]
        lib.orc_phi_many.restype = None
        lib.orc_phi_many.argtypes = [i64p, i64, dp, i64, dp]
        lib.orc_lattice_sum.restype = None
        lib.orc_lattice_sum.argtypes = [i32p, i64, dp, i32p, i64, dp, i64, dp]
        lib.orc_near_sum.restype = None
        lib.orc_near_sum.argtypes = [i32p, i64, dp, i32p, i64, i64, i64, i64, dp, i64, dp]
        lib.orc_num_threads.restype = ctypes.c_int
        lib.orc_num_threads.argtypes = []
        _lib = lib
    return _lib


def _ptr(a, ctype):
    return a.ctypes.data_as(ctypes.POINTER(ctype))


def _xy(a) -> np.ndarray:
    a = np.ascontiguousarray(a, dtype=np.int32)
    if a.ndim != 2 or a.shape[1] != 2:
        raise ValueError("coordinates must have shape (n, 2)")
    return a


def num_threads() -> int:
    return int(_load().orc_num_threads())


def phi_asym(d) -> np.ndarray:
    """eq. 3.1 (remainder dropped) at offsets d of shape (n, 2); d != 0."""
    d = np.asarray(d, dtype=np.float64).reshape(-1, 2)
    lib = _load()
    return np.array([lib.orc_phi_asym(float(a), float(b)) for a, b in d])


def phi(d, R: int = DEFAULT_R) -> np.ndarray:
    """phi at integer offsets d of shape (n, 2): exact table for |d|_inf <= R, else eq. 3.1."""
    d = np.ascontiguousarray(np.asarray(d, dtype=np.int64).reshape(-1, 2))
    oct_ = phi_octant(R)
    out = np.empty(d.shape[0], dtype=np.float64)
    _load().orc_phi_many(_ptr(d, ctypes.c_int64), d.shape[0], _ptr(oct_, ctypes.c_double), R,
                         _ptr(out, ctypes.c_double))
    return out


def lattice_sum(src, f, tgt, R: int = DEFAULT_R) -> np.ndarray:
    """u_i = sum_j phi(tgt_i - src_j) f_j in binary64 with Neumaier summation (eq. 1.7)."""
    src, tgt = _xy(src), _xy(tgt)
    f = np.ascontiguousarray(f, dtype=np.float64)
    if f.shape != (src.shape[0],):
        raise ValueError("f must have one value per source")
    oct_ = phi_octant(R)
    u = np.empty(tgt.shape[0], dtype=np.float64)
    _load().orc_lattice_sum(_ptr(src, ctypes.c_int32), src.shape[0], _ptr(f, ctypes.c_double),
                            _ptr(tgt, ctypes.c_int32), tgt.shape[0],
                            _ptr(oct_, ctypes.c_double), R, _ptr(u, ctypes.c_double))
    return u


def near_sum(src, f, tgt, x0: int, y0: int, s: int, R: int = DEFAULT_R) -> np.ndarray:
    """Near field of eq. 2.2: sources in the target's leaf or an adjacent leaf of a
    uniform tree with leaf side s and root corner (x0, y0)."""
    src, tgt = _xy(src), _xy(tgt)
    f = np.ascontiguousarray(f, dtype=np.float64)
    oct_ = phi_octant(R)
    u = np.empty(tgt.shape[0], dtype=np.float64)
    _load().orc_near_sum(_ptr(src, ctypes.c_int32), src.shape[0], _ptr(f, ctypes.c_double),
                         _ptr(tgt, ctypes.c_int32), tgt.shape[0], int(x0), int(y0), int(s),
                         _ptr(oct_, ctypes.c_double), R, _ptr(u, ctypes.c_double))
    return u


def uniform_tree(src, tgt, n_leaf: int, max_leaf_side: int = 64):
    """Root box and leaf level of the uniform quadtree (Sec. 6).

    The root is the square of side 2^K anchored at the lower-left corner
    (min x, min y) of all sources and targets, K the smallest integer with
    2^K >= the larger extent.  The leaf level L is the smallest level whose
    4^L boxes each hold at most n_leaf sources and at most n_leaf targets,
    subject to leaf side 2^(K-L) <= max_leaf_side; if no level qualifies
    (coincident points) L = K.

    Returns dict(x0, y0, K, L, side) with side = 2^(K-L)."""
    src, tgt = _xy(src), _xy(tgt)
    pts = np.concatenate([src, tgt]).astype(np.int64)
    x0, y0 = int(pts[:, 0].min()), int(pts[:, 1].min())
    ext = int(max(pts[:, 0].max() - x0, pts[:, 1].max() - y0)) + 1
    K = 0
    while (1 << K) < ext:
        K += 1
    smax_log = int(max_leaf_side).bit_length() - 1
    L_lo = max(0, K - smax_log)
    L = K
    for level in range(L_lo, K + 1):
        shift = K - level
        ok = True
        for arr in (src, tgt):
            bx = (arr[:, 0].astype(np.int64) - x0) >> shift
            by = (arr[:, 1].astype(np.int64) - y0) >> shift
            _, counts = np.unique(bx * (1 << level) + by, return_counts=True)
            if counts.size and counts.max() > n_leaf:
                ok = False
                break
        if ok:
            L = level
            break
    return dict(x0=x0, y0=y0, K=K, L=L, side=1 << (K - L))


def apply_A(u_of: dict, m) -> float:
    """(A u)(m) = 4u(m) - u(m+e1) - u(m-e1) - u(m+e2) - u(m-e2)   (eq. 1.2)."""
    x, y = m
    return (4.0 * u_of[(x, y)] - u_of[(x + 1, y)] - u_of[(x - 1, y)]
            - u_of[(x, y + 1)] - u_of[(x, y - 1)])


__all__ = ["phi_octant", "octant_index", "phi_exact_fraction", "phi", "phi_asym",
           "lattice_sum", "near_sum", "uniform_tree", "apply_A", "num_threads", "DEFAULT_R"]

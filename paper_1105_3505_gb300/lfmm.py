"""Thin ctypes binding of liblfmm.so (C ABI in include/lfmm.h).

Argument marshalling only: every step of the method runs inside the library.
Arrays may be numpy arrays (host) or torch tensors (host or CUDA); pointers are
passed straight through and the library copies host data itself.  The library
must have been built (``paper_1105_3505_gb300.build.build()``); loading fails
loudly otherwise - there is no fallback implementation.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from .build import LIB

(LFMM_OK, LFMM_EINVAL, LFMM_ENOMEM, LFMM_ECUDA, LFMM_ETIMEOUT, LFMM_EUNSUPPORTED, LFMM_EINTERNAL, LFMM_EBUSY,
 LFMM_ECANCELED) = range(9)
LFMM_FP64, LFMM_MIXED, LFMM_DF = 0, 1, 2
LFMM_TREE_AUTO, LFMM_TREE_UNIFORM, LFMM_TREE_PRUNED = 0, 1, 2
LFMM_FLAG_GRAPH, LFMM_FLAG_SERIAL, LFMM_FLAG_PERSISTENT = 1, 2, 4

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "lfmm.h")


class LfmmError(RuntimeError):
    def __init__(self, status: int, where: str, detail: str):
        super().__init__(f"{where}: {detail or 'status ' + str(status)} (status {status})")
        self.status = status


class lfmm_opts(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int32), ("p", ctypes.c_int32), ("leaf_size", ctypes.c_int32),
                ("max_leaf_side", ctypes.c_int32), ("proxies_per_edge", ctypes.c_int32),
                ("tc_min_level", ctypes.c_int32), ("tree", ctypes.c_int32), ("flags", ctypes.c_int32),
                ("m2l_tile", ctypes.c_int32), ("m2l_stages", ctypes.c_int32), ("m2l_split", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]


class lfmm_plan_info(ctypes.Structure):
    _fields_ = [("n_src", ctypes.c_int64), ("n_tgt", ctypes.c_int64), ("x0", ctypes.c_int64),
                ("y0", ctypes.c_int64), ("K", ctypes.c_int32), ("L", ctypes.c_int32),
                ("leaf_side", ctypes.c_int32), ("P", ctypes.c_int32), ("P_pad", ctypes.c_int32),
                ("precision", ctypes.c_int32), ("max_leaf_src", ctypes.c_int32),
                ("max_leaf_tgt", ctypes.c_int32), ("device_bytes", ctypes.c_int64), ("tree", ctypes.c_int32),
                ("n_problems", ctypes.c_int32), ("n_boxes", ctypes.c_int64)]


class lfmm_request(ctypes.Structure):
    _fields_ = [("src_xy", ctypes.c_void_p), ("n_src", ctypes.c_int64), ("tgt_xy", ctypes.c_void_p),
                ("n_tgt", ctypes.c_int64), ("f", ctypes.c_void_p), ("u", ctypes.c_void_p), ("tol", ctypes.c_double)]


class lfmm_request_stats(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("precision", ctypes.c_int32), ("queue_ms", ctypes.c_double),
                ("run_ms", ctypes.c_double), ("total_ms", ctypes.c_double), ("device_bytes", ctypes.c_int64)]


class lfmm_tune_result(ctypes.Structure):
    _fields_ = [("opts", lfmm_opts), ("rel_err", ctypes.c_double), ("ms", ctypes.c_double),
                ("candidates", ctypes.c_int32), ("from_cache", ctypes.c_int32)]


_lib = None


def load(path: str | None = None) -> ctypes.CDLL:
    """Load liblfmm.so (raises OSError if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or LIB
    if not os.path.exists(path):
        raise OSError(f"liblfmm.so not found at {path}; build it with paper_1105_3505_gb300.build.build()")
    lib = ctypes.CDLL(path)
    vp, i32, i64, dp = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_void_p
    sig = {
        "lfmm_opts_default": (None, [ctypes.POINTER(lfmm_opts)]),
        "lfmm_plan_create": (ctypes.c_int, [ctypes.POINTER(vp), vp, i64, vp, i64, ctypes.POINTER(lfmm_opts), vp]),
        "lfmm_forest_create": (ctypes.c_int, [ctypes.POINTER(vp), vp, vp, vp, vp, i64, ctypes.POINTER(lfmm_opts),
                                              vp]),
        "lfmm_eval": (ctypes.c_int, [vp, vp, vp, vp]),
        "lfmm_eval_parts": (ctypes.c_int, [vp, vp, vp, vp, vp]),
        "lfmm_plan_destroy": (ctypes.c_int, [vp]),
        "lfmm_plan_set_flags": (ctypes.c_int, [vp, i32]),
        "lfmm_solve": (ctypes.c_int, [vp, i64, vp, i64, vp, vp, ctypes.POINTER(lfmm_opts), vp]),
        "lfmm_eval_multi": (ctypes.c_int, [vp, vp, i32, vp, vp]),
        "lfmm_phi_quadrature": (ctypes.c_int, [vp, vp, i32, i32, vp, vp]),
        "lfmm_plan_status": (ctypes.c_int, [vp, vp]),
        "lfmm_plan_get_info": (ctypes.c_int, [vp, ctypes.POINTER(lfmm_plan_info)]),
        "lfmm_status_string": (ctypes.c_char_p, [ctypes.c_int]),
        "lfmm_last_error": (ctypes.c_char_p, []),
        "lfmm_phi_table": (ctypes.c_int, [i32, dp]),
        "lfmm_phi": (ctypes.c_int, [vp, i64, dp]),
        "lfmm_model_skeleton": (ctypes.c_int, [i32, i32, i32, i32, vp, ctypes.POINTER(i32)]),
        "lfmm_model_tofs": (ctypes.c_int, [i32, i32, i32, dp]),
        "lfmm_model_s": (ctypes.c_int, [i32, i32, i32, i32, dp]),
        "lfmm_profile_enable": (ctypes.c_int, [ctypes.c_int]),
        "lfmm_profile_read": (ctypes.c_int, [vp, vp, ctypes.c_int]),
        "lfmm_launch_count": (ctypes.c_int64, []),
        "lfmm_plan_shape_noalloc": (ctypes.c_int, [vp, i64, vp, i64, ctypes.POINTER(lfmm_opts),
                                                   ctypes.POINTER(lfmm_plan_info), vp]),
        "lfmm_server_create": (ctypes.c_int, [ctypes.POINTER(vp), i32, i64]),
        "lfmm_server_submit": (ctypes.c_int, [vp, ctypes.POINTER(lfmm_request), ctypes.POINTER(i64)]),
        "lfmm_server_wait": (ctypes.c_int, [vp, i64, ctypes.POINTER(lfmm_request_stats)]),
        "lfmm_server_destroy": (ctypes.c_int, [vp]),
        "lfmm_server_set_limits": (ctypes.c_int, [vp, i32, ctypes.c_double]),
        "lfmm_server_cancel": (ctypes.c_int, [vp, i64]),
        "lfmm_plan_set_wait_budget": (ctypes.c_int, [vp, i32]),
        "lfmm_plan_inject_barrier_stall": (ctypes.c_int, [vp]),
        "lfmm_pool_used_bytes": (ctypes.c_int, [ctypes.POINTER(i64)]),
        "lfmm_fault_inject_alloc": (ctypes.c_int, [i64]),
        "lfmm_autotune": (ctypes.c_int, [vp, i64, vp, vp, i64, vp, i64, ctypes.c_double, ctypes.POINTER(lfmm_opts),
                                         ctypes.POINTER(lfmm_tune_result), vp]),
        "lfmm_tune_cache_clear": (ctypes.c_int, []),
        "lfmm_tune_cache_save": (ctypes.c_int, [ctypes.c_char_p]),
        "lfmm_tune_cache_load": (ctypes.c_int, [ctypes.c_char_p]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _check(status: int, where: str):
    if status != LFMM_OK:
        lib = load()
        raise LfmmError(status, where, lib.lfmm_last_error().decode())


def _ptr(a) -> int:
    """Raw address of a numpy array or torch tensor (must be contiguous)."""
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return a.ctypes.data
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return a.data_ptr()
    raise TypeError(f"unsupported array type {type(a)}")


def _stream_handle(stream) -> int | None:
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream  # torch.cuda.Stream


def lfmm_opts_default() -> lfmm_opts:
    o = lfmm_opts()
    load().lfmm_opts_default(ctypes.byref(o))
    return o


def make_opts(precision: int = LFMM_MIXED, p: int = 8, leaf_size: int = 64, max_leaf_side: int = 32,
              proxies_per_edge: int = 64, tc_min_level: int = 0, tree: int = LFMM_TREE_AUTO,
              graph: bool = False, serial: bool = False, m2l_tile: int = 0, m2l_stages: int = 0,
              m2l_split: int = 0, persistent: bool = False) -> lfmm_opts:
    o = lfmm_opts_default()
    o.precision, o.p, o.leaf_size = precision, p, leaf_size
    o.max_leaf_side, o.proxies_per_edge, o.tc_min_level = max_leaf_side, proxies_per_edge, tc_min_level
    o.tree = tree
    o.flags = (LFMM_FLAG_GRAPH if graph else 0) | (LFMM_FLAG_SERIAL if serial else 0) | \
        (LFMM_FLAG_PERSISTENT if persistent else 0)
    o.m2l_tile, o.m2l_stages, o.m2l_split = m2l_tile, m2l_stages, m2l_split
    return o


def lfmm_plan_create(src_xy, n_src: int, tgt_xy, n_tgt: int, opts: lfmm_opts | None, stream=None) -> int:
    h = ctypes.c_void_p()
    st = load().lfmm_plan_create(ctypes.byref(h), _ptr(src_xy), int(n_src), _ptr(tgt_xy), int(n_tgt),
                                 ctypes.byref(opts) if opts is not None else None, _stream_handle(stream))
    _check(st, "lfmm_plan_create")
    return h.value


def lfmm_forest_create(src_xy, src_offsets, tgt_xy, tgt_offsets, opts: lfmm_opts | None, stream=None) -> int:
    """src_offsets, tgt_offsets: n_problems + 1 int64 offsets (host numpy)."""
    so = np.ascontiguousarray(np.asarray(src_offsets, dtype=np.int64))
    to = np.ascontiguousarray(np.asarray(tgt_offsets, dtype=np.int64))
    if so.shape != to.shape or so.ndim != 1 or so.shape[0] < 2:
        raise ValueError("offsets must be two 1-D arrays of n_problems + 1 entries")
    h = ctypes.c_void_p()
    st = load().lfmm_forest_create(ctypes.byref(h), _ptr(src_xy), so.ctypes.data, _ptr(tgt_xy), to.ctypes.data,
                                   so.shape[0] - 1, ctypes.byref(opts) if opts is not None else None,
                                   _stream_handle(stream))
    _check(st, "lfmm_forest_create")
    return h.value


def lfmm_eval(plan: int, f, u, stream=None) -> None:
    _check(load().lfmm_eval(plan, _ptr(f), _ptr(u), _stream_handle(stream)), "lfmm_eval")


def lfmm_eval_parts(plan: int, f, u_near, u_far, stream=None) -> None:
    _check(load().lfmm_eval_parts(plan, _ptr(f), _ptr(u_near), _ptr(u_far), _stream_handle(stream)),
           "lfmm_eval_parts")


def lfmm_plan_destroy(plan: int) -> None:
    _check(load().lfmm_plan_destroy(plan), "lfmm_plan_destroy")


def lfmm_plan_status(plan: int, stream=None) -> None:
    """Raise LfmmError(LFMM_ETIMEOUT) if a bounded device-side wait of the plan gave up."""
    _check(load().lfmm_plan_status(plan, _stream_handle(stream)), "lfmm_plan_status")


def lfmm_plan_get_info(plan: int) -> dict:
    info = lfmm_plan_info()
    _check(load().lfmm_plan_get_info(plan, ctypes.byref(info)), "lfmm_plan_get_info")
    return {name: getattr(info, name) for name, _ in lfmm_plan_info._fields_}


def lfmm_plan_shape_noalloc(src_xy, n_src: int, tgt_xy, n_tgt: int, opts: lfmm_opts | None,
                            stream=None) -> dict:
    """Tree shape and device footprint of a would-be plan, computed without allocating
    (see include/lfmm.h); coordinates must be CUDA tensors."""
    info = lfmm_plan_info()
    _check(load().lfmm_plan_shape_noalloc(_ptr(src_xy), int(n_src), _ptr(tgt_xy), int(n_tgt),
                                          ctypes.byref(opts) if opts is not None else None,
                                          ctypes.byref(info), _stream_handle(stream)),
           "lfmm_plan_shape_noalloc")
    return {name: getattr(info, name) for name, _ in lfmm_plan_info._fields_}


def lfmm_status_string(status: int) -> str:
    return load().lfmm_status_string(int(status)).decode()


def lfmm_last_error() -> str:
    return load().lfmm_last_error().decode()


def lfmm_phi_table(R: int) -> np.ndarray:
    out = np.empty((R + 1) * (R + 2) // 2, dtype=np.float64)
    _check(load().lfmm_phi_table(int(R), out.ctypes.data), "lfmm_phi_table")
    return out


def lfmm_phi(d) -> np.ndarray:
    d = np.ascontiguousarray(np.asarray(d, dtype=np.int64).reshape(-1, 2))
    out = np.empty(d.shape[0], dtype=np.float64)
    _check(load().lfmm_phi(d.ctypes.data, d.shape[0], out.ctypes.data), "lfmm_phi")
    return out


def lfmm_model_skeleton(leaf_side: int, p: int, proxies_per_edge: int, level_above_leaf: int) -> np.ndarray:
    xy = np.zeros(2 * 64, dtype=np.int32)
    n = ctypes.c_int32()
    _check(load().lfmm_model_skeleton(leaf_side, p, proxies_per_edge, level_above_leaf, xy.ctypes.data,
                                      ctypes.byref(n)), "lfmm_model_skeleton")
    return xy[: 2 * n.value].reshape(-1, 2).copy()


def lfmm_model_tofs(leaf_side: int, p: int, proxies_per_edge: int) -> np.ndarray:
    P0 = lfmm_model_skeleton(leaf_side, p, proxies_per_edge, 0).shape[0]
    out = np.empty((P0, leaf_side * leaf_side), dtype=np.float64)
    _check(load().lfmm_model_tofs(leaf_side, p, proxies_per_edge, out.ctypes.data), "lfmm_model_tofs")
    return out


def lfmm_model_s(leaf_side: int, p: int, proxies_per_edge: int, level_above_leaf: int) -> np.ndarray:
    Pp = lfmm_model_skeleton(leaf_side, p, proxies_per_edge, level_above_leaf).shape[0]
    Pc = lfmm_model_skeleton(leaf_side, p, proxies_per_edge, level_above_leaf - 1).shape[0]
    out = np.empty((Pp, 4 * Pc), dtype=np.float64)
    _check(load().lfmm_model_s(leaf_side, p, proxies_per_edge, level_above_leaf, out.ctypes.data), "lfmm_model_s")
    return out


PHASES = ("tree", "operators", "p2m", "m2m", "m2l", "p2p", "copy", "m2l_tc", "l2p")


def lfmm_profile_enable(enable: bool) -> None:
    _check(load().lfmm_profile_enable(1 if enable else 0), "lfmm_profile_enable")


def lfmm_profile_read(reset: bool = False) -> dict:
    """{phase: (milliseconds, kernel launches)} accumulated by the library's phase timers."""
    ms = np.zeros(len(PHASES), dtype=np.float64)
    n = np.zeros(len(PHASES), dtype=np.int64)
    _check(load().lfmm_profile_read(ms.ctypes.data, n.ctypes.data, 1 if reset else 0), "lfmm_profile_read")
    return {k: (float(ms[i]), int(n[i])) for i, k in enumerate(PHASES)}


def lfmm_plan_set_wait_budget(plan: int, polls: int) -> None:
    _check(load().lfmm_plan_set_wait_budget(plan, int(polls)), "lfmm_plan_set_wait_budget")


def lfmm_plan_inject_barrier_stall(plan: int) -> None:
    _check(load().lfmm_plan_inject_barrier_stall(plan), "lfmm_plan_inject_barrier_stall")


def lfmm_pool_used_bytes() -> int:
    v = ctypes.c_int64()
    _check(load().lfmm_pool_used_bytes(ctypes.byref(v)), "lfmm_pool_used_bytes")
    return v.value


def lfmm_fault_inject_alloc(nth: int) -> None:
    _check(load().lfmm_fault_inject_alloc(int(nth)), "lfmm_fault_inject_alloc")


def lfmm_launch_count() -> int:
    return int(load().lfmm_launch_count())


def lfmm_phi_quadrature(offsets, weights, R: int, stream=None) -> np.ndarray:
    """phi of the operator sum_k w_k (2u(m) - u(m+d_k) - u(m-d_k)) on |m|_inf <= R by the
    GPU quadrature; returns a (2R+1, 2R+1) array indexed [y + R, x + R]."""
    d = np.ascontiguousarray(np.asarray(offsets, dtype=np.int32).reshape(-1, 2))
    w = np.ascontiguousarray(np.asarray(weights, dtype=np.float64).reshape(-1))
    out = np.empty((2 * R + 1, 2 * R + 1), dtype=np.float64)
    _check(load().lfmm_phi_quadrature(d.ctypes.data, w.ctypes.data, int(d.shape[0]), int(R), out.ctypes.data,
                                      _stream_handle(stream)), "lfmm_phi_quadrature")
    return out


def lfmm_plan_set_flags(handle: int, flags: int) -> None:
    _check(load().lfmm_plan_set_flags(handle, int(flags)), "lfmm_plan_set_flags")


def lfmm_solve(src, tgt, f, u, opts: lfmm_opts | None = None, stream=None) -> None:
    """One-shot solve (plan create + eval + destroy); host f uploads beside the tree build."""
    st = load().lfmm_solve(_ptr(src), int(src.shape[0]), _ptr(tgt), int(tgt.shape[0]), _ptr(f), _ptr(u),
                           ctypes.byref(opts) if opts is not None else None, _stream_handle(stream))
    _check(st, "lfmm_solve")


def autotune(src, tgt, tol: float, src_offsets=None, tgt_offsets=None, base: lfmm_opts | None = None,
             stream=None) -> tuple[lfmm_opts, dict]:
    """lfmm_autotune: (chosen opts, {rel_err, ms, candidates, from_cache}).  With offsets
    (host int64 arrays, as for Forest) the points are a forest of problems."""
    r = lfmm_tune_result()
    so = to = None
    n_prob = 1
    if src_offsets is not None:
        so = np.ascontiguousarray(src_offsets, dtype=np.int64)
        to = np.ascontiguousarray(tgt_offsets, dtype=np.int64)
        n_prob = so.shape[0] - 1
    st = load().lfmm_autotune(_ptr(src), int(src.shape[0]), so.ctypes.data if so is not None else None, _ptr(tgt),
                              int(tgt.shape[0]), to.ctypes.data if to is not None else None, n_prob, float(tol),
                              ctypes.byref(base) if base is not None else None, ctypes.byref(r),
                              _stream_handle(stream))
    _check(st, "lfmm_autotune")
    return r.opts, {"rel_err": r.rel_err, "ms": r.ms, "candidates": int(r.candidates),
                    "from_cache": bool(r.from_cache), "p": int(r.opts.p), "leaf_size": int(r.opts.leaf_size),
                    "tc_min_level": int(r.opts.tc_min_level), "precision": int(r.opts.precision),
                    "m2l_tile": int(r.opts.m2l_tile), "m2l_stages": int(r.opts.m2l_stages),
                    "m2l_split": int(r.opts.m2l_split)}


def tune_cache_clear() -> None:
    _check(load().lfmm_tune_cache_clear(), "lfmm_tune_cache_clear")


def tune_cache_save(path: str) -> None:
    _check(load().lfmm_tune_cache_save(path.encode()), "lfmm_tune_cache_save")


def tune_cache_load(path: str) -> None:
    _check(load().lfmm_tune_cache_load(path.encode()), "lfmm_tune_cache_load")


class Plan:
    """Convenience owner of an lfmm plan: ``Plan(src, tgt, ...).eval(f) -> u``.

    src, tgt: (n, 2) int32 numpy arrays or torch tensors (host or CUDA).
    eval(f): f float64 of length n_src (host or CUDA); returns u in the same kind of
    memory as f (numpy for numpy input, torch CUDA tensor for CUDA input)."""

    def __init__(self, src, tgt, precision: int = LFMM_MIXED, p: int = 8, leaf_size: int = 64,
                 max_leaf_side: int = 32, proxies_per_edge: int = 64, tc_min_level: int = 0,
                 tree: int = LFMM_TREE_AUTO, graph: bool = False, stream=None, opts: lfmm_opts | None = None):
        self.n_src, self.n_tgt = int(src.shape[0]), int(tgt.shape[0])
        self.stream = stream
        if opts is None:
            opts = make_opts(precision, p, leaf_size, max_leaf_side, proxies_per_edge, tc_min_level, tree, graph)
        self.handle = lfmm_plan_create(src, self.n_src, tgt, self.n_tgt, opts, stream)

    def status(self):
        lfmm_plan_status(self.handle, self.stream)

    def set_flags(self, graph: bool = False, serial: bool = False, persistent: bool = False):
        """lfmm_plan_set_flags: graph replay, serial order and (pruned trees, forests) one
        persistent launch per sweep for later evaluations."""
        lfmm_plan_set_flags(self.handle, (LFMM_FLAG_GRAPH if graph else 0) | (LFMM_FLAG_SERIAL if serial else 0) |
                            (LFMM_FLAG_PERSISTENT if persistent else 0))

    def info(self) -> dict:
        return lfmm_plan_get_info(self.handle)

    def eval(self, f, out=None):
        if out is None:
            if isinstance(f, np.ndarray):
                out = np.empty(self.n_tgt, dtype=np.float64)
            else:
                import torch
                out = torch.empty(self.n_tgt, dtype=torch.float64, device=f.device)
        lfmm_eval(self.handle, f, out, self.stream)
        return out

    def eval_multi(self, F, out=None):
        """lfmm_eval_multi: F of shape (k, n_src) -> U of shape (k, n_tgt), same kind of memory."""
        k = int(F.shape[0])
        if out is None:
            if isinstance(F, np.ndarray):
                out = np.empty((k, self.n_tgt), dtype=np.float64)
            else:
                import torch
                out = torch.empty((k, self.n_tgt), dtype=torch.float64, device=F.device)
        _check(load().lfmm_eval_multi(self.handle, _ptr(F), k, _ptr(out), _stream_handle(self.stream)),
               "lfmm_eval_multi")
        return out

    def eval_parts(self, f):
        if isinstance(f, np.ndarray):
            un, uf = np.empty(self.n_tgt), np.empty(self.n_tgt)
        else:
            import torch
            un = torch.empty(self.n_tgt, dtype=torch.float64, device=f.device)
            uf = torch.empty_like(un)
        lfmm_eval_parts(self.handle, f, un, uf, self.stream)
        return un, uf

    def close(self):
        if getattr(self, "handle", None):
            lfmm_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


class Forest(Plan):
    """Many independent problems in one plan: ``Forest(src, src_offsets, tgt, tgt_offsets)``.

    src, tgt: concatenated (n, 2) int32 points of all problems; problem i owns rows
    src_offsets[i]:src_offsets[i+1] (and likewise for targets).  eval(f) takes f of all
    sources and returns u of all targets, concatenated in the same order."""

    def __init__(self, src, src_offsets, tgt, tgt_offsets, precision: int = LFMM_MIXED, p: int = 8,
                 leaf_size: int = 64, max_leaf_side: int = 32, proxies_per_edge: int = 64, tc_min_level: int = 0,
                 graph: bool = False, stream=None, opts: lfmm_opts | None = None):
        self.n_src, self.n_tgt = int(src.shape[0]), int(tgt.shape[0])
        self.stream = stream
        if opts is None:
            opts = make_opts(precision, p, leaf_size, max_leaf_side, proxies_per_edge, tc_min_level,
                             LFMM_TREE_AUTO, graph)
        self.handle = lfmm_forest_create(src, src_offsets, tgt, tgt_offsets, opts, stream)


class Server:
    """Request loop with continuous admission (lfmm_server_* in include/lfmm.h).

    submit(src, tgt, f, tol) queues a solve and returns a ticket; wait(ticket) blocks
    until it is done and returns (u, stats).  The arrays passed to submit are kept
    referenced here until the ticket has been waited for."""

    def __init__(self, n_slots: int = 4, hbm_budget_bytes: int = 0):
        h = ctypes.c_void_p()
        _check(load().lfmm_server_create(ctypes.byref(h), int(n_slots), int(hbm_budget_bytes)),
               "lfmm_server_create")
        self.handle = h.value
        self._live = {}

    def submit(self, src, tgt, f, tol: float, out=None) -> int:
        if out is None:
            if isinstance(f, np.ndarray):
                out = np.empty(int(tgt.shape[0]), dtype=np.float64)
            else:
                import torch
                out = torch.empty(int(tgt.shape[0]), dtype=torch.float64, device=f.device)
        req = lfmm_request(_ptr(src), int(src.shape[0]), _ptr(tgt), int(tgt.shape[0]), _ptr(f), _ptr(out),
                           float(tol))
        t = ctypes.c_int64()
        _check(load().lfmm_server_submit(self.handle, ctypes.byref(req), ctypes.byref(t)), "lfmm_server_submit")
        self._live[t.value] = (src, tgt, f, out)
        return t.value

    def wait(self, ticket: int):
        out, stats = self.wait_stats(ticket)
        _check(stats["status"], "lfmm_server_wait")
        return out, stats

    def wait_stats(self, ticket: int):
        """(u or None, stats) without raising for the request's own failure (a refused,
        shed or cancelled request has stats["status"] != LFMM_OK)."""
        st = lfmm_request_stats()
        status = load().lfmm_server_wait(self.handle, int(ticket), ctypes.byref(st))
        _, _, _, out = self._live.pop(ticket)
        stats = {name: getattr(st, name) for name, _ in lfmm_request_stats._fields_}
        if status != LFMM_OK and stats["status"] == LFMM_OK:
            stats["status"] = status
        return (out if status == LFMM_OK else None), stats

    def set_limits(self, max_pending: int = 0, max_queue_ms: float = 0.0):
        _check(load().lfmm_server_set_limits(self.handle, int(max_pending), float(max_queue_ms)),
               "lfmm_server_set_limits")

    def cancel(self, ticket: int):
        _check(load().lfmm_server_cancel(self.handle, int(ticket)), "lfmm_server_cancel")

    def close(self):
        if getattr(self, "handle", None):
            _check(load().lfmm_server_destroy(self.handle), "lfmm_server_destroy")
            self.handle = None
            self._live.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

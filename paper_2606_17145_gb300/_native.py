"""ctypes declarations of the libog.so C ABI (include/og.h).

Argument marshalling only.  If the library is missing this module raises at
import time: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

from . import build as _build

OG_OK, OG_EINVAL, OG_ENOSPACE, OG_ECUDA, OG_EWALK, OG_ETREE, OG_ENOTIMPL = range(7)
OG_FP32_KAHAN, OG_FP64 = 0, 1


class og_params(C.Structure):
    _fields_ = [("leaf_size", C.c_int32), ("deep_stack", C.c_int32), ("rcut_factor", C.c_double),
                ("node_capacity", C.c_int64), ("max_walk_iters", C.c_int64)]


class og_tree(C.Structure):
    _fields_ = [("n", C.c_int64), ("n_groups", C.c_int64), ("node_capacity", C.c_int64), ("box", C.c_double),
                ("rcut_factor", C.c_double), ("leaf_size", C.c_int32), ("built", C.c_int32),
                ("mem", C.c_void_p), ("mem_bytes", C.c_size_t), ("max_walk_iters", C.c_int64),
                ("deep_stack", C.c_int32), ("reserved1", C.c_int32)]


# symbol -> (restype, argtypes)
SIGNATURES = {
    "og_params_default": (None, [C.POINTER(og_params)]),
    "og_keys_sort_ws_bytes": (C.c_size_t, [C.c_int64]),
    "og_tree_bytes": (C.c_size_t, [C.c_int64, C.POINTER(og_params)]),
    "og_accel_ws_bytes": (C.c_size_t, [C.POINTER(og_tree), C.c_int]),
    "og_adjoint_ws_bytes": (C.c_size_t, [C.POINTER(og_tree), C.c_int]),
    "og_keys_sort": (C.c_int, [C.c_void_p, C.c_int64, C.c_double, C.c_void_p, C.c_void_p, C.c_void_p, C.c_size_t,
                               C.c_void_p]),
    "og_tree_build": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_double, C.c_int64,
                                C.c_double, C.POINTER(og_params), C.c_void_p, C.c_size_t, C.POINTER(og_tree),
                                C.c_void_p]),
    "og_shortrange_accel": (C.c_int, [C.POINTER(og_tree), C.c_double, C.c_double, C.c_int, C.c_void_p, C.c_void_p,
                                      C.c_void_p, C.c_void_p, C.c_size_t, C.c_void_p]),
    "og_shortrange_adjoint": (C.c_int, [C.POINTER(og_tree), C.c_double, C.c_double, C.c_int, C.c_void_p,
                                        C.c_void_p, C.c_void_p, C.c_int, C.c_void_p, C.c_size_t, C.c_void_p]),
    "og_shortrange_accel_range": (C.c_int, [C.POINTER(og_tree), C.c_double, C.c_double, C.c_int, C.c_int64,
                                            C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_size_t,
                                            C.c_void_p]),
    "og_shortrange_adjoint_range": (C.c_int, [C.POINTER(og_tree), C.c_double, C.c_double, C.c_int, C.c_void_p,
                                              C.c_int64, C.c_int64, C.c_void_p, C.c_void_p, C.c_int, C.c_void_p,
                                              C.c_size_t, C.c_void_p]),
    "og_shortrange_accel_adjoint": (C.c_int, [C.POINTER(og_tree), C.c_double, C.c_double, C.c_int, C.c_void_p,
                                              C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                              C.c_void_p, C.c_size_t, C.c_void_p]),
    "og_keys_sort_noalloc": (C.c_int, [C.c_void_p, C.c_int64, C.c_double, C.c_void_p, C.c_void_p, C.c_void_p]),
    "og_poll_status": (C.c_int, [C.c_void_p, C.c_void_p]),
    "og_tree_node_count": (C.c_int64, [C.POINTER(og_tree), C.c_void_p]),
    "og_tree_copy_nodes": (C.c_int, [C.POINTER(og_tree)] + [C.c_void_p] * 9 + [C.c_void_p]),
    "og_status_str": (C.c_char_p, [C.c_int]),
    "og_pm_plan_create": (C.c_int, [C.c_int32, C.POINTER(C.c_void_p)]),
    "og_pm_plan_destroy": (None, [C.c_void_p]),
    "og_pm_ws_bytes": (C.c_size_t, [C.c_void_p]),
    "og_pm_accel": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64, C.c_double, C.c_double, C.c_void_p,
                              C.c_size_t, C.c_void_p, C.c_void_p]),
    "og_kick": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64, C.c_double, C.c_void_p]),
    "og_drift": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_double, C.c_void_p]),
    "og_sph_ws_bytes": (C.c_size_t, []),
    "og_probe_pipe": (C.c_int, [C.c_int32, C.c_int32, C.c_void_p, C.POINTER(C.c_uint64), C.c_void_p]),
    "og_sph_density": (C.c_int, [C.POINTER(og_tree), C.c_double, C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p,
                                 C.c_void_p, C.c_void_p]),
}


def header_symbols() -> list[str]:
    """Function names declared in include/og.h."""
    import re
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "..", "include", "og.h")
    text = open(path).read()
    return sorted(set(re.findall(r"^\s*(?:[\w\s\*]+?)\b(og_\w+)\s*\(", text, flags=re.M)))


def load(path: str | None = None) -> C.CDLL:
    path = path or _build.LIB
    if not os.path.exists(path):
        raise ImportError(f"libog.so not found at {path}; build it with paper_2606_17145_gb300.build.build() "
                          "(the library has no CPU fallback)")
    lib = C.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib

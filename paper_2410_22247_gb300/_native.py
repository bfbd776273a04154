"""ctypes binding of ``libaaqaoa.so`` (include/aaqaoa.h).

Only argument marshalling lives here: every step of the computation runs in
the CUDA library. The functions keep the C names. A missing or unloadable
library raises immediately; there is no fallback path.
"""
from __future__ import annotations

import ctypes
import os

from . import build as _build

_lib = None

AAQAOA_C64 = 0
AAQAOA_C128 = 1
AAQAOA_OBS_FULL = 0
AAQAOA_OBS_RED = 1
AAQAOA_AGG_FUSED = 0
AAQAOA_AGG_PERTERM = 1
AAQAOA_AGG_SINGLEPASS = 2
AAQAOA_AGG_PERORBIT = AAQAOA_AGG_SINGLEPASS
AAQAOA_FAULT_DROP_TILE = 1
AAQAOA_OK = 0
ERRORS = {
    -1: "AAQAOA_ERR_INVALID_ARG", -2: "AAQAOA_ERR_BAD_ORBITS", -3: "AAQAOA_ERR_WORKSPACE",
    -4: "AAQAOA_ERR_CUDA", -5: "AAQAOA_ERR_TIMEOUT", -6: "AAQAOA_ERR_UNSUPPORTED",
}

class Stats(ctypes.Structure):
    """aaqaoa_stats_t"""
    _fields_ = [("launches", ctypes.c_int * 5), ("ms", ctypes.c_double * 5), ("bytes", ctypes.c_double * 5)]


class GraphDesc(ctypes.Structure):
    """aaqaoa_graph_desc"""
    _fields_ = [("n", ctypes.c_int), ("num_edges", ctypes.c_int), ("edges", ctypes.POINTER(ctypes.c_int32)),
                ("num_orbits", ctypes.c_int), ("orbit_rep", ctypes.POINTER(ctypes.c_int32)),
                ("orbit_weight", ctypes.POINTER(ctypes.c_int32)), ("edge_orbit", ctypes.POINTER(ctypes.c_int32))]


# (name, restype, argtypes)
_i32p = ctypes.POINTER(ctypes.c_int32)
_f64p = ctypes.POINTER(ctypes.c_double)
_vp = ctypes.c_void_p
_PROTOS = [
    ("aaqaoa_prepare", ctypes.c_int, [ctypes.c_int, ctypes.c_int, _i32p, ctypes.c_int, _i32p, _i32p, _i32p,
                                      ctypes.c_int, ctypes.c_uint, _vp, ctypes.POINTER(_vp)]),
    ("aaqaoa_prepare_weighted", ctypes.c_int, [ctypes.c_int, ctypes.c_int, _i32p, _i32p, ctypes.c_int, _i32p, _i32p,
                                               _i32p, ctypes.c_int, ctypes.c_uint, _vp, ctypes.POINTER(_vp)]),
    ("aaqaoa_prepare_ising", ctypes.c_int, [ctypes.c_int, ctypes.c_int, _i32p, _f64p, _f64p, ctypes.c_int, _i32p,
                                            _i32p, _i32p, ctypes.c_int, _i32p, _i32p, _i32p, ctypes.c_int,
                                            ctypes.c_uint, _vp, ctypes.POINTER(_vp)]),
    ("aaqaoa_workspace_bytes", ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_size_t)]),
    ("aaqaoa_set_workspace", ctypes.c_int, [_vp, _vp, ctypes.c_size_t, ctypes.c_int, ctypes.c_int]),
    ("aaqaoa_set_stream", ctypes.c_int, [_vp, _vp]),
    ("aaqaoa_expect", ctypes.c_int, [_vp, _f64p, _f64p, ctypes.c_int, ctypes.c_int, _f64p]),
    ("aaqaoa_grad", ctypes.c_int, [_vp, _f64p, _f64p, ctypes.c_int, _f64p, _f64p, _f64p]),
    ("aaqaoa_expect_batch", ctypes.c_int, [_vp, ctypes.c_int, _f64p, _f64p, ctypes.c_int, _f64p]),
    ("aaqaoa_expect_device", ctypes.c_int, [_vp, ctypes.c_int, _vp, _vp, ctypes.c_int, _vp]),
    ("aaqaoa_grad_device", ctypes.c_int, [_vp, _vp, _vp, ctypes.c_int, _vp]),
    ("aaqaoa_grad_batch", ctypes.c_int, [_vp, ctypes.c_int, _f64p, _f64p, ctypes.c_int, _f64p, _f64p, _f64p]),
    ("aaqaoa_grad_batch_device", ctypes.c_int, [_vp, ctypes.c_int, _vp, _vp, ctypes.c_int, _vp]),
    ("aaqaoa_sync", ctypes.c_int, [_vp]),
    ("aaqaoa_edge_zz", ctypes.c_int, [_vp, _f64p, _f64p, _f64p]),
    ("aaqaoa_verify_orbits", ctypes.c_int, [_vp, _f64p, _f64p, ctypes.c_double, ctypes.POINTER(ctypes.c_int)]),
    ("aaqaoa_max_cut", ctypes.c_int, [_vp, _i32p, ctypes.POINTER(ctypes.c_uint64)]),
    ("aaqaoa_sample", ctypes.c_int, [_vp, _f64p, _f64p, ctypes.c_int, _f64p, ctypes.POINTER(ctypes.c_uint64), _i32p]),
    ("aaqaoa_statevector", ctypes.c_int, [_vp, _f64p, _f64p, _vp]),
    ("aaqaoa_aggregate_only", ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_int, _f64p]),
    ("aaqaoa_expect_static", ctypes.c_int, [_vp, _f64p, _f64p, ctypes.c_int, _f64p]),
    ("aaqaoa_prepare_multi", ctypes.c_int, [ctypes.c_int, ctypes.POINTER(GraphDesc), ctypes.c_int, ctypes.c_uint,
                                            _vp, ctypes.POINTER(_vp)]),
    ("aaqaoa_multi_workspace_bytes", ctypes.c_int, [_vp, ctypes.POINTER(ctypes.c_size_t)]),
    ("aaqaoa_multi_set_workspace", ctypes.c_int, [_vp, _vp, ctypes.c_size_t]),
    ("aaqaoa_expect_multi", ctypes.c_int, [_vp, _f64p, _f64p, ctypes.c_int, _f64p]),
    ("aaqaoa_multi_info", ctypes.c_int, [_vp, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                         ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]),
    ("aaqaoa_destroy_multi", None, [_vp]),
    ("aaqaoa_inject_fault", ctypes.c_int, [_vp, ctypes.c_int]),
    ("aaqaoa_ising_orbits", ctypes.c_int, [ctypes.c_int, ctypes.c_int, _i32p, _f64p, _f64p, _i32p, _i32p, _i32p,
                                           _i32p, _i32p, _i32p, _i32p, _i32p]),
    ("aaqaoa_edge_orbits", ctypes.c_int, [ctypes.c_int, ctypes.c_int, _i32p, _i32p, _i32p, _i32p, _i32p, _i32p]),
    ("aaqaoa_get_pass_plan", ctypes.c_int, [_vp, _i32p]),
    ("aaqaoa_set_pass_plan", ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int]),
    ("aaqaoa_autotune", ctypes.c_int, [_vp, _i32p]),
    ("aaqaoa_set_layer_fusion", ctypes.c_int, [_vp, ctypes.c_int]),
    ("aaqaoa_get_layer_fusion", ctypes.c_int, [_vp, ctypes.POINTER(ctypes.c_int)]),
    ("aaqaoa_get_schedule", ctypes.c_int, [_vp, ctypes.c_int, _i32p, ctypes.c_int, ctypes.POINTER(ctypes.c_int)]),
    ("aaqaoa_plan_info", ctypes.c_int, [_vp, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                        ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                        ctypes.POINTER(ctypes.c_uint)]),
    ("aaqaoa_launch_count", ctypes.c_int, [_vp, ctypes.POINTER(ctypes.c_int)]),
    ("aaqaoa_profile_enable", ctypes.c_int, [_vp, ctypes.c_int]),
    ("aaqaoa_profile_read", ctypes.c_int, [_vp, ctypes.c_int, _f64p, ctypes.POINTER(ctypes.c_int), _f64p]),
    ("aaqaoa_stats", ctypes.c_int, [_vp, ctypes.POINTER(Stats)]),
    ("aaqaoa_profile_launches", ctypes.c_int, [_vp, ctypes.c_int, ctypes.POINTER(ctypes.c_int), _i32p, _i32p, _f64p,
                                               _f64p]),
    ("aaqaoa_destroy", None, [_vp]),
    ("aaqaoa_strerror", ctypes.c_char_p, [ctypes.c_int]),
    ("aaqaoa_last_error_detail", ctypes.c_char_p, []),
]
EXPORTED = [p[0] for p in _PROTOS]


class AAQAOAError(RuntimeError):
    def __init__(self, code: int, where: str, detail: str):
        self.code = code
        super().__init__(f"{where}: {ERRORS.get(code, code)}: {detail}")


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load (building first if needed) and bind the CUDA library."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if build_if_missing and (not os.path.exists(path) or _build._stale()):
        _build.build()
    if not os.path.exists(path):
        raise ImportError(f"CUDA library {path} is missing; run paper_2410_22247_gb300.build.build()")
    lib = ctypes.CDLL(path)
    for name, res, args in _PROTOS:
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def check(code: int, where: str) -> None:
    if code != AAQAOA_OK:
        detail = load().aaqaoa_last_error_detail().decode(errors="replace")
        raise AAQAOAError(code, where, detail)


def _call(name):
    def f(*args):
        return getattr(load(), name)(*args)
    f.__name__ = name
    return f


for _name in EXPORTED:
    globals()[_name] = _call(_name)

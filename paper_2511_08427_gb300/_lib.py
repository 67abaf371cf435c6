"""ctypes binding of libpyronn.so (argument marshalling only; every operator runs in the CUDA library).

There is no fallback: if the library has not been built, importing the operators raises.
"""
from __future__ import annotations

import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libpyronn.so")

F32, BF16, F16 = 0, 1, 2
BP_PLAIN, BP_INV_W2 = 0, 1

STATUS = {0: "OK", -1: "INVALID_ARG", -2: "UNSUPPORTED_DTYPE", -3: "MISALIGNED", -4: "CUDA_ERROR", -5: "OOM",
          -6: "SINGULAR", -7: "DEVICE_CHECK_FAILED"}


class PyronnError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"pyronn {STATUS.get(code, code)}: {msg}")
        self.code = code


class VolDesc(ctypes.Structure):
    _fields_ = [("ndim", ctypes.c_int), ("shape", ctypes.c_int * 3), ("spacing", ctypes.c_double * 3),
                ("offset", ctypes.c_double * 3)]


class DetDesc(ctypes.Structure):
    _fields_ = [("shape", ctypes.c_int * 2), ("spacing", ctypes.c_double * 2), ("offset", ctypes.c_double * 2)]


_lib = None

# (name, restype, argtypes)
_c_int, _c_double, _vp, _dp = ctypes.c_int, ctypes.c_double, ctypes.c_void_p, ctypes.POINTER(ctypes.c_double)
_geomp = ctypes.POINTER(ctypes.c_void_p)
SIGNATURES = [
    ("pyronn_geom_create_parallel2d", _c_int, [ctypes.POINTER(VolDesc), ctypes.POINTER(DetDesc), _c_int, _c_double, _geomp]),
    ("pyronn_geom_create_fan2d", _c_int, [ctypes.POINTER(VolDesc), ctypes.POINTER(DetDesc), _c_int, _c_double, _c_double,
                                          _c_double, _geomp]),
    ("pyronn_geom_create_cone_circular", _c_int, [ctypes.POINTER(VolDesc), ctypes.POINTER(DetDesc), _c_int, _c_double,
                                                  _c_double, _c_double, _c_double, _geomp]),
    ("pyronn_geom_create_from_positions", _c_int, [ctypes.POINTER(VolDesc), ctypes.POINTER(DetDesc), _c_int, _dp, _dp,
                                                   _dp, _dp, _geomp]),
    ("pyronn_geom_create_cone_matrices", _c_int, [ctypes.POINTER(VolDesc), ctypes.POINTER(DetDesc), _c_int, _dp, _geomp]),
    ("pyronn_geom_create_matrices2d", _c_int, [ctypes.POINTER(VolDesc), ctypes.POINTER(DetDesc), _c_int, _dp, _geomp]),
    ("pyronn_geom_destroy", _c_int, [_vp]),
    ("pyronn_geom_set_step", _c_int, [_vp, _c_double]),
    ("pyronn_geom_get_step", _c_int, [_vp, _dp]),
    ("pyronn_geom_info", _c_int, [_vp, ctypes.POINTER(_c_int), ctypes.POINTER(_c_int), ctypes.POINTER(_c_int)]),
    ("pyronn_geom_get_views", _c_int, [_vp, _dp]),
    ("pyronn_geom_count_samples", _c_int, [_vp, ctypes.POINTER(ctypes.c_int64)]),
    ("pyronn_geom_set_variant", _c_int, [_vp, _c_int, _c_int]),
    ("pyronn_autotune", _c_int, [_vp, _c_int, _vp, _vp, _c_int, _c_int, _vp, _dp]),
    ("pyronn_geom_set_tuning", _c_int, [_vp, _c_int, _c_int]),
    ("pyronn_fp", _c_int, [_vp, _vp, _vp, _c_int, _c_int, _vp]),
    ("pyronn_adjoint", _c_int, [_vp, _vp, _vp, _c_int, _c_int, _vp]),
    ("pyronn_adjoint_update", _c_int, [_vp, _vp, _vp, ctypes.c_double, _vp, _c_int, _c_int, _vp]),
    ("pyronn_fbp_filter", _c_int, [_vp, _vp, _vp, _c_int, _c_int, _c_int, _vp]),
    ("pyronn_sim_detector_jitter", _c_int, [_vp, _vp, _vp, _vp, _c_int, _c_int, _c_int, _vp]),
    ("pyronn_sim_gaussian_noise", _c_int, [_vp, _vp, _vp, _vp, ctypes.c_double, ctypes.c_double, _c_int, _c_int, _vp]),
    ("pyronn_sim_ring", _c_int, [_vp, _vp, _vp, _vp, _vp, _c_int, _c_int, _c_int, _c_int, _c_int, _vp]),
    ("pyronn_sim_motion_blur", _c_int, [_vp, _vp, _vp, _vp, _c_int, _c_int, _c_int, _vp]),
    ("pyronn_bp", _c_int, [_vp, _vp, _vp, _c_int, _c_int, _c_int, _vp]),
    ("pyronn_bp_transpose", _c_int, [_vp, _vp, _vp, _c_int, _c_int, _c_int, _vp]),
    ("pyronn_adjoint_noalloc", _c_int, [_vp, _vp, _vp, _c_int, _c_int, _vp]),
    ("pyronn_plan_create", _c_int, [_c_int, ctypes.POINTER(ctypes.c_void_p), _c_int, _geomp]),
    ("pyronn_plan_destroy", _c_int, [_vp]),
    ("pyronn_plan_info", _c_int, [_vp, ctypes.POINTER(_c_int), ctypes.POINTER(ctypes.c_int64),
                                  ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(_c_int)]),
    ("pyronn_plan_fp", _c_int, [_vp, ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(ctypes.c_void_p), _vp]),
    ("pyronn_plan_adjoint", _c_int, [_vp, ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(ctypes.c_void_p), _vp]),
    ("pyronn_plan_bp", _c_int, [_vp, ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(ctypes.c_void_p), _c_int, _vp]),
    ("pyronn_fp_host", _c_int, [_vp, _vp, _vp, _c_int, _c_int, _vp]),
    ("pyronn_adjoint_host", _c_int, [_vp, _vp, _vp, _c_int, _c_int, _vp]),
    ("pyronn_geom_read_flags", _c_int, [_vp, ctypes.POINTER(_c_int), _c_int]),
    ("pyronn_geom_fp_config", _c_int, [_vp, _c_int, ctypes.POINTER(_c_int)]),
    ("pyronn_geom_adjoint_config", _c_int, [_vp, ctypes.POINTER(_c_int)]),
    ("pyronn_geom_bp_config", _c_int, [_vp, _c_int, ctypes.POINTER(_c_int)]),
    ("pyronn_last_error", ctypes.c_char_p, []),
    ("pyronn_version", _c_int, []),
]


def lib():
    """Load libpyronn.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: build it with `python -c 'import __graft_entry__ as g; "
                              f"g.build()'` (or python paper_2511_08427_gb300/build.py)")
        L = ctypes.CDLL(LIB_PATH)
        for name, res, args in SIGNATURES:
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def check(rc: int) -> None:
    if rc != 0:
        msg = lib().pyronn_last_error()
        raise PyronnError(rc, msg.decode() if msg else "")


def exported_symbols():
    return [name for name, _, _ in SIGNATURES]

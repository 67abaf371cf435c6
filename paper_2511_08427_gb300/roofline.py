"""Measured on-chip peaks: the denominators of the roofline fractions of the projector kernels.

None of the operators is a dense contraction or HBM-bound at the benchmark sizes; their binding units
are on the SM: shared-memory loads (forward projector), shared-memory int32 reductions (matched
adjoint), L1-hit global loads (voxel-driven back-projector), the FP32 pipe, and for the hardware-
filtered texture projector the texture unit's trilinear fetch. ``measure()`` runs the probes of
roofline_peaks.cu on the current device and returns their rates per SM clock cycle (counted on the SM
with clock64, so they do not depend on the clock the GPU happens to run at) and the clock it saw.
``peak(rates, key, mhz)`` turns one rate into a whole-GPU peak per second at a given SM clock.
"""
from __future__ import annotations

import ctypes

from . import build as _build

KEYS = ("red_shared_s32", "red_shared_f32", "ld_shared_b32", "ffma", "ld_global_l1_b32", "tex_fetch", "tex3d_trilinear")

_lib = None


def _load():
    global _lib
    if _lib is None:
        path = _build.build_roofline()
        lib = ctypes.CDLL(path)
        lib.pyronn_roofline_measure.restype = ctypes.c_int
        lib.pyronn_roofline_measure.argtypes = [ctypes.POINTER(ctypes.c_double), ctypes.c_int]
        _lib = lib
    return _lib


def measure() -> dict:
    """Rates per SM clock cycle on the current CUDA device (lanes, i.e. thread-level operations), plus
    'sms' and 'sm_mhz' (the clock during the probes). Raises RuntimeError on a CUDA error."""
    out = (ctypes.c_double * 10)()
    rc = _load().pyronn_roofline_measure(out, 10)
    if rc != 0:
        raise RuntimeError(f"roofline probes failed with CUDA error {rc}")
    res = {"sms": int(out[0]), "sm_mhz": float(out[1])}
    for i, k in enumerate(KEYS):
        res[k + "_per_clk_sm"] = float(out[2 + i])
    return res


def peak(rates: dict, key: str, mhz: float) -> float:
    """Whole-GPU rate in operations per second of unit ``key`` at SM clock ``mhz``."""
    return rates[key + "_per_clk_sm"] * rates["sms"] * mhz * 1e6

"""Front end of the library's autotuner (pyronn_autotune): tile and brick shapes chosen by measurement.

``tune(g, op)`` lets the library time every candidate configuration of one operator of a geometry
(forward projection: slab depth x buffers of the TMA-staged projector; matched adjoint: slab depth x
row pitch of the slab-ordered adjoint; back-projection: brick depth of the L1-path bricks, or the bricks
with staged detector shadows) with CUDA events on the current
stream and apply the fastest. The choice is cached in a JSON file keyed by the device name, the
operator and a signature of the geometry (shapes, spacings, views, step, element type), so a later
process re-applies it through pyronn_geom_set_tuning without timing. Every candidate computes the same
operator.
"""
from __future__ import annotations

import ctypes
import hashlib
import json
import os

import numpy as np
import torch

from . import _lib
from .operators import (_DTYPES, TUNE_ADJ_DEPTH, TUNE_ADJ_PITCH, TUNE_BP_BRICK_Z, TUNE_FP_BUFFERS,
                        TUNE_FP_DEPTH)

OPS = {"fp": 0, "adjoint": 1, "bp": 2}
# the two settings each operator's result sets (the back-projector's second one is its kernel variant)
_KNOBS = {0: (TUNE_FP_DEPTH, TUNE_FP_BUFFERS), 1: (TUNE_ADJ_DEPTH, TUNE_ADJ_PITCH), 2: (TUNE_BP_BRICK_Z, "variant")}


def _cache_path() -> str:
    return os.environ.get("PYRONN_TUNE_CACHE", os.path.join(os.path.expanduser("~"), ".cache", "pyronn_tune.json"))


def signature(g, dtype) -> str:
    views = g.views()
    h = hashlib.sha1(np.ascontiguousarray(views).tobytes()).hexdigest()[:16]
    return json.dumps([g.volume_shape, g.volume_spacing, g.detector_shape, g.detector_spacing, g.n_views,
                       round(g.step, 9), str(dtype), h])


def _load():
    try:
        with open(_cache_path()) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _store(db):
    path = _cache_path()
    try:
        os.makedirs(os.path.dirname(path), exist_ok=True)
        tmp = path + ".tmp"
        with open(tmp, "w") as f:
            json.dump(db, f, indent=1)
        os.replace(tmp, path)
    except OSError:
        pass


def apply(g, op: int, a: int, b: int) -> None:
    k1, k2 = _KNOBS[op]
    g.set_tuning(k1, int(a))
    if k2 == "variant":
        g.set_variant(2, int(b))
    else:
        g.set_tuning(k2, int(b))


def tune(g, op: str = "fp", dtype=torch.float32, repeats: int = 2, use_cache: bool = True, device=None) -> dict:
    """Tune one operator ('fp', 'adjoint' or 'bp') of geometry g and apply the choice.

    Returns {"op", "params": [a, b], "ms", "candidates", "cached"}. The timing buffers are allocated here
    (torch) and freed on return; the library allocates nothing for the tuning itself."""
    o = OPS[op]
    device = torch.device(device or "cuda")
    key = "|".join([torch.cuda.get_device_name(device), op, signature(g, dtype)])
    db = _load() if use_cache else {}
    if use_cache and key in db:
        best = db[key]
        apply(g, o, *best["params"])
        return dict(best, cached=True)
    vol = torch.zeros(g.volume_shape, dtype=dtype, device=device)
    sino = torch.zeros(g.sinogram_shape, dtype=dtype, device=device)
    if o == 0:
        vol.uniform_(0.0, 1.0)
        src, dst = vol, sino
    else:
        sino.normal_()
        src, dst = sino, vol
    res = (ctypes.c_double * 4)()
    stream = torch.cuda.current_stream(device).cuda_stream
    _lib.check(_lib.lib().pyronn_autotune(g.handle, o, ctypes.c_void_p(src.data_ptr()), ctypes.c_void_p(dst.data_ptr()),
                                          _DTYPES[dtype], int(repeats), ctypes.c_void_p(stream), res))
    best = {"op": op, "params": [int(res[1]), int(res[2])], "ms": float(res[0]), "candidates": int(res[3])}
    if use_cache:
        db[key] = best
        _store(db)
    return dict(best, cached=False)


def tune_forward(g, dtype=torch.float32, repeats: int = 2, use_cache: bool = True, device=None) -> dict:
    """Forward projector only (slab depth and buffer count); {"depth", "buffers", "ms", "cached"}."""
    r = tune(g, "fp", dtype, repeats, use_cache, device)
    return {"depth": r["params"][0], "buffers": r["params"][1], "ms": r["ms"], "cached": r["cached"]}

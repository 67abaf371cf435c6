"""Autotuner for the kernel knobs of a geometry (slab depth and buffer count of the TMA-staged
forward projector).

Every candidate computes the same operator; the tuner times each with CUDA events on the current
stream (after a warm-up launch) and keeps the fastest. Results are cached in a JSON file keyed by
the device name and a signature of the geometry (shapes, spacings, views, step, element type), so
a later process re-applies the choice without timing.
"""
from __future__ import annotations

import hashlib
import json
import os

import numpy as np
import torch

from ._lib import PyronnError
from .operators import TUNE_FP_BUFFERS as FP_BUFFERS, TUNE_FP_DEPTH as FP_DEPTH

DEFAULT_CANDIDATES = [(8, 2), (8, 1), (4, 2), (4, 1), (12, 1), (16, 1)]


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


def apply(g, depth: int, nbuf: int) -> None:
    g.set_tuning(FP_DEPTH, int(depth))
    g.set_tuning(FP_BUFFERS, int(nbuf))


def tune_forward(g, dtype=torch.float32, candidates=None, repeats: int = 3, use_cache: bool = True,
                 device=None) -> dict:
    """Time the forward projector for each (depth, buffers) candidate and apply the fastest.

    Returns {"depth", "buffers", "ms", "timings": {...}, "cached": bool}.
    """
    from . import operators as ops
    device = torch.device(device or "cuda")
    key = torch.cuda.get_device_name(device) + "|" + signature(g, dtype)
    db = _load() if use_cache else {}
    if use_cache and key in db:
        best = db[key]
        apply(g, best["depth"], best["buffers"])
        return dict(best, cached=True)
    vol = torch.zeros(g.volume_shape, dtype=dtype, device=device)
    sino = torch.empty(g.sinogram_shape, dtype=dtype, device=device)
    stream = torch.cuda.current_stream(device)
    timings = {}
    for depth, nbuf in (candidates or DEFAULT_CANDIDATES):
        try:
            apply(g, depth, nbuf)
            if g.fp_config(dtype)["kernel"] != 3:
                continue
            ops.forward_project(vol, g, out=sino)
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
            ev[0].record(stream)
            for _ in range(repeats):
                ops.forward_project(vol, g, out=sino)
            ev[1].record(stream)
            torch.cuda.synchronize(device)
            timings[f"{depth}x{nbuf}"] = ev[0].elapsed_time(ev[1]) / repeats
        except PyronnError:
            continue
    if not timings:
        apply(g, 0, 0)
        return {"depth": 0, "buffers": 0, "ms": None, "timings": {}, "cached": False}
    best_key = min(timings, key=timings.get)
    depth, nbuf = (int(x) for x in best_key.split("x"))
    apply(g, depth, nbuf)
    best = {"depth": depth, "buffers": nbuf, "ms": timings[best_key], "timings": timings}
    if use_cache:
        db[key] = best
        _store(db)
    return dict(best, cached=False)

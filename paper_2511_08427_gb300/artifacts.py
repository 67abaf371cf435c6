"""Acquisition-artifact simulation on sinograms (Sec. 2.4): detector jitter, Gaussian noise, ring
artifacts and gantry motion blur, each one CUDA kernel of libpyronn.so (pyronn_sim_*). Random
quantities are arguments (see `inputs` for seeded recipes); Poisson noise is `inputs.poisson_log_sinogram`
and `inputs.poisson_log_sinogram_torch`.
"""
from __future__ import annotations

import torch

from ._lib import check, lib
from .operators import Geometry, _batch, _check, _check_like, _sino_dims, _stream_ptr


def _prep(sino: torch.Tensor, g: Geometry):
    dt = _check(sino, "sinogram")
    sino = sino.contiguous()
    lead, nb = _batch(sino, _sino_dims(g), "sinogram")
    return sino, dt, nb


def _dev_array(x, dtype, device):
    t = torch.as_tensor(x, dtype=dtype, device=device).contiguous()
    return t


def detector_jitter(sino: torch.Tensor, g: Geometry, shifts, axis: int = 0) -> torch.Tensor:
    """Every detector row (axis 0) or column (axis 1) shifted by its integer shift (zero fill); shifts
    shaped [batch, V, Nv] (axis 0) or [batch, V, Nu] (axis 1) (batch dimension optional)."""
    sino, dt, nb = _prep(sino, g)
    sh = _dev_array(shifts, torch.int32, sino.device)
    want = nb * g.n_views * (g.detector_shape[0] if (axis == 0 and g.ndim == 3) else
                             (1 if axis == 0 else g.detector_shape[-1]))
    if sh.numel() != want:
        raise ValueError(f"expected {want} shifts, got {sh.numel()}")
    out = torch.empty_like(sino)
    with torch.cuda.device(sino.device):
        check(lib().pyronn_sim_detector_jitter(g.handle, sino.data_ptr(), out.data_ptr(), sh.data_ptr(), int(axis), dt,
                                               nb, _stream_ptr(sino.device)))
    return out


def gaussian_noise(sino: torch.Tensor, g: Geometry, noise: torch.Tensor, mean: float = 0.0, std: float = 1.0,
                   out: torch.Tensor | None = None) -> torch.Tensor:
    """sino + mean + std * noise (noise: standard-normal samples shaped like sino)."""
    sino, dt, nb = _prep(sino, g)
    nz = _dev_array(noise, torch.float32, sino.device)
    if nz.numel() != sino.numel():
        raise ValueError("noise must have one sample per sinogram element")
    if out is None:
        out = torch.empty_like(sino)
    _check_like(out, sino.shape, sino.dtype, sino.device, "out")
    with torch.cuda.device(sino.device):
        check(lib().pyronn_sim_gaussian_noise(g.handle, sino.data_ptr(), out.data_ptr(), nz.data_ptr(), float(mean),
                                              float(std), dt, nb, _stream_ptr(sino.device)))
    return out


def ring_artifacts(sino: torch.Tensor, g: Geometry, columns, gains, view_begin: int = 0, view_end: int | None = None,
                   out: torch.Tensor | None = None) -> torch.Tensor:
    """Detector columns `columns` scaled by `gains` (0: dead element) over views [view_begin, view_end)."""
    sino, dt, nb = _prep(sino, g)
    cols = _dev_array(columns, torch.int32, sino.device)
    gs = _dev_array(gains, torch.float32, sino.device)
    if cols.numel() != gs.numel():
        raise ValueError("one gain per column")
    if out is None:
        out = torch.empty_like(sino)
    _check_like(out, sino.shape, sino.dtype, sino.device, "out")
    ve = g.n_views if view_end is None else int(view_end)
    with torch.cuda.device(sino.device):
        check(lib().pyronn_sim_ring(g.handle, sino.data_ptr(), out.data_ptr(), cols.data_ptr(), gs.data_ptr(),
                                    cols.numel(), int(view_begin), ve, dt, nb, _stream_ptr(sino.device)))
    return out


def motion_blur(sino: torch.Tensor, g: Geometry, angles, length: int) -> torch.Tensor:
    """Each projection blurred by a `length`-sample line kernel rotated to its view angle (radians)."""
    sino, dt, nb = _prep(sino, g)
    ang = _dev_array(angles, torch.float32, sino.device)
    if ang.numel() != g.n_views:
        raise ValueError("one angle per view")
    out = torch.empty_like(sino)
    with torch.cuda.device(sino.device):
        check(lib().pyronn_sim_motion_blur(g.handle, sino.data_ptr(), out.data_ptr(), ang.data_ptr(), int(length), dt,
                                           nb, _stream_ptr(sino.device)))
    return out

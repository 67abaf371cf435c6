"""PyTorch front end of libpyronn.so: geometries, operators, autograd functions and layers.

PyTorch supplies device memory and the current CUDA stream; every operator runs in the CUDA
library through the C ABI (pyronn_fp / pyronn_adjoint / pyronn_bp / pyronn_bp_transpose).

Layer names follow Listing 1 of the paper (ConeProjectionFor3D, ConeBackProjectionFor3D, and the
2D parallel / fan analogues of Sec. 2.1). Gradients (Sec. 2.1: "analytical gradients for all
operators"): the projector's backward is the matched adjoint A^T (exact transpose of the sampled
projector); the voxel-driven back-projector's backward is its own exact transpose.
"""
from __future__ import annotations

import ctypes
import math
from typing import Sequence

import numpy as np
import torch

from . import _lib
from ._lib import BF16, BP_INV_W2, BP_PLAIN, F16, F32, DetDesc, VolDesc, check, lib

_DTYPES = {torch.float32: F32, torch.bfloat16: BF16, torch.float16: F16}

# tuning parameters of Geometry.set_tuning (pyronn_tuning_param)
(TUNE_FP_DEPTH, TUNE_FP_BUFFERS, TUNE_ADJ_ACCUM, TUNE_FP_CTAS_PER_SM, TUNE_FP_TRANSPOSE, TUNE_ADJ_PITCH, TUNE_ADJ_DEPTH,
 TUNE_BP_BRICK_Z, TUNE_ADJ_LANES, TUNE_FP_PACKED) = 0, 1, 2, 3, 4, 5, 6, 7, 8, 9


def _dp(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


class Geometry:
    """A projection geometry (owns a pyronn_geom handle).

    Volume arrays are [Nz, Ny, Nx] (2D: [Ny, Nx]); sinograms are [V, Nv, Nu] (2D: [V, Nu]); leading
    dimensions are a batch. Spacings and offsets follow the same (z, y, x) / (v, u) order.
    """

    def __init__(self, handle, ndim: int, volume_shape, volume_spacing, detector_shape, detector_spacing,
                 n_views: int, kind: int):
        self._h = handle
        self.ndim = ndim
        self.volume_shape = tuple(int(x) for x in volume_shape)
        self.volume_spacing = tuple(float(x) for x in volume_spacing)
        self.detector_shape = tuple(int(x) for x in detector_shape)
        self.detector_spacing = tuple(float(x) for x in detector_spacing)
        self.n_views = int(n_views)
        self.kind = kind

    # -- construction ------------------------------------------------------------------------
    @staticmethod
    def _descs(ndim, volume_shape, volume_spacing, volume_offset, detector_shape, detector_spacing,
               detector_offset):
        vd = VolDesc()
        dd = DetDesc()
        vd.ndim = ndim
        if ndim == 2:
            vs = (1,) + tuple(volume_shape)
            sp = (1.0,) + tuple(volume_spacing)
            of = (0.0,) + tuple(volume_offset or (0.0, 0.0))
            ds = (1, int(_as_seq(detector_shape)[-1]))
            dsp = (1.0, float(_as_seq(detector_spacing)[-1]))
            dof = (0.0, float(_as_seq(detector_offset if detector_offset is not None else 0.0)[-1]))
        else:
            vs, sp, of = tuple(volume_shape), tuple(volume_spacing), tuple(volume_offset or (0.0, 0.0, 0.0))
            ds, dsp, dof = tuple(detector_shape), tuple(detector_spacing), tuple(detector_offset or (0.0, 0.0))
        for i in range(3):
            vd.shape[i] = int(vs[i]); vd.spacing[i] = float(sp[i]); vd.offset[i] = float(of[i])
        for i in range(2):
            dd.shape[i] = int(ds[i]); dd.spacing[i] = float(dsp[i]); dd.offset[i] = float(dof[i])
        return vd, dd, vs, sp, ds, dsp

    @classmethod
    def _make(cls, fn, ndim, volume_shape, volume_spacing, volume_offset, detector_shape, detector_spacing,
              detector_offset, n_views, *args):
        vd, dd, vs, sp, ds, dsp = cls._descs(ndim, volume_shape, volume_spacing, volume_offset, detector_shape,
                                            detector_spacing, detector_offset)
        h = ctypes.c_void_p()
        check(fn(ctypes.byref(vd), ctypes.byref(dd), int(n_views), *args, ctypes.byref(h)))
        kind = ctypes.c_int()
        lib().pyronn_geom_info(h, None, ctypes.byref(kind), None)
        vshape = vs[1:] if ndim == 2 else vs
        vspac = sp[1:] if ndim == 2 else sp
        dshape = ds[1:] if ndim == 2 else ds
        dspac = dsp[1:] if ndim == 2 else dsp
        return cls(h, ndim, vshape, vspac, dshape, dspac, n_views, kind.value)

    @classmethod
    def parallel2d(cls, volume_shape, volume_spacing, detector_shape, detector_spacing, number_of_projections,
                   angular_range=math.pi, volume_offset=None, detector_offset=None):
        return cls._make(lib().pyronn_geom_create_parallel2d, 2, volume_shape, volume_spacing, volume_offset,
                         _as_seq(detector_shape), _as_seq(detector_spacing), detector_offset, number_of_projections,
                         float(angular_range))

    @classmethod
    def fan2d(cls, volume_shape, volume_spacing, detector_shape, detector_spacing, number_of_projections,
              angular_range, sid, sdd, volume_offset=None, detector_offset=None):
        return cls._make(lib().pyronn_geom_create_fan2d, 2, volume_shape, volume_spacing, volume_offset,
                         _as_seq(detector_shape), _as_seq(detector_spacing), detector_offset, number_of_projections,
                         float(angular_range), float(sid), float(sdd))

    @classmethod
    def cone_circular(cls, volume_shape, volume_spacing, detector_shape, detector_spacing, number_of_projections,
                      angular_range, sid, sdd, helical_pitch=0.0, volume_offset=None, detector_offset=None):
        return cls._make(lib().pyronn_geom_create_cone_circular, 3, volume_shape, volume_spacing, volume_offset,
                         detector_shape, detector_spacing, detector_offset, number_of_projections,
                         float(angular_range), float(sid), float(sdd), float(helical_pitch))

    @classmethod
    def cone_from_positions(cls, volume_shape, volume_spacing, detector_shape, detector_spacing, src, det_centre,
                            eu, ev, volume_offset=None, detector_offset=None):
        arrs = [np.ascontiguousarray(np.asarray(a, dtype=np.float64).reshape(-1, 3)) for a in (src, det_centre, eu, ev)]
        n = arrs[0].shape[0]
        if any(a.shape[0] != n for a in arrs):
            raise ValueError("src, det_centre, eu, ev must have the same number of views")
        g = cls._make(lib().pyronn_geom_create_from_positions, 3, volume_shape, volume_spacing, volume_offset,
                      detector_shape, detector_spacing, detector_offset, n, *[_dp(a) for a in arrs])
        return g

    @classmethod
    def cone_from_matrices(cls, volume_shape, volume_spacing, detector_shape, detector_spacing, matrices,
                           volume_offset=None):
        P = np.ascontiguousarray(np.asarray(matrices, dtype=np.float64).reshape(-1, 12))
        return cls._make(lib().pyronn_geom_create_cone_matrices, 3, volume_shape, volume_spacing, volume_offset,
                         detector_shape, detector_spacing, None, P.shape[0], _dp(P))

    @classmethod
    def from_matrices2d(cls, volume_shape, volume_spacing, detector_shape, detector_spacing, matrices,
                        volume_offset=None):
        P = np.ascontiguousarray(np.asarray(matrices, dtype=np.float64).reshape(-1, 6))
        return cls._make(lib().pyronn_geom_create_matrices2d, 2, volume_shape, volume_spacing, volume_offset,
                         _as_seq(detector_shape), _as_seq(detector_spacing), None, P.shape[0], _dp(P))

    # -- properties --------------------------------------------------------------------------
    @property
    def handle(self):
        return self._h

    @property
    def sinogram_shape(self):
        return (self.n_views,) + self.detector_shape

    @property
    def step(self) -> float:
        d = ctypes.c_double()
        check(lib().pyronn_geom_get_step(self._h, ctypes.byref(d)))
        return d.value

    @step.setter
    def step(self, dt_mm: float):
        check(lib().pyronn_geom_set_step(self._h, float(dt_mm)))

    def views(self) -> np.ndarray:
        out = np.zeros((self.n_views, 12))
        check(lib().pyronn_geom_get_views(self._h, _dp(out)))
        return out

    def count_samples(self) -> int:
        n = ctypes.c_int64()
        check(lib().pyronn_geom_count_samples(self._h, ctypes.byref(n)))
        return int(n.value)

    def read_flags(self, reset: bool = True) -> list:
        out = (ctypes.c_int * 8)()
        check(lib().pyronn_geom_read_flags(self._h, out, int(reset)))
        return list(out)

    def fp_config(self, dtype=torch.float32) -> dict:
        out = (ctypes.c_int * 20)()
        check(lib().pyronn_geom_fp_config(self._h, _DTYPES[dtype], out))
        o = list(out)
        return {"kernel": o[0], "depth": o[1], "guard": o[2], "slab0": o[3],
                "box": [o[4:7], o[7:10], o[10:13]], "buf_elems": o[13], "smem_bytes": o[14],
                "thread_box_capacity": o[15], "y_fastest_x_march": bool(o[16])}

    def bp_config(self, dtype=torch.float32) -> dict:
        out = (ctypes.c_int * 8)()
        check(lib().pyronn_geom_bp_config(self._h, _DTYPES[dtype], out))
        return {"kernel": out[0], "box": [out[1], out[2]], "brick_z": out[3], "views_per_stage": out[4],
                "slot_elems": out[5]}

    def adjoint_config(self) -> dict:
        out = (ctypes.c_int * 8)()
        check(lib().pyronn_geom_adjoint_config(self._h, out))
        return {"kernel": out[0], "depth": out[1], "guard": out[2], "box_floats": out[3], "odd_pitch": bool(out[4]),
                "max_slabs": out[5], "pitch32": bool(out[6])}

    def set_tuning(self, param: int, value: int) -> None:
        check(lib().pyronn_geom_set_tuning(self._h, int(param), int(value)))

    def set_variant(self, op: int, variant: int) -> None:
        check(lib().pyronn_geom_set_variant(self._h, int(op), int(variant)))

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and _lib._lib is not None:
            _lib._lib.pyronn_geom_destroy(h)
            self._h = None


def _as_seq(x) -> Sequence:
    return tuple(x) if np.ndim(x) else (x,)


# ------------------------------------------------------------------------------------------------
# tensor plumbing
# ------------------------------------------------------------------------------------------------

def _vol_dims(g: Geometry):
    return g.volume_shape if g.ndim == 3 else g.volume_shape


def _sino_dims(g: Geometry):
    return (g.n_views,) + (g.detector_shape if g.ndim == 3 else g.detector_shape)


def _batch(t: torch.Tensor, dims, what: str) -> tuple:
    nd = len(dims)
    if t.dim() < nd or tuple(t.shape[-nd:]) != tuple(dims):
        raise ValueError(f"{what} must end with shape {tuple(dims)}, got {tuple(t.shape)}")
    lead = tuple(t.shape[:-nd])
    return lead, int(np.prod(lead)) if lead else 1


def _check(t: torch.Tensor, what: str) -> int:
    if not t.is_cuda:
        raise ValueError(f"{what} must be a CUDA tensor (the operators run only in the CUDA library)")
    if t.dtype not in _DTYPES:
        raise TypeError(f"{what}: unsupported dtype {t.dtype} (float32, bfloat16, float16)")
    return _DTYPES[t.dtype]


def _check_like(t: torch.Tensor, shape, dtype, device, what: str) -> torch.Tensor:
    """A caller-supplied tensor the library writes (or reads in place) must match exactly: the library
    sees only a pointer, so a wrong size, type, device or layout would let it run past the tensor."""
    if t.device != device:
        raise ValueError(f"{what} must be on {device}, got {t.device}")
    if t.dtype != dtype:
        raise TypeError(f"{what} must be {dtype}, got {t.dtype}")
    if tuple(t.shape) != tuple(shape):
        raise ValueError(f"{what} must have shape {tuple(shape)}, got {tuple(t.shape)}")
    if not t.is_contiguous():
        raise ValueError(f"{what} must be contiguous")
    return t


def _stream_ptr(device) -> int:
    return torch.cuda.current_stream(device).cuda_stream


def forward_project(vol: torch.Tensor, g: Geometry, out: torch.Tensor | None = None) -> torch.Tensor:
    """p = A vol (ray-driven forward projection, Sec. 2.1)."""
    dt = _check(vol, "volume")
    vol = vol.contiguous()
    lead, nb = _batch(vol, _vol_dims(g), "volume")
    if out is None:
        out = torch.empty(lead + _sino_dims(g), dtype=vol.dtype, device=vol.device)
    _check_like(out, lead + _sino_dims(g), vol.dtype, vol.device, "out")
    with torch.cuda.device(vol.device):
        check(lib().pyronn_fp(g.handle, vol.data_ptr(), out.data_ptr(), dt, nb, _stream_ptr(vol.device)))
    return out


def adjoint(sino: torch.Tensor, g: Geometry, out: torch.Tensor | None = None) -> torch.Tensor:
    """vol = A^T sino (matched adjoint: exact transpose of forward_project, Sec. 2.2)."""
    dt = _check(sino, "sinogram")
    sino = sino.contiguous()
    lead, nb = _batch(sino, _sino_dims(g), "sinogram")
    if out is None:
        out = torch.empty(lead + _vol_dims(g), dtype=sino.dtype, device=sino.device)
    _check_like(out, lead + _vol_dims(g), sino.dtype, sino.device, "out")
    with torch.cuda.device(sino.device):
        check(lib().pyronn_adjoint(g.handle, sino.data_ptr(), out.data_ptr(), dt, nb, _stream_ptr(sino.device)))
    return out


def adjoint_update(vol: torch.Tensor, sino: torch.Tensor, g: Geometry, alpha: float,
                   sino_b: torch.Tensor | None = None) -> torch.Tensor:
    """vol += alpha A^T (sino - sino_b) in place (sino_b optional): the fused data-term update of a
    gradient step (pyronn_adjoint_update). Returns vol."""
    dt = _check(sino, "sinogram")
    sino = sino.contiguous()
    lead, nb = _batch(sino, _sino_dims(g), "sinogram")
    _check_like(vol, lead + _vol_dims(g), sino.dtype, sino.device, "the updated volume")
    sb = 0
    if sino_b is not None:
        sino_b = _check_like(sino_b.contiguous(), sino.shape, sino.dtype, sino.device, "sino_b")
        sb = sino_b.data_ptr()
    with torch.cuda.device(sino.device):
        check(lib().pyronn_adjoint_update(g.handle, sino.data_ptr(), sb, float(alpha), vol.data_ptr(), dt, nb,
                                          _stream_ptr(sino.device)))
    return vol


FILTER_RAM_LAK, FILTER_SHEPP_LOGAN = 0, 1


def fbp_filter(sino: torch.Tensor, g: Geometry, filter: int = FILTER_RAM_LAK,
               out: torch.Tensor | None = None) -> torch.Tensor:
    """Cosine-weighted (divergent beams), ramp-filtered and scaled sinogram (pyronn_fbp_filter): its
    back-projection with weight BP_INV_W2 (divergent) or BP_PLAIN (parallel) is the filtered
    back-projection (Sec. 2.2). out may be sino itself."""
    dt = _check(sino, "sinogram")
    sino = sino.contiguous()
    lead, nb = _batch(sino, _sino_dims(g), "sinogram")
    if out is None:
        out = torch.empty_like(sino)
    _check_like(out, sino.shape, sino.dtype, sino.device, "out")
    with torch.cuda.device(sino.device):
        check(lib().pyronn_fbp_filter(g.handle, sino.data_ptr(), out.data_ptr(), int(filter), dt, nb,
                                      _stream_ptr(sino.device)))
    return out


def fbp(sino: torch.Tensor, g: Geometry, filter: int = FILTER_RAM_LAK) -> torch.Tensor:
    """Filtered back-projection (FDK for divergent beams) of a full scan: fbp_filter, then the voxel-driven
    back-projection with the matching weight."""
    return back_project(fbp_filter(sino, g, filter), g, BP_INV_W2 if g.kind == 1 else BP_PLAIN)


def back_project(sino: torch.Tensor, g: Geometry, weight: int = BP_PLAIN, out: torch.Tensor | None = None):
    """vol = BP sino (voxel-driven back-projection, Sec. 2.1); weight BP_PLAIN or BP_INV_W2."""
    dt = _check(sino, "sinogram")
    sino = sino.contiguous()
    lead, nb = _batch(sino, _sino_dims(g), "sinogram")
    if out is None:
        out = torch.empty(lead + _vol_dims(g), dtype=sino.dtype, device=sino.device)
    _check_like(out, lead + _vol_dims(g), sino.dtype, sino.device, "out")
    with torch.cuda.device(sino.device):
        check(lib().pyronn_bp(g.handle, sino.data_ptr(), out.data_ptr(), dt, nb, int(weight),
                              _stream_ptr(sino.device)))
    return out


def back_project_transpose(vol: torch.Tensor, g: Geometry, weight: int = BP_PLAIN,
                           out: torch.Tensor | None = None):
    """sino = BP^T vol (exact transpose of back_project; the gradient of the back-projector)."""
    dt = _check(vol, "volume")
    vol = vol.contiguous()
    lead, nb = _batch(vol, _vol_dims(g), "volume")
    if out is None:
        out = torch.empty(lead + _sino_dims(g), dtype=vol.dtype, device=vol.device)
    _check_like(out, lead + _sino_dims(g), vol.dtype, vol.device, "out")
    with torch.cuda.device(vol.device):
        check(lib().pyronn_bp_transpose(g.handle, vol.data_ptr(), out.data_ptr(), dt, nb, int(weight),
                                        _stream_ptr(vol.device)))
    return out


# ------------------------------------------------------------------------------------------------
# batched plans
# ------------------------------------------------------------------------------------------------

class Plan:
    """Several volumes with their own geometries, one persistent launch per operator.

    Calls allocate nothing on the device (outputs passed in), so they can be captured in a CUDA graph
    (torch.cuda.graph) after the plan has been created.
    """

    def __init__(self, geometries, dtype=torch.float32):
        self.geometries = list(geometries)
        self.dtype = dtype
        arr = (ctypes.c_void_p * len(self.geometries))(*[g.handle.value if isinstance(g.handle, ctypes.c_void_p)
                                                          else g.handle for g in self.geometries])
        h = ctypes.c_void_p()
        check(lib().pyronn_plan_create(len(self.geometries), arr, _DTYPES[dtype], ctypes.byref(h)))
        self._h = h

    def info(self) -> dict:
        n = ctypes.c_int()
        a = ctypes.c_int64()
        b = ctypes.c_int64()
        gr = (ctypes.c_int * 3)()
        check(lib().pyronn_plan_info(self._h, ctypes.byref(n), ctypes.byref(a), ctypes.byref(b), gr))
        return {"n": n.value, "items_fp": a.value, "items_brick": b.value, "grids": list(gr)}

    def _ptrs(self, tensors, shapes, what):
        if len(tensors) != len(self.geometries):
            raise ValueError(f"expected {len(self.geometries)} {what} tensors")
        for t, shp in zip(tensors, shapes):
            _check(t, what)
            if t.dtype != self.dtype or tuple(t.shape) != tuple(shp) or not t.is_contiguous():
                raise ValueError(f"{what}: expected contiguous {self.dtype} of shape {tuple(shp)}, got "
                                 f"{t.dtype} {tuple(t.shape)}")
            if t.device != tensors[0].device:
                raise ValueError(f"{what}: all tensors of a plan call must be on one device")
        return (ctypes.c_void_p * len(tensors))(*[t.data_ptr() for t in tensors])

    def forward_project(self, vols, sinos):
        v = self._ptrs(vols, [g.volume_shape for g in self.geometries], "volume")
        s = self._ptrs(sinos, [g.sinogram_shape for g in self.geometries], "sinogram")
        check(lib().pyronn_plan_fp(self._h, v, s, _stream_ptr(vols[0].device)))
        return sinos

    def adjoint(self, sinos, vols):
        s = self._ptrs(sinos, [g.sinogram_shape for g in self.geometries], "sinogram")
        v = self._ptrs(vols, [g.volume_shape for g in self.geometries], "volume")
        check(lib().pyronn_plan_adjoint(self._h, s, v, _stream_ptr(vols[0].device)))
        return vols

    def back_project(self, sinos, vols, weight: int = BP_PLAIN):
        s = self._ptrs(sinos, [g.sinogram_shape for g in self.geometries], "sinogram")
        v = self._ptrs(vols, [g.volume_shape for g in self.geometries], "volume")
        check(lib().pyronn_plan_bp(self._h, s, v, int(weight), _stream_ptr(vols[0].device)))
        return vols

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and _lib._lib is not None:
            _lib._lib.pyronn_plan_destroy(h)
            self._h = None


# ------------------------------------------------------------------------------------------------
# autograd
# ------------------------------------------------------------------------------------------------

class ForwardProjectFn(torch.autograd.Function):
    """A with backward A^T (matched adjoint)."""

    @staticmethod
    def forward(ctx, vol, g):
        ctx.g = g
        return forward_project(vol, g)

    @staticmethod
    def backward(ctx, grad):
        return adjoint(grad.contiguous(), ctx.g), None


class AdjointFn(torch.autograd.Function):
    """A^T with backward A."""

    @staticmethod
    def forward(ctx, sino, g):
        ctx.g = g
        return adjoint(sino, g)

    @staticmethod
    def backward(ctx, grad):
        return forward_project(grad.contiguous(), ctx.g), None


class BackProjectFn(torch.autograd.Function):
    """Voxel-driven BP with backward BP^T (its exact transpose)."""

    @staticmethod
    def forward(ctx, sino, g, weight):
        ctx.g, ctx.weight = g, weight
        return back_project(sino, g, weight)

    @staticmethod
    def backward(ctx, grad):
        return back_project_transpose(grad.contiguous(), ctx.g, ctx.weight), None, None


class GradientStepFn(torch.autograd.Function):
    """x_next = x - alpha A^T (A x - p) with the fused update kernel (one projection, one fused adjoint).
    Backward: grad_x = g - alpha A^T A g (fused again), grad_p = alpha A g,
    grad_alpha = -<A g, A x - p>."""

    @staticmethod
    def forward(ctx, x, p, alpha, g):
        pm = forward_project(x.contiguous(), g)
        # the fused kernel takes the step as a host scalar: a Python float or a CPU tensor costs nothing, a
        # CUDA tensor is read back once here (the backward reuses this value)
        a = float(alpha)
        out = adjoint_update(x.detach().clone(memory_format=torch.contiguous_format), pm, g, -a, sino_b=p)
        ctx.g = g
        ctx.alpha = a
        ctx.alpha_is_tensor = isinstance(alpha, torch.Tensor)
        ctx.alpha_like = alpha if ctx.alpha_is_tensor else None
        ctx.save_for_backward(pm, p)
        return out

    @staticmethod
    def backward(ctx, grad):
        pm, p = ctx.saved_tensors
        g, a = ctx.g, ctx.alpha
        grad = grad.contiguous()
        ag = forward_project(grad, g)
        gx = adjoint_update(grad.clone(), ag, g, -a) if ctx.needs_input_grad[0] else None
        gp = a * ag if ctx.needs_input_grad[1] else None
        galpha = None
        if ctx.needs_input_grad[2] and ctx.alpha_is_tensor:
            al = ctx.alpha_like
            galpha = (-torch.sum(ag * (pm - p), dtype=torch.float64)).to(al.dtype).reshape(al.shape)
        return gx, gp, galpha, None


def gradient_step(x, p, alpha, g):
    """x - alpha A^T (A x - p) (fused update, differentiable in x, p and alpha). alpha: a Python float, or a
    tensor of one element (a gradient reaches it when it requires one); a CUDA tensor is read back once per
    call, since the fused kernel takes the step as a scalar argument."""
    return GradientStepFn.apply(x, p, alpha, g)


def project(vol, g):
    return ForwardProjectFn.apply(vol, g)


def project_adjoint(sino, g):
    return AdjointFn.apply(sino, g)


def backproject(sino, g, weight=BP_PLAIN):
    return BackProjectFn.apply(sino, g, weight)


# ------------------------------------------------------------------------------------------------
# layers (Listing 1 names)
# ------------------------------------------------------------------------------------------------

class _Projection(torch.nn.Module):
    def forward(self, vol, geometry: Geometry):
        return project(vol, geometry)


class _BackProjection(torch.nn.Module):
    def __init__(self, weight: int = BP_PLAIN):
        super().__init__()
        self.weight = weight

    def forward(self, sino, geometry: Geometry):
        return backproject(sino, geometry, self.weight)


class ParallelProjectionFor2D(_Projection):
    pass


class FanProjectionFor2D(_Projection):
    pass


class ConeProjectionFor3D(_Projection):
    pass


class ParallelBackProjectionFor2D(_BackProjection):
    pass


class FanBackProjectionFor2D(_BackProjection):
    pass


class ConeBackProjectionFor3D(_BackProjection):
    pass

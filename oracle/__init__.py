"""FP64 CPU oracle (ctypes wrapper around oracle/pyronn_oracle.c).

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the benchmark's CPU-baseline leg
may use this package; the product path never does. It shares no code with the CUDA library.

Geometry conventions (the paper leaves them open; these are the project's readings):
  * volume arrays are [Nz, Ny, Nx] (x fastest), spacing and offsets given in (z, y, x) order;
    voxel i along an axis sits at (i - (N-1)/2) * s + o (mm);
  * detector arrays are [V, Nv, Nu] (u fastest); pixel (u, v) of a view sits at
    Dc + ((u - (Nu-1)/2) du + ou) eu + ((v - (Nv-1)/2) dv + ov) ev;
  * circular orbit (Listing 1: sdd, sid, number_of_projections, angular_range): view n at
    angle n * range / V, source sid (cos, sin, 0), detector centre -(sdd - sid) (cos, sin, 0),
    eu = (-sin, cos, 0), ev = (0, 0, 1);
  * 2D geometries are the z = 0 plane of a volume with Nz = 1 and a detector with Nv = 1;
  * parallel beam: rays along -(cos t, sin t), detector axis (-sin t, cos t) through the origin;
  * rays are sampled at (k + 1/2) dt from their point closest to the volume centre,
    dt = 0.5 * (smallest voxel spacing) unless given.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pyronn_oracle.c")
_LIB_PATH = os.path.join(_HERE, "_build", "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2, OpenMP, no FMA contraction)."""
    os.makedirs(os.path.dirname(_LIB_PATH), exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        cmd = ["gcc", "-O2", "-std=c11", "-D_GNU_SOURCE", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared",
               "-o", _LIB_PATH, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
    return _LIB_PATH


class _OG(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("sx", ctypes.c_double), ("sy", ctypes.c_double), ("sz", ctypes.c_double),
                ("ox", ctypes.c_double), ("oy", ctypes.c_double), ("oz", ctypes.c_double),
                ("nu", ctypes.c_int), ("nv", ctypes.c_int),
                ("du", ctypes.c_double), ("dv", ctypes.c_double),
                ("ou", ctypes.c_double), ("ov", ctypes.c_double),
                ("n_views", ctypes.c_int), ("kind", ctypes.c_int),
                ("views", ctypes.POINTER(ctypes.c_double)), ("dt", ctypes.c_double)]


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB_PATH)
        dp = ctypes.POINTER(ctypes.c_double)
        ip = ctypes.POINTER(ctypes.c_int64)
        og = ctypes.POINTER(_OG)
        L.or_set_threads.argtypes = [ctypes.c_int]
        L.or_max_threads.restype = ctypes.c_int
        L.or_frames_circular.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                         ctypes.c_double, dp, dp, dp, dp]
        L.or_pmat_from_frames.argtypes = [ctypes.c_int, dp, dp, dp, dp, ctypes.c_int, ctypes.c_int,
                                          ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_double, dp]
        L.or_pmat_from_frames.restype = ctypes.c_int
        L.or_normalise_pmat.argtypes = [ctypes.c_int, dp, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                        ctypes.c_double, dp]
        L.or_normalise_pmat.restype = ctypes.c_int
        L.or_fp.argtypes = [og, dp, dp]
        L.or_fp_rays.argtypes = [og, dp, ctypes.c_long, ip, dp]
        L.or_count_samples.argtypes = [og, ip]
        L.or_adjoint_rays.argtypes = [og, ctypes.c_long, ip, dp, dp]
        L.or_adjoint.argtypes = [og, dp, dp]
        L.or_adjoint.restype = ctypes.c_int
        L.or_bp.argtypes = [og, dp, ctypes.c_int, dp]
        L.or_bp_voxels.argtypes = [og, dp, ctypes.c_int, ctypes.c_long, ip, dp]
        L.or_fbp_filter.argtypes = [og, ctypes.c_int, dp, dp]
        L.or_fbp_filter.restype = ctypes.c_int
        _lib = L
    return _lib


def _dp(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _ip(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))


def set_threads(n: int) -> None:
    lib().or_set_threads(int(n))


def max_threads() -> int:
    return int(lib().or_max_threads())


@dataclass
class Geometry:
    """Oracle geometry. kind 1: per-view normalised 3x4 projection matrices; kind 0: parallel views
    given as [Dc(3), eu(3), ev(3), d(3)]."""
    vol_shape: tuple            # (nz, ny, nx)
    vol_spacing: tuple          # (sz, sy, sx)
    vol_offset: tuple           # (oz, oy, ox)
    det_shape: tuple            # (nv, nu)
    det_spacing: tuple          # (dv, du)
    det_offset: tuple           # (ov, ou)
    kind: int
    views: np.ndarray           # (V, 12) float64
    dt: float
    ndim: int = 3
    _keep: list = field(default_factory=list, repr=False)

    @property
    def n_views(self) -> int:
        return int(self.views.shape[0])

    @property
    def sino_shape(self):
        return (self.n_views, self.det_shape[0], self.det_shape[1])

    def struct(self) -> _OG:
        v = np.ascontiguousarray(self.views, dtype=np.float64)
        self._keep = [v]
        nz, ny, nx = self.vol_shape
        sz, sy, sx = self.vol_spacing
        oz, oy, ox = self.vol_offset
        nv, nu = self.det_shape
        dv, du = self.det_spacing
        ov, ou = self.det_offset
        return _OG(nx, ny, nz, sx, sy, sz, ox, oy, oz, nu, nv, du, dv, ou, ov,
                   self.n_views, self.kind, _dp(v), self.dt)


def default_dt(vol_spacing, ndim: int) -> float:
    sp = list(vol_spacing)
    return 0.5 * (min(sp[1:]) if ndim == 2 else min(sp))


def circular_frames(n_views: int, angular_range: float, sid: float, sdd: float, pitch: float = 0.0):
    src = np.zeros((n_views, 3)); det = np.zeros((n_views, 3))
    eu = np.zeros((n_views, 3)); ev = np.zeros((n_views, 3))
    lib().or_frames_circular(n_views, angular_range, sid, sdd, pitch, _dp(src), _dp(det), _dp(eu), _dp(ev))
    return src, det, eu, ev


def pmat_from_frames(src, det, eu, ev, det_shape, det_spacing, det_offset=(0.0, 0.0)) -> np.ndarray:
    src, det, eu, ev = (np.ascontiguousarray(a, dtype=np.float64) for a in (src, det, eu, ev))
    n = src.shape[0]
    P = np.zeros((n, 12))
    rc = lib().or_pmat_from_frames(n, _dp(src), _dp(det), _dp(eu), _dp(ev), int(det_shape[1]), int(det_shape[0]),
                                   float(det_spacing[1]), float(det_spacing[0]),
                                   float(det_offset[1]), float(det_offset[0]), _dp(P))
    if rc:
        raise ValueError("singular detector frame")
    return P


def normalise_pmat(P, du: float, centre_xyz) -> np.ndarray:
    P = np.ascontiguousarray(np.asarray(P, dtype=np.float64).reshape(-1, 12))
    out = np.zeros_like(P)
    rc = lib().or_normalise_pmat(P.shape[0], _dp(P), float(du), float(centre_xyz[0]), float(centre_xyz[1]),
                                 float(centre_xyz[2]), _dp(out))
    if rc:
        raise ValueError("projection matrix cannot be normalised")
    return out


def cone_circular(vol_shape, vol_spacing, det_shape, det_spacing, n_views, angular_range, sid, sdd,
                  pitch=0.0, vol_offset=(0.0, 0.0, 0.0), det_offset=(0.0, 0.0), dt=None) -> Geometry:
    src, det, eu, ev = circular_frames(n_views, angular_range, sid, sdd, pitch)
    P = pmat_from_frames(src, det, eu, ev, det_shape, det_spacing, det_offset)
    dt = default_dt(vol_spacing, 3) if dt is None else dt
    return Geometry(tuple(vol_shape), tuple(vol_spacing), tuple(vol_offset), tuple(det_shape), tuple(det_spacing),
                    tuple(det_offset), 1, P, dt)


def cone_from_positions(vol_shape, vol_spacing, det_shape, det_spacing, src, det, eu, ev,
                        vol_offset=(0.0, 0.0, 0.0), det_offset=(0.0, 0.0), dt=None) -> Geometry:
    P = pmat_from_frames(src, det, eu, ev, det_shape, det_spacing, det_offset)
    dt = default_dt(vol_spacing, 3) if dt is None else dt
    return Geometry(tuple(vol_shape), tuple(vol_spacing), tuple(vol_offset), tuple(det_shape), tuple(det_spacing),
                    tuple(det_offset), 1, P, dt)


def cone_from_matrices(vol_shape, vol_spacing, det_shape, det_spacing, P, vol_offset=(0.0, 0.0, 0.0),
                       dt=None) -> Geometry:
    c = (vol_offset[2], vol_offset[1], vol_offset[0])
    Pn = normalise_pmat(P, det_spacing[1], c)
    dt = default_dt(vol_spacing, 3) if dt is None else dt
    return Geometry(tuple(vol_shape), tuple(vol_spacing), tuple(vol_offset), tuple(det_shape), tuple(det_spacing),
                    (0.0, 0.0), 1, Pn, dt)


def fan_circular(img_shape, img_spacing, n_bins, du, n_views, angular_range, sid, sdd,
                 img_offset=(0.0, 0.0), det_offset=0.0, dt=None) -> Geometry:
    """2D fan beam as the z = 0 plane: volume (1, Ny, Nx), detector (1, Nu)."""
    vol_shape = (1, img_shape[0], img_shape[1])
    vol_spacing = (1.0, img_spacing[0], img_spacing[1])
    vol_offset = (0.0, img_offset[0], img_offset[1])
    src, det, eu, ev = circular_frames(n_views, angular_range, sid, sdd, 0.0)
    P = pmat_from_frames(src, det, eu, ev, (1, n_bins), (1.0, du), (0.0, det_offset))
    dt = default_dt(vol_spacing, 2) if dt is None else dt
    return Geometry(vol_shape, vol_spacing, vol_offset, (1, n_bins), (1.0, du), (0.0, det_offset), 1, P, dt, ndim=2)


def parallel2d(img_shape, img_spacing, n_bins, du, n_views, angular_range=math.pi,
               img_offset=(0.0, 0.0), det_offset=0.0, dt=None) -> Geometry:
    """2D parallel beam: view n at angle t = n * range / V, rays along -(cos t, sin t),
    bin u at signed distance (u - (Nu-1)/2) du + ou along (-sin t, cos t)."""
    vol_shape = (1, img_shape[0], img_shape[1])
    vol_spacing = (1.0, img_spacing[0], img_spacing[1])
    vol_offset = (0.0, img_offset[0], img_offset[1])
    views = np.zeros((n_views, 12))
    for n in range(n_views):
        t = n * angular_range / n_views
        c, s = math.cos(t), math.sin(t)
        views[n, 0:3] = 0.0
        views[n, 3:6] = (-s, c, 0.0)
        views[n, 6:9] = (0.0, 0.0, 1.0)
        views[n, 9:12] = (-c, -s, 0.0)
    dt = default_dt(vol_spacing, 2) if dt is None else dt
    return Geometry(vol_shape, vol_spacing, vol_offset, (1, n_bins), (1.0, du), (0.0, det_offset), 0, views, dt,
                    ndim=2)


def parallel_from_views(vol_shape, vol_spacing, det_shape, det_spacing, views, vol_offset=(0.0, 0.0, 0.0),
                        det_offset=(0.0, 0.0), dt=None, ndim=3) -> Geometry:
    views = np.ascontiguousarray(np.asarray(views, dtype=np.float64).reshape(-1, 12))
    dt = default_dt(vol_spacing, ndim) if dt is None else dt
    return Geometry(tuple(vol_shape), tuple(vol_spacing), tuple(vol_offset), tuple(det_shape), tuple(det_spacing),
                    tuple(det_offset), 0, views, dt, ndim=ndim)


# ------------------------------------------------------------------------------------------------
# operators
# ------------------------------------------------------------------------------------------------

def _vol3(g: Geometry, x) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(x, dtype=np.float64).reshape(g.vol_shape))


def fp(g: Geometry, vol) -> np.ndarray:
    """Forward projection, returns [V, Nv, Nu] float64."""
    v = _vol3(g, vol)
    out = np.zeros(g.sino_shape)
    s = g.struct()
    lib().or_fp(ctypes.byref(s), _dp(v), _dp(out))
    return out


def fp_rays(g: Geometry, vol, ray_ids) -> np.ndarray:
    v = _vol3(g, vol)
    ids = np.ascontiguousarray(np.asarray(ray_ids, dtype=np.int64))
    out = np.zeros(ids.shape[0])
    s = g.struct()
    lib().or_fp_rays(ctypes.byref(s), _dp(v), ids.shape[0], _ip(ids), _dp(out))
    return out


def adjoint(g: Geometry, sino) -> np.ndarray:
    """Exact transpose of fp, returns [Nz, Ny, Nx] float64."""
    y = np.ascontiguousarray(np.asarray(sino, dtype=np.float64).reshape(g.sino_shape))
    out = np.zeros(g.vol_shape)
    s = g.struct()
    if lib().or_adjoint(ctypes.byref(s), _dp(y), _dp(out)):
        raise MemoryError("oracle adjoint buffers")
    return out


def adjoint_rays(g: Geometry, ray_ids, values) -> np.ndarray:
    ids = np.ascontiguousarray(np.asarray(ray_ids, dtype=np.int64))
    val = np.ascontiguousarray(np.asarray(values, dtype=np.float64))
    out = np.zeros(g.vol_shape)
    s = g.struct()
    lib().or_adjoint_rays(ctypes.byref(s), ids.shape[0], _ip(ids), _dp(val), _dp(out))
    return out


def bp(g: Geometry, sino, weight: int = 0) -> np.ndarray:
    """Voxel-driven back-projection; weight 0: plain sum, 1: 1 / w^2 distance weight."""
    y = np.ascontiguousarray(np.asarray(sino, dtype=np.float64).reshape(g.sino_shape))
    out = np.zeros(g.vol_shape)
    s = g.struct()
    lib().or_bp(ctypes.byref(s), _dp(y), int(weight), _dp(out))
    return out


def fbp_filter(g: Geometry, sino, filt: int = 0) -> np.ndarray:
    """Cosine-weighted (divergent beams), ramp-filtered and scaled sinogram: its BP (weight 1 for
    perspective geometries, 0 for parallel) is the filtered back-projection. filt 0: Ram-Lak,
    1: Shepp-Logan."""
    y = np.ascontiguousarray(np.asarray(sino, dtype=np.float64).reshape(g.sino_shape))
    out = np.zeros(g.sino_shape)
    s = g.struct()
    if lib().or_fbp_filter(ctypes.byref(s), int(filt), _dp(y), _dp(out)) != 0:
        raise ValueError("singular view")
    return out


def fbp(g: Geometry, sino, filt: int = 0) -> np.ndarray:
    """Filtered back-projection (FDK for perspective geometries)."""
    return bp(g, fbp_filter(g, sino, filt), 1 if g.kind == 1 else 0)


def bp_voxels(g: Geometry, sino, voxel_ids, weight: int = 0) -> np.ndarray:
    y = np.ascontiguousarray(np.asarray(sino, dtype=np.float64).reshape(g.sino_shape))
    ids = np.ascontiguousarray(np.asarray(voxel_ids, dtype=np.int64))
    out = np.zeros(ids.shape[0])
    s = g.struct()
    lib().or_bp_voxels(ctypes.byref(s), _dp(y), int(weight), ids.shape[0], _ip(ids), _dp(out))
    return out


def count_samples(g: Geometry) -> np.ndarray:
    """In-support sample count per view (int64)."""
    out = np.zeros(g.n_views, dtype=np.int64)
    s = g.struct()
    lib().or_count_samples(ctypes.byref(s), _ip(out))
    return out

"""Seeded synthetic inputs shared by the tests, the benchmark and the smoke run.

This module holds input recipes only: random phantoms (ellipses / ellipsoids
voxelised at voxel centres), random cotangents, trajectory perturbations and
photon noise. It contains none of the projector arithmetic (no ray sampling,
no interpolation, no projection matrices), so the CUDA path and the FP64
oracle can both consume its outputs without sharing any operator code.

The paper evaluates on a Shepp-Logan phantom (Listing 1, Fig. 1); its
coefficient table is not reproduced here. Random ellipse / ellipsoid phantoms
with the same structure (overlapping constant-density ellipsoids, additive
densities) stand in for it.

Voxel-centre convention (shared by every part of this project): voxel index
i along an axis with N voxels of spacing s and origin offset o has its centre
at world coordinate (i - (N - 1) / 2) * s + o, in millimetres.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np


def _centres(n: int, s: float, o: float = 0.0) -> np.ndarray:
    return (np.arange(n, dtype=np.float64) - (n - 1) / 2.0) * s + o


# ----------------------------------------------------------------------------------------------
# 2D ellipse phantoms
# ----------------------------------------------------------------------------------------------

def random_ellipses(n: int, half_fov_mm: float, seed: int,
                    centre_frac: float = 0.45, axis_lo: float = 0.05, axis_hi: float = 0.35) -> np.ndarray:
    """Random ellipses as an (n, 6) float64 array: cx, cy, a, b, phi, density.

    Centres are uniform in a disk of radius centre_frac * half_fov_mm, semi-axes
    uniform in [axis_lo, axis_hi] * half_fov_mm, rotation phi uniform in [0, pi),
    density uniform in [0, 1). With the defaults every ellipse lies inside the
    inscribed circle of the field of view (0.45 + 0.35 < 1).
    """
    rng = np.random.default_rng(seed)
    r = centre_frac * half_fov_mm * np.sqrt(rng.random(n))
    ang = rng.random(n) * 2.0 * math.pi
    out = np.empty((n, 6), dtype=np.float64)
    out[:, 0] = r * np.cos(ang)
    out[:, 1] = r * np.sin(ang)
    out[:, 2] = (axis_lo + (axis_hi - axis_lo) * rng.random(n)) * half_fov_mm
    out[:, 3] = (axis_lo + (axis_hi - axis_lo) * rng.random(n)) * half_fov_mm
    out[:, 4] = rng.random(n) * math.pi
    out[:, 5] = rng.random(n)
    return out


def rasterise_ellipses(ell: np.ndarray, shape_yx, spacing_yx, offset_yx=(0.0, 0.0)) -> np.ndarray:
    """Sum of ellipse densities at each pixel centre; returns float32 [Ny, Nx]."""
    ny, nx = shape_yx
    y = _centres(ny, spacing_yx[0], offset_yx[0])[:, None]
    x = _centres(nx, spacing_yx[1], offset_yx[1])[None, :]
    img = np.zeros((ny, nx), dtype=np.float64)
    for cx, cy, a, b, phi, rho in ell:
        c, s = math.cos(phi), math.sin(phi)
        xr = (x - cx) * c + (y - cy) * s
        yr = -(x - cx) * s + (y - cy) * c
        img += rho * (((xr / a) ** 2 + (yr / b) ** 2) <= 1.0)
    return img.astype(np.float32)


# ----------------------------------------------------------------------------------------------
# 3D ellipsoid phantoms
# ----------------------------------------------------------------------------------------------

def euler_zyz(alpha: float, beta: float, gamma: float) -> np.ndarray:
    """Rotation matrix Rz(alpha) @ Ry(beta) @ Rz(gamma)."""
    ca, sa = math.cos(alpha), math.sin(alpha)
    cb, sb = math.cos(beta), math.sin(beta)
    cg, sg = math.cos(gamma), math.sin(gamma)
    rz1 = np.array([[ca, -sa, 0.0], [sa, ca, 0.0], [0.0, 0.0, 1.0]])
    ry = np.array([[cb, 0.0, sb], [0.0, 1.0, 0.0], [-sb, 0.0, cb]])
    rz2 = np.array([[cg, -sg, 0.0], [sg, cg, 0.0], [0.0, 0.0, 1.0]])
    return rz1 @ ry @ rz2


def random_ellipsoids(n: int, half_fov_mm: float, seed: int,
                      centre_frac: float = 0.45, axis_lo: float = 0.05, axis_hi: float = 0.35) -> np.ndarray:
    """Random ellipsoids as an (n, 10) float64 array: cx, cy, cz, a, b, c, alpha, beta, gamma, density.

    Centres are uniform in a ball of radius centre_frac * half_fov_mm, semi-axes
    uniform in [axis_lo, axis_hi] * half_fov_mm, ZYZ Euler angles uniform in
    [0, 2 pi), density uniform in [0, 1).
    """
    rng = np.random.default_rng(seed)
    out = np.empty((n, 10), dtype=np.float64)
    v = rng.normal(size=(n, 3))
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    r = centre_frac * half_fov_mm * np.cbrt(rng.random(n))
    out[:, 0:3] = v * r[:, None]
    out[:, 3:6] = (axis_lo + (axis_hi - axis_lo) * rng.random((n, 3))) * half_fov_mm
    out[:, 6:9] = rng.random((n, 3)) * 2.0 * math.pi
    out[:, 9] = rng.random(n)
    return out


def rasterise_ellipsoids(ell: np.ndarray, shape_zyx, spacing_zyx, offset_zyx=(0.0, 0.0, 0.0)) -> np.ndarray:
    """Sum of ellipsoid densities at each voxel centre; returns float32 [Nz, Ny, Nx]."""
    nz, ny, nx = shape_zyx
    zc = _centres(nz, spacing_zyx[0], offset_zyx[0])
    yc = _centres(ny, spacing_zyx[1], offset_zyx[1])
    xc = _centres(nx, spacing_zyx[2], offset_zyx[2])
    vol = np.zeros((nz, ny, nx), dtype=np.float32)
    for e in ell:
        cen, axes, rho = e[0:3], e[3:6], float(e[9])
        rot = euler_zyz(*e[6:9])
        rmax = float(axes.max())
        # bounding box of the ellipsoid's circumscribed sphere, in index space
        sl = []
        for coords, cc in ((zc, cen[2]), (yc, cen[1]), (xc, cen[0])):
            idx = np.nonzero(np.abs(coords - cc) <= rmax)[0]
            sl.append(slice(int(idx[0]), int(idx[-1]) + 1) if idx.size else slice(0, 0))
        if any(s.stop <= s.start for s in sl):
            continue
        z = zc[sl[0]][:, None, None] - cen[2]
        y = yc[sl[1]][None, :, None] - cen[1]
        x = xc[sl[2]][None, None, :] - cen[0]
        # local = R^T (X - c)
        lx = rot[0, 0] * x + rot[1, 0] * y + rot[2, 0] * z
        ly = rot[0, 1] * x + rot[1, 1] * y + rot[2, 1] * z
        lz = rot[0, 2] * x + rot[1, 2] * y + rot[2, 2] * z
        inside = (lx / axes[0]) ** 2 + (ly / axes[1]) ** 2 + (lz / axes[2]) ** 2 <= 1.0
        vol[sl[0], sl[1], sl[2]] += np.float32(rho) * inside.astype(np.float32)
    return vol


# ----------------------------------------------------------------------------------------------
# cotangents, noise, trajectories
# ----------------------------------------------------------------------------------------------

def gaussian(shape, seed: int, dtype=np.float32) -> np.ndarray:
    """Standard-normal array (e.g. a random cotangent for gradient checks)."""
    return np.random.default_rng(seed).standard_normal(size=shape).astype(dtype)


def uniform(shape, seed: int, dtype=np.float32) -> np.ndarray:
    return np.random.default_rng(seed).random(size=shape).astype(dtype)


def poisson_log_sinogram(p: np.ndarray, i0: float, seed: int, scale_to_max: float | None = 3.0) -> np.ndarray:
    """Photon-noise model of Sec. 2.4 ("Poisson noise"): counts ~ Poisson(I0 * exp(-p)).

    p is first scaled so that max(p) == scale_to_max (when given), because line
    integrals of [0, 1]-density phantoms over ~100 mm chords would otherwise
    starve every count. Zero counts are clamped to one photon before the log.
    Returns the noisy line integrals -ln(max(c, 1) / I0) as float32.
    """
    p = np.asarray(p, dtype=np.float64)
    if scale_to_max is not None and p.max() > 0:
        p = p * (scale_to_max / p.max())
    c = np.random.default_rng(seed).poisson(i0 * np.exp(-p))
    return (-np.log(np.maximum(c, 1.0) / i0)).astype(np.float32)


def poisson_log_sinogram_torch(p, i0: float, seed: int, scale_to_max: float | None = 3.0):
    """The photon-noise recipe of poisson_log_sinogram on a torch tensor (for sinograms too large for the
    host): same model and clamping, counts drawn by torch.poisson with a generator seeded by seed on the
    tensor's device. Returns FP32 noisy line integrals."""
    import torch
    gen = torch.Generator(device=p.device).manual_seed(seed)
    p = p.float()
    if scale_to_max is not None:
        pmax = p.max()
        if pmax > 0:
            p = p * (scale_to_max / pmax)
    c = torch.poisson(i0 * torch.exp(-p), generator=gen)
    return -torch.log(torch.clamp(c, min=1.0) / i0)


def jitter_shifts(shape, max_shift: int, seed: int) -> np.ndarray:
    """Integer detector shifts uniform in [-max_shift, max_shift] (int32), e.g. shape (V, Nv) per row."""
    return np.random.default_rng(seed).integers(-max_shift, max_shift + 1, size=shape).astype(np.int32)


def ring_columns(nu: int, count: int, seed: int, gain_lo: float = 0.0, gain_hi: float = 1.2):
    """`count` distinct detector columns and their gains uniform in [gain_lo, gain_hi]."""
    rng = np.random.default_rng(seed)
    cols = rng.choice(nu, size=count, replace=False).astype(np.int32)
    return cols, (gain_lo + (gain_hi - gain_lo) * rng.random(count)).astype(np.float32)


@dataclass
class Trajectory:
    """Per-view source position, detector centre and detector axes, world mm (float64, V x 3 each)."""
    src: np.ndarray
    det_centre: np.ndarray
    eu: np.ndarray
    ev: np.ndarray


def jittered_circular_trajectory(n_views: int, angular_range: float, sid: float, sdd: float,
                                 sigma_mm: float, sigma_deg: float, seed: int) -> Trajectory:
    """A circular orbit (source at sid (cos t, sin t, 0), detector centre at -(sdd - sid) (cos t, sin t, 0),
    detector axes eu = (-sin t, cos t, 0), ev = (0, 0, 1), t = n * range / V) perturbed per view:
    source and detector centre move by N(0, sigma_mm) in each coordinate, the detector axes are
    rotated about the detector centre by ZYZ Euler angles drawn from N(0, sigma_deg).
    """
    rng = np.random.default_rng(seed)
    t = np.arange(n_views, dtype=np.float64) * (angular_range / n_views)
    c, s = np.cos(t), np.sin(t)
    src = np.stack([sid * c, sid * s, np.zeros_like(t)], axis=1)
    det = np.stack([-(sdd - sid) * c, -(sdd - sid) * s, np.zeros_like(t)], axis=1)
    eu = np.stack([-s, c, np.zeros_like(t)], axis=1)
    ev = np.tile(np.array([0.0, 0.0, 1.0]), (n_views, 1))
    src = src + rng.normal(0.0, sigma_mm, size=(n_views, 3))
    det = det + rng.normal(0.0, sigma_mm, size=(n_views, 3))
    ang = np.deg2rad(rng.normal(0.0, sigma_deg, size=(n_views, 3)))
    for n in range(n_views):
        r = euler_zyz(*ang[n])
        eu[n] = r @ eu[n]
        ev[n] = r @ ev[n]
    return Trajectory(src, det, eu, ev)


def batched_cone_workload(n_volumes: int = 16, voxel_mm: float = 0.5, sid: float = 750.0, sdd: float = 1200.0):
    """Parameters of the uneven batched cone-beam workload (16 volumes, 96^3 ... 256^3).

    Volume i: cube side 8 * round((96 + i * 160 / 15) / 8) (uneven sizes; rows a multiple of 16
    bytes even in BF16, so that tensor copies apply to every storage type), views 180 + round(i * 360 / 15),
    detector side 256 + 16 * round(i * 16 / 15); circular orbit for even i, one-turn helix for
    odd i with pitch = half the detector height at the isocentre. The pixel size is chosen so
    that the volume's xy diagonal, magnified by sdd / sid, fills 90 % of the detector width.
    """
    out = []
    last = max(n_volumes - 1, 1)
    for i in range(n_volumes):
        side = int(8 * round((96 + i * 160 / last) / 8))
        views = int(180 + round(i * 360 / last))
        ndet = int(256 + 16 * round(i * 16 / last))
        mag = sdd / sid
        du = mag * side * voxel_mm * math.sqrt(2.0) / (0.9 * ndet)
        pitch = 0.0 if i % 2 == 0 else 0.5 * ndet * du / mag
        out.append(dict(index=i, side=side, voxel_mm=voxel_mm, views=views, det=ndet, du=du,
                        sid=sid, sdd=sdd, angular_range=2.0 * math.pi, pitch=pitch, seed=4 + i))
    return out

"""Geometry cases built twice from the same parameters: once through the library's C ABI
(paper_2511_08427_gb300.operators.Geometry) and once through the FP64 oracle."""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

import oracle
from paper_2511_08427_gb300 import inputs


@dataclass
class Case:
    name: str
    params: dict
    ndim: int

    def oracle_geometry(self):
        p = self.params
        k = p["kind"]
        if k == "parallel2d":
            return oracle.parallel2d(p["vol_shape"], p["vol_spacing"], p["nu"], p["du"], p["views"], p["range"],
                                     det_offset=p.get("ou", 0.0))
        if k == "fan2d":
            return oracle.fan_circular(p["vol_shape"], p["vol_spacing"], p["nu"], p["du"], p["views"], p["range"],
                                       p["sid"], p["sdd"], det_offset=p.get("ou", 0.0))
        if k == "cone":
            return oracle.cone_circular(p["vol_shape"], p["vol_spacing"], p["det_shape"], p["det_spacing"],
                                        p["views"], p["range"], p["sid"], p["sdd"], pitch=p.get("pitch", 0.0),
                                        vol_offset=p.get("vol_offset", (0.0, 0.0, 0.0)),
                                        det_offset=p.get("det_offset", (0.0, 0.0)))
        if k == "positions":
            tr = self.trajectory()
            return oracle.cone_from_positions(p["vol_shape"], p["vol_spacing"], p["det_shape"], p["det_spacing"],
                                              tr.src, tr.det_centre, tr.eu, tr.ev)
        raise ValueError(k)

    def trajectory(self):
        p = self.params
        return inputs.jittered_circular_trajectory(p["views"], p["range"], p["sid"], p["sdd"], p["sigma_mm"],
                                                   p["sigma_deg"], p["seed"])

    def library_geometry(self):
        from paper_2511_08427_gb300.operators import Geometry
        p = self.params
        k = p["kind"]
        if k == "parallel2d":
            return Geometry.parallel2d(p["vol_shape"], p["vol_spacing"], p["nu"], p["du"], p["views"], p["range"],
                                       detector_offset=p.get("ou", 0.0))
        if k == "fan2d":
            return Geometry.fan2d(p["vol_shape"], p["vol_spacing"], p["nu"], p["du"], p["views"], p["range"],
                                  p["sid"], p["sdd"], detector_offset=p.get("ou", 0.0))
        if k == "cone":
            return Geometry.cone_circular(p["vol_shape"], p["vol_spacing"], p["det_shape"], p["det_spacing"],
                                          p["views"], p["range"], p["sid"], p["sdd"], helical_pitch=p.get("pitch", 0.0),
                                          volume_offset=p.get("vol_offset"), detector_offset=p.get("det_offset"))
        if k == "positions":
            tr = self.trajectory()
            return Geometry.cone_from_positions(p["vol_shape"], p["vol_spacing"], p["det_shape"], p["det_spacing"],
                                                tr.src, tr.det_centre, tr.eu, tr.ev)
        raise ValueError(k)

    @property
    def vol_shape3(self):
        s = self.params["vol_shape"]
        return (1,) + tuple(s) if self.ndim == 2 else tuple(s)

    def phantom(self, seed=7) -> np.ndarray:
        p = self.params
        if self.ndim == 2:
            half = 0.5 * min(p["vol_shape"][0] * p["vol_spacing"][0], p["vol_shape"][1] * p["vol_spacing"][1])
            return inputs.rasterise_ellipses(inputs.random_ellipses(10, half, seed), p["vol_shape"], p["vol_spacing"])
        half = 0.5 * min(a * b for a, b in zip(p["vol_shape"], p["vol_spacing"]))
        return inputs.rasterise_ellipsoids(inputs.random_ellipsoids(12, half, seed), p["vol_shape"], p["vol_spacing"],
                                           p.get("vol_offset", (0.0, 0.0, 0.0)))


# Small cases: several tiles and a ragged tail in every dimension; the oracle finishes in seconds.
SMALL = [
    Case("parallel2d", dict(kind="parallel2d", vol_shape=(37, 45), vol_spacing=(1.0, 0.9), nu=61, du=1.1,
                            views=23, range=math.pi, ou=0.3), 2),
    Case("fan2d", dict(kind="fan2d", vol_shape=(41, 39), vol_spacing=(0.5, 0.55), nu=77, du=1.0, views=29,
                       range=2 * math.pi, sid=100.0, sdd=150.0, ou=-0.4), 2),
    Case("cone", dict(kind="cone", vol_shape=(21, 26, 30), vol_spacing=(0.5, 0.5, 0.5), det_shape=(19, 37),
                      det_spacing=(0.6, 0.6), views=13, range=2 * math.pi, sid=75.0, sdd=120.0,
                      det_offset=(0.7, -0.5)), 3),
    Case("cone_aniso_offset", dict(kind="cone", vol_shape=(18, 25, 22), vol_spacing=(0.6, 0.4, 0.5),
                                   det_shape=(23, 29), det_spacing=(0.7, 0.55), views=11, range=1.5 * math.pi,
                                   sid=60.0, sdd=100.0, vol_offset=(0.8, -0.6, 0.3)), 3),
    Case("helical", dict(kind="cone", vol_shape=(24, 20, 20), vol_spacing=(0.5, 0.5, 0.5), det_shape=(17, 33),
                         det_spacing=(0.6, 0.6), views=17, range=2 * math.pi, sid=75.0, sdd=120.0, pitch=6.0), 3),
    Case("cone_tma_rows", dict(kind="cone", vol_shape=(19, 23, 32), vol_spacing=(0.45, 0.5, 0.5), det_shape=(21, 35),
                               det_spacing=(0.55, 0.6), views=10, range=2 * math.pi, sid=70.0, sdd=115.0,
                               det_offset=(-0.4, 0.9)), 3),
    Case("jittered_positions", dict(kind="positions", vol_shape=(20, 22, 24), vol_spacing=(0.5, 0.5, 0.5),
                                    det_shape=(21, 27), det_spacing=(0.6, 0.6), views=9, range=2 * math.pi,
                                    sid=75.0, sdd=120.0, sigma_mm=0.5, sigma_deg=0.2, seed=5), 3),
]

def _aligned(case: Case) -> Case:
    """The same 3D geometry with the detector widened to a multiple of 8 pixels (rows of whole 16-byte
    groups in every storage type), so that the kernels that copy detector boxes with tensor copies apply."""
    p = dict(case.params)
    nv, nu = p["det_shape"]
    p["det_shape"] = (nv, (nu + 7) // 8 * 8)
    return Case(case.name + "_det8", p, case.ndim)


# Small 3D cases whose detector rows are whole 16-byte groups.
SMALL_DET8 = [_aligned(c) for c in SMALL if c.ndim == 3]

# The workloads of the benchmark configurations (full sizes).
CFG1 = Case("cfg1_parallel2d", dict(kind="parallel2d", vol_shape=(128, 128), vol_spacing=(1.0, 1.0), nu=183, du=1.0,
                                    views=180, range=math.pi), 2)
CFG2 = Case("cfg2_fan2d", dict(kind="fan2d", vol_shape=(256, 256), vol_spacing=(0.5, 0.5), nu=512, du=1.0,
                               views=360, range=2 * math.pi, sid=1000.0, sdd=1500.0), 2)
CFG3 = Case("cfg3_cone256", dict(kind="cone", vol_shape=(256, 256, 256), vol_spacing=(0.5, 0.5, 0.5),
                                 det_shape=(512, 512), det_spacing=(0.6, 0.6), views=360, range=2 * math.pi,
                                 sid=750.0, sdd=1200.0), 3)
CFG5 = Case("cfg5_cone512_jitter", dict(kind="positions", vol_shape=(512, 512, 512), vol_spacing=(0.4, 0.4, 0.4),
                                        det_shape=(1024, 1024), det_spacing=(0.4, 0.4), views=720, range=2 * math.pi,
                                        sid=750.0, sdd=1200.0, sigma_mm=0.5, sigma_deg=0.2, seed=5), 3)


def cfg_phantom(case: Case) -> np.ndarray:
    """The configuration's phantom: 10 ellipses (2D) or 20 ellipsoids (3D), seeded per configuration."""
    p = case.params
    seed = {"cfg1_parallel2d": 1, "cfg2_fan2d": 2, "cfg3_cone256": 3, "cfg5_cone512_jitter": 5}[case.name]
    if case.ndim == 2:
        half = 0.5 * p["vol_shape"][0] * p["vol_spacing"][0]
        return inputs.rasterise_ellipses(inputs.random_ellipses(10, half, seed), p["vol_shape"], p["vol_spacing"])
    half = 0.5 * p["vol_shape"][0] * p["vol_spacing"][0]
    return inputs.rasterise_ellipsoids(inputs.random_ellipsoids(20, half, seed), p["vol_shape"], p["vol_spacing"])


def rel_l2(a, b) -> float:
    a = np.asarray(a, dtype=np.float64).ravel()
    b = np.asarray(b, dtype=np.float64).ravel()
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / (nb if nb > 0 else 1.0))

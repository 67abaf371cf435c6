"""Filtered back-projection on the GPU (pyronn_fbp_filter + the voxel-driven BP) against the FP64
oracle: every small geometry and both filters, the 2D configurations at full size, in-place
filtering, BF16 storage, and an FDK reconstruction of an analytic ball."""
import math

import numpy as np
import pytest
import torch

import oracle
from paper_2511_08427_gb300 import inputs

from cases import CFG1, CFG2, SMALL, cfg_phantom, rel_l2

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


@pytest.fixture(scope="module")
def ops():
    from paper_2511_08427_gb300 import build
    build.build()
    from paper_2511_08427_gb300 import operators
    return operators


def host(t):
    return t.detach().float().cpu().numpy().astype(np.float64)


def lib_sino(case, a):
    og = case.oracle_geometry()
    return torch.from_numpy(np.ascontiguousarray(a, np.float32).reshape((og.n_views, -1) if case.ndim == 2
                                                                          else og.sino_shape)).to(DEV)


@pytest.mark.parametrize("filt", [0, 1])
@pytest.mark.parametrize("case", SMALL, ids=lambda c: c.name)
def test_fbp_filter_matches_oracle(ops, case, filt):
    g = case.library_geometry()
    og = case.oracle_geometry()
    y = inputs.uniform(og.sino_shape, seed=60)
    q = host(ops.fbp_filter(lib_sino(case, y), g, filt))
    assert rel_l2(q.ravel(), oracle.fbp_filter(og, y, filt).ravel()) <= 1e-5


@pytest.mark.parametrize("case", [CFG1, CFG2], ids=lambda c: c.name)
def test_fbp_2d_configs_full(ops, case):
    """Projection of the configuration's phantom by the oracle, reconstruction on the GPU vs the oracle."""
    g = case.library_geometry()
    og = case.oracle_geometry()
    p = oracle.fp(og, cfg_phantom(case))
    rec = host(ops.fbp(lib_sino(case, p), g))
    assert rel_l2(rec.ravel(), oracle.fbp(og, p).ravel()) <= 1e-5


def test_fbp_filter_in_place_and_bf16(ops):
    case = next(c for c in SMALL if c.name == "cone")
    g = case.library_geometry()
    og = case.oracle_geometry()
    y = inputs.uniform(og.sino_shape, seed=61)
    ref = oracle.fbp_filter(og, y)
    s = lib_sino(case, y)
    ops.fbp_filter(s, g, out=s)
    assert rel_l2(host(s).ravel(), ref.ravel()) <= 1e-5
    sb = lib_sino(case, y).bfloat16()
    qb = host(ops.fbp_filter(sb, g))
    assert rel_l2(qb.ravel(), oracle.fbp_filter(og, host(sb)).ravel()) <= 4e-3


def test_fdk_reconstructs_an_analytic_ball(ops):
    n, nd, views, R, sid, sdd, du = 64, 128, 360, 18.0, 300.0, 600.0, 1.0
    g = ops.Geometry.cone_circular((n, n, n), (1.0, 1.0, 1.0), (nd, nd), (du, du), views, 2 * math.pi, sid, sdd)
    og = oracle.cone_circular((n, n, n), (1.0, 1.0, 1.0), (nd, nd), (du, du), views, 2 * math.pi, sid, sdd)
    p = np.zeros(og.sino_shape)
    uu, vv = np.meshgrid(np.arange(nd), np.arange(nd), indexing="xy")
    for k in range(views):
        t = k * 2 * math.pi / views
        S = np.array([sid * math.cos(t), sid * math.sin(t), 0.0])
        Dc = -(sdd - sid) * np.array([math.cos(t), math.sin(t), 0.0])
        eu, ev = np.array([-math.sin(t), math.cos(t), 0.0]), np.array([0.0, 0.0, 1.0])
        P = Dc + ((uu - (nd - 1) / 2) * du)[..., None] * eu + ((vv - (nd - 1) / 2) * du)[..., None] * ev
        d = P - S
        d /= np.linalg.norm(d, axis=-1, keepdims=True)
        tt = -(d * S).sum(-1)
        p[k] = 2.0 * np.sqrt(np.maximum(R * R - np.maximum((S * S).sum() - tt * tt, 0.0), 0.0))
    rec = host(ops.fbp(torch.from_numpy(p.astype(np.float32)).to(DEV), g))
    mid = rec[n // 2 - 1:n // 2 + 1].mean(axis=0)
    yy, xx = np.meshgrid(np.arange(n) - (n - 1) / 2, np.arange(n) - (n - 1) / 2, indexing="ij")
    r = np.hypot(xx, yy)
    assert abs(mid[r < R - 3].mean() - 1.0) < 0.02
    assert abs(mid[r > R + 3].mean()) < 0.02
    vids = np.random.default_rng(3).choice(n ** 3, size=400, replace=False)
    ref = oracle.bp_voxels(og, oracle.fbp_filter(og, p.astype(np.float32)), vids, 1)
    assert rel_l2(rec.ravel()[vids], ref) <= 1e-5


def test_fdk_error_decreases_with_views(ops):
    """FDK of a random-ellipsoid phantom (128^3 at 0.5 mm, circular cone beam, SID 750 / SDD 1200): the
    reconstruction error against the phantom, over the central slices inside the scanned cylinder,
    falls as the number of views goes from 90 to 180 to 360 (fewer angular-undersampling streaks)."""
    n, sp = 128, 0.5
    x = inputs.rasterise_ellipsoids(inputs.random_ellipsoids(12, 0.5 * n * sp, 21), (n, n, n), (sp, sp, sp))
    xt = torch.from_numpy(x).to(DEV)
    zz, yy, xx = np.meshgrid(*(np.arange(n) - (n - 1) / 2,) * 3, indexing="ij")
    mask = (np.abs(zz) < 8) & (np.hypot(xx, yy) < 0.4 * n)
    errs = []
    for views in (90, 180, 360):
        g = ops.Geometry.cone_circular((n, n, n), (sp,) * 3, (256, 256), (0.6, 0.6), views, 2 * math.pi, 750.0, 1200.0)
        with torch.no_grad():
            rec = host(ops.fbp(ops.forward_project(xt, g), g))
        errs.append(float(np.linalg.norm((rec - x)[mask]) / np.linalg.norm(x[mask])))
    print("FDK rel-L2 against the phantom, 90 / 180 / 360 views:", ", ".join(f"{e:.4f}" for e in errs))
    assert errs[0] > errs[1] > errs[2]
    assert errs[2] < 0.5


def test_listing1_fdk_pipeline(ops):
    """Listing 1's filtered back-projection (Sec. 2.3) with the listing's parameters (read from the
    golden file): a 256^3 volume at 0.5 mm, 400 x 600 detector at 1 mm, 360 views over 2 pi, SDD 1200,
    SID 750. A random-ellipsoid phantom replaces the listing's Shepp-Logan phantom; it is projected with
    the ConeProjectionFor3D layer, filtered (cosine weights, ramp) and back-projected with the
    ConeBackProjectionFor3D layer (1/w^2 weights). The reconstruction matches the oracle's FDK on sampled
    voxels and approximates the phantom; its error is printed."""
    import json
    import os
    prm = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "listing1_params.json")))
    shape, spacing = tuple(prm["volume_shape"]), tuple(float(s) for s in prm["volume_spacing"])
    det, dsp = tuple(prm["detector_shape"]), tuple(float(s) for s in prm["detector_spacing"])
    V, sdd, sid = prm["number_of_projections"], float(prm["sdd"]), float(prm["sid"])
    assert prm["angular_range"] == "2*pi"
    g = ops.Geometry.cone_circular(shape, spacing, det, dsp, V, 2 * math.pi, sid, sdd)
    og = oracle.cone_circular(shape, spacing, det, dsp, V, 2 * math.pi, sid, sdd)
    x = inputs.rasterise_ellipsoids(inputs.random_ellipsoids(20, 0.5 * shape[0] * spacing[0], 17), shape, spacing)
    with torch.no_grad():
        sino = ops.ConeProjectionFor3D()(torch.from_numpy(x).to(DEV), g)
        filtered = ops.fbp_filter(sino, g)
        rec = ops.ConeBackProjectionFor3D(ops.BP_INV_W2)(filtered, g)
    rec = host(rec)
    # the filter is compared with the oracle's on every geometry above; here the sampled rays of the
    # projection and the back-projection of the GPU-filtered sinogram
    rng = np.random.default_rng(9)
    rids = rng.choice(sino.numel(), size=500, replace=False)
    assert rel_l2(host(sino).ravel()[rids], oracle.fp_rays(og, x, rids)) <= 1e-5
    vids = rng.choice(x.size, size=300, replace=False)
    ref = oracle.bp_voxels(og, host(filtered), vids, 1)
    assert rel_l2(rec.ravel()[vids], ref) <= 1e-5
    zz, yy, xx = np.meshgrid(*(np.arange(n) - (n - 1) / 2 for n in shape), indexing="ij")
    mask = (np.abs(zz) < 16) & (np.hypot(xx, yy) < 0.4 * shape[1])
    err = float(np.linalg.norm((rec - x)[mask]) / np.linalg.norm(x[mask]))
    print(f"Listing 1 FDK: rel-L2 against the phantom over the central slices {err:.4f}")
    assert err < 0.5

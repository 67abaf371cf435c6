"""Batched plans (one persistent launch per operator over volumes with their own sizes and
geometries) against the per-geometry operators and the FP64 oracle, and under CUDA-graph capture."""
import math

import numpy as np
import pytest
import torch

import oracle
from paper_2511_08427_gb300 import inputs

from cases import rel_l2

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


@pytest.fixture(scope="module")
def ops():
    from paper_2511_08427_gb300 import build
    build.build()
    from paper_2511_08427_gb300 import operators
    return operators


def small_batch(ops):
    """Four volumes: circular / helical / jittered-positions cone beams of different sizes, one with
    rows that are not a multiple of 16 bytes (forward projection outside the persistent launch)."""
    specs = [
        dict(kind="circ", shape=(20, 24, 32), sp=0.5, det=(19, 37), V=11, pitch=0.0),
        dict(kind="circ", shape=(24, 28, 24), sp=0.45, det=(23, 29), V=9, pitch=5.0),
        dict(kind="pos", shape=(16, 20, 40), sp=0.5, det=(21, 35), V=7),
        dict(kind="circ", shape=(18, 22, 26), sp=0.5, det=(17, 31), V=8, pitch=0.0),
    ]
    lib_g, ora_g, vols = [], [], []
    for k, s in enumerate(specs):
        spz = (s["sp"],) * 3
        if s["kind"] == "circ":
            lib_g.append(ops.Geometry.cone_circular(s["shape"], spz, s["det"], (0.6, 0.6), s["V"], 2 * math.pi, 75.0,
                                                    120.0, helical_pitch=s["pitch"]))
            ora_g.append(oracle.cone_circular(s["shape"], spz, s["det"], (0.6, 0.6), s["V"], 2 * math.pi, 75.0, 120.0,
                                              pitch=s["pitch"]))
        else:
            tr = inputs.jittered_circular_trajectory(s["V"], 2 * math.pi, 75.0, 120.0, 0.5, 0.2, seed=5)
            lib_g.append(ops.Geometry.cone_from_positions(s["shape"], spz, s["det"], (0.6, 0.6), tr.src,
                                                          tr.det_centre, tr.eu, tr.ev))
            ora_g.append(oracle.cone_from_positions(s["shape"], spz, s["det"], (0.6, 0.6), tr.src, tr.det_centre,
                                                    tr.eu, tr.ev))
        half = 0.5 * min(a * s["sp"] for a in s["shape"])
        vols.append(inputs.rasterise_ellipsoids(inputs.random_ellipsoids(8, half, 10 + k), s["shape"], spz))
    return lib_g, ora_g, vols


def host(t):
    return t.float().cpu().numpy().astype(np.float64)


def test_plan_matches_single_operators_and_oracle(ops):
    lib_g, ora_g, vols = small_batch(ops)
    plan = ops.Plan(lib_g)
    info = plan.info()
    assert info["n"] == 4 and min(info["grids"]) > 0
    xs = [torch.from_numpy(v).to(DEV) for v in vols]
    sinos = [torch.full(g.sinogram_shape, float("nan"), device=DEV) for g in lib_g]
    plan.forward_project(xs, sinos)
    ys = [torch.from_numpy(inputs.gaussian(g.sinogram_shape, seed=30 + i)).to(DEV) for i, g in enumerate(lib_g)]
    adj = [torch.full(g.volume_shape, float("nan"), device=DEV) for g in lib_g]
    plan.adjoint(ys, adj)
    bps = [torch.full(g.volume_shape, float("nan"), device=DEV) for g in lib_g]
    plan.back_project(ys, bps, weight=1)
    torch.cuda.synchronize()
    for i, (g, og) in enumerate(zip(lib_g, ora_g)):
        ref_fp = ops.forward_project(xs[i], g)
        assert rel_l2(host(sinos[i]), host(ref_fp)) <= 1e-6, i
        assert rel_l2(host(sinos[i]), oracle.fp(og, vols[i])) <= 1e-5, i
        # the plan's persistent slab adjoint and the single-geometry launch add the boxes to the volume
        # in different orders: both within the oracle tolerance
        assert rel_l2(host(adj[i]), host(ops.adjoint(ys[i], g))) <= 1e-5, i
        assert rel_l2(host(adj[i]), oracle.adjoint(og, host(ys[i]))) <= 1e-5, i
        assert rel_l2(host(bps[i]), host(ops.back_project(ys[i], g, 1))) <= 1e-6, i
        assert rel_l2(host(bps[i]), oracle.bp(og, host(ys[i]), 1)) <= 1e-5, i
        assert g.read_flags()[:4] == [0, 0, 0, 0]


def test_plan_bf16_storage(ops):
    lib_g, ora_g, vols = small_batch(ops)
    plan = ops.Plan(lib_g, dtype=torch.bfloat16)
    xs = [torch.from_numpy(v).to(DEV).to(torch.bfloat16) for v in vols]
    sinos = [torch.empty(g.sinogram_shape, device=DEV, dtype=torch.bfloat16) for g in lib_g]
    plan.forward_project(xs, sinos)
    adj = [torch.empty(g.volume_shape, device=DEV, dtype=torch.bfloat16) for g in lib_g]
    plan.adjoint(sinos, adj)
    torch.cuda.synchronize()
    for i, og in enumerate(ora_g):
        assert rel_l2(host(sinos[i]), oracle.fp(og, host(xs[i]))) <= 4e-3, i
        assert rel_l2(host(adj[i]), oracle.adjoint(og, host(sinos[i]))) <= 4e-3, i


def test_plan_mixes_y_fastest_and_plain_staging(ops):
    """One persistent FP launch over volumes whose x-march slabs come from a y-fastest copy and volumes
    staged from the volume itself (PYRONN_TUNE_FP_TRANSPOSE set per geometry before the plan is made):
    every volume matches its per-geometry projection."""
    lib_g, _, vols = small_batch(ops)
    for i, g in enumerate(lib_g):
        g.set_tuning(ops.TUNE_FP_TRANSPOSE, i % 2)
    assert any(g.fp_config()["y_fastest_x_march"] for g in lib_g)
    assert any(g.fp_config()["kernel"] == 3 and not g.fp_config()["y_fastest_x_march"] for g in lib_g)
    plan = ops.Plan(lib_g)
    xs = [torch.from_numpy(v).to(DEV) for v in vols]
    sinos = [torch.full(g.sinogram_shape, float("nan"), device=DEV) for g in lib_g]
    plan.forward_project(xs, sinos)
    torch.cuda.synchronize()
    for i, g in enumerate(lib_g):
        assert rel_l2(host(sinos[i]), host(ops.forward_project(xs[i], g))) <= 1e-6, i


def test_plan_under_cuda_graph(ops):
    lib_g, _, vols = small_batch(ops)
    plan = ops.Plan(lib_g)
    xs = [torch.from_numpy(v).to(DEV) for v in vols]
    sinos = [torch.empty(g.sinogram_shape, device=DEV) for g in lib_g]
    adj = [torch.empty(g.volume_shape, device=DEV) for g in lib_g]
    plan.forward_project(xs, sinos)    # warm-up outside capture
    plan.adjoint(sinos, adj)
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        with torch.cuda.graph(graph, stream=s):
            plan.forward_project(xs, sinos)
            plan.adjoint(sinos, adj)
    torch.cuda.current_stream().wait_stream(s)
    for rep in range(2):
        for i, x in enumerate(xs):
            x.copy_(torch.from_numpy(inputs.rasterise_ellipsoids(inputs.random_ellipsoids(6, 4.0, 50 + 10 * rep + i),
                                                                 tuple(x.shape), (0.5,) * 3)).to(DEV))
        graph.replay()
        torch.cuda.synchronize()
        for i, g in enumerate(lib_g):
            ref = ops.forward_project(xs[i], g)
            assert rel_l2(host(sinos[i]), host(ref)) <= 1e-6
            assert rel_l2(host(adj[i]), host(ops.adjoint(ref, g))) <= 1e-5


def test_batched_workload_16_volumes(ops):
    """The 16-volume uneven workload (96^3 ... 256^3, circular / helical, 180-540 views, 256^2-512^2
    detectors) through plans in FP32 and BF16 storage, against the oracle per volume: sampled rays of
    the forward projection, the matched adjoint of a sparse cotangent over the whole volume, and
    sampled voxels of the voxel-driven back-projection of the plan's sinogram (the oracle reads the same,
    rounded, inputs). FP32 plans also equal the per-geometry operators. The per-volume errors are
    printed."""
    from paper_2511_08427_gb300.inputs import batched_cone_workload
    specs = batched_cone_workload()
    lib_g, ora_g, vols = [], [], []
    for w in specs:
        n = w["side"]
        sp = (w["voxel_mm"],) * 3
        lib_g.append(ops.Geometry.cone_circular((n, n, n), sp, (w["det"], w["det"]), (w["du"], w["du"]), w["views"],
                                                w["angular_range"], w["sid"], w["sdd"], helical_pitch=w["pitch"]))
        ora_g.append(oracle.cone_circular((n, n, n), sp, (w["det"], w["det"]), (w["du"], w["du"]), w["views"],
                                          w["angular_range"], w["sid"], w["sdd"], pitch=w["pitch"]))
        vols.append(inputs.rasterise_ellipsoids(inputs.random_ellipsoids(20, 0.5 * n * w["voxel_mm"], w["seed"]),
                                                (n, n, n), sp))
    tol = {torch.float32: 1e-5, torch.bfloat16: 4e-3}
    rng = np.random.default_rng(0)
    for dtype in (torch.float32, torch.bfloat16):
        plan = ops.Plan(lib_g, dtype=dtype)
        xs = [torch.from_numpy(v).to(DEV).to(dtype) for v in vols]
        sinos = [torch.empty(g.sinogram_shape, device=DEV, dtype=dtype) for g in lib_g]
        plan.forward_project(xs, sinos)
        # sparse cotangents: 200 random rays per volume
        ys, picks = [], []
        for g, og in zip(lib_g, ora_g):
            nr = og.n_views * og.det_shape[0] * og.det_shape[1]
            ids = np.sort(rng.choice(nr, size=200, replace=False))
            vals = rng.standard_normal(ids.size).astype(np.float32)
            y = torch.zeros(nr, device=DEV, dtype=dtype)
            y[torch.from_numpy(ids).to(DEV)] = torch.from_numpy(vals).to(DEV).to(dtype)
            ys.append(y.view(g.sinogram_shape))
            picks.append((ids, y.float().cpu().numpy()[ids].astype(np.float64)))
        adj = [torch.empty(g.volume_shape, device=DEV, dtype=dtype) for g in lib_g]
        plan.adjoint(ys, adj)
        bps = [torch.empty(g.volume_shape, device=DEV, dtype=dtype) for g in lib_g]
        plan.back_project(sinos, bps)
        torch.cuda.synchronize()
        rows = []
        for i, (g, og) in enumerate(zip(lib_g, ora_g)):
            xh = host(xs[i])
            nr = og.n_views * og.det_shape[0] * og.det_shape[1]
            rid = rng.choice(nr, size=150, replace=False)
            e_fp = rel_l2(host(sinos[i]).ravel()[rid], oracle.fp_rays(og, xh, rid))
            e_adj = rel_l2(host(adj[i]), oracle.adjoint_rays(og, picks[i][0], picks[i][1]))
            vid = rng.choice(xh.size, size=300, replace=False)
            e_bp = rel_l2(host(bps[i]).ravel()[vid], oracle.bp_voxels(og, host(sinos[i]), vid, 0))
            rows.append((i, e_fp, e_adj, e_bp))
            if dtype == torch.float32:
                assert torch.equal(sinos[i], ops.forward_project(xs[i], g)), i
            assert e_fp <= tol[dtype] and e_adj <= tol[dtype] and e_bp <= tol[dtype], (dtype, rows[-1])
        print(f"16-volume plan, {dtype}: per-volume rel-L2 against the oracle (FP rays / adjoint / BP voxels)")
        for i, a, b, c in rows:
            print(f"  volume {i:2d} ({specs[i]['side']}^3, {specs[i]['views']} views): {a:.2e} {b:.2e} {c:.2e}")
        del plan, xs, sinos, ys, adj, bps
        torch.cuda.empty_cache()

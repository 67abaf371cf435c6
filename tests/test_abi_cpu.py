"""CPU-side checks of the C ABI (no kernel launches): the library loads and exports every entry
point that include/pyronn.h declares, the host geometry code matches the FP64 oracle's
geometry, the sample count matches the oracle's count, and invalid arguments are rejected."""
import ctypes
import math
import os
import re

import numpy as np
import pytest

import oracle
from paper_2511_08427_gb300 import _lib, inputs

from cases import SMALL, Case

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    from paper_2511_08427_gb300 import build
    build.build()
    return _lib.lib()


def declared_symbols():
    text = open(os.path.join(ROOT, "include", "pyronn.h")).read()
    return sorted(set(re.findall(r"PYRONN_API\s+(?:const\s+char\s*\*|int)\s*(pyronn_\w+)\s*\(", text)))


def test_every_declared_symbol_is_exported(L):
    decl = declared_symbols()
    assert len(decl) >= 20
    for name in decl:
        assert hasattr(L, name), name
    # and the binding marshals exactly the declared set
    assert sorted(_lib.exported_symbols()) == decl


def test_version_and_error_string(L):
    assert L.pyronn_version() >= 100
    assert isinstance(L.pyronn_last_error(), bytes)


@pytest.mark.parametrize("case", SMALL, ids=lambda c: c.name)
def test_library_views_match_oracle(L, case: Case):
    g = case.library_geometry()
    og = case.oracle_geometry()
    assert g.kind == og.kind
    assert np.allclose(g.views(), og.views, rtol=1e-12, atol=1e-12)
    assert abs(g.step - og.dt) < 1e-15


@pytest.mark.parametrize("case", SMALL, ids=lambda c: c.name)
def test_sample_count_matches_oracle(L, case: Case):
    g = case.library_geometry()
    og = case.oracle_geometry()
    assert g.count_samples() == int(oracle.count_samples(og).sum())


def test_matrices_paths_match_oracle(L):
    from paper_2511_08427_gb300.operators import Geometry
    vs, sp, ds, dsp = (10, 12, 14), (0.5, 0.6, 0.7), (9, 11), (0.8, 0.9)
    og = oracle.cone_circular(vs, sp, ds, dsp, 7, 2 * math.pi, 70.0, 110.0)
    scale = np.linspace(-3.0, 5.0, 7)
    scale[scale == 0] = 1.0
    g = Geometry.cone_from_matrices(vs, sp, ds, dsp, og.views * scale[:, None])
    assert np.allclose(g.views(), og.views, rtol=1e-12, atol=1e-13)
    # 2D fan from 2 x 3 matrices: the (u, w) rows of the 3D fan embedding
    of = oracle.fan_circular((20, 22), (0.5, 0.5), 31, 1.0, 5, 2 * math.pi, 100.0, 150.0)
    P2 = of.views.reshape(-1, 3, 4)[:, [0, 2], :][:, :, [0, 1, 3]] * 2.5
    gf = Geometry.from_matrices2d((20, 22), (0.5, 0.5), 31, 1.0, P2)
    assert gf.kind == 1
    assert np.allclose(gf.views(), of.views, rtol=1e-12, atol=1e-13)
    # 2D parallel from affine 2 x 3 matrices u = (X . eu) / du + (Nu - 1) / 2 - ou / du
    op = oracle.parallel2d((20, 22), (0.5, 0.5), 31, 0.8, 6, math.pi, det_offset=0.25)
    rows = []
    for n in range(6):
        eu = op.views[n, 3:5]
        rows.append([[eu[0] / 0.8, eu[1] / 0.8, 15.0 - 0.25 / 0.8], [0.0, 0.0, 1.0]])
    gp = Geometry.from_matrices2d((20, 22), (0.5, 0.5), 31, 0.8, np.array(rows))
    assert gp.kind == 0
    v = gp.views()
    # same rays (origin line and direction up to sign) as the oracle's parallel geometry
    for n in range(6):
        eu, d = v[n, 3:6], v[n, 9:12]
        assert np.allclose(eu, op.views[n, 3:6], atol=1e-12)
        assert abs(abs(np.dot(d, op.views[n, 9:12])) - 1.0) < 1e-12
        # the detector-centre offsets agree along eu
        assert abs(np.dot(v[n, 0:3], eu) - (np.dot(op.views[n, 0:3], eu) + 0.25)) < 1e-12


def test_positions_path_matches_oracle(L):
    from paper_2511_08427_gb300.operators import Geometry
    tr = inputs.jittered_circular_trajectory(8, 2 * math.pi, 750.0, 1200.0, 0.5, 0.2, seed=5)
    vs, sp, ds, dsp = (16, 16, 16), (0.4, 0.4, 0.4), (12, 14), (0.4, 0.4)
    g = Geometry.cone_from_positions(vs, sp, ds, dsp, tr.src, tr.det_centre, tr.eu, tr.ev)
    og = oracle.cone_from_positions(vs, sp, ds, dsp, tr.src, tr.det_centre, tr.eu, tr.ev)
    assert np.allclose(g.views(), og.views, rtol=1e-12, atol=1e-12)


def test_invalid_arguments_are_rejected(L):
    from paper_2511_08427_gb300.operators import Geometry
    with pytest.raises(_lib.PyronnError) as e:
        Geometry.cone_circular((0, 4, 4), (1, 1, 1), (4, 4), (1, 1), 3, 1.0, 10.0, 20.0)
    assert e.value.code == -1
    with pytest.raises(_lib.PyronnError):
        Geometry.cone_circular((4, 4, 4), (1, 1, 1), (4, 4), (1, 1), 3, 1.0, 30.0, 20.0)   # sdd < sid
    with pytest.raises(_lib.PyronnError) as e:
        Geometry.cone_from_matrices((4, 4, 4), (1, 1, 1), (4, 4), (1, 1), np.zeros((2, 12)))
    assert e.value.code == -6
    g = Geometry.cone_circular((4, 4, 4), (1, 1, 1), (4, 4), (1, 1), 3, 1.0, 10.0, 20.0)
    with pytest.raises(_lib.PyronnError):
        g.step = -1.0
    with pytest.raises(_lib.PyronnError):
        g.set_variant(0, 7)
    # operator calls validate before touching the device
    assert L.pyronn_fp(g.handle, None, None, 0, 1, None) != 0
    assert L.pyronn_fp(g.handle, ctypes.c_void_p(16), ctypes.c_void_p(32), 9, 1, None) == -2
    assert L.pyronn_bp(None, None, None, 0, 1, 0, None) == -1
    assert b"null" in L.pyronn_last_error()


def test_values_outside_the_device_tables_are_rejected(L):
    """Non-finite offsets, spacings whose value or reciprocal is not finite in FP32, orbits whose
    FP32 view tables would overflow, and steps that give more than 2^22 samples across the volume are
    rejected at create / set time with INVALID_ARG; a step of 2^16 voxels or more is accepted and
    routed to the generic projector and adjoint instead of the slab-staged ones."""
    from paper_2511_08427_gb300.operators import Geometry
    nan, inf = float("nan"), float("inf")
    bad = [dict(volume_offset=(0.0, nan, 0.0)), dict(volume_offset=(inf, 0.0, 0.0)),
           dict(detector_offset=(0.0, nan)), dict(volume_spacing=(1.0, 1e-300, 1.0)),
           dict(volume_spacing=(1e300, 1.0, 1.0)), dict(detector_spacing=(1.0, 1e-60)),
           dict(sid=1e300, sdd=2e300)]
    for kw in bad:
        args = dict(volume_shape=(8, 8, 8), volume_spacing=(1.0, 1.0, 1.0), detector_shape=(8, 8),
                    detector_spacing=(1.0, 1.0), number_of_projections=3, angular_range=2 * math.pi,
                    sid=100.0, sdd=200.0)
        args.update(kw)
        with pytest.raises(_lib.PyronnError) as e:
            Geometry.cone_circular(**args)
        assert e.value.code == -1, kw
    g = Geometry.cone_circular((8, 16, 16), (1.0, 1.0, 1.0), (8, 8), (1.0, 1.0), 3, 2 * math.pi, 100.0, 200.0)
    diag = math.sqrt(17 ** 2 + 17 ** 2 + 9 ** 2)           # support box (-1, N) on every axis, in mm
    with pytest.raises(_lib.PyronnError) as e:
        g.step = diag / 2 ** 22 * 0.99
    assert e.value.code == -1 and b"2^22" in L.pyronn_last_error()
    g.step = diag / 2 ** 22 * 1.01
    assert g.count_samples() > 0
    g.step = 0.5
    assert g.fp_config()["kernel"] in (2, 3) and g.adjoint_config()["kernel"] == 3
    g.step = 70000.0                                         # more than 2^16 voxels per sample
    assert g.fp_config()["kernel"] == 1 and g.adjoint_config()["kernel"] == 2
    assert g.count_samples() <= 3 * 8 * 8                    # at most one sample per ray


def test_step_changes_sample_count(L):
    from paper_2511_08427_gb300.operators import Geometry
    g = Geometry.parallel2d((8, 20), (1.0, 1.0), 5, 1.0, 1)
    assert g.count_samples() == 5 * (2 * 20 + 2)     # closed form of the symmetric lattice
    g.step = 0.25
    assert g.count_samples() == 5 * (4 * 20 + 4)


@pytest.mark.parametrize("dtype_size,dtype", [(4, "float32"), (2, "bfloat16")])
def test_fp_config_invariants(L, dtype_size, dtype):
    """TMA boxes: at most 256 per dimension, innermost extent a multiple of 16 bytes (x, or y for
    x-march boxes staged from the y-fastest copy), first slab plane minus the guard aligned (so
    x-march boxes of the x-fastest volume start aligned), double buffer within 200 KB."""
    import torch
    from paper_2511_08427_gb300.operators import TUNE_BP_BRICK_Z, TUNE_FP_TRANSPOSE, Geometry
    td = getattr(torch, dtype)
    g = Geometry.cone_circular((64, 96, 128), (0.5, 0.5, 0.5), (100, 130), (0.6, 0.6), 40, 2 * math.pi, 750.0, 1200.0)
    for transpose in (0, 1):
        g.set_tuning(TUNE_FP_TRANSPOSE, transpose)
        c = g.fp_config(td)
        assert c["kernel"] == 3
        assert c["y_fastest_x_march"] == (transpose == 0)     # ny * dtype_size is a multiple of 16
        align = 16 // dtype_size
        for m, box in enumerate(c["box"]):
            assert all(1 <= e <= 256 for e in box)
            inner = 1 if (m == 0 and c["y_fastest_x_march"]) else 0
            assert (box[inner] * dtype_size) % 16 == 0
        assert (c["slab0"] - c["guard"]) % align == 0
        assert c["smem_bytes"] <= 200 * 1024 + 128
    # a y extent that is not a multiple of 16 bytes keeps x-march boxes on the volume itself
    g3 = Geometry.cone_circular((64, 90, 128), (0.5, 0.5, 0.5), (100, 130), (0.6, 0.6), 8, 2 * math.pi, 750.0, 1200.0)
    assert g3.fp_config(td)["kernel"] == 3 and not g3.fp_config(td)["y_fastest_x_march"]
    # rows that are not a multiple of 16 bytes cannot use tensor copies
    g2 = Geometry.cone_circular((20, 20, 30), (0.5, 0.5, 0.5), (30, 30), (0.6, 0.6), 8, 2 * math.pi, 75.0, 120.0)
    assert g2.fp_config(td)["kernel"] == 2
    g2.set_variant(0, 1)
    assert g2.fp_config(td)["kernel"] == 1


def test_config_invariants_over_random_geometries(L):
    """The TMA alignment and shared-memory budgets hold for every geometry, not only the hand-picked
    ones: 120 seeded random cone geometries (sizes, anisotropic spacings, offsets, helices, detector
    sizes, steps), each storage type and both x-march staging choices. Wherever the TMA projector is
    chosen, x-march boxes start and stay 16-byte aligned along their innermost axis and fit 200 KB;
    wherever the slab adjoint is chosen, its box (at most 160 KB) and slab table fit 200 KB; wherever the
    staged back-projector is chosen, its detector boxes follow the tensor-copy rules."""
    import random
    import torch
    from paper_2511_08427_gb300.operators import TUNE_BP_BRICK_Z, TUNE_FP_TRANSPOSE, Geometry
    rnd = random.Random(2024)
    seen_tma = seen_adj = seen_bp = 0
    for _ in range(120):
        shape = tuple(rnd.choice([8, 12, 16, 24, 32, 40, 48, 64, 96]) for _ in range(3))
        sp = tuple(rnd.choice([0.25, 0.4, 0.5, 0.8, 1.0, 2.0]) for _ in range(3))
        det = (rnd.choice([8, 16, 24, 40, 64]), rnd.choice([8, 16, 33, 64, 100]))
        dsp = (rnd.choice([0.3, 0.6, 1.2]), rnd.choice([0.3, 0.6, 1.2, 3.0]))
        sid = rnd.choice([20.0, 60.0, 150.0, 750.0])
        g = Geometry.cone_circular(shape, sp, det, dsp, rnd.choice([1, 5, 12]), 2 * math.pi, sid,
                                   sid * rnd.choice([1.3, 1.6, 2.5]), helical_pitch=rnd.choice([0.0, 0.0, 6.0]),
                                   volume_offset=tuple(rnd.choice([0.0, 2.5, -4.0]) for _ in range(3)))
        if rnd.random() < 0.5:
            g.step = min(sp) * rnd.choice([0.25, 0.5, 1.0, 2.5])
        for td, size in ((torch.float32, 4), (torch.bfloat16, 2), (torch.float16, 2)):
            align = 16 // size
            for transpose in (0, 1):
                g.set_tuning(TUNE_FP_TRANSPOSE, transpose)
                c = g.fp_config(td)
                if c["kernel"] != 3:
                    assert (shape[2] * size) % 16 != 0 or c["kernel"] in (1, 2)
                    continue
                seen_tma += 1
                assert (shape[2] * size) % 16 == 0
                assert c["depth"] % align == 0 and (c["slab0"] - c["guard"]) % align == 0
                assert c["slab0"] - c["guard"] <= -1 - c["guard"]
                assert c["y_fastest_x_march"] == (transpose == 0 and (shape[1] * size) % 16 == 0)
                for m, box in enumerate(c["box"]):
                    assert all(1 <= e <= 256 for e in box), box
                    inner = 1 if (m == 0 and c["y_fastest_x_march"]) else 0
                    assert (box[inner] * size) % 16 == 0, (m, box)
                assert c["smem_bytes"] <= 200 * 1024 + 128
            g.set_variant(2, 3)
            for bz in (8, 16):
                g.set_tuning(TUNE_BP_BRICK_Z, bz)
                b = g.bp_config(td)
                if b["kernel"] == 3:
                    seen_bp += 1
                    bu, bv = b["box"]
                    # tensor-copy rules: the box's inner extent a multiple of 16 bytes, every extent at
                    # most 256, each view's slot in shared memory a multiple of 128 bytes (its destination
                    # must be 128-byte aligned), two stages within the kernel's shared memory
                    assert b["brick_z"] == bz
                    assert (det[1] * size) % 16 == 0
                    assert (bu * size) % 16 == 0 and 1 <= bu <= 256 and 3 <= bv <= 256
                    assert b["slot_elems"] >= bu * bv and (b["slot_elems"] * size) % 128 == 0
                    assert 1 <= b["views_per_stage"] <= 4
                    assert 2 * b["views_per_stage"] * b["slot_elems"] * size <= 100 * 1024
                else:
                    assert (det[1] * size) % 16 != 0 or b["kernel"] == 2
            g.set_tuning(TUNE_BP_BRICK_Z, 0)
            g.set_variant(2, 0)
        a = g.adjoint_config()
        if a["kernel"] == 3:
            seen_adj += 1
            assert a["depth"] in (8, 6, 5, 4) and a["guard"] >= 1
            assert a["max_slabs"] == (max(shape) + 2 + a["depth"] - 1) // a["depth"]
            # the box itself at most 160 KB; box and slab table within the 200 KB the kernel is given
            assert a["box_floats"] <= 40 * 1024
            assert 4 * ((a["box_floats"] + 3) // 4 * 4) + 104 * a["max_slabs"] <= 200 * 1024
    assert seen_tma > 100 and seen_adj > 60 and seen_bp > 60


def test_adjoint_config_invariants(L):
    """Slab adjoint: the slab table holds every slab of the longest axis at the chosen depth; box and
    table fit the two-CTAs-per-SM budget (112 KB each); the odd x-march pitch is on by default and the
    16-byte pitch (PYRONN_TUNE_ADJ_PITCH = 1) needs no larger box."""
    from paper_2511_08427_gb300.operators import TUNE_ADJ_PITCH, Geometry
    g = Geometry.cone_circular((64, 96, 128), (0.5, 0.5, 0.5), (100, 130), (0.6, 0.6), 40, 2 * math.pi, 750.0, 1200.0)
    c = g.adjoint_config()
    assert c["kernel"] == 3 and c["odd_pitch"]
    assert c["depth"] in (8, 6, 5, 4)
    assert c["max_slabs"] == (128 + 2 + c["depth"] - 1) // c["depth"]
    assert 4 * ((c["box_floats"] + 3) // 4 * 4) + 104 * c["max_slabs"] <= 112 * 1024
    g.set_tuning(TUNE_ADJ_PITCH, 1)
    c1 = g.adjoint_config()
    assert c1["kernel"] == 3 and not c1["odd_pitch"]
    assert c1["depth"] < c["depth"] or c1["box_floats"] <= c["box_floats"]
    g.set_tuning(TUNE_ADJ_PITCH, 0)
    assert g.adjoint_config() == c


def test_argument_checks_precede_the_device(L):
    """Every entry point rejects bad arguments before touching the device (these run without a GPU):
    empty batches, volumes too large for 32-bit indexing, unknown filters, non-finite steps, jitter
    axes and in-place use, blur lengths, ring view ranges."""
    from paper_2511_08427_gb300.operators import Geometry
    g = Geometry.cone_circular((4, 5, 6), (1, 1, 1), (3, 4), (1, 1), 3, 1.0, 10.0, 20.0)
    a, b = ctypes.c_void_p(256), ctypes.c_void_p(512)
    h = g.handle
    assert L.pyronn_fp(h, a, b, 0, 0, None) == -1                       # batch 0
    assert b"batch" in L.pyronn_last_error()
    big = Geometry.cone_circular((1024, 2048, 1024), (1, 1, 1), (4, 4), (1, 1), 2, 1.0, 5000.0, 9000.0)
    assert L.pyronn_adjoint(big.handle, a, b, 0, 1, None) == -1          # 2^31 voxels
    assert b"too large" in L.pyronn_last_error()
    assert L.pyronn_fbp_filter(h, a, b, 7, 0, 1, None) == -1             # unknown filter
    assert L.pyronn_adjoint_update(h, a, None, float("nan"), b, 0, 1, None) == -1
    assert L.pyronn_sim_detector_jitter(h, a, b, a, 2, 0, 1, None) == -1  # axis
    assert L.pyronn_sim_detector_jitter(h, a, a, b, 0, 0, 1, None) == -1  # in place
    assert L.pyronn_sim_motion_blur(h, a, b, a, 0, 0, 1, None) == -1      # length 0
    assert L.pyronn_sim_ring(h, a, b, a, a, 1, 2, 9, 0, 1, None) == -1    # views [2, 9) of 3
    assert L.pyronn_sim_gaussian_noise(h, a, b, None, 0.0, 1.0, 0, 1, None) == -1
    assert L.pyronn_fp(h, ctypes.c_void_p(8), b, 0, 1, None) == -3        # misaligned
    res = (ctypes.c_double * 4)()
    assert L.pyronn_autotune(h, 3, a, b, 0, 2, None, res) == -1          # unknown operator
    assert L.pyronn_autotune(h, 0, a, b, 0, 0, None, res) == -1          # no timed launch
    assert L.pyronn_autotune(h, 1, a, b, 5, 2, None, res) == -2          # unknown element type
    assert L.pyronn_autotune(h, 2, None, b, 0, 2, None, res) == -1       # null buffer
    assert L.pyronn_autotune(h, 2, a, b, 0, 2, None, None) == -1         # null result


def test_tuning_knobs_of_the_autotuner(L):
    """The knobs pyronn_autotune sets: an adjoint slab depth is taken as given (two CTAs per SM where its
    box fits, one otherwise), 0 restores the automatic choice, and out-of-range values are refused."""
    from paper_2511_08427_gb300 import PyronnError
    from paper_2511_08427_gb300.operators import TUNE_ADJ_DEPTH, TUNE_BP_BRICK_Z, Geometry
    g = Geometry.cone_circular((64, 96, 128), (0.5, 0.5, 0.5), (100, 130), (0.6, 0.6), 40, 2 * math.pi, 750.0, 1200.0)
    auto = g.adjoint_config()
    for d in (3, 4, 5, 6, 8):
        g.set_tuning(TUNE_ADJ_DEPTH, d)
        c = g.adjoint_config()
        assert c["kernel"] == 3 and c["depth"] == d
        assert c["max_slabs"] == (128 + 2 + d - 1) // d
    g.set_tuning(TUNE_ADJ_DEPTH, 0)
    assert g.adjoint_config() == auto
    for knob, bad in ((TUNE_ADJ_DEPTH, 1), (TUNE_ADJ_DEPTH, 17), (TUNE_BP_BRICK_Z, 5), (TUNE_BP_BRICK_Z, 32)):
        with pytest.raises(PyronnError):
            g.set_tuning(knob, bad)
    for bz in (0, 4, 8, 16):
        g.set_tuning(TUNE_BP_BRICK_Z, bz)


def test_caller_tensors_are_checked_before_the_library_sees_them(L):
    """The library sees only pointers, so the binding checks every tensor it hands over: inputs must be
    CUDA tensors of a supported type, and caller-supplied outputs or in-place operands must match the
    expected shape, type and device and be contiguous. These checks run before any device work."""
    import torch
    from paper_2511_08427_gb300 import operators as ops
    g = ops.Geometry.cone_circular((4, 6, 8), (1.0, 1.0, 1.0), (5, 7), (1.0, 1.0), 3, 2 * math.pi, 50.0, 90.0)
    with pytest.raises(ValueError, match="CUDA tensor"):
        ops.forward_project(torch.zeros(4, 6, 8), g)
    with pytest.raises(ValueError, match="CUDA tensor"):
        ops.adjoint_update(torch.zeros(4, 6, 8), torch.zeros(3, 5, 7), g, 0.5)
    cpu = torch.device("cpu")
    good = torch.zeros(2, 3, 5, 7)
    assert ops._check_like(good, (2, 3, 5, 7), torch.float32, cpu, "out") is good
    with pytest.raises(ValueError, match="shape"):
        ops._check_like(torch.zeros(2, 3, 5, 6), (2, 3, 5, 7), torch.float32, cpu, "out")
    with pytest.raises(TypeError):
        ops._check_like(good.to(torch.bfloat16), (2, 3, 5, 7), torch.float32, cpu, "out")
    with pytest.raises(ValueError, match="contiguous"):
        ops._check_like(torch.zeros(2, 3, 7, 5).transpose(-1, -2), (2, 3, 5, 7), torch.float32, cpu, "out")
    with pytest.raises(ValueError, match="must be on"):
        ops._check_like(good, (2, 3, 5, 7), torch.float32, torch.device("cuda", 0), "out")


def test_concurrent_queries_on_one_geometry_agree(L):
    """Eight host threads query one fresh geometry at once (ctypes releases the interpreter lock, so
    the library calls overlap): the lazily built configurations and the cached sample count are set
    up under the geometry's lock, and every thread sees the serial results."""
    import threading
    import torch
    from paper_2511_08427_gb300.operators import Geometry
    args = ((24, 32, 40), (0.5, 0.5, 0.5), (20, 28), (0.8, 0.8), 16, 2 * math.pi, 100.0, 160.0)
    ref = Geometry.cone_circular(*args)
    want = (ref.count_samples(), ref.fp_config(torch.float32), ref.fp_config(torch.bfloat16), ref.adjoint_config())
    for _ in range(3):
        g = Geometry.cone_circular(*args)
        got, errs = [], []
        start = threading.Barrier(8)

        def work():
            try:
                start.wait()
                got.append((g.count_samples(), g.fp_config(torch.float32), g.fp_config(torch.bfloat16),
                            g.adjoint_config()))
            except Exception as e:      # surfaced below
                errs.append(e)

        th = [threading.Thread(target=work) for _ in range(8)]
        for t in th:
            t.start()
        for t in th:
            t.join()
        assert not errs and len(got) == 8
        assert all(r == want for r in got)


def test_plan_arguments_are_checked_before_the_device(L):
    """Batched plans: the geometry count (1 to 16), null arrays and handles and the element type are
    checked before any device work; plan operators reject a null plan."""
    from paper_2511_08427_gb300.operators import Geometry
    g = Geometry.cone_circular((8, 8, 8), (1.0, 1.0, 1.0), (8, 8), (1.0, 1.0), 4, 2 * math.pi, 50.0, 90.0)
    h = ctypes.c_void_p()
    arr = (ctypes.c_void_p * 17)(*([g.handle.value] * 17))
    assert L.pyronn_plan_create(0, arr, 0, ctypes.byref(h)) == -1
    assert L.pyronn_plan_create(17, arr, 0, ctypes.byref(h)) == -1 and b"1 to 16" in L.pyronn_last_error()
    assert L.pyronn_plan_create(2, None, 0, ctypes.byref(h)) == -1
    assert L.pyronn_plan_create(2, arr, 0, None) == -1
    assert L.pyronn_plan_create(2, arr, 7, ctypes.byref(h)) == -2
    nulls = (ctypes.c_void_p * 2)(None, None)
    assert L.pyronn_plan_create(2, nulls, 0, ctypes.byref(h)) == -1 and b"null" in L.pyronn_last_error()
    assert not h.value
    ptrs = (ctypes.c_void_p * 1)(16)
    assert L.pyronn_plan_fp(None, ptrs, ptrs, None) == -1
    assert L.pyronn_plan_adjoint(None, ptrs, ptrs, None) == -1
    assert L.pyronn_plan_bp(None, ptrs, ptrs, 0, None) == -1
    assert L.pyronn_plan_destroy(None) == 0


def test_size_limits_at_their_edges(L):
    """Volume sides up to 16384, detector sides up to 65536 and up to 2^20 views are accepted; one more
    is rejected before anything is allocated. The largest accepted volume and detector are created
    (host tables only) and report their shapes."""
    from paper_2511_08427_gb300.operators import Geometry
    g = Geometry.parallel2d((16384, 16384), (0.1, 0.1), 65536, 0.05, 2)
    assert g.volume_shape == (16384, 16384) and g.sinogram_shape == (2, 65536)
    for kw in (dict(shape=(16385, 8)), dict(nb=65537), dict(views=(1 << 20) + 1), dict(views=0), dict(nb=0)):
        with pytest.raises(_lib.PyronnError) as e:
            Geometry.parallel2d(kw.get("shape", (8, 8)), (1.0, 1.0), kw.get("nb", 8), 1.0, kw.get("views", 4))
        assert e.value.code == -1, kw
    with pytest.raises(_lib.PyronnError):
        Geometry.cone_circular((16385, 4, 4), (1.0, 1.0, 1.0), (4, 4), (1.0, 1.0), 2, 1.0, 50.0, 90.0)


def test_sample_count_matches_oracle_over_random_geometries(L):
    """The library's sample count (per ray, the support box's slab intersection turned into a lattice
    count in closed form) equals the oracle's, which tests every lattice sample against the box, over
    40 seeded random geometries: 2D parallel and fan, 3D cone with offsets, helices, anisotropic voxels,
    fans up to about 100 degrees and steps from 0.3 to 2.5 voxels."""
    import random
    from paper_2511_08427_gb300.operators import Geometry
    rnd = random.Random(77)
    for it in range(40):
        kind = ("par", "fan", "cone", "cone")[it % 4]
        step = rnd.choice([0.3, 0.5, 1.0, 2.5])
        if kind == "cone":
            shape = tuple(rnd.choice([5, 8, 11, 16]) for _ in range(3))
            sp = tuple(rnd.choice([0.5, 0.8, 1.0, 1.7]) for _ in range(3))
            det, dsp = (rnd.choice([6, 9, 13]), rnd.choice([7, 10, 15])), (rnd.choice([0.7, 1.3]), rnd.choice([0.9, 2.0]))
            sid = rnd.choice([12.0, 30.0, 90.0])
            sdd = sid * rnd.choice([1.4, 2.0])
            pitch = rnd.choice([0.0, 0.0, 4.0])
            off = tuple(rnd.choice([0.0, 1.5, -2.5]) for _ in range(3))
            V = rnd.choice([2, 5])
            g = Geometry.cone_circular(shape, sp, det, dsp, V, 2 * math.pi, sid, sdd, helical_pitch=pitch,
                                       volume_offset=off)
            og = oracle.cone_circular(shape, sp, det, dsp, V, 2 * math.pi, sid, sdd, pitch=pitch, vol_offset=off)
        else:
            shape = (rnd.choice([6, 9, 14]), rnd.choice([7, 10, 15]))
            sp = (rnd.choice([0.5, 1.0, 1.5]), rnd.choice([0.6, 1.0]))
            nb, du, V = rnd.choice([9, 17, 31]), rnd.choice([0.5, 1.1]), rnd.choice([3, 7])
            if kind == "par":
                g = Geometry.parallel2d(shape, sp, nb, du, V, math.pi, detector_offset=0.3)
                og = oracle.parallel2d(shape, sp, nb, du, V, math.pi, det_offset=0.3)
            else:
                g = Geometry.fan2d(shape, sp, nb, du, V, 2 * math.pi, 20.0, 45.0)
                og = oracle.fan_circular(shape, sp, nb, du, V, 2 * math.pi, 20.0, 45.0)
        dt = step * min(sp)
        g.step = dt
        og.dt = dt
        assert g.count_samples() == int(oracle.count_samples(og).sum()), (it, kind)


def test_views_match_oracle_over_random_geometries(L):
    """The library's normalised per-view matrices (FP64) equal the oracle's over seeded random
    geometries: circular and helical cones with volume and detector offsets, jittered source /
    detector positions, user matrices under random non-zero rescaling, fans and parallel beams."""
    import random
    from paper_2511_08427_gb300.operators import Geometry
    rnd = random.Random(91)
    for it in range(30):
        shape = tuple(rnd.choice([6, 9, 12]) for _ in range(3))
        sp = tuple(rnd.choice([0.4, 0.7, 1.0]) for _ in range(3))
        det, dsp = (rnd.choice([5, 8]), rnd.choice([7, 12])), (rnd.choice([0.6, 1.1]), rnd.choice([0.5, 0.9]))
        doff = (rnd.choice([0.0, 0.35]), rnd.choice([0.0, -0.6]))
        off = tuple(rnd.choice([0.0, 2.0, -1.0]) for _ in range(3))
        V, sid = rnd.choice([3, 6]), rnd.choice([40.0, 200.0])
        sdd = sid * rnd.choice([1.5, 1.9])
        k = it % 5
        if k == 0:
            pitch = rnd.choice([0.0, 3.0])
            g = Geometry.cone_circular(shape, sp, det, dsp, V, 2 * math.pi, sid, sdd, helical_pitch=pitch,
                                       volume_offset=off, detector_offset=doff)
            og = oracle.cone_circular(shape, sp, det, dsp, V, 2 * math.pi, sid, sdd, pitch=pitch, vol_offset=off,
                                      det_offset=doff)
        elif k == 1:
            tr = inputs.jittered_circular_trajectory(V, 2 * math.pi, sid, sdd, 0.5, 0.3, seed=it)
            g = Geometry.cone_from_positions(shape, sp, det, dsp, tr.src, tr.det_centre, tr.eu, tr.ev,
                                             volume_offset=off, detector_offset=doff)
            og = oracle.cone_from_positions(shape, sp, det, dsp, tr.src, tr.det_centre, tr.eu, tr.ev, vol_offset=off,
                                            det_offset=doff)
        elif k == 2:
            og0 = oracle.cone_circular(shape, sp, det, dsp, V, 2 * math.pi, sid, sdd, vol_offset=off)
            scale = np.array([rnd.choice([-3.0, -0.2, 0.5, 7.0]) for _ in range(V)])
            g = Geometry.cone_from_matrices(shape, sp, det, dsp, og0.views * scale[:, None], volume_offset=off)
            og = og0
        elif k == 3:
            g = Geometry.fan2d(shape[1:], sp[1:], det[1], dsp[1], V, 2 * math.pi, sid, sdd)
            og = oracle.fan_circular(shape[1:], sp[1:], det[1], dsp[1], V, 2 * math.pi, sid, sdd)
        else:
            g = Geometry.parallel2d(shape[1:], sp[1:], det[1], dsp[1], V, math.pi, detector_offset=doff[1])
            og = oracle.parallel2d(shape[1:], sp[1:], det[1], dsp[1], V, math.pi, det_offset=doff[1])
        assert g.kind == og.kind, it
        assert np.allclose(g.views(), og.views, rtol=1e-12, atol=1e-12), it
        assert abs(g.step - og.dt) < 1e-15, it


def test_projector_automatic_depth_by_storage_type(L):
    """The TMA projector's automatic slab depth: 12 planes for FP32 and 16 for 2-byte storage where four
    CTAs still share an SM (else 8); an explicit depth is kept for every type."""
    import torch
    from paper_2511_08427_gb300.operators import TUNE_FP_DEPTH, Geometry
    g = Geometry.cone_circular((64, 96, 128), (0.5, 0.5, 0.5), (96, 128), (0.6, 0.6), 40, 2 * math.pi, 750.0, 1200.0)
    c = g.fp_config(torch.float32)
    assert c["kernel"] == 3 and c["depth"] == 12 and 4 * (c["smem_bytes"] + 512 + 1024) <= 228 * 1024
    for td in (torch.bfloat16, torch.float16):
        c = g.fp_config(td)
        assert c["kernel"] == 3 and c["depth"] == 16
        assert 4 * (c["smem_bytes"] + 512 + 1024) <= 228 * 1024
    g.set_tuning(TUNE_FP_DEPTH, 8)
    assert g.fp_config(torch.bfloat16)["depth"] == 8 and g.fp_config(torch.float32)["depth"] == 8

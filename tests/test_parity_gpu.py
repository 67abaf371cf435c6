"""GPU parity: the CUDA operators (through the C ABI) against the FP64 oracle.

Tolerances. FP32 storage: relative L2 <= 1e-5 per output tensor (the target the operators are
held to); FP32 arithmetic with FP32 per-view geometry gives ~1e-7..1e-6 in practice. BF16 / FP16
storage: the oracle is fed the same rounded inputs, so the remaining error is the output rounding
(2^-9 relative for BF16, 2^-12 for FP16) plus FP32 arithmetic: rel-L2 <= 4e-3 (BF16) and
<= 5e-4 (FP16). Dot-product (adjoint) test: |<Ax, y> - <x, A^T y>| <= 1e-6 |<Ax, y>| with the
inner products accumulated in FP64 on the host.
"""
import math

import numpy as np
import pytest
import torch

import oracle
from paper_2511_08427_gb300 import inputs

from cases import CFG1, CFG2, CFG3, SMALL, SMALL_DET8, Case, cfg_phantom, rel_l2

pytestmark = pytest.mark.gpu

TOL = {torch.float32: 1e-5, torch.bfloat16: 4e-3, torch.float16: 5e-4}


@pytest.fixture(scope="module")
def ops():
    from paper_2511_08427_gb300 import build
    build.build()
    from paper_2511_08427_gb300 import operators
    return operators


DEV = "cuda:0"


def to_dev(a, dtype=torch.float32):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).to(DEV).to(dtype)


def host(t):
    return t.float().cpu().numpy().astype(np.float64)


def sino3(case: Case, s):
    """Library 2D sinograms are [V, Nu]; the oracle's are [V, 1, Nu]."""
    s = np.asarray(s)
    return s.reshape(s.shape[0], 1, s.shape[1]) if case.ndim == 2 else s


_oracle_cache = {}


def oracle_fp(case, x):
    key = ("fp", case.name, x.tobytes().__hash__())
    if key not in _oracle_cache:
        _oracle_cache[key] = oracle.fp(case.oracle_geometry(), x)
    return _oracle_cache[key]


# ------------------------------------------------------------------------------------------------
# small cases: every geometry, every kernel variant, every storage type
# ------------------------------------------------------------------------------------------------

@pytest.mark.parametrize("variant", [0, 1, 2, 3, 4])
@pytest.mark.parametrize("case", SMALL, ids=lambda c: c.name)
def test_fp_matches_oracle(ops, case, variant):
    g = case.library_geometry()
    g.set_variant(0, variant)
    x = case.phantom()
    p = host(ops.forward_project(to_dev(x), g))
    assert rel_l2(sino3(case, p), oracle_fp(case, x)) <= 1e-5
    assert g.read_flags()[:4] == [0, 0, 0, 0]


YFAN = Case("fan_extreme", dict(kind="fan2d"), 2)   # only its ndim is used (sinogram reshaping)

# y and x extents of 16-byte multiples in FP32 and BF16, so that x-march boxes of the TMA-staged
# projector can come from the y-fastest copy of the volume; ragged detector, offsets
YFAST = Case("cone_y_fastest", dict(kind="cone", vol_shape=(22, 24, 32), vol_spacing=(0.5, 0.45, 0.5),
                                    det_shape=(23, 37), det_spacing=(0.6, 0.6), views=14, range=2 * math.pi,
                                    sid=70.0, sdd=115.0, det_offset=(0.3, -0.6), vol_offset=(0.4, -0.2, 0.3)), 3)


@pytest.mark.parametrize("transpose", [0, 1])
@pytest.mark.parametrize("dtype", [torch.float32, torch.bfloat16])
def test_fp_x_march_boxes_from_y_fastest_copy(ops, dtype, transpose):
    """TMA-staged projector with the x-march boxes staged from the y-fastest copy of the volume
    (transpose 0) and from the volume itself (1): both match the oracle on a batch of two volumes (the
    copy covers every volume of the batch), and the two agree to rounding."""
    g = YFAST.library_geometry()
    g.set_variant(0, 3)
    g.set_tuning(ops.TUNE_FP_TRANSPOSE, transpose)
    cfg = g.fp_config(dtype)
    assert cfg["kernel"] == 3 and cfg["y_fastest_x_march"] == (transpose == 0)
    og = YFAST.oracle_geometry()
    xs = np.stack([YFAST.phantom(seed=s) for s in (1, 2)])
    xd = to_dev(xs, dtype)
    xr = host(xd)
    g.read_flags(reset=True)
    p = host(ops.forward_project(xd, g))
    assert g.read_flags()[:4] == [0, 0, 0, 0]
    for i in range(2):
        assert rel_l2(p[i], oracle.fp(og, xr[i])) <= TOL[dtype]
    g.set_tuning(ops.TUNE_FP_TRANSPOSE, 1 - transpose)
    q = host(ops.forward_project(xd, g))
    # FP32 storage: the two differ by the order of the lerps only; BF16: also by output roundings
    assert rel_l2(q, p) <= (1e-6 if dtype == torch.float32 else TOL[dtype])


@pytest.mark.parametrize("variant", [1, 2, 3])
@pytest.mark.parametrize("case", SMALL, ids=lambda c: c.name)
def test_adjoint_matches_oracle(ops, case, variant):
    g = case.library_geometry()
    g.set_variant(1, variant)
    og = case.oracle_geometry()
    y = inputs.gaussian(og.sino_shape, seed=22)
    a = host(ops.adjoint(to_dev(y.reshape((og.n_views, -1)) if case.ndim == 2 else y), g))
    ref = oracle.adjoint(og, y)
    assert rel_l2(a.reshape(ref.shape), ref) <= 1e-5
    assert g.read_flags()[:4] == [0, 0, 0, 0]


SMALL3 = [c for c in SMALL if c.ndim == 3]


@pytest.mark.parametrize("accum", [0, 1, 2])
@pytest.mark.parametrize("case", SMALL3, ids=lambda c: c.name)
def test_slab_adjoint_accumulation_modes(ops, case, accum):
    """Slab-ordered adjoint with int32 fixed-point boxes (automatic: per-sample reductions; 2: cell
    accumulation) and FP32 boxes only: all match the oracle; the diagnostic counters say which boxes
    were used."""
    g = case.library_geometry()
    g.set_variant(1, 3)
    g.set_tuning(ops.TUNE_ADJ_ACCUM, accum)
    og = case.oracle_geometry()
    ref_y = inputs.gaussian(og.sino_shape, seed=23)
    g.read_flags(reset=True)
    a = host(ops.adjoint(to_dev(ref_y), g))
    assert rel_l2(a, oracle.adjoint(og, ref_y)) <= 1e-5
    f = g.read_flags()
    assert f[:4] == [0, 0, 0, 0]
    if accum == 1:
        assert f[4] == 0 and f[5] > 0
    else:
        assert f[4] > 0


@pytest.mark.parametrize("c", [1.999, -1.999, 1.0])
@pytest.mark.parametrize("case", SMALL3, ids=lambda c: c.name)
def test_slab_adjoint_fixed_point_range_edge(ops, case, c):
    """Constant sinograms with y dt = c: the fixed-point scale puts the largest single contribution
    (a sample on a lattice point) at |c| 2^e, just below 2^22 for |c| = 1.999 (the end of the range
    that one FFMA rounds exactly) and at 2^21 for c = 1 (a power of two). The adjoint matches the
    oracle and every box stays in fixed point."""
    g = case.library_geometry()
    g.set_variant(1, 3)
    og = case.oracle_geometry()
    y = np.full(og.sino_shape, c / og.dt)
    g.read_flags(reset=True)
    a = host(ops.adjoint(to_dev(y), g))
    assert rel_l2(a, oracle.adjoint(og, y)) <= 1e-5
    f = g.read_flags()
    assert f[:4] == [0, 0, 0, 0] and f[4] > 0 and f[5] == 0


def test_slab_adjoint_spiky_sinogram(ops):
    """One value per 32 x 32 detector tile 10^3 times the others (the tile's fixed-point quantum is set
    by its largest value): the adjoint of the small values, read as A^T y - A^T spikes, stays within
    the error the quantum allows, and the full adjoint matches the oracle."""
    case = [c for c in SMALL3 if c.name.startswith("cone")][0]
    g = case.library_geometry()
    g.set_variant(1, 3)
    og = case.oracle_geometry()
    base = inputs.gaussian(og.sino_shape, seed=25)
    spikes = np.zeros_like(base)
    spikes[:, 5::32, 7::32] = 1.0e3
    y = base + spikes
    a = host(ops.adjoint(to_dev(y), g))
    assert rel_l2(a, oracle.adjoint(og, y)) <= 1e-5
    small = a - host(ops.adjoint(to_dev(spikes), g))
    # per contribution at most half a quantum (2^-22 of the tile's largest |y| dt); a voxel collects
    # contributions from every view, so compare in the L2 sense against the small part's own norm
    assert rel_l2(small, oracle.adjoint(og, base)) <= 5e-3


def test_slab_adjoint_high_dynamic_range_cotangent(ops):
    """Cotangent magnitudes spread log-uniformly over four decades inside every detector tile, signs
    random. The fixed-point boxes round each contribution to a quantum of at most 2^-21 of the tile's
    largest |y| dt, so the error of a voxel is bounded by that quantum times the number of contributions
    it receives, not by its own value: voxels reached only by small cotangent values carry a larger
    relative error than the FP32 path would give them. The test holds the whole result to the FP32
    parity bound and every voxel to 1e-5 of the largest value, and prints the relative error of the
    voxels whose values are below 1e-3 of the largest (the trade-off the fixed-point boxes make)."""
    case = [c for c in SMALL3 if c.name.startswith("cone")][0]
    g = case.library_geometry()
    g.set_variant(1, 3)
    og = case.oracle_geometry()
    rng = np.random.default_rng(26)
    mag = 10.0 ** rng.uniform(-4.0, 0.0, size=og.sino_shape)
    y = (mag * rng.choice([-1.0, 1.0], size=og.sino_shape)).astype(np.float32)
    a = host(ops.adjoint(to_dev(y), g))
    ref = oracle.adjoint(og, y)
    assert rel_l2(a, ref) <= 1e-5
    err = np.abs(a - ref)
    top = np.abs(ref).max()
    assert err.max() <= 1e-5 * top
    small = (np.abs(ref) < 1e-3 * top) & (np.abs(ref) > 0)
    if small.any():
        print(f"high-dynamic-range cotangent: rel-L2 {rel_l2(a, ref):.2e}; voxels below 1e-3 of the maximum: "
              f"rel-L2 {rel_l2(a[small], ref[small]):.2e}, max error / max value {err.max() / top:.2e}")
    assert g.read_flags()[4] > 0   # the slabs did accumulate in fixed point


@pytest.mark.parametrize("pitch", [0, 1, 2])
@pytest.mark.parametrize("case", SMALL3, ids=lambda c: c.name)
def test_slab_adjoint_box_pitch(ops, case, pitch):
    """Box row pitches: 0 (automatic: odd x-march pitch, 32-word y- and z-march pitch where it fits), 1
    (rows of whole 16-byte groups) and 2 (odd x-march pitch only): all match the oracle."""
    g = case.library_geometry()
    g.set_variant(1, 3)
    g.set_tuning(ops.TUNE_ADJ_PITCH, pitch)
    c = g.adjoint_config()
    assert c["odd_pitch"] == (pitch != 1) and c["pitch32"] == (pitch == 0)
    og = case.oracle_geometry()
    y = inputs.gaussian(og.sino_shape, seed=26)
    g.read_flags(reset=True)
    a = host(ops.adjoint(to_dev(y), g))
    assert rel_l2(a, oracle.adjoint(og, y)) <= 1e-5
    assert g.read_flags()[:4] == [0, 0, 0, 0]


def test_extreme_fan_direct_rays(ops):
    """A ~160-degree fan (source 20 mm from the centre of a 16 mm volume, 61 columns of 5 mm pixels 30 mm
    from the source, views every 45 degrees): in the views along the axes the central pixel column looks
    exactly across one axis, and a detector tile (16 columns for the projector, 32 for the adjoint) spreads
    its rays by more than 45 degrees, so that column's rays barely advance along their tile's march axis
    while crossing the volume. Both the slab-staged projector and adjoint route them through their
    direct global-memory paths (flag 1, set by each); FP, matched adjoint and BP match the oracle. The
    tiles' slab boxes, built from their corner rays, do not bound such rays, so the sample loops' exact
    per-axis box tests are exercised too."""
    kw = dict(vol_shape=(16, 16, 16), vol_spacing=(1.0, 1.0, 1.0), det_shape=(16, 61), det_spacing=(2.5, 5.0),
              views=8, range=2 * math.pi, sid=20.0, sdd=30.0)
    args = (kw["vol_shape"], kw["vol_spacing"], kw["det_shape"], kw["det_spacing"], kw["views"], kw["range"],
            kw["sid"], kw["sdd"])
    g = ops.Geometry.cone_circular(*args)
    og = oracle.cone_circular(*args)
    x = inputs.uniform(og.vol_shape, seed=71)
    g.set_variant(0, 3)
    g.set_variant(1, 3)
    g.read_flags(reset=True)
    p = host(ops.forward_project(to_dev(x), g))
    assert rel_l2(p, oracle.fp(og, x)) <= 1e-5
    assert g.read_flags(reset=True)[1] > 0
    y = inputs.gaussian(og.sino_shape, seed=72)
    a = host(ops.adjoint(to_dev(y), g))
    assert rel_l2(a, oracle.adjoint(og, y)) <= 1e-5
    assert g.read_flags()[1] > 0
    for w in (0, 1):
        b = host(ops.back_project(to_dev(y), g, w))
        assert rel_l2(b, oracle.bp(og, y, w)) <= 1e-5


@pytest.mark.parametrize("variant", [1, 2])
def test_extreme_fan_other_variants(ops, variant):
    """The extreme-fan geometry through the other projector variants (1 one thread per ray, 2 thread-staged
    slabs) and adjoint variants (1 atomic scatter, 2 output-stationary bricks): all match the oracle."""
    args = ((16, 16, 16), (1.0, 1.0, 1.0), (16, 61), (2.5, 5.0), 8, 2 * math.pi, 20.0, 30.0)
    g = ops.Geometry.cone_circular(*args)
    og = oracle.cone_circular(*args)
    g.set_variant(0, variant)
    g.set_variant(1, variant)
    x = inputs.uniform(og.vol_shape, seed=73)
    assert rel_l2(host(ops.forward_project(to_dev(x), g)), oracle.fp(og, x)) <= 1e-5
    y = inputs.gaussian(og.sino_shape, seed=74)
    assert rel_l2(host(ops.adjoint(to_dev(y), g)), oracle.adjoint(og, y)) <= 1e-5


@pytest.mark.parametrize("variant", [0, 1, 2])
def test_extreme_fan_2d(ops, variant):
    """2D fan beam with a ~160-degree fan (source 20 mm from the centre of a 16 mm image, 61 bins of 5 mm
    30 mm away): every projector and adjoint variant matches the oracle, and so does the BP."""
    args = ((16, 16), (1.0, 1.0), 61, 5.0, 8, 2 * math.pi, 20.0, 30.0)
    g = ops.Geometry.fan2d(*args)
    og = oracle.fan_circular(*args)
    g.set_variant(0, variant)
    g.set_variant(1, variant)
    x = inputs.uniform(og.vol_shape, seed=75).reshape(16, 16)
    p = host(ops.forward_project(to_dev(x), g))
    assert rel_l2(sino3(YFAN, p), oracle.fp(og, x.reshape(og.vol_shape))) <= 1e-5
    y = inputs.gaussian(og.sino_shape, seed=76)
    a = host(ops.adjoint(to_dev(y.reshape(og.n_views, -1)), g))
    ref = oracle.adjoint(og, y)
    assert rel_l2(a.reshape(ref.shape), ref) <= 1e-5
    b = host(ops.back_project(to_dev(y.reshape(og.n_views, -1)), g, 0))
    refb = oracle.bp(og, y, 0)
    assert rel_l2(b.reshape(refb.shape), refb) <= 1e-5


def test_strongly_anisotropic_voxels(ops):
    """Voxel spacings 3.0 / 0.25 / 1.0 mm (z, y, x) and an offset volume: the step (half the smallest
    spacing) is 1/24 of a z voxel, slab boxes are thin along y and the fixed-point bound of the adjoint
    sees many samples per voxel; FP, matched adjoint and BP match the oracle, and the dot-product test
    holds."""
    kw = dict(vol_shape=(10, 40, 24), vol_spacing=(3.0, 0.25, 1.0), det_shape=(22, 34), det_spacing=(1.2, 0.9),
              views=12, range=2 * math.pi, sid=80.0, sdd=130.0)
    args = (kw["vol_shape"], kw["vol_spacing"], kw["det_shape"], kw["det_spacing"], kw["views"], kw["range"],
            kw["sid"], kw["sdd"])
    g = ops.Geometry.cone_circular(*args, volume_offset=(1.5, -0.7, 2.0))
    og = oracle.cone_circular(*args, vol_offset=(1.5, -0.7, 2.0))
    x = inputs.uniform(og.vol_shape, seed=81)
    g.read_flags(reset=True)
    p = host(ops.forward_project(to_dev(x), g))
    assert rel_l2(p, oracle.fp(og, x)) <= 1e-5
    y = inputs.gaussian(og.sino_shape, seed=82)
    a = host(ops.adjoint(to_dev(y), g))
    assert rel_l2(a, oracle.adjoint(og, y)) <= 1e-5
    assert g.read_flags()[:4] == [0, 0, 0, 0]
    lhs = float(np.vdot(p.ravel(), y.astype(np.float64).ravel()))
    rhs = float(np.vdot(x.astype(np.float64).ravel(), a.ravel()))
    assert abs(lhs - rhs) <= 1e-6 * np.linalg.norm(p) * np.linalg.norm(y)
    for w in (0, 1):
        assert rel_l2(host(ops.back_project(to_dev(y), g, w)), oracle.bp(og, y, w)) <= 1e-5


def test_slab_adjoint_dense_rays_keep_fp32_boxes(ops):
    """Detector pixels much smaller than the voxels (many rays per voxel support): the bound on the
    box values exceeds the fixed-point budget and the boxes stay FP32; the operator is unchanged."""
    kw = dict(vol_shape=(16, 18, 20), vol_spacing=(0.8, 0.8, 0.8), det_shape=(48, 64), det_spacing=(0.12, 0.12),
              views=5, range=2 * math.pi, sid=75.0, sdd=120.0)
    g = ops.Geometry.cone_circular(kw["vol_shape"], kw["vol_spacing"], kw["det_shape"], kw["det_spacing"], kw["views"],
                                   kw["range"], kw["sid"], kw["sdd"])
    og = oracle.cone_circular(kw["vol_shape"], kw["vol_spacing"], kw["det_shape"], kw["det_spacing"], kw["views"],
                              kw["range"], kw["sid"], kw["sdd"])
    g.set_variant(1, 3)
    y = inputs.gaussian(og.sino_shape, seed=24)
    g.read_flags(reset=True)
    a = host(ops.adjoint(to_dev(y), g))
    assert rel_l2(a, oracle.adjoint(og, y)) <= 1e-5
    f = g.read_flags()
    assert f[:4] == [0, 0, 0, 0] and f[5] > 0


@pytest.mark.parametrize("variant", [1, 2, 3])
@pytest.mark.parametrize("weight", [0, 1])
@pytest.mark.parametrize("case", SMALL, ids=lambda c: c.name)
def test_bp_matches_oracle(ops, case, weight, variant):
    g = case.library_geometry()
    g.set_variant(2, variant)
    og = case.oracle_geometry()
    for q in (inputs.uniform(og.sino_shape, seed=9), inputs.gaussian(og.sino_shape, seed=10)):
        b = host(ops.back_project(to_dev(q.reshape((og.n_views, -1)) if case.ndim == 2 else q), g, weight))
        ref = oracle.bp(og, q, weight)
        assert rel_l2(b.reshape(ref.shape), ref) <= 1e-5
    assert g.read_flags()[:4] == [0, 0, 0, 0]


@pytest.mark.parametrize("bz", [8, 16])
@pytest.mark.parametrize("dtype", [torch.float32, torch.bfloat16, torch.float16])
@pytest.mark.parametrize("weight", [0, 1])
@pytest.mark.parametrize("case", SMALL_DET8, ids=lambda c: c.name)
def test_staged_bp_matches_oracle_and_l1_path(ops, case, weight, dtype, bz):
    """The back-projector with TMA-staged detector shadows (variant 3; columns of 8 or 16 voxels) against
    the oracle (fed the same rounded sinogram) and against the L1-path brick kernel, in every storage type;
    the staged box is the one the geometry reports."""
    g = case.library_geometry()
    og = case.oracle_geometry()
    q = to_dev(inputs.uniform(og.sino_shape, seed=11), dtype)
    g.set_tuning(ops.TUNE_BP_BRICK_Z, bz)
    g.set_variant(2, 3)
    c = g.bp_config(dtype)
    assert c["kernel"] == 3 and c["brick_z"] == bz
    assert c["box"][0] * q.element_size() % 16 == 0 and c["box"][1] >= 3
    staged = host(ops.back_project(q, g, weight))
    g.set_variant(2, 2)
    l1 = host(ops.back_project(q, g, weight))
    ref = oracle.bp(og, host(q), weight)
    tol = TOL[dtype]
    assert rel_l2(staged, ref) <= tol
    assert rel_l2(staged, l1) <= (1e-6 if dtype == torch.float32 else tol)
    assert g.read_flags()[:4] == [0, 0, 0, 0]


@pytest.mark.parametrize("case", SMALL, ids=lambda c: c.name)
def test_dot_product_adjoint_gpu(ops, case):
    g = case.library_geometry()
    og = case.oracle_geometry()
    x = inputs.uniform(case.vol_shape3, seed=31).reshape(
        case.params["vol_shape"] if case.ndim == 2 else case.vol_shape3)
    sshape = (og.n_views, -1) if case.ndim == 2 else og.sino_shape
    ax = host(ops.forward_project(to_dev(x), g))
    # non-negative x and y: <Ax, y> has no cancellation, so the relative test is well conditioned
    y = inputs.uniform(og.sino_shape, seed=32).reshape(sshape)
    aty = host(ops.adjoint(to_dev(y), g))
    lhs = float(np.vdot(ax.ravel(), y.astype(np.float64).ravel()))
    rhs = float(np.vdot(x.astype(np.float64).ravel(), aty.ravel()))
    assert abs(lhs - rhs) <= 1e-6 * abs(lhs)
    # signed cotangent: bounded by the Cauchy-Schwarz scale of the two inner products
    y = inputs.gaussian(og.sino_shape, seed=33).reshape(sshape)
    aty = host(ops.adjoint(to_dev(y), g))
    lhs = float(np.vdot(ax.ravel(), y.astype(np.float64).ravel()))
    rhs = float(np.vdot(x.astype(np.float64).ravel(), aty.ravel()))
    assert abs(lhs - rhs) <= 1e-6 * np.linalg.norm(ax) * np.linalg.norm(y)


@pytest.mark.parametrize("weight", [0, 1])
@pytest.mark.parametrize("case", SMALL, ids=lambda c: c.name)
def test_bp_transpose_against_oracle_bp(ops, case, weight):
    """<BP q, x> (oracle BP, FP64) equals <q, BP^T x> (GPU transpose)."""
    g = case.library_geometry()
    og = case.oracle_geometry()
    q = inputs.gaussian(og.sino_shape, seed=41)
    x = inputs.uniform(og.vol_shape, seed=42)
    xt = x.reshape(case.params["vol_shape"]) if case.ndim == 2 else x
    bt = host(ops.back_project_transpose(to_dev(xt), g, weight))
    bq = oracle.bp(og, q, weight)
    lhs = float(np.vdot(bq.ravel(), x.astype(np.float64).ravel()))
    rhs = float(np.vdot(q.astype(np.float64).ravel(), bt.ravel()))
    # the Gaussian q makes <BP q, x> a cancelling sum: bound by the Cauchy-Schwarz scale
    assert abs(lhs - rhs) <= 1e-6 * np.linalg.norm(q) * np.linalg.norm(bt)


@pytest.mark.parametrize("dtype", [torch.bfloat16, torch.float16])
@pytest.mark.parametrize("case", SMALL, ids=lambda c: c.name)
def test_reduced_precision_storage(ops, case, dtype):
    """BF16 / FP16 storage with FP32 arithmetic; the oracle sees the same rounded inputs."""
    g = case.library_geometry()
    og = case.oracle_geometry()
    x = case.phantom()
    xd = to_dev(x, dtype)
    xr = host(xd)
    p = host(ops.forward_project(xd, g))
    assert rel_l2(sino3(case, p), oracle.fp(og, xr)) <= TOL[dtype]
    y = inputs.gaussian(og.sino_shape, seed=22)
    yd = to_dev(y.reshape((og.n_views, -1)) if case.ndim == 2 else y, dtype)
    a = host(ops.adjoint(yd, g))
    ref = oracle.adjoint(og, host(yd).reshape(og.sino_shape))
    assert rel_l2(a.reshape(ref.shape), ref) <= TOL[dtype]
    b = host(ops.back_project(yd, g))
    refb = oracle.bp(og, host(yd).reshape(og.sino_shape))
    assert rel_l2(b.reshape(refb.shape), refb) <= TOL[dtype]


@pytest.mark.parametrize("case", SMALL[:3], ids=lambda c: c.name)
def test_batch_equals_single_calls(ops, case):
    g = case.library_geometry()
    xs = np.stack([case.phantom(seed=s) for s in (1, 2, 3)])
    pb = host(ops.forward_project(to_dev(xs), g))
    for i in range(3):
        assert np.array_equal(pb[i], host(ops.forward_project(to_dev(xs[i]), g)))
    y = inputs.gaussian(pb.shape, seed=5)
    ab = host(ops.adjoint(to_dev(y), g))
    for i in range(3):
        assert rel_l2(ab[i], host(ops.adjoint(to_dev(y[i]), g))) <= 1e-6


def test_autograd_backward_is_matched_adjoint(ops):
    case = SMALL[2]
    g = case.library_geometry()
    og = case.oracle_geometry()
    x = to_dev(case.phantom()).requires_grad_(True)
    p = ops.project(x, g)
    yc = inputs.gaussian(tuple(p.shape), seed=22)
    (p * to_dev(yc)).sum().backward()
    assert rel_l2(host(x.grad), oracle.adjoint(og, yc)) <= 1e-5
    # back-projector gradient is its exact transpose; projector-adjoint gradient is the projector
    q = to_dev(inputs.uniform(tuple(p.shape), seed=3)).requires_grad_(True)
    b = ops.backproject(q, g)
    xc = to_dev(inputs.gaussian(tuple(b.shape), seed=4))
    (b * xc).sum().backward()
    assert rel_l2(host(q.grad), host(ops.back_project_transpose(xc, g))) <= 1e-6
    y2 = to_dev(yc).requires_grad_(True)
    a = ops.project_adjoint(y2, g)
    (a * xc).sum().backward()
    assert torch.equal(y2.grad, ops.forward_project(xc, g))


def test_layers_follow_listing1(ops):
    """Listing 1 flow: ConeProjectionFor3D().forward(phantom[None], geom), then
    ConeBackProjectionFor3D().forward(sinogram, geom), with a leading batch dimension."""
    case = SMALL[2]
    g = case.library_geometry()
    og = case.oracle_geometry()
    x = case.phantom()
    sino = ops.ConeProjectionFor3D().forward(to_dev(x[None]), g)
    assert tuple(sino.shape) == (1,) + og.sino_shape
    reco = ops.ConeBackProjectionFor3D().forward(sino, g)
    assert tuple(reco.shape) == (1,) + tuple(x.shape)
    assert rel_l2(host(reco[0]), oracle.bp(og, host(sino[0]))) <= 1e-5


# ------------------------------------------------------------------------------------------------
# edge cases
# ------------------------------------------------------------------------------------------------

def test_rays_missing_the_volume_give_zero(ops):
    from paper_2511_08427_gb300.operators import Geometry
    g = Geometry.cone_circular((8, 8, 8), (1, 1, 1), (6, 6), (1, 1), 4, 2 * math.pi, 50.0, 80.0,
                               detector_offset=(500.0, 0.0))
    p = ops.forward_project(torch.ones((8, 8, 8), device=DEV), g)
    assert torch.count_nonzero(p) == 0
    assert torch.count_nonzero(ops.adjoint(torch.ones_like(p), g)) == 0


def test_degenerate_single_voxel_single_pixel(ops):
    from paper_2511_08427_gb300.operators import Geometry
    g = Geometry.cone_circular((1, 1, 1), (1.0, 1.0, 1.0), (1, 1), (1.0, 1.0), 1, 2 * math.pi, 10.0, 20.0)
    og = oracle.cone_circular((1, 1, 1), (1.0, 1.0, 1.0), (1, 1), (1.0, 1.0), 1, 2 * math.pi, 10.0, 20.0)
    p = host(ops.forward_project(torch.full((1, 1, 1), 2.0, device=DEV), g))
    # a unit-hat voxel on the central ray: dt * sum_k hat((k + 1/2) dt) = 1 for dt = 1/2 voxel
    assert abs(p.item() - 2.0) < 1e-6
    assert abs(p.item() - oracle.fp(og, np.full((1, 1, 1), 2.0)).item()) < 1e-6


@pytest.mark.parametrize("dt", [0.2, 1.3])
def test_custom_step(ops, dt):
    case = SMALL[2]
    g = case.library_geometry()
    g.step = dt
    og = case.oracle_geometry()
    og.dt = dt
    x = case.phantom()
    for variant in (1, 2, 3):
        g.set_variant(0, variant)
        assert rel_l2(host(ops.forward_project(to_dev(x), g)), oracle.fp(og, x)) <= 1e-5
    y = inputs.gaussian(og.sino_shape, seed=2)
    assert rel_l2(host(ops.adjoint(to_dev(y), g)), oracle.adjoint(og, y)) <= 1e-5


def test_texture_gather_projector_batch(ops):
    """Texture-gather forward projector (variant 4): a batch of two volumes (each plane a tile of one
    gather texture, with zero tiles between the volumes) equals the per-volume projections and the
    oracle."""
    case = SMALL[2]
    g = case.library_geometry()
    g.set_variant(0, 4)
    assert g.fp_config()["kernel"] == 4
    x1, x2 = case.phantom(seed=7), case.phantom(seed=8)
    pb = host(ops.forward_project(to_dev(np.stack([x1, x2])), g))
    for i, x in enumerate((x1, x2)):
        assert rel_l2(pb[i], oracle_fp(case, x)) <= 1e-5
        assert rel_l2(pb[i], host(ops.forward_project(to_dev(x), g))) <= 1e-7
    assert g.read_flags()[:4] == [0, 0, 0, 0]


def test_many_views_times_batch_splits_launches(ops):
    from paper_2511_08427_gb300.operators import Geometry
    V, B = 3000, 25            # V * B > 65535 grid rows: the launcher splits the batch
    g = Geometry.parallel2d((6, 7), (1.0, 1.0), 5, 1.0, V)
    x = torch.rand((B, 6, 7), device=DEV)
    p = ops.forward_project(x, g)
    for i in (0, 12, 24):
        assert torch.equal(p[i], ops.forward_project(x[i].contiguous(), g))


def test_many_views_times_batch_splits_tma_launches(ops):
    """3D, 3000 views x 25 volumes: the TMA projector makes the y-fastest copies of the whole batch and
    every volume equals its single projection; the slab adjoint's batched and single calls each match
    the oracle at the FP32 parity bound. They are not compared with each other bit for bit, because the
    boxes reach the volume through FP32 global reductions whose order depends on scheduling (each result
    carries its own rounding, about 1e-6 relative on a Gaussian cotangent over 3000 views)."""
    from paper_2511_08427_gb300.operators import Geometry
    V, B = 3000, 25
    g = Geometry.cone_circular((8, 8, 8), (1.0, 1.0, 1.0), (4, 4), (1.0, 1.0), V, 2 * math.pi, 30.0, 50.0)
    og = oracle.cone_circular((8, 8, 8), (1.0, 1.0, 1.0), (4, 4), (1.0, 1.0), V, 2 * math.pi, 30.0, 50.0)
    cfg = g.fp_config()
    assert cfg["kernel"] == 3 and cfg["y_fastest_x_march"]
    x = torch.rand((B, 8, 8, 8), device=DEV, generator=torch.Generator(device=DEV).manual_seed(3))
    p = ops.forward_project(x, g)
    y = torch.randn_like(p)
    a = ops.adjoint(y, g)
    for i in (0, 20, 21, 24):
        assert torch.equal(p[i], ops.forward_project(x[i].contiguous(), g)), i
        want = oracle.adjoint(og, host(y[i]))
        assert rel_l2(host(a[i]), want) <= 1e-5, i
        assert rel_l2(host(ops.adjoint(y[i].contiguous(), g)), want) <= 1e-5, i


def test_more_views_than_grid_rows_split_launches(ops):
    """70000 views (more than the 65535 grid rows the slab kernels put views on): the TMA projector and
    the slab adjoint split the views into launches whose tables and sinogram start at the launch's first
    view; both match the oracle."""
    from paper_2511_08427_gb300.operators import Geometry
    V = 70000
    args = ((8, 8, 8), (1.0, 1.0, 1.0), (4, 4), (1.0, 1.0), V, 2 * math.pi, 30.0, 50.0)
    g = Geometry.cone_circular(*args)
    og = oracle.cone_circular(*args)
    assert g.fp_config()["kernel"] == 3 and g.adjoint_config()["kernel"] == 3
    x = inputs.uniform((8, 8, 8), seed=31)
    p = host(ops.forward_project(to_dev(x), g))
    assert rel_l2(p, oracle.fp(og, x)) <= 1e-5
    y = inputs.gaussian(og.sino_shape, seed=32)
    assert rel_l2(host(ops.adjoint(to_dev(y), g)), oracle.adjoint(og, y)) <= 1e-5
    assert g.read_flags()[:4] == [0, 0, 0, 0]


def test_batch_times_tile_rows_split_launches(ops):
    """One view on a 2048-row detector (128 tile rows of the projector, 64 of the adjoint) and 1100
    volumes: tile rows x batch items exceed the 65535 grid layers, so both kernels split the batch;
    every volume's projection equals its single projection and the adjoints match the oracle."""
    from paper_2511_08427_gb300.operators import Geometry
    B = 1100
    args = ((8, 8, 8), (1.0, 1.0, 1.0), (2048, 8), (0.01, 2.0), 1, 2 * math.pi, 30.0, 50.0)
    g = Geometry.cone_circular(*args)
    og = oracle.cone_circular(*args)
    assert g.fp_config()["kernel"] == 3 and g.adjoint_config()["kernel"] == 3
    x = torch.rand((B, 8, 8, 8), device=DEV, generator=torch.Generator(device=DEV).manual_seed(4))
    p = ops.forward_project(x, g)
    y = torch.randn_like(p)
    a = ops.adjoint(y, g)
    for i in (0, 510, 511, 1022, 1023, 1099):
        assert torch.equal(p[i], ops.forward_project(x[i].contiguous(), g)), i
        assert rel_l2(host(p[i]), oracle.fp(og, host(x[i]))) <= 1e-5, i
        assert rel_l2(host(a[i]), oracle.adjoint(og, host(y[i]))) <= 1e-5, i


def test_misaligned_pointer_is_rejected(ops):
    from paper_2511_08427_gb300 import PyronnError
    case = SMALL[0]
    g = case.library_geometry()
    n = int(np.prod(case.params["vol_shape"]))
    buf = torch.zeros(n + 1, device=DEV)
    with pytest.raises(PyronnError) as e:
        ops.forward_project(buf[1:].view(case.params["vol_shape"]), g)
    assert e.value.code == -3


def test_host_buffer_entry_point(ops):
    import ctypes
    from paper_2511_08427_gb300 import _lib
    case = SMALL[2]
    g = case.library_geometry()
    x = case.phantom().astype(np.float32)
    out = np.zeros(case.oracle_geometry().sino_shape, dtype=np.float32)
    _lib.check(_lib.lib().pyronn_fp_host(g.handle, x.ctypes.data_as(ctypes.c_void_p),
                                         out.ctypes.data_as(ctypes.c_void_p), 0, 1, None))
    assert rel_l2(out, oracle_fp(case, x)) <= 1e-5


@pytest.mark.parametrize("dtype", [torch.float32, torch.bfloat16])
@pytest.mark.parametrize("transpose", [0, 1])
def test_host_buffer_fp_overlapped_download(ops, transpose, dtype):
    """pyronn_fp_host on the TMA projector projects the views in chunks and downloads each chunk's rows
    on a second stream while the next chunk runs (14 views: chunks of one and two views). A batch of two,
    from pageable and from pinned host buffers, equals the device-buffer projection exactly (every ray's
    arithmetic is independent of how the views are split into launches)."""
    import ctypes
    from paper_2511_08427_gb300 import _lib
    g = YFAST.library_geometry()
    g.set_variant(0, 3)
    g.set_tuning(ops.TUNE_FP_TRANSPOSE, transpose)
    assert g.fp_config()["kernel"] == 3
    xs = torch.from_numpy(np.stack([YFAST.phantom(seed=s) for s in (3, 4)]).astype(np.float32)).to(dtype)
    ref = ops.forward_project(xs.to(DEV), g).cpu()
    code = {torch.float32: _lib.F32, torch.bfloat16: _lib.BF16}[dtype]
    for pinned in (False, True):
        hx = xs.clone()
        ho = torch.full(tuple(ref.shape), float("nan"), dtype=dtype)
        if pinned:
            hx, ho = hx.pin_memory(), ho.pin_memory()
        _lib.check(_lib.lib().pyronn_fp_host(g.handle, ctypes.c_void_p(hx.data_ptr()), ctypes.c_void_p(ho.data_ptr()),
                                             code, 2, None))
        assert torch.equal(ho, ref), pinned


def test_host_buffer_adjoint(ops):
    """pyronn_adjoint_host (FP32, slab adjoint), a batch of two from pageable and pinned host buffers:
    matches the device-buffer adjoint and the oracle."""
    import ctypes
    from paper_2511_08427_gb300 import _lib
    g = YFAST.library_geometry()
    og = YFAST.oracle_geometry()
    y = np.stack([inputs.gaussian(og.sino_shape, seed=s) for s in (61, 62)]).astype(np.float32)
    ref = host(ops.adjoint(to_dev(y), g))
    for pinned in (False, True):
        hy = torch.from_numpy(y)
        ho = torch.full(tuple(ref.shape), float("nan"))
        if pinned:
            hy, ho = hy.pin_memory(), ho.pin_memory()
        _lib.check(_lib.lib().pyronn_adjoint_host(g.handle, ctypes.c_void_p(hy.data_ptr()),
                                                  ctypes.c_void_p(ho.data_ptr()), 0, 2, None))
        a = ho.numpy().astype(np.float64)
        assert rel_l2(a, ref) <= 1e-6, pinned
        for i in range(2):
            assert rel_l2(a[i], oracle.adjoint(og, y[i].astype(np.float64))) <= 1e-5, (pinned, i)


# ------------------------------------------------------------------------------------------------
# benchmark configurations at full size
# ------------------------------------------------------------------------------------------------

@pytest.mark.parametrize("case", [CFG1, CFG2], ids=lambda c: c.name)
def test_2d_configs_full(ops, case):
    g = case.library_geometry()
    og = case.oracle_geometry()
    x = cfg_phantom(case)
    p = host(ops.forward_project(to_dev(x), g))
    assert rel_l2(sino3(case, p), oracle.fp(og, x)) <= 1e-5
    y = inputs.gaussian(og.sino_shape, seed=22)
    a = host(ops.adjoint(to_dev(y.reshape(og.n_views, -1)), g))
    assert rel_l2(a.reshape(og.vol_shape), oracle.adjoint(og, y)) <= 1e-5
    b = host(ops.back_project(to_dev(y.reshape(og.n_views, -1)), g))
    assert rel_l2(b.reshape(og.vol_shape), oracle.bp(og, y)) <= 1e-5


def test_cone256_config_sampled(ops):
    """256^3 cone beam, 360 views, 512^2 detector: sampled rays / voxels, sparse cotangent."""
    case = CFG3
    g = case.library_geometry()
    og = case.oracle_geometry()
    x = cfg_phantom(case)
    xd = to_dev(x)
    p = ops.forward_project(xd, g)
    rng = np.random.default_rng(0)
    n_rays = og.n_views * og.det_shape[0] * og.det_shape[1]
    ids = rng.choice(n_rays, size=3000, replace=False)
    ref = oracle.fp_rays(og, x, ids)
    got = host(p).ravel()[ids]
    assert rel_l2(got, ref) <= 1e-5
    # matched adjoint of a sparse cotangent, compared over the whole volume
    sid = rng.choice(n_rays, size=400, replace=False)
    vals = rng.standard_normal(400)
    y = torch.zeros(n_rays, device=DEV)
    y[torch.from_numpy(sid).to(DEV)] = torch.from_numpy(vals.astype(np.float32)).to(DEV)
    a = host(ops.adjoint(y.view(og.sino_shape), g))
    refa = oracle.adjoint_rays(og, sid, vals.astype(np.float32).astype(np.float64))
    assert rel_l2(a, refa) <= 1e-5
    # voxel-driven BP of the projection, sampled voxels
    b = host(ops.back_project(p, g, 1))
    vids = rng.choice(x.size, size=3000, replace=False)
    refb = oracle.bp_voxels(og, host(p), vids, 1)
    assert rel_l2(b.ravel()[vids], refb) <= 1e-5
    # dot-product test at full size: non-negative cotangent (no cancellation, relative bound) and a
    # signed one (bounded by the Cauchy-Schwarz scale of the inner products)
    yc = torch.rand(og.sino_shape, device=DEV)
    lhs = float(np.vdot(host(p).ravel(), host(yc).ravel()))
    rhs = float(np.vdot(x.astype(np.float64).ravel(), host(ops.adjoint(yc, g)).ravel()))
    assert abs(lhs - rhs) <= 1e-6 * abs(lhs)
    yc = torch.randn(og.sino_shape, device=DEV)
    lhs = float(np.vdot(host(p).ravel(), host(yc).ravel()))
    rhs = float(np.vdot(x.astype(np.float64).ravel(), host(ops.adjoint(yc, g)).ravel()))
    assert abs(lhs - rhs) <= 1e-6 * np.linalg.norm(host(p)) * np.linalg.norm(host(yc))


def test_variants_agree_at_full_size(ops):
    case = CFG3
    g = case.library_geometry()
    x = to_dev(cfg_phantom(case))
    g.set_variant(0, 1)
    p1 = ops.forward_project(x, g)
    for variant in (2, 3):
        g.set_variant(0, variant)
        p2 = ops.forward_project(x, g)
        assert rel_l2(host(p2), host(p1)) <= 2e-6
        assert g.read_flags()[:4] == [0, 0, 0, 0]


@pytest.mark.parametrize("dtype", [torch.float32, torch.bfloat16])
@pytest.mark.parametrize("case", [c for c in SMALL if c.ndim == 3], ids=lambda c: c.name)
def test_packed_interpolation_is_bit_identical(ops, case, dtype):
    """The TMA projector's packed FP32x2 arithmetic (lerps: the default; lerps and positions) and its
    scalar form round every lane the same way, so the projections are identical bit for bit."""
    g = case.library_geometry()
    if g.fp_config(dtype)["kernel"] != 3:
        pytest.skip("the TMA-staged projector does not apply to this geometry")
    x = to_dev(case.phantom(), dtype)
    g.set_tuning(ops.TUNE_FP_PACKED, 1)
    scalar = ops.forward_project(x, g)
    for mode in (2, 3):
        g.set_tuning(ops.TUNE_FP_PACKED, mode)
        assert torch.equal(ops.forward_project(x, g), scalar), mode


@pytest.mark.parametrize("depth", [12, 16, 24])
@pytest.mark.parametrize("name", ["helical", "jittered_positions"])
def test_projector_slabs_deeper_than_the_volume(ops, name, depth):
    """TMA projector slabs deeper than the volume along the march axis (the first slab starts below plane
    -1 at an x-aligned plane, so its box spans more than N + 2 guard + 2 planes): every slab fits its
    box (no overflow flag) and the projection matches the oracle."""
    case = next(c for c in SMALL if c.name == name)
    g = case.library_geometry()
    g.set_tuning(ops.TUNE_FP_DEPTH, depth)
    assert g.fp_config()["kernel"] == 3
    og = case.oracle_geometry()
    x = case.phantom()
    g.read_flags(reset=True)
    p = host(ops.forward_project(to_dev(x), g))
    assert rel_l2(p, oracle.fp(og, x)) <= 1e-5
    assert g.read_flags()[:4] == [0, 0, 0, 0]

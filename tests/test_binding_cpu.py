"""The PyTorch binding's marshalling, checked on the CPU against a stand-in for the operator entry
points: every call hands the C ABI the tensors' own pointers, the element-type code, the batch count
and the stream, allocates outputs of the documented shapes, and refuses mismatched outputs before
calling the library. Geometry creation and queries use the real library (host code only); the
operator entry points, which need a GPU, are replaced by recorders. CPU tensors stand in for device
tensors, so the CUDA-device checks are relaxed here and only here."""
import contextlib
import ctypes
import math

import pytest
import torch

from paper_2511_08427_gb300 import _lib, artifacts, operators as ops

STUBBED = ("pyronn_fp", "pyronn_adjoint", "pyronn_adjoint_update", "pyronn_bp", "pyronn_bp_transpose",
           "pyronn_fbp_filter", "pyronn_plan_create", "pyronn_plan_fp", "pyronn_plan_adjoint", "pyronn_plan_bp",
           "pyronn_sim_detector_jitter", "pyronn_sim_gaussian_noise", "pyronn_sim_ring", "pyronn_sim_motion_blur")


class _Recorder:
    def __init__(self, real):
        self.real, self.calls = real, []

    def __getattr__(self, name):
        if name not in STUBBED:
            return getattr(self.real, name)

        def call(*args):
            self.calls.append((name, args))
            return 0
        return call


@pytest.fixture
def rec(monkeypatch):
    from paper_2511_08427_gb300 import build
    build.build()
    r = _Recorder(_lib.lib())
    monkeypatch.setattr(ops, "lib", lambda: r)
    monkeypatch.setattr(artifacts, "lib", lambda: r)
    relaxed = lambda t, what: ops._DTYPES[t.dtype]       # noqa: E731  (CPU tensors stand in for device ones)
    monkeypatch.setattr(ops, "_check", relaxed)
    monkeypatch.setattr(artifacts, "_check", relaxed)
    monkeypatch.setattr(ops, "_stream_ptr", lambda d: 0)
    monkeypatch.setattr(artifacts, "_stream_ptr", lambda d: 0)
    monkeypatch.setattr(torch.cuda, "device", lambda d: contextlib.nullcontext())
    return r


def _cone():
    return ops.Geometry.cone_circular((4, 6, 8), (1.0, 1.0, 1.0), (5, 7), (1.0, 1.0), 3, 2 * math.pi, 50.0, 90.0)


def test_operators_pass_pointers_types_and_batches(rec):
    g = _cone()
    vol = torch.rand(2, 4, 6, 8)
    p = ops.forward_project(vol, g)
    assert p.shape == (2, 3, 5, 7) and p.dtype == torch.float32
    name, a = rec.calls[-1]
    assert name == "pyronn_fp" and a[1:] == (vol.data_ptr(), p.data_ptr(), _lib.F32, 2, 0)
    s = torch.rand(3, 5, 7, dtype=torch.bfloat16)
    v = ops.adjoint(s, g)
    assert v.shape == (4, 6, 8) and v.dtype == torch.bfloat16
    assert rec.calls[-1][0] == "pyronn_adjoint" and rec.calls[-1][1][1:] == (s.data_ptr(), v.data_ptr(), _lib.BF16, 1, 0)
    b = ops.back_project(s.half(), g, ops.BP_INV_W2)
    assert b.dtype == torch.float16 and rec.calls[-1][1][4:6] == (1, ops.BP_INV_W2)
    t = ops.back_project_transpose(vol, g)
    assert t.shape == (2, 3, 5, 7) and rec.calls[-1][0] == "pyronn_bp_transpose"
    # outputs supplied by the caller are used as given, in place where documented
    out = torch.empty(2, 3, 5, 7)
    assert ops.forward_project(vol, g, out=out) is out and rec.calls[-1][1][2] == out.data_ptr()
    f = ops.fbp_filter(p, g, out=p)
    assert f is p and rec.calls[-1][1][1] == rec.calls[-1][1][2] == p.data_ptr()
    y = torch.rand(3, 5, 7)
    yb = torch.rand(3, 5, 7)
    x = torch.rand(4, 6, 8)
    assert ops.adjoint_update(x, y, g, 0.25, sino_b=yb) is x
    name, a = rec.calls[-1]
    assert name == "pyronn_adjoint_update" and a[1:] == (y.data_ptr(), yb.data_ptr(), 0.25, x.data_ptr(), _lib.F32, 1, 0)


def test_mismatched_outputs_never_reach_the_library(rec):
    g = _cone()
    vol = torch.rand(2, 4, 6, 8)
    n = len(rec.calls)
    for bad in (torch.empty(2, 3, 5, 6), torch.empty(2, 3, 5, 7, dtype=torch.float16),
                torch.empty(2, 3, 7, 5).transpose(-1, -2), torch.empty(3, 5, 7)):
        with pytest.raises((ValueError, TypeError)):
            ops.forward_project(vol, g, out=bad)
    with pytest.raises(ValueError):
        ops.adjoint_update(torch.rand(4, 6, 7), torch.rand(3, 5, 7), g, 1.0)
    with pytest.raises(TypeError):
        ops.adjoint_update(torch.rand(4, 6, 8), torch.rand(3, 5, 7), g, 1.0, sino_b=torch.rand(3, 5, 7).half())
    with pytest.raises(ValueError):
        artifacts.gaussian_noise(torch.rand(3, 5, 7), g, torch.rand(3, 5, 7), out=torch.empty(3, 5, 8))
    assert len(rec.calls) == n


def test_gradient_step_and_layers_route_through_the_abi(rec):
    """The fused gradient step (forward and backward) and the Listing 1 layers call the library with
    consistent shapes; with recorders the values are meaningless, the plumbing is what is checked."""
    g = _cone()
    x = torch.zeros(4, 6, 8, requires_grad=True)
    p = torch.zeros(3, 5, 7, requires_grad=True)
    alpha = torch.tensor(0.1, requires_grad=True)
    y = ops.gradient_step(x, p, alpha, g)
    y.sum().backward()
    assert x.grad.shape == x.shape and p.grad.shape == p.shape and alpha.grad.shape == alpha.shape
    names = [c[0] for c in rec.calls]
    assert names.count("pyronn_fp") == 2 and names.count("pyronn_adjoint_update") == 2
    # a plain Python step: no gradient for it, the others as before
    x2 = torch.zeros(4, 6, 8, requires_grad=True)
    ops.gradient_step(x2, p, 0.1, g).sum().backward()
    assert x2.grad.shape == x2.shape
    names = [c[0] for c in rec.calls]
    assert names.count("pyronn_fp") == 4 and names.count("pyronn_adjoint_update") == 4
    q = ops.ConeProjectionFor3D()(torch.zeros(4, 6, 8), g)
    assert q.shape == (3, 5, 7)
    bq = ops.ConeBackProjectionFor3D()(q, g)
    assert bq.shape == (4, 6, 8)


def test_plan_and_artifacts_marshal_lists(rec):
    g1, g2 = _cone(), ops.Geometry.cone_circular((8, 8, 8), (1.0,) * 3, (6, 6), (1.0, 1.0), 2, 2 * math.pi, 40.0, 80.0)
    plan = ops.Plan([g1, g2])
    vols = [torch.rand(4, 6, 8), torch.rand(8, 8, 8)]
    sinos = [torch.empty(3, 5, 7), torch.empty(2, 6, 6)]
    assert plan.forward_project(vols, sinos) is sinos
    name, a = rec.calls[-1]
    assert name == "pyronn_plan_fp" and list(a[1]) == [v.data_ptr() for v in vols]
    assert list(a[2]) == [s.data_ptr() for s in sinos]
    with pytest.raises(ValueError):
        plan.adjoint(sinos, [torch.rand(4, 6, 8), torch.rand(8, 8, 7)])
    s = torch.rand(3, 5, 7)
    out = artifacts.ring_artifacts(s, g1, [1, 4], [0.0, 1.5], 0, 2)
    name, a = rec.calls[-1]
    assert name == "pyronn_sim_ring" and a[1] == s.data_ptr() and a[2] == out.data_ptr() and a[5:8] == (2, 0, 2)
    plan._h = ctypes.c_void_p()     # the recorder created no plan


def test_remaining_call_patterns(rec):
    """The other patterns the GPU tests use: artifact calls (noise written in place), valid plan adjoint and
    back-projection calls, and the unrolled reconstruction (checkpointed, fused and unfused) forward and
    backward."""
    from paper_2511_08427_gb300.unrolled import UnrolledGD
    g = _cone()
    s = torch.rand(2, 3, 5, 7)
    j = artifacts.detector_jitter(s, g, torch.zeros(2, 3, 5, dtype=torch.int32), 0)
    assert j.shape == s.shape and rec.calls[-1][0] == "pyronn_sim_detector_jitter" and rec.calls[-1][1][6] == 2
    n = artifacts.gaussian_noise(s, g, torch.zeros_like(s), 0.1, 0.05, out=s)
    assert n is s and rec.calls[-1][1][1] == rec.calls[-1][1][2] == s.data_ptr()
    b = artifacts.motion_blur(s, g, [0.1, 0.2, 0.3], 3)
    assert b.shape == s.shape and rec.calls[-1][0] == "pyronn_sim_motion_blur"
    g2 = ops.Geometry.cone_circular((8, 8, 8), (1.0,) * 3, (6, 6), (1.0, 1.0), 2, 2 * math.pi, 40.0, 80.0)
    plan = ops.Plan([g, g2])
    sinos = [torch.rand(3, 5, 7), torch.rand(2, 6, 6)]
    vols = [torch.empty(4, 6, 8), torch.empty(8, 8, 8)]
    assert plan.adjoint(sinos, vols) is vols and rec.calls[-1][0] == "pyronn_plan_adjoint"
    assert plan.back_project(sinos, vols, ops.BP_INV_W2) is vols and rec.calls[-1][1][3] == ops.BP_INV_W2
    plan._h = ctypes.c_void_p()
    cpu = torch.device("cpu")
    for fused in (True, False):
        net = UnrolledGD(g, iterations=3, alpha0=0.1, checkpoint=True, device=cpu, fused=fused)
        p = torch.zeros(3, 5, 7)
        x = net(p)
        assert x.shape == (4, 6, 8)
        x.sum().backward()
        assert net.alpha.grad.shape == (3,)

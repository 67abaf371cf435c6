"""Acquisition-artifact kernels (Sec. 2.4) against the FP64 references of oracle.artifacts."""
import math

import numpy as np
import pytest
import torch

from oracle import artifacts as A
from paper_2511_08427_gb300 import inputs

from cases import SMALL, rel_l2

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


@pytest.fixture(scope="module")
def art():
    from paper_2511_08427_gb300 import build
    build.build()
    from paper_2511_08427_gb300 import artifacts, operators
    return artifacts, operators


def host(t):
    return t.detach().float().cpu().numpy().astype(np.float64)


def setup(ops, name="cone"):
    case = next(c for c in SMALL if c.name == name)
    g = case.library_geometry()
    og = case.oracle_geometry()
    p = inputs.uniform(og.sino_shape, seed=70)
    return g, og, p, torch.from_numpy(p).to(DEV)


@pytest.mark.parametrize("axis", [0, 1])
def test_detector_jitter(art, axis):
    A_, ops = art
    g, og, p, pd = setup(ops)
    V, Nv, Nu = og.sino_shape
    s = inputs.jitter_shifts((V, Nv if axis == 0 else Nu), 3, seed=71)
    out = host(A_.detector_jitter(pd, g, s, axis))
    assert np.array_equal(out.astype(np.float32), A.detector_jitter(p, s, axis).astype(np.float32))


def test_gaussian_noise_in_place(art):
    A_, ops = art
    g, og, p, pd = setup(ops)
    nz = inputs.gaussian(og.sino_shape, seed=72)
    out = A_.gaussian_noise(pd, g, torch.from_numpy(nz).to(DEV), 0.1, 0.05, out=pd)
    assert rel_l2(host(out), A.gaussian_noise(p, nz, 0.1, 0.05)) <= 1e-7


def test_ring_artifacts(art):
    A_, ops = art
    g, og, p, pd = setup(ops)
    cols, gains = inputs.ring_columns(og.sino_shape[2], 4, seed=73)
    out = host(A_.ring_artifacts(pd, g, cols, gains, 2, 9))
    assert rel_l2(out, A.ring_artifacts(p, cols, gains, 2, 9)) <= 1e-7


@pytest.mark.parametrize("length", [1, 4, 7])
def test_motion_blur(art, length):
    A_, ops = art
    g, og, p, pd = setup(ops)
    ang = np.linspace(0, 2 * math.pi, og.n_views, endpoint=False).astype(np.float32)
    out = host(A_.motion_blur(pd, g, ang, length))
    assert rel_l2(out, A.motion_blur(p, ang, length)) <= 1e-6


def test_artifacts_on_a_2d_sinogram_and_bf16(art):
    A_, ops = art
    case = next(c for c in SMALL if c.name == "fan2d")
    g = case.library_geometry()
    og = case.oracle_geometry()
    p = inputs.uniform(og.sino_shape, seed=74)
    pd = torch.from_numpy(p.reshape(og.n_views, -1)).to(DEV)
    s = inputs.jitter_shifts((og.n_views, 1), 2, seed=75)
    out = host(A_.detector_jitter(pd, g, s, 0)).reshape(og.sino_shape)
    assert np.array_equal(out.astype(np.float32), A.detector_jitter(p, s, 0).astype(np.float32))
    pb = pd.bfloat16()
    ang = np.zeros(og.n_views, np.float32)
    ob = host(A_.motion_blur(pb, g, ang, 3)).reshape(og.sino_shape)
    assert rel_l2(ob, A.motion_blur(host(pb).reshape(og.sino_shape), ang, 3)) <= 4e-3

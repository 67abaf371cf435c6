"""Gradients through the operators: finite differences and the oracle's gradient (2D fan-beam
configuration, full size), the 512^3 arbitrary-trajectory configuration (sampled parity at full size
and a 10-iteration checkpointed unrolled gradient-descent reconstruction from a Poisson-noised
sinogram), and checkpointed vs stored autograd on a small unrolled solver."""
import math

import numpy as np
import pytest
import torch

import oracle
from paper_2511_08427_gb300 import inputs

from cases import CFG2, CFG5, cfg_phantom, rel_l2

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


def test_fan2d_config_gradient_finite_difference_and_oracle(ops):
    """256^2 fan beam, 360 views, 512 bins: the autograd gradient of L(x) = 0.5 ||A x - y||^2 equals
    the oracle's A^T (A x - y) and the central finite difference along a random direction (exact for a
    quadratic up to FP32 rounding of A x)."""
    case = CFG2
    g = case.library_geometry()
    og = case.oracle_geometry()
    xt = cfg_phantom(case)
    y = oracle.fp(og, xt).reshape(og.n_views, -1)
    y = y + 0.05 * inputs.gaussian(y.shape, seed=40).astype(np.float64) * np.abs(y).max()
    x0 = 0.5 * xt
    x = torch.from_numpy(x0.astype(np.float32)).to(DEV).requires_grad_(True)
    yd = torch.from_numpy(y.astype(np.float32)).to(DEV)
    r = ops.project(x, g) - yd
    (0.5 * (r.double() ** 2).sum()).backward()
    # oracle gradient from the oracle's own residual
    ro = oracle.fp(og, x0.astype(np.float32).astype(np.float64)).reshape(og.n_views, -1) - y.astype(np.float32)
    go = oracle.adjoint(og, ro.reshape(og.sino_shape)).reshape(x0.shape)
    assert rel_l2(host(x.grad), go) <= 1e-5

    def loss(xv):
        with torch.no_grad():
            rr = ops.forward_project(xv, g).double() - yd.double()
            return 0.5 * float((rr ** 2).sum())

    half = 0.5 * case.params["vol_shape"][0] * case.params["vol_spacing"][0]
    d = torch.from_numpy(inputs.rasterise_ellipses(inputs.random_ellipses(10, half, 41), case.params["vol_shape"],
                                                   case.params["vol_spacing"])).to(DEV)
    gd = float((x.grad.double() * d.double()).sum())
    base = x.detach()
    eps = 0.02 * float(base.norm()) / float(d.norm())
    fd = (loss(base + eps * d) - loss(base - eps * d)) / (2 * eps)
    assert abs(fd - gd) <= 1e-3 * abs(gd)


@pytest.fixture(scope="module")
def cfg5(ops):
    case = CFG5
    g = case.library_geometry()
    og = case.oracle_geometry()
    xt = cfg_phantom(case)
    return case, g, og, xt


def test_cfg5_full_size_sampled_parity(ops, cfg5):
    """512^3 at 0.4 mm, 720 jittered views, 1024^2 detector: sampled rays, a sparse-cotangent adjoint over
    the whole volume, sampled back-projected voxels, against the oracle."""
    case, g, og, xt = cfg5
    x = torch.from_numpy(xt).to(DEV)
    p = ops.forward_project(x, g)
    rng = np.random.default_rng(5)
    n_rays = og.n_views * og.det_shape[0] * og.det_shape[1]
    ids = rng.choice(n_rays, size=2000, replace=False)
    ph = host(p)
    assert rel_l2(ph.ravel()[ids], oracle.fp_rays(og, xt, ids)) <= 1e-5
    sid = rng.choice(n_rays, size=300, replace=False)
    vals = rng.standard_normal(300).astype(np.float32)
    y = torch.zeros(n_rays, device=DEV)
    y[torch.from_numpy(sid).to(DEV)] = torch.from_numpy(vals).to(DEV)
    a = host(ops.adjoint(y.view(og.sino_shape), g))
    assert rel_l2(a, oracle.adjoint_rays(og, sid, vals.astype(np.float64))) <= 1e-5
    del y, a
    b = ops.back_project(p, g, 1)
    vids = rng.choice(xt.size, size=1500, replace=False)
    assert rel_l2(host(b).ravel()[vids], oracle.bp_voxels(og, ph, vids, 1)) <= 1e-5
    assert g.read_flags()[:4] == [0, 0, 0, 0]


def test_cfg5_unrolled_gd_checkpointed(ops, cfg5):
    """10 learnable-step gradient-descent iterations from a Poisson-noised sinogram (1e5 photons) with
    checkpointed autograd through the projector and the matched adjoint: the data term decreases at
    every iteration (steps below 1 / ||A||^2), and the step sizes receive finite gradients."""
    from paper_2511_08427_gb300.unrolled import UnrolledGD
    case, g, og, xt = cfg5
    x_true = torch.from_numpy(xt).to(DEV)
    with torch.no_grad():
        p_clean = ops.forward_project(x_true, g)
        scale = 3.0 / float(p_clean.max())
        p_noisy = inputs.poisson_log_sinogram_torch(p_clean, 1e5, seed=5)
        del p_clean
    x_true = x_true * scale   # the reconstruction target in the units of the scaled sinogram
    model = UnrolledGD(g, iterations=10, checkpoint=True)
    assert 0.0 < float(model.alpha.detach()[0]) < math.inf
    x10, xs = model(p_noisy, return_all=True)
    loss = ((x10 - x_true) ** 2).mean()
    loss.backward()
    grad = model.alpha.grad
    assert grad is not None and torch.isfinite(grad).all() and float(grad.abs().max()) > 0.0
    with torch.no_grad():
        data = [0.5 * float(((ops.forward_project(xk, g) - p_noisy).double() ** 2).sum()) for xk in xs]
    data0 = 0.5 * float((p_noisy.double() ** 2).sum())
    seq = [data0] + data
    assert all(b < a for a, b in zip(seq, seq[1:])), seq
    assert g.read_flags()[:4] == [0, 0, 0, 0]


def test_unrolled_gd_checkpoint_matches_stored_and_finite_difference(ops):
    """Small jittered cone beam: checkpointed and stored autograd give the same step-size gradients, and
    the gradient of the loss with respect to one step size matches its central finite difference (the
    iterate is affine in each step size, so the loss is quadratic in it)."""
    from paper_2511_08427_gb300.unrolled import UnrolledGD
    tr = inputs.jittered_circular_trajectory(40, 2 * math.pi, 75.0, 120.0, 0.5, 0.2, seed=8)
    shape, sp = (40, 44, 48), (0.5, 0.5, 0.5)
    g = ops.Geometry.cone_from_positions(shape, sp, (48, 64), (0.6, 0.6), tr.src, tr.det_centre, tr.eu, tr.ev)
    xt = inputs.rasterise_ellipsoids(inputs.random_ellipsoids(8, 10.0, 11), shape, sp)
    x_true = torch.from_numpy(xt).to(DEV)
    with torch.no_grad():
        p = ops.forward_project(x_true, g)
        p = p + 0.01 * float(p.max()) * torch.from_numpy(inputs.gaussian(tuple(p.shape), seed=12)).to(DEV)
    grads = []
    for ck in (True, False):
        m = UnrolledGD(g, iterations=6, checkpoint=ck)
        ((m(p) - x_true) ** 2).sum().backward()
        grads.append(m.alpha.grad.clone())
    assert rel_l2(host(grads[0]), host(grads[1])) <= 1e-5
    m = UnrolledGD(g, iterations=6, checkpoint=False)
    base = m.alpha.detach().clone()

    def loss(alpha):
        with torch.no_grad():
            m.alpha.copy_(alpha)
            return float(((m(p) - x_true).double() ** 2).sum())

    k = 3
    h = 0.2 * float(base[k])
    ap, am = base.clone(), base.clone()
    ap[k] += h
    am[k] -= h
    fd = (loss(ap) - loss(am)) / (2 * h)
    assert abs(fd - float(grads[1][k])) <= 2e-3 * abs(float(grads[1][k])) + 1e-9


@pytest.mark.parametrize("name", ["cone", "jittered_positions", "fan2d"])
@pytest.mark.parametrize("with_b", [True, False])
def test_adjoint_update_matches_composition_and_oracle(ops, name, with_b):
    """vol += alpha A^T (a - b): fused (3D: slab adjoint) or through work buffers (2D), against the
    unfused composition and the oracle."""
    from cases import SMALL
    case = next(c for c in SMALL if c.name == name)
    g = case.library_geometry()
    og = case.oracle_geometry()
    sshape = (og.n_views, -1) if case.ndim == 2 else og.sino_shape
    a = inputs.gaussian(og.sino_shape, seed=50)
    b = inputs.gaussian(og.sino_shape, seed=51) if with_b else np.zeros(og.sino_shape, np.float32)
    v0 = inputs.gaussian(og.vol_shape, seed=52).reshape(case.params["vol_shape"] if case.ndim == 2 else og.vol_shape)
    alpha = -0.37
    vol = torch.from_numpy(v0).to(DEV)
    ad = torch.from_numpy(a.reshape(sshape)).to(DEV)
    bd = torch.from_numpy(b.reshape(sshape)).to(DEV) if with_b else None
    ops.adjoint_update(vol, ad, g, alpha, sino_b=bd)
    ref = torch.from_numpy(v0).to(DEV) + alpha * ops.adjoint(ad - bd if with_b else ad, g)
    assert rel_l2(host(vol), host(ref)) <= 1e-6
    ora = v0.astype(np.float64).ravel() + alpha * oracle.adjoint(og, (a.astype(np.float64) - b)).ravel()
    assert rel_l2(host(vol).ravel(), ora) <= 1e-5


def test_adjoint_update_bf16(ops):
    from cases import SMALL
    case = next(c for c in SMALL if c.name == "cone")
    g = case.library_geometry()
    og = case.oracle_geometry()
    a = torch.from_numpy(inputs.gaussian(og.sino_shape, seed=53)).to(DEV).bfloat16()
    b = torch.from_numpy(inputs.gaussian(og.sino_shape, seed=54)).to(DEV).bfloat16()
    v = torch.from_numpy(inputs.gaussian(og.vol_shape, seed=55)).to(DEV).bfloat16()
    ref = v.double().cpu().numpy().ravel() + 0.5 * oracle.adjoint(og, host(a) - host(b)).ravel()
    ops.adjoint_update(v, a, g, 0.5, sino_b=b)
    assert rel_l2(host(v).ravel(), ref) <= 4e-3


def test_fused_gradient_step_autograd(ops):
    """operators.gradient_step (fused forward and backward) gives the values and the gradients of the
    unfused x - alpha A^T (A x - p) composed from the autograd operators."""
    tr = inputs.jittered_circular_trajectory(24, 2 * math.pi, 75.0, 120.0, 0.5, 0.2, seed=9)
    shape, sp = (28, 30, 32), (0.5, 0.5, 0.5)
    g = ops.Geometry.cone_from_positions(shape, sp, (32, 40), (0.6, 0.6), tr.src, tr.det_centre, tr.eu, tr.ev)
    x0 = torch.from_numpy(inputs.rasterise_ellipsoids(inputs.random_ellipsoids(6, 7.0, 13), shape, sp)).to(DEV)
    p0 = torch.from_numpy(inputs.uniform(g.sinogram_shape, seed=14)).to(DEV)
    w = torch.from_numpy(inputs.gaussian(shape, seed=15)).to(DEV)
    outs, grads = [], []
    for fused in (True, False):
        x = x0.clone().requires_grad_(True)
        p = p0.clone().requires_grad_(True)
        alpha = torch.tensor(0.01, device=DEV, requires_grad=True)
        if fused:
            y = ops.gradient_step(x, p, alpha, g)
        else:
            y = x - alpha * ops.project_adjoint(ops.project(x, g) - p, g)
        (y * w).sum().backward()
        outs.append(y.detach())
        grads.append((x.grad, p.grad, alpha.grad))
    assert rel_l2(host(outs[0]), host(outs[1])) <= 1e-6
    for a, b in zip(grads[0], grads[1]):
        assert rel_l2(host(a), host(b)) <= 1e-5


def test_unrolled_fused_matches_unfused(ops):
    from paper_2511_08427_gb300.unrolled import UnrolledGD
    tr = inputs.jittered_circular_trajectory(30, 2 * math.pi, 75.0, 120.0, 0.5, 0.2, seed=10)
    shape, sp = (32, 36, 40), (0.5, 0.5, 0.5)
    g = ops.Geometry.cone_from_positions(shape, sp, (40, 48), (0.6, 0.6), tr.src, tr.det_centre, tr.eu, tr.ev)
    x_true = torch.from_numpy(inputs.rasterise_ellipsoids(inputs.random_ellipsoids(8, 8.0, 16), shape, sp)).to(DEV)
    with torch.no_grad():
        p = ops.forward_project(x_true, g)
    res = []
    for fused in (True, False):
        m = UnrolledGD(g, iterations=5, checkpoint=True, fused=fused)
        x5 = m(p)
        ((x5 - x_true) ** 2).sum().backward()
        res.append((x5.detach(), m.alpha.grad.clone()))
    assert rel_l2(host(res[0][0]), host(res[1][0])) <= 1e-6
    assert rel_l2(host(res[0][1]), host(res[1][1])) <= 1e-5

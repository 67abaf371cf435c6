"""Pins of the FP64 oracle against facts that do not come from the oracle itself.

Each test checks the oracle (oracle/pyronn_oracle.c) against a closed form, an invariant, an
independent geometric construction or a brute-force system matrix, chosen so that a dropped
term, a wrong sign or index, or a transposed operand fails at least one of them:

  * geometry: P [S; 1] = 0, the isocentre maps to the detector centre with w = sid / sdd,
    positions-built matrices equal the circular ones, rescaled matrices normalise back, and
    u, v agree with an independent line-plane intersection (Sec. 2.4, Listing 1);
  * forward projection: axis-aligned rays give the exact discrete line sum (the hat function's
    Fourier transform sinc^2 vanishes at non-zero integers, so sampling at a step dividing the
    voxel integrates the hat basis exactly), the parallel-beam symmetry p(t + pi, u) =
    p(t, Nu - 1 - u), convergence to analytic chord lengths of ellipses / ellipsoids, and a
    brute-force system matrix on tiny grids (Sec. 2.1, ray-driven projection);
  * matched adjoint: <A x, y> = <x, A^T y> and the brute-force matrix transposed (Sec. 2.2);
  * voxel-driven back-projection: partition of unity, 1 / w^2 weights from independent depths,
    single-pixel footprints from an independent intersection (Sec. 2.1, voxel-driven);
  * filtered back-projection (Sec. 2.2, x = A^T F^T K F p): the filter taps are the inverse Fourier
    transform of the band-limited ramp (numerical integration), its DC and Nyquist responses, the
    divergent-beam cosine weight and scale from an independent source / pixel construction, and
    reconstructions of an analytic disk (parallel) and ball (FDK). Planted mistakes (no cosine
    weight, unsquared distance ratio, a tap sign) each fail at least one of them.
"""
import json
import math
import os

import numpy as np
import pytest

from paper_2511_08427_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ------------------------------------------------------------------------------------------------
# independent helpers (test-side geometry; no oracle code)
# ------------------------------------------------------------------------------------------------

def circ_frame(t, sid, sdd):
    c, s = math.cos(t), math.sin(t)
    S = np.array([sid * c, sid * s, 0.0])
    Dc = np.array([-(sdd - sid) * c, -(sdd - sid) * s, 0.0])
    eu = np.array([-s, c, 0.0])
    ev = np.array([0.0, 0.0, 1.0])
    return S, Dc, eu, ev


def detector_coords(X, S, Dc, eu, ev, nu, nv, du, dv):
    """(u, v) of the intersection of the line S -> X with the detector plane, and the depth ratio."""
    n = np.cross(eu, ev)
    lam = np.dot(Dc - S, n) / np.dot(X - S, n)
    I = S + lam * (X - S)
    u = np.dot(I - Dc, eu) / du + (nu - 1) / 2
    v = np.dot(I - Dc, ev) / dv + (nv - 1) / 2
    return u, v, 1.0 / lam


def voxel_centres(shape_zyx, spacing_zyx, offset_zyx=(0, 0, 0)):
    nz, ny, nx = shape_zyx
    z = (np.arange(nz) - (nz - 1) / 2) * spacing_zyx[0] + offset_zyx[0]
    y = (np.arange(ny) - (ny - 1) / 2) * spacing_zyx[1] + offset_zyx[1]
    x = (np.arange(nx) - (nx - 1) / 2) * spacing_zyx[2] + offset_zyx[2]
    Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
    return np.stack([X, Y, Z], axis=-1)  # (..., 3) world xyz


def hat(s):
    return np.maximum(0.0, 1.0 - np.abs(s))


def rays_from_geometry(g):
    """Per-ray (origin, unit direction) computed here from the views array (numpy inverses)."""
    nv, nu = g.det_shape
    out = []
    for n in range(g.n_views):
        r = g.views[n]
        for v in range(nv):
            for u in range(nu):
                if g.kind == 1:
                    P = r.reshape(3, 4)
                    Mi = np.linalg.inv(P[:, :3])
                    a = -Mi @ P[:, 3]
                    d = Mi @ np.array([u, v, 1.0])
                else:
                    Dc, eu, ev, d = r[0:3], r[3:6], r[6:9], r[9:12].copy()
                    su = (u - (nu - 1) / 2) * g.det_spacing[1] + g.det_offset[1]
                    sv = (v - (nv - 1) / 2) * g.det_spacing[0] + g.det_offset[0]
                    a = Dc + su * eu + sv * ev
                out.append((a, d / np.linalg.norm(d)))
    return out


def brute_system_matrix(g):
    """A[r, voxel] = dt * sum_k prod_a hat(q_a(k) - idx_a), with k over a generous range and every
    voxel visited explicitly (no floor / corner logic, no support-box test)."""
    nz, ny, nx = g.vol_shape
    sz, sy, sx = g.vol_spacing
    oz, oy, ox = g.vol_offset
    C = np.array([ox, oy, oz])
    ext = np.array([(nx + 1) * sx, (ny + 1) * sy, (nz + 1) * sz])
    K = int(np.ceil(np.linalg.norm(ext) / g.dt)) + 4
    ks = np.arange(-K, K + 1)
    ii, jj, kk = np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz), indexing="ij")
    rows = []
    for a, d in rays_from_geometry(g):
        c = a + np.dot(C - a, d) * d
        X = c[None, :] + ((ks + 0.5) * g.dt)[:, None] * d[None, :]
        qx = (X[:, 0] - ox) / sx + (nx - 1) / 2
        qy = (X[:, 1] - oy) / sy + (ny - 1) / 2
        qz = (X[:, 2] - oz) / sz + (nz - 1) / 2
        w = (hat(qx[:, None, None, None] - ii[None]) * hat(qy[:, None, None, None] - jj[None])
             * hat(qz[:, None, None, None] - kk[None])).sum(axis=0)       # (nx, ny, nz)
        rows.append(g.dt * np.transpose(w, (2, 1, 0)).ravel())
    return np.array(rows)


def ellipse_chords(ell, a, d):
    """Sum over ellipses of density * chord length of the line a + t d (2D, d unit)."""
    tot = 0.0
    for cx, cy, ax, bx, phi, rho in ell:
        c, s = math.cos(phi), math.sin(phi)
        px, py = a[0] - cx, a[1] - cy
        p0 = np.array([px * c + py * s, -px * s + py * c])
        q = np.array([d[0] * c + d[1] * s, -d[0] * s + d[1] * c])
        A = (q[0] / ax) ** 2 + (q[1] / bx) ** 2
        B = 2 * (p0[0] * q[0] / ax ** 2 + p0[1] * q[1] / bx ** 2)
        Cc = (p0[0] / ax) ** 2 + (p0[1] / bx) ** 2 - 1
        disc = B * B - 4 * A * Cc
        if disc > 0:
            tot += rho * math.sqrt(disc) / A
    return tot


def ellipsoid_chords(ell, a, d):
    tot = 0.0
    for e in ell:
        cen, axes, rho = e[0:3], e[3:6], e[9]
        R = inputs.euler_zyz(*e[6:9])
        p0 = R.T @ (a - cen)
        q = R.T @ d
        A = np.sum((q / axes) ** 2)
        B = 2 * np.sum(p0 * q / axes ** 2)
        Cc = np.sum((p0 / axes) ** 2) - 1
        disc = B * B - 4 * A * Cc
        if disc > 0:
            tot += rho * math.sqrt(disc) / A
    return tot


def rel_l2(a, b):
    return float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / np.linalg.norm(np.ravel(b)))


# ------------------------------------------------------------------------------------------------
# geometry pins (Sec. 2.4, Listing 1)
# ------------------------------------------------------------------------------------------------

def test_listing1_geometry_pins(oracle_lib):
    o = oracle_lib
    p = json.load(open(os.path.join(GOLDEN, "listing1_params.json")))
    assert p["angular_range"] == "2*pi"
    V, sid, sdd = p["number_of_projections"], p["sid"], p["sdd"]
    nv, nu = p["detector_shape"]
    dv, du = p["detector_spacing"]
    g = o.cone_circular(tuple(p["volume_shape"]), tuple(p["volume_spacing"]), (nv, nu), (dv, du),
                        V, 2 * math.pi, sid, sdd)
    src, det, eu, ev = o.circular_frames(V, 2 * math.pi, sid, sdd)
    for n in range(0, V, 37):
        P = g.views[n].reshape(3, 4)
        # the source is the projection centre: P [S; 1] = 0
        assert np.allclose(P @ np.append(src[n], 1.0), 0.0, atol=1e-9)
        # the isocentre projects to the detector centre with depth ratio sid / sdd
        a, b, w = P @ np.array([0.0, 0.0, 0.0, 1.0])
        assert abs(a / w - (nu - 1) / 2) < 1e-9 and abs(b / w - (nv - 1) / 2) < 1e-9
        assert abs(w - sid / sdd) < 1e-12
        # the detector centre itself has w = 1
        a, b, w = P @ np.append(det[n], 1.0)
        assert abs(w - 1.0) < 1e-12 and abs(a / w - (nu - 1) / 2) < 1e-9
        # frames follow the stated orbit
        t = n * 2 * math.pi / V
        S, Dc, e1, e2 = circ_frame(t, sid, sdd)
        assert np.allclose(src[n], S, atol=1e-12) and np.allclose(det[n], Dc, atol=1e-12)
        assert np.allclose(eu[n], e1, atol=1e-15) and np.allclose(ev[n], e2)


def test_projection_matches_independent_intersection(oracle_lib):
    o = oracle_lib
    nv, nu, dv, du = 9, 13, 0.7, 0.9
    g = o.cone_circular((5, 6, 7), (0.5, 0.6, 0.7), (nv, nu), (dv, du), 7, 2 * math.pi, 60.0, 100.0)
    rng = np.random.default_rng(3)
    for n in range(g.n_views):
        S, Dc, eu, ev = circ_frame(n * 2 * math.pi / 7, 60.0, 100.0)
        P = g.views[n].reshape(3, 4)
        for _ in range(5):
            X = rng.uniform(-3, 3, size=3)
            a, b, w = P @ np.append(X, 1.0)
            u, v, ww = detector_coords(X, S, Dc, eu, ev, nu, nv, du, dv)
            assert abs(a / w - u) < 1e-9 and abs(b / w - v) < 1e-9 and abs(w - ww) < 1e-12


def test_positions_equal_circular_and_normalisation(oracle_lib):
    o = oracle_lib
    V = 24
    tr = inputs.jittered_circular_trajectory(V, 2 * math.pi, 750.0, 1200.0, 0.0, 0.0, seed=5)
    g1 = o.cone_circular((8, 8, 8), (1, 1, 1), (6, 10), (0.8, 0.7), V, 2 * math.pi, 750.0, 1200.0)
    g2 = o.cone_from_positions((8, 8, 8), (1, 1, 1), (6, 10), (0.8, 0.7), tr.src, tr.det_centre, tr.eu, tr.ev)
    assert np.allclose(g1.views, g2.views, rtol=0, atol=1e-12)
    # any non-zero rescaling (including a sign flip) normalises back to the same matrices
    scale = np.random.default_rng(1).uniform(0.1, 10.0, size=V) * np.where(np.arange(V) % 2 == 0, 1, -1)
    g3 = o.cone_from_matrices((8, 8, 8), (1, 1, 1), (6, 10), (0.8, 0.7), g1.views * scale[:, None])
    assert np.allclose(g3.views, g1.views, rtol=1e-12, atol=1e-14)


def test_helical_orbit_advance_and_centring(oracle_lib):
    """Helical orbit (pitch h): the source and detector centre rise by h per full turn, linearly in the
    view index, the trajectory is centred on z = 0, and the in-plane frames equal the circular ones."""
    o = oracle_lib
    V, rng_, sid, sdd, h = 30, 4 * math.pi, 600.0, 1000.0, 7.5
    src, det, eu, ev = o.circular_frames(V, rng_, sid, sdd, h)
    src0, det0, eu0, ev0 = o.circular_frames(V, rng_, sid, sdd, 0.0)
    rise = h * (rng_ / V) / (2 * math.pi)            # pitch x fraction of a turn per view
    assert np.allclose(np.diff(src[:, 2]), rise, rtol=0, atol=1e-12)
    assert abs(src[:, 2].mean()) < 1e-12
    assert abs(src[-1, 2] - src[0, 2] - h * (V - 1) / V * 2) < 1e-12      # two turns, V - 1 steps
    assert np.array_equal(det[:, 2], src[:, 2])
    assert np.allclose(src[:, :2], src0[:, :2], atol=0) and np.allclose(det[:, :2], det0[:, :2], atol=0)
    assert np.array_equal(eu, eu0) and np.array_equal(ev, ev0)


# ------------------------------------------------------------------------------------------------
# forward projection pins (Sec. 2.1)
# ------------------------------------------------------------------------------------------------

def test_axis_aligned_rays_are_exact_discrete_line_sums(oracle_lib):
    """Parallel view at t = 0: rays along -x at height y_u. With dt dividing the voxel, the sampled
    sum of the x-hat basis is exactly 1 per voxel, so p(u) = sx * sum_{i,j} f[j, i] hat(q_y - j)."""
    o = oracle_lib
    ny, nx, sy, sx = 11, 9, 1.3, 1.0
    for dt in (0.5, 0.25, 1.0 / 3.0):
        g = o.parallel2d((ny, nx), (sy, sx), 17, 0.9, 1, math.pi, det_offset=0.137, dt=dt * sx)
        f = np.random.default_rng(0).random((ny, nx))
        p = o.fp(g, f)[0, 0]
        for u in range(17):
            yu = (u - 8) * 0.9 + 0.137          # eu = (0, 1) at t = 0
            qy = yu / sy + (ny - 1) / 2
            expect = sx * sum(f[j, :].sum() * hat(qy - j) for j in range(ny))
            assert abs(p[u] - expect) < 1e-12 * max(1.0, abs(expect))


def test_axis_aligned_3d_rays_trilinear(oracle_lib):
    """3D parallel rays along -z and along +x: exact sums of the bilinear cross-section interpolant."""
    o = oracle_lib
    nz, ny, nx = 7, 6, 5
    sp = (0.5, 0.8, 1.1)
    f = np.random.default_rng(2).random((nz, ny, nx))
    views = np.array([[0, 0, 0, 1, 0, 0, 0, 1, 0, 0, 0, -1.0],       # rays along -z, eu = x, ev = y
                      [0, 0, 0, 0, 1, 0, 0, 0, 1, 1.0, 0, 0]])       # rays along +x, eu = y, ev = z
    g = o.parallel_from_views((nz, ny, nx), sp, (5, 7), (0.61, 0.47), views, det_offset=(0.05, -0.11),
                              dt=0.25 * 0.5)
    p = o.fp(g, f)
    for u in range(7):
        for v in range(5):
            su = (u - 3) * 0.47 - 0.11
            sv = (v - 2) * 0.61 + 0.05
            # view 0: x = su, y = sv; sum along z
            qx, qy = su / sp[2] + (nx - 1) / 2, sv / sp[1] + (ny - 1) / 2
            e0 = sp[0] * sum(f[:, j, i].sum() * hat(qx - i) * hat(qy - j) for j in range(ny) for i in range(nx))
            assert abs(p[0, v, u] - e0) < 1e-12
    g2 = o.parallel_from_views((nz, ny, nx), sp, (5, 7), (0.61, 0.47), views, det_offset=(0.05, -0.11),
                               dt=1.1 / 4)
    p2 = o.fp(g2, f)
    for u in range(7):
        for v in range(5):
            su = (u - 3) * 0.47 - 0.11
            sv = (v - 2) * 0.61 + 0.05
            qy, qz = su / sp[1] + (ny - 1) / 2, sv / sp[0] + (nz - 1) / 2
            e1 = sp[2] * sum(f[k, j, :].sum() * hat(qy - j) * hat(qz - k) for k in range(nz) for j in range(ny))
            assert abs(p2[1, v, u] - e1) < 1e-12


def test_constant_volume_axis_ray_and_sample_count(oracle_lib):
    o = oracle_lib
    nx = 20
    g = o.parallel2d((8, nx), (1.0, 1.0), 5, 1.0, 1)
    p = o.fp(g, np.ones((8, nx)))[0, 0]
    assert abs(p[2] - nx * 1.0) < 1e-12            # central ray, fully inside
    # symmetric lattice: samples at (Nx-1)/2 +- (k + 1/2) dt inside (-1, Nx) -> 2 Nx + 2 per inner ray
    cnt = o.count_samples(g)
    assert cnt[0] == 5 * (2 * nx + 2)


def test_parallel_symmetry(oracle_lib):
    o = oracle_lib
    V = 12
    g = o.parallel2d((21, 19), (1.0, 0.9), 27, 0.95, V, 2 * math.pi)
    f = inputs.rasterise_ellipses(inputs.random_ellipses(6, 9.0, seed=8), (21, 19), (1.0, 0.9))
    p = o.fp(g, f)[:, 0, :]
    assert np.max(np.abs(p[V // 2:] - p[:V // 2, ::-1])) < 1e-12 * np.abs(p).max()


def test_volume_offset_is_a_world_translation(oracle_lib):
    """Moving the volume centre to o and the source and detector by the same o changes nothing: FP,
    matched adjoint and the weighted BP of an offset volume equal those of the centred volume seen
    from the source and detector translated by -o. This fixes where the offset enters the voxel
    centres, the sample positions and the ray's reference point (the point closest to the volume
    centre, which sets the sampling phase)."""
    o = oracle_lib
    rng = np.random.default_rng(8)
    shape, sp, off = (6, 7, 8), (0.9, 0.7, 0.8), (2.3, -4.1, 3.7)        # (z, y, x)
    oxyz = np.array([off[2], off[1], off[0]])
    V = 5
    src, det, eu, ev = o.circular_frames(V, 2 * math.pi, 40.0, 70.0)
    src, det = src + oxyz, det + oxyz          # the orbit follows the volume
    g1 = o.cone_from_positions(shape, sp, (9, 11), (0.9, 0.8), src, det, eu, ev, vol_offset=off)
    g0 = o.cone_from_positions(shape, sp, (9, 11), (0.9, 0.8), src - oxyz, det - oxyz, eu, ev)
    f = rng.random(shape)
    y = rng.random(g1.sino_shape)
    p1, p0 = o.fp(g1, f), o.fp(g0, f)
    assert p0.max() > 1.0 and rel_l2(p1, p0) < 1e-12
    assert rel_l2(o.adjoint(g1, y), o.adjoint(g0, y)) < 1e-12
    assert rel_l2(o.bp(g1, y, 1), o.bp(g0, y, 1)) < 1e-12
    # 2D parallel beam: the detector line through o instead of through the origin
    t = 0.4
    base = np.array([0, 0, 0, -math.sin(t), math.cos(t), 0, 0, 0, 1, -math.cos(t), -math.sin(t), 0])
    moved = base.copy()
    moved[0:3] = (oxyz[0], oxyz[1], 0.0)
    h1 = o.parallel_from_views((1, 7, 8), (1.0, 0.7, 0.8), (1, 13), (1.0, 0.6), [moved],
                               vol_offset=(0.0, off[1], off[2]), ndim=2)
    h0 = o.parallel_from_views((1, 7, 8), (1.0, 0.7, 0.8), (1, 13), (1.0, 0.6), [base], ndim=2)
    f2 = rng.random((1, 7, 8))
    q2 = rng.random(h1.sino_shape)
    assert o.fp(h0, f2).max() > 1.0 and rel_l2(o.fp(h1, f2), o.fp(h0, f2)) < 1e-12
    assert rel_l2(o.bp(h1, q2), o.bp(h0, q2)) < 1e-12


def test_fp_is_continuous_in_the_geometry(oracle_lib):
    """Sample weights vanish on the boundary of the open support box and the hat basis is continuous,
    so the forward projection is a continuous function of the geometry: rays lying exactly on a row
    boundary, through row centres, or on the support's edge (index -1 and N) agree with rays shifted a
    nanometre either way, to first order in the shift (parallel beam at t = 0, rays along -x)."""
    o = oracle_lib
    ny, nx = 7, 9
    f = np.random.default_rng(9).random((ny, nx)) + 0.5
    # bin u = 0 of a one-bin detector sits at y = ou; row j's centre is y = j - (ny - 1) / 2
    for yq in (-1.0, -0.5, 0.0, 0.5, 2.0, 3.5, 6.0, 7.0):
        y0 = yq - (ny - 1) / 2                      # index coordinate yq -> world y
        vals = []
        for eps in (-1e-9, 0.0, 1e-9):
            g = o.parallel2d((ny, nx), (1.0, 1.0), 1, 1.0, 1, math.pi, det_offset=y0 + eps, dt=0.25)
            vals.append(o.fp(g, f)[0, 0, 0])
        assert abs(vals[1] - vals[0]) < 1e-7 and abs(vals[2] - vals[1]) < 1e-7, (yq, vals)
        if yq in (-1.0, 7.0):                       # the support's edge: the line sum is zero there
            assert abs(vals[1]) < 1e-12
    # oblique cone rays: a small change of the source distance moves the projection a little
    g1 = o.cone_circular((6, 7, 8), (1.0, 1.0, 1.0), (9, 11), (1.0, 1.0), 3, 2 * math.pi, 40.0, 70.0)
    g2 = o.cone_circular((6, 7, 8), (1.0, 1.0, 1.0), (9, 11), (1.0, 1.0), 3, 2 * math.pi, 40.0 + 1e-9, 70.0)
    x = np.random.default_rng(10).random((6, 7, 8))
    assert np.max(np.abs(o.fp(g1, x) - o.fp(g2, x))) < 1e-6


def test_fp_converges_to_ellipse_chords(oracle_lib):
    """2D parallel beam, 10 random ellipses: rel-L2 to the analytic chord sums is small at 128^2
    and shrinks when the grid is refined (orientation or offset mistakes give O(1) errors)."""
    o = oracle_lib
    ell = inputs.random_ellipses(10, 64.0, seed=1)
    V, nb = 30, 91
    errs = []
    for n, s in ((128, 1.0), (256, 0.5)):
        img = inputs.rasterise_ellipses(ell, (n, n), (s, s))
        g = o.parallel2d((n, n), (s, s), nb, 1.4, V)
        p = o.fp(g, img)[:, 0, :]
        ref = np.zeros_like(p)
        for k in range(V):
            t = k * math.pi / V
            eu = np.array([-math.sin(t), math.cos(t)])
            d = -np.array([math.cos(t), math.sin(t)])
            for u in range(nb):
                ref[k, u] = ellipse_chords(ell, ((u - (nb - 1) / 2) * 1.4) * eu, d)
        errs.append(rel_l2(p, ref))
    assert errs[0] < 0.03, errs
    assert errs[1] < 0.7 * errs[0], errs


def test_cone_fp_converges_to_ellipsoid_chords(oracle_lib):
    o = oracle_lib
    ell = inputs.random_ellipsoids(8, 24.0, seed=3)
    V, nv, nu, du = 6, 24, 28, 3.0
    sid, sdd = 150.0, 250.0
    errs = []
    for n, s in ((32, 1.5), (64, 0.75)):
        vol = inputs.rasterise_ellipsoids(ell, (n, n, n), (s, s, s))
        g = o.cone_circular((n, n, n), (s, s, s), (nv, nu), (du, du), V, 2 * math.pi, sid, sdd)
        p = o.fp(g, vol)
        ref = np.zeros_like(p)
        for k in range(V):
            S, Dc, eu, ev = circ_frame(k * 2 * math.pi / V, sid, sdd)
            for v in range(nv):
                for u in range(nu):
                    X = Dc + (u - (nu - 1) / 2) * du * eu + (v - (nv - 1) / 2) * du * ev
                    d = (X - S) / np.linalg.norm(X - S)
                    ref[k, v, u] = ellipsoid_chords(ell, S, d)
        errs.append(rel_l2(p, ref))
    assert errs[0] < 0.12, errs
    assert errs[1] < 0.7 * errs[0], errs


@pytest.mark.parametrize("case", ["fan", "parallel", "cone", "cone_wide_fan"])
def test_brute_force_system_matrix(oracle_lib, case):
    o = oracle_lib
    if case == "fan":
        g = o.fan_circular((8, 8), (1.0, 1.1), 11, 1.7, 6, 2 * math.pi, 20.0, 35.0)
    elif case == "parallel":
        g = o.parallel2d((8, 7), (1.0, 1.2), 11, 1.1, 6, math.pi, det_offset=0.21)
    elif case == "cone_wide_fan":
        # ~100-degree fan (source 8 mm from the centre of a 6 mm volume, 3 mm pixels 12 mm away): the
        # regime of the GPU's extreme-fan tests, pinned here by the explicit matrix
        g = o.cone_circular((6, 6, 6), (1.0, 1.0, 1.0), (5, 9), (2.0, 3.0), 4, 2 * math.pi, 8.0, 12.0)
    else:
        g = o.cone_circular((6, 6, 6), (1.0, 0.9, 1.2), (5, 7), (1.6, 1.5), 4, 2 * math.pi, 25.0, 40.0,
                            det_offset=(0.3, -0.2))
    A = brute_system_matrix(g)
    rng = np.random.default_rng(4)
    x = rng.random(g.vol_shape)
    y = rng.standard_normal(g.sino_shape)
    assert np.max(np.abs(A @ x.ravel() - o.fp(g, x).ravel())) < 1e-12 * max(1, np.abs(A @ x.ravel()).max())
    aty = A.T @ y.ravel()
    assert np.max(np.abs(aty - o.adjoint(g, y).ravel())) < 1e-12 * max(1, np.abs(aty).max())


# ------------------------------------------------------------------------------------------------
# matched adjoint pins (Sec. 2.2)
# ------------------------------------------------------------------------------------------------

@pytest.mark.parametrize("case", ["parallel", "fan", "cone", "cone_matrices"])
def test_dot_product_adjoint(oracle_lib, case):
    o = oracle_lib
    if case == "parallel":
        g = o.parallel2d((33, 29), (1.0, 1.0), 45, 1.0, 17)
    elif case == "fan":
        g = o.fan_circular((32, 32), (0.5, 0.5), 40, 1.0, 19, 2 * math.pi, 100.0, 150.0)
    elif case == "cone":
        g = o.cone_circular((12, 14, 16), (0.5, 0.5, 0.5), (11, 13), (0.6, 0.6), 9, 2 * math.pi, 75.0, 120.0,
                            pitch=3.0)
    else:
        tr = inputs.jittered_circular_trajectory(7, 2 * math.pi, 75.0, 120.0, 0.5, 0.2, seed=5)
        g = o.cone_from_positions((10, 12, 14), (0.5, 0.5, 0.5), (12, 12), (0.6, 0.6), tr.src, tr.det_centre,
                                  tr.eu, tr.ev)
    rng = np.random.default_rng(11)
    x = rng.random(g.vol_shape)
    y = rng.standard_normal(g.sino_shape)
    lhs = float(np.vdot(o.fp(g, x), y))
    rhs = float(np.vdot(x, o.adjoint(g, y)))
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)
    # finite differences of <y, A x> along a random direction equal <A^T y, h> (the map is linear)
    h = rng.standard_normal(g.vol_shape)
    fd = (float(np.vdot(y, o.fp(g, x + 1e-3 * h))) - lhs) / 1e-3
    assert abs(fd - float(np.vdot(o.adjoint(g, y), h))) <= 1e-8 * max(1.0, abs(fd))


def test_adjoint_rays_subset_matches_full(oracle_lib):
    o = oracle_lib
    g = o.cone_circular((10, 10, 10), (1, 1, 1), (8, 9), (1.2, 1.2), 5, 2 * math.pi, 60.0, 100.0)
    y = np.zeros(g.sino_shape)
    ids = np.array([3, 77, 150, 222, 359])
    y.ravel()[ids] = [1.0, -2.0, 0.5, 3.0, 1.5]
    assert np.allclose(o.adjoint(g, y), o.adjoint_rays(g, ids, y.ravel()[ids]), atol=1e-13)


def test_fp_rays_and_bp_voxels_subsets_match_full(oracle_lib):
    """The sampled entry points used for full-size parity address rays as (view * Nv + v) * Nu + u and
    voxels as (k * Ny + j) * Nx + i, and return exactly the full operators' values there."""
    o = oracle_lib
    rng = np.random.default_rng(12)
    g = o.cone_circular((7, 9, 10), (1.0, 0.8, 1.1), (8, 11), (1.2, 1.0), 5, 2 * math.pi, 60.0, 100.0)
    x = rng.random(g.vol_shape)
    full = o.fp(g, x)
    ids = np.unique(rng.integers(0, full.size - 1, 60))      # below the last, so a planted "+ 1" stays in range
    assert np.array_equal(o.fp_rays(g, x, ids), full.ravel()[ids])
    q = rng.random(g.sino_shape)
    vids = np.unique(rng.integers(0, x.size - 1, 60))
    for w in (0, 1):
        assert np.array_equal(o.bp_voxels(g, q, vids, w), o.bp(g, q, w).ravel()[vids])


# ------------------------------------------------------------------------------------------------
# voxel-driven back-projection pins (Sec. 2.1)
# ------------------------------------------------------------------------------------------------

def test_bp_partition_of_unity_and_depth_weights(oracle_lib):
    o = oracle_lib
    sid, sdd, V = 80.0, 130.0, 8
    g = o.cone_circular((6, 7, 8), (1.0, 1.0, 1.0), (40, 50), (1.0, 1.0), V, 2 * math.pi, sid, sdd)
    ones = np.ones(g.sino_shape)
    assert np.allclose(o.bp(g, ones, 0), V, atol=1e-12)
    b = o.bp(g, ones, 1)
    Xs = voxel_centres(g.vol_shape, g.vol_spacing)
    expect = np.zeros(g.vol_shape)
    for n in range(V):
        S, Dc, eu, ev = circ_frame(n * 2 * math.pi / V, sid, sdd)
        nrm = np.cross(eu, ev)
        w = ((Xs - S) @ nrm) / np.dot(Dc - S, nrm)
        expect += 1.0 / w ** 2
    assert np.allclose(b, expect, rtol=1e-12)


def test_bp_single_pixel_footprint(oracle_lib):
    o = oracle_lib
    sid, sdd, nv, nu, dv, du = 50.0, 90.0, 9, 11, 0.8, 0.7
    g = o.cone_circular((7, 8, 9), (0.6, 0.5, 0.4), (nv, nu), (dv, du), 3, 2 * math.pi, sid, sdd)
    q = np.zeros(g.sino_shape)
    q[1, 4, 6] = 1.0
    b = o.bp(g, q, 0)
    Xs = voxel_centres(g.vol_shape, g.vol_spacing)
    S, Dc, eu, ev = circ_frame(1 * 2 * math.pi / 3, sid, sdd)
    expect = np.zeros(g.vol_shape)
    for idx in np.ndindex(*g.vol_shape):
        u, v, _ = detector_coords(Xs[idx], S, Dc, eu, ev, nu, nv, du, dv)
        expect[idx] = hat(u - 6) * hat(v - 4)
    assert expect.max() > 0.5
    assert np.allclose(b, expect, atol=1e-12)


def test_bp_voxels_behind_the_source_receive_nothing(oracle_lib):
    """Source inside the volume (sid 2.5 mm, voxels at x = -4 ... 4 mm): one view, an all-ones
    sinogram. A voxel in front of the source gets the bilinear interpolant of the ones (zero outside
    the detector) at its independently intersected (u, v), times 1 / w^2 in the weighted mode; a voxel
    behind the source plane, whose central projection lands on the detector through the source, gets
    nothing."""
    o = oracle_lib
    sid, sdd, nv, nu, dv, du = 2.5, 10.0, 31, 41, 1.0, 1.0
    g = o.cone_circular((5, 9, 9), (1.0, 1.0, 1.0), (nv, nu), (dv, du), 1, 2 * math.pi, sid, sdd)
    q = np.ones(g.sino_shape)
    Xs = voxel_centres(g.vol_shape, g.vol_spacing)
    S, Dc, eu, ev = circ_frame(0.0, sid, sdd)
    axis = (Dc - S) / np.linalg.norm(Dc - S)

    def ones_interp(s, n):
        return sum(hat(s - m) for m in range(n))

    for weight in (0, 1):
        b = o.bp(g, q, weight)
        n_behind = n_front = 0
        for idx in np.ndindex(*g.vol_shape):
            X = Xs[idx]
            if np.dot(X - S, axis) <= 0:
                assert b[idx] == 0.0
                u, v, _ = detector_coords(X, S, Dc, eu, ev, nu, nv, du, dv)
                n_behind += ones_interp(u, nu) * ones_interp(v, nv) > 0.5
                continue
            u, v, w = detector_coords(X, S, Dc, eu, ev, nu, nv, du, dv)
            expect = ones_interp(u, nu) * ones_interp(v, nv) * (1.0 / (w * w) if weight else 1.0)
            n_front += expect > 0
            assert abs(b[idx] - expect) < 1e-12 * max(1.0, expect)
        # the case is live: behind-source voxels that would land on the detector, and lit voxels in front
        assert n_behind > 10 and n_front > 100


def test_parallel_bp_constant_along_rays(oracle_lib):
    o = oracle_lib
    g = o.parallel2d((9, 12), (1.0, 1.0), 15, 1.0, 1)
    q = np.random.default_rng(0).random(g.sino_shape)
    b = o.bp(g, q)[0]
    # t = 0: rays along -x, so the back-projection is constant along x and equals the sinogram
    # linearly interpolated at the row height y_j (bins centred: u = y_j + (15 - 1) / 2)
    assert np.allclose(b, b[:, :1], atol=1e-14)
    for j in range(9):
        u = (j - 4) + 7
        assert abs(b[j, 0] - q[0, 0, u]) < 1e-14


def test_parallel_bp_detector_offset(oracle_lib):
    """Parallel beam with the detector shifted by ou along eu: a voxel at signed distance s along eu
    reads bin (s - ou) / du + (Nu - 1) / 2, at t = 0 (s = y) and at an oblique angle."""
    o = oracle_lib
    ny, nx, nu, du, ou = 9, 12, 19, 0.8, 1.37
    for t in (0.0, 0.7):
        view = [0, 0, 0, -math.sin(t), math.cos(t), 0, 0, 0, 1, -math.cos(t), -math.sin(t), 0]
        g = o.parallel_from_views((1, ny, nx), (1.0, 1.0, 1.0), (1, nu), (1.0, du), [view], det_offset=(0.0, ou),
                                  ndim=2)
        q = np.random.default_rng(4).random(g.sino_shape)
        b = o.bp(g, q)[0]
        Xs = voxel_centres(g.vol_shape, g.vol_spacing)[0]
        for j in range(ny):
            for i in range(nx):
                s_ = Xs[j, i, 0] * -math.sin(t) + Xs[j, i, 1] * math.cos(t)
                uc = (s_ - ou) / du + (nu - 1) / 2
                expect = sum(q[0, 0, m] * hat(uc - m) for m in range(nu))
                assert abs(b[j, i] - expect) < 1e-13


# ------------------------------------------------------------------------------------------------
# filtered back-projection (Sec. 2.2: x = A^T F^T K F p)
# ------------------------------------------------------------------------------------------------

def _impulse_response(o, filt, nu=41):
    """Filter output of a unit impulse at the centre bin of a 1-view parallel geometry (du = 1), with
    the oracle's scale pi / V = pi removed: the taps h(u - c)."""
    g = o.parallel2d((8, 8), (1.0, 1.0), nu, 1.0, 1)
    p = np.zeros(g.sino_shape)
    p[0, 0, nu // 2] = 1.0
    return o.fbp_filter(g, p, filt)[0, 0] / math.pi


@pytest.mark.parametrize("filt", [0, 1])
def test_ramp_taps_are_the_band_limited_ramp(oracle_lib, filt):
    """The taps at unit spacing are the inverse Fourier transform of the ramp |f| band-limited to the
    detector's Nyquist frequency (times the sinc window for Shepp-Logan), evaluated at the bins."""
    from scipy.integrate import quad
    h = _impulse_response(oracle_lib, filt)
    c = h.size // 2
    for k in range(-6, 7):
        if filt == 0:
            ref = 2 * quad(lambda f: f * math.cos(2 * math.pi * f * k), 0.0, 0.5, limit=200)[0]
        else:
            ref = 2 * quad(lambda f: f * (math.sin(math.pi * f) / (math.pi * f) if f > 0 else 1.0) *
                           math.cos(2 * math.pi * f * k), 0.0, 0.5, limit=200)[0]
        assert abs(h[c + k] - ref) < 1e-10, (k, h[c + k], ref)


@pytest.mark.parametrize("filt", [0, 1])
def test_ramp_filter_dc_and_nyquist_response(oracle_lib, filt):
    """A constant row is annihilated (the ramp vanishes at f = 0) and an alternating row is scaled by
    the response at the Nyquist frequency: 1/2 (Ram-Lak) or 1/pi (Shepp-Logan), up to the truncation
    of the taps at the row ends (checked at the centre of a long row)."""
    o = oracle_lib
    nu = 4001
    g = o.parallel2d((8, 8), (1.0, 1.0), nu, 1.0, 1)
    c = nu // 2
    dc = o.fbp_filter(g, np.ones(g.sino_shape), filt)[0, 0, c] / math.pi
    alt = o.fbp_filter(g, ((-1.0) ** np.arange(nu)).reshape(g.sino_shape), filt)[0, 0, c] / math.pi
    assert abs(dc) < 2e-4
    assert abs(alt - (0.5 if filt == 0 else 1.0 / math.pi)) < 2e-4


def test_fbp_parallel_reconstructs_a_disk(oracle_lib):
    """Parallel-beam FBP of the analytic projections 2 sqrt(R^2 - s^2) of a centred unit disk gives the
    disk: ~1 inside, ~0 outside (discretisation error only)."""
    o = oracle_lib
    n, nb, views, R = 128, 183, 300, 40.0
    g = o.parallel2d((n, n), (1.0, 1.0), nb, 1.0, views)
    s = np.arange(nb) - (nb - 1) / 2
    row = np.where(np.abs(s) < R, 2.0 * np.sqrt(np.maximum(R * R - s * s, 0.0)), 0.0)
    p = np.tile(row, (views, 1)).reshape(g.sino_shape)
    rec = o.fbp(g, p)[0]
    yy, xx = np.meshgrid(np.arange(n) - (n - 1) / 2, np.arange(n) - (n - 1) / 2, indexing="ij")
    r = np.hypot(xx, yy)
    assert abs(rec[r < R - 4].mean() - 1.0) < 0.01
    assert abs(rec[r > R + 4].mean()) < 0.01
    assert np.abs(rec[r < R - 4] - 1.0).max() < 0.05


def test_fdk_reconstructs_a_ball(oracle_lib):
    """FDK (cosine weights, ramp, 1/w^2 back-projection) of analytic cone-beam line integrals of a
    centred unit ball, computed from an independent source / pixel construction: ~1 inside the
    central slice, ~0 outside."""
    o = oracle_lib
    n, nd, views, R, sid, sdd, du = 48, 96, 240, 14.0, 200.0, 400.0, 1.0
    g = o.cone_circular((n, n, n), (1.0, 1.0, 1.0), (nd, nd), (du, du), views, 2 * math.pi, sid, sdd)
    p = np.zeros(g.sino_shape)
    uu, vv = np.meshgrid(np.arange(nd), np.arange(nd), indexing="xy")
    for k in range(views):
        S, Dc, eu, ev = circ_frame(k * 2 * math.pi / views, sid, sdd)
        P = Dc[None, None] + ((uu - (nd - 1) / 2) * du)[..., None] * eu + ((vv - (nd - 1) / 2) * du)[..., None] * ev
        d = P - S
        d /= np.linalg.norm(d, axis=-1, keepdims=True)
        t = -(S[None, None] * d).sum(-1)
        dist2 = np.maximum((S * S).sum() - t * t, 0.0)
        p[k] = 2.0 * np.sqrt(np.maximum(R * R - dist2, 0.0))
    rec = o.fbp(g, p)
    mid = rec[n // 2 - 1:n // 2 + 1].mean(axis=0)
    yy, xx = np.meshgrid(np.arange(n) - (n - 1) / 2, np.arange(n) - (n - 1) / 2, indexing="ij")
    r = np.hypot(xx, yy)
    assert abs(mid[r < R - 3].mean() - 1.0) < 0.02
    assert abs(mid[r > R + 3].mean()) < 0.02


def test_fdk_cosine_weight_from_independent_geometry(oracle_lib):
    """The pre-weight of divergent beams is the cosine of each pixel's ray to the detector normal, and
    the output scale is (pi / V) r^2 / tau with r = sid / sdd and tau = du r: rows equal to 1 / cos
    (computed here from the source and pixel positions) become rows of ones after weighting, so the
    output is the ones-row convolved with the impulse response (pinned above) times that scale."""
    o = oracle_lib
    nd, sid, sdd, du = 101, 100.0, 150.0, 0.7
    g = o.cone_circular((8, 8, 8), (1.0, 1.0, 1.0), (3, nd), (du, du), 1, 2 * math.pi, sid, sdd)
    S, Dc, eu, ev = circ_frame(0.0, sid, sdd)
    u = np.arange(nd)
    for v in range(3):
        P = Dc[None] + ((u - (nd - 1) / 2) * du)[:, None] * eu[None] + ((v - 1) * du) * ev[None]
        cosw = sdd / np.linalg.norm(P - S, axis=1)
        p = np.zeros(g.sino_shape)
        p[0, v] = 1.0 / cosw
        q = o.fbp_filter(g, p)[0, v]
        h = _impulse_response(o, 0, nu=2 * nd + 1)   # taps at offsets -nd .. nd
        r = sid / sdd
        conv = np.array([h[nd + (k - np.arange(nd))].sum() for k in range(nd)])
        expected = math.pi * r * r / (du * r) * conv
        assert np.abs(q - expected).max() < 1e-10 * np.abs(expected).max(), v


# ------------------------------------------------------------------------------------------------
# acquisition-artifact simulations (Sec. 2.4)
# ------------------------------------------------------------------------------------------------

def test_artifact_references():
    from oracle import artifacts
    check_artifact_references(artifacts)


def check_artifact_references(A):
    """Jitter by zero is the identity and by s moves every value s pixels (zero fill); noise adds mean
    plus std times the sample; ring gains touch only the chosen columns and views; the blur kernel has
    unit weight (interior sums preserved), blurs a point into a segment of L pixels of weight 1/L along
    the view angle (u at 0, v at pi/2, the diagonal at pi/4), leaves a linear ramp unchanged away from
    the edges at any angle (a symmetric average of a linear function, sampled bilinearly, is its
    centre value), and L = 1 is the identity."""
    rng = np.random.default_rng(0)
    p = rng.random((3, 9, 11))
    assert np.array_equal(A.detector_jitter(p, np.zeros((3, 9), int), 0), p)
    s = np.full((3, 9), 2)
    j = A.detector_jitter(p, s, 0)
    assert np.array_equal(j[:, :, 2:], p[:, :, :-2]) and not j[:, :, :2].any()
    j = A.detector_jitter(p, np.full((3, 11), -1), 1)
    assert np.array_equal(j[:, :-1, :], p[:, 1:, :]) and not j[:, -1, :].any()
    r = A.ring_artifacts(p, [3, 7], [0.0, 1.5], 1, 3)
    assert np.array_equal(r[0], p[0]) and not r[1:, :, 3].any()
    assert np.allclose(r[1:, :, 7], 1.5 * p[1:, :, 7]) and np.array_equal(r[:, :, 5], p[:, :, 5])
    assert np.allclose(A.motion_blur(p, [0.3, 1.0, 2.0], 1), p)
    d = np.zeros((2, 15, 15))
    d[:, 7, 7] = 1.0
    b = A.motion_blur(d, [0.0, math.pi / 2], 5)
    row = np.zeros(15)
    row[5:10] = 0.2
    assert np.allclose(b[0, 7], row) and np.allclose(b[0].sum(), 1.0)
    assert np.allclose(b[1][:, 7], row) and np.allclose(b[1].sum(), 1.0)
    b = A.motion_blur(d, [0.7, 2.1], 4)
    assert np.allclose(b.sum(axis=(1, 2)), 1.0)
    # pi / 4, L = 3 (t = -1, 0, 1): only t = -1 from (8, 8) and t = 1 from (6, 6) reach the point, each
    # with bilinear weight (1 / sqrt 2)^2 = 1/2; at (7, 7) t = 0 hits it and t = +-1 each add
    # (1 - 1 / sqrt 2)^2; the anti-diagonal neighbours get nothing
    b = A.motion_blur(d[:1], [math.pi / 4], 3)[0]
    assert abs(b[8, 8] - 1 / 6) < 1e-12 and abs(b[6, 6] - 1 / 6) < 1e-12
    assert abs(b[7, 7] - (1 + 2 * (1 - 1 / math.sqrt(2)) ** 2) / 3) < 1e-12
    assert b[6, 8] == 0.0 and b[8, 6] == 0.0
    vv, uu = np.meshgrid(np.arange(15.0), np.arange(15.0), indexing="ij")
    ramp = np.broadcast_to(0.3 * uu - 0.7 * vv + 2.0, (3, 15, 15))
    b = A.motion_blur(ramp, [0.4, 1.9, 3.5], 5)
    assert np.allclose(b[:, 3:12, 3:12], ramp[:, 3:12, 3:12], rtol=0, atol=1e-12)
    z = rng.standard_normal(p.shape)
    assert np.allclose(A.gaussian_noise(p, np.zeros_like(p), 0.25, 3.0), p + 0.25, rtol=0, atol=1e-15)
    assert np.allclose(A.gaussian_noise(p, z, 0.0, 2.0) - p, 2.0 * z, rtol=0, atol=1e-14)
    r = A.ring_artifacts(p, [4], [0.5], 0, 2)
    assert np.allclose(r[:2, :, 4], 0.5 * p[:2, :, 4]) and np.array_equal(r[2], p[2])

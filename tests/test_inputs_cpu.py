"""The seeded input generators follow the stated workload recipe: they are deterministic per seed,
their phantoms lie where the recipe puts them and rasterise to the right sizes, the jittered
trajectory reduces to the circular orbit at zero jitter and keeps orthonormal detector axes, and the
batched workload has the listed sizes. (The generators hold no operator arithmetic.)"""
import math

import numpy as np

from paper_2511_08427_gb300 import inputs


def test_generators_are_deterministic_per_seed():
    assert np.array_equal(inputs.random_ellipsoids(20, 64.0, seed=3), inputs.random_ellipsoids(20, 64.0, seed=3))
    assert not np.array_equal(inputs.random_ellipsoids(20, 64.0, seed=3), inputs.random_ellipsoids(20, 64.0, seed=4))
    assert np.array_equal(inputs.gaussian((5, 7), seed=1), inputs.gaussian((5, 7), seed=1))
    assert inputs.gaussian((5, 7), seed=1).dtype == np.float32


def test_phantoms_lie_inside_the_field_of_view():
    e2 = inputs.random_ellipses(200, 50.0, seed=1)
    r = np.hypot(e2[:, 0], e2[:, 1])
    assert np.all(r <= 0.45 * 50.0) and np.all(r + np.maximum(e2[:, 2], e2[:, 3]) < 50.0)
    assert np.all((e2[:, 5] >= 0) & (e2[:, 5] < 1)) and np.all((e2[:, 4] >= 0) & (e2[:, 4] < math.pi))
    e3 = inputs.random_ellipsoids(200, 50.0, seed=2)
    r = np.linalg.norm(e3[:, 0:3], axis=1)
    assert np.all(r <= 0.45 * 50.0)
    assert np.all((e3[:, 3:6] >= 0.05 * 50.0) & (e3[:, 3:6] <= 0.35 * 50.0))


def test_rasterised_sizes_match_areas_and_volumes():
    # one axis-aligned ellipse (a = 20, b = 10 mm, density 0.7) on a 0.25 mm grid: area pi a b
    ell = np.array([[3.0, -2.0, 20.0, 10.0, 0.0, 0.7]])
    img = inputs.rasterise_ellipses(ell, (200, 240), (0.25, 0.25))
    assert abs((img > 0).sum() * 0.25 ** 2 / (math.pi * 20 * 10) - 1) < 0.01
    assert set(np.unique(img)) <= {0.0, np.float32(0.7)}
    # a rotated ellipsoid (8, 5, 3 mm): volume 4/3 pi a b c, unchanged by the rotation
    for ang in ((0.0, 0.0, 0.0), (0.7, 1.1, 2.3)):
        e = np.array([[1.0, -0.5, 0.25, 8.0, 5.0, 3.0, *ang, 1.0]])
        vol = inputs.rasterise_ellipsoids(e, (48, 64, 64), (0.4, 0.4, 0.4))
        assert abs(vol.sum() * 0.4 ** 3 / (4 / 3 * math.pi * 8 * 5 * 3) - 1) < 0.02


def test_jittered_trajectory():
    V, sid, sdd = 240, 750.0, 1200.0
    tr0 = inputs.jittered_circular_trajectory(V, 2 * math.pi, sid, sdd, 0.0, 0.0, seed=5)
    t = np.arange(V) * 2 * math.pi / V
    assert np.allclose(tr0.src, np.stack([sid * np.cos(t), sid * np.sin(t), 0 * t], 1), atol=1e-12)
    assert np.allclose(tr0.det_centre, np.stack([-(sdd - sid) * np.cos(t), -(sdd - sid) * np.sin(t), 0 * t], 1),
                       atol=1e-12)
    tr = inputs.jittered_circular_trajectory(V, 2 * math.pi, sid, sdd, 0.5, 0.2, seed=5)
    d = tr.src - tr0.src
    assert 0.4 < d.std() < 0.6 and abs(d.mean()) < 0.1           # N(0, 0.5 mm) per coordinate
    for n in range(V):
        assert abs(np.dot(tr.eu[n], tr.ev[n])) < 1e-12
        assert abs(np.linalg.norm(tr.eu[n]) - 1) < 1e-12 and abs(np.linalg.norm(tr.ev[n]) - 1) < 1e-12
    tilt = np.degrees(np.arccos(np.clip(tr.ev[:, 2], -1, 1)))
    assert 0.05 < np.median(tilt) < 0.6                          # axes rotated by angles ~ N(0, 0.2 deg)


def test_batched_workload_sizes():
    w = inputs.batched_cone_workload()
    sides = [x["side"] for x in w]
    assert len(w) == 16 and sides[0] == 96 and sides[-1] == 256 and sides == sorted(sides)
    assert all(s % 8 == 0 for s in sides)                        # BF16 rows a multiple of 16 bytes
    assert [x["views"] for x in w][::5] == [180, 300, 420, 540]
    assert all((x["pitch"] == 0) == (x["index"] % 2 == 0) for x in w)
    for x in w:                                                  # the shadow fills 90 % of the detector
        mag = x["sdd"] / x["sid"]
        assert abs(mag * x["side"] * x["voxel_mm"] * math.sqrt(2) / (x["det"] * x["du"]) - 0.9) < 1e-12

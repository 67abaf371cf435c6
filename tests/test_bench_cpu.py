"""Host logic of bench.py on CPU: the reference arm's JSON line, and the oracle sub-geometries its CPU
legs time (a subset of views, a band of detector rows)."""
import json
import math
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def test_reference_arm_line_on_rank_zero(monkeypatch, capsys):
    """Rank 0 prints one JSON line with the reference arm's keys: the timed steps' rate as value, e2e with
    no host-device bytes, and a cpu_baseline that carries the all-core and the single-core oracle rates.
    The oracle timings are replaced by fixed numbers here; the line's arithmetic is what is checked."""
    import bench
    import oracle
    monkeypatch.setenv("RANK", "0")
    monkeypatch.setattr(bench, "build_volume", lambda name, rank=0: np.zeros((2, 2, 2), np.float32))

    class G:
        n_views = 720

    monkeypatch.setattr(bench, "oracle_geometry", lambda name: G())
    calls = []

    def fake_views(og, vol64, ids):
        calls.append(list(ids))
        return None, 1_500_000 * len(ids), 1.0 * len(ids)   # 1.5e6 samples per view, 1 s per view

    monkeypatch.setattr(bench, "oracle_fp_views", fake_views)
    monkeypatch.setattr(bench, "oracle_single_core_rate", lambda og, vol, view: (0.001, 1_000_000, 1.0))
    monkeypatch.setattr(oracle, "max_threads", lambda: 8)

    class A:
        warmup, steps, gpus, ref_seconds, workload = 3, 2, 1, 4.0, "cone512_jitter"

    assert bench.run_reference(A()) == 0
    lines = [ln for ln in capsys.readouterr().out.splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    # one sizing call of one view, then warmup + steps calls of round(4 s / 1 s) = 4 views each
    assert len(calls) == 1 + 5 and calls[0] == [1] and all(len(c) == 4 for c in calls[1:])
    assert all(0 <= v < 720 for c in calls for v in c)
    assert d["impl"] == "reference" and d["steps"] == 2 and d["warmup"] == 3
    assert abs(d["value"] - 1.5e-3) < 1e-12 and d["unit"] == "G ray-samples/s"
    assert d["config"]["workload"].startswith("arbitrary-trajectory cone beam 512^3")
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] == 8 and cb["value"] == d["value"]
    assert cb["single_core"]["cores"] == 1 and abs(cb["single_core"]["value"] - 0.001) < 1e-15


def test_reference_arm_skips_other_ranks(monkeypatch):
    import bench
    monkeypatch.setenv("RANK", "1")

    class A:
        warmup, steps, gpus, ref_seconds, workload = 3, 2, 2, 1.0, "cone512_jitter"

    assert bench.run_reference(A()) == 0


def test_oracle_subset_views_and_row_band_equal_the_full_projection(oracle_lib):
    """The CPU legs time the oracle on whole views and on a band of detector rows of one view: both
    sub-geometries give exactly the corresponding entries of the full forward projection and sample
    counts that add up (a jittered trajectory, so every view has its own matrix)."""
    import bench
    import oracle
    from paper_2511_08427_gb300 import inputs
    tr = inputs.jittered_circular_trajectory(6, 2 * math.pi, 75.0, 120.0, 0.5, 0.2, seed=3)
    og = oracle.cone_from_positions((10, 12, 14), (0.5, 0.5, 0.5), (9, 11), (0.6, 0.6), tr.src, tr.det_centre, tr.eu,
                                    tr.ev)
    x = inputs.rasterise_ellipsoids(inputs.random_ellipsoids(5, 3.0, 4), (10, 12, 14), (0.5, 0.5, 0.5))
    full = oracle.fp(og, x)
    sub, samples, _ = bench.oracle_fp_views(og, np.asarray(x, np.float64), [4, 1])
    assert np.array_equal(sub, full[[4, 1]])
    assert samples == int(oracle.count_samples(og)[[4, 1]].sum())
    band = bench.oracle_subset(og, [2], rows=(3, 7))
    assert band.det_shape == (4, 11)
    np.testing.assert_allclose(oracle.fp(band, x)[0], full[2, 3:7], rtol=1e-12, atol=1e-12)

"""The library's autotuner (pyronn_autotune through autotune.tune) on the GPU: for each operator it
times at least one candidate, leaves the chosen configuration applied, the tuned operator still matches
the FP64 oracle, and a second process-level call re-applies the cached choice without timing. Every
value of the knobs it sets (adjoint slab depth, back-projector brick depth) computes the same operator."""
import numpy as np
import pytest
import torch

import oracle
from paper_2511_08427_gb300 import inputs

from cases import SMALL, rel_l2

pytestmark = pytest.mark.gpu
DEV = "cuda:0"
CASE = next(c for c in SMALL if c.name == "cone_tma_rows")


@pytest.fixture(scope="module")
def ops():
    from paper_2511_08427_gb300 import build
    build.build()
    from paper_2511_08427_gb300 import operators
    return operators


def host(t):
    return t.float().cpu().numpy().astype(np.float64)


def _check_operator(ops, g, og, op):
    if op == "fp":
        x = CASE.phantom()
        got = host(ops.forward_project(torch.from_numpy(x).to(DEV), g))
        assert rel_l2(got, oracle.fp(og, x)) <= 1e-5
    elif op == "adjoint":
        y = inputs.gaussian(og.sino_shape, seed=81)
        got = host(ops.adjoint(torch.from_numpy(y).to(DEV), g))
        assert rel_l2(got, oracle.adjoint(og, y)) <= 1e-5
    else:
        y = inputs.uniform(og.sino_shape, seed=82)
        got = host(ops.back_project(torch.from_numpy(y).to(DEV), g))
        assert rel_l2(got, oracle.bp(og, y)) <= 1e-5


@pytest.mark.parametrize("op", ["fp", "adjoint", "bp"])
def test_autotune_applies_its_choice_and_keeps_the_operator(ops, op, tmp_path, monkeypatch):
    from paper_2511_08427_gb300 import autotune
    monkeypatch.setenv("PYRONN_TUNE_CACHE", str(tmp_path / "tune.json"))
    g = CASE.library_geometry()
    og = CASE.oracle_geometry()
    r = autotune.tune(g, op, repeats=2)
    assert not r["cached"] and r["candidates"] >= 1 and r["ms"] > 0.0
    a, b = r["params"]
    if op == "fp":
        assert g.fp_config()["kernel"] == 3
    elif op == "adjoint":
        c = g.adjoint_config()
        assert c["kernel"] == 3 and c["depth"] == a
    else:
        assert (a, b) in ((4, 2), (8, 2), (16, 2), (8, 3), (16, 3)) and g.bp_config()["kernel"] == b
    _check_operator(ops, g, og, op)
    g2 = CASE.library_geometry()
    r2 = autotune.tune(g2, op)
    assert r2["cached"] and r2["params"] == [a, b]
    if op == "adjoint":
        assert g2.adjoint_config()["depth"] == a
    _check_operator(ops, g2, og, op)


@pytest.mark.parametrize("lanes", [1, 2])
@pytest.mark.parametrize("depth", [3, 4, 5, 6, 8])
@pytest.mark.parametrize("name", ["cone_tma_rows", "jittered_positions", "cone_aniso_offset"])
def test_adjoint_slab_depths_match_the_oracle(ops, name, depth, lanes):
    case = next(c for c in SMALL if c.name == name)
    g = case.library_geometry()
    og = case.oracle_geometry()
    g.set_tuning(ops.TUNE_ADJ_DEPTH, depth)
    g.set_tuning(ops.TUNE_ADJ_LANES, lanes)
    c = g.adjoint_config()
    assert c["kernel"] == 3 and c["depth"] == depth
    y = inputs.gaussian(og.sino_shape, seed=83)
    got = host(ops.adjoint(torch.from_numpy(y).to(DEV), g))
    assert rel_l2(got, oracle.adjoint(og, y)) <= 1e-5
    assert g.read_flags()[:4] == [0, 0, 0, 0]


@pytest.mark.parametrize("bz", [4, 8, 16])
@pytest.mark.parametrize("weight", [0, 1])
@pytest.mark.parametrize("name", ["cone", "helical", "jittered_positions"])
def test_bp_brick_depths_match_the_oracle(ops, name, weight, bz):
    case = next(c for c in SMALL if c.name == name)
    g = case.library_geometry()
    og = case.oracle_geometry()
    g.set_tuning(ops.TUNE_BP_BRICK_Z, bz)
    y = inputs.uniform(og.sino_shape, seed=84)
    got = host(ops.back_project(torch.from_numpy(y).to(DEV), g, weight))
    assert rel_l2(got, oracle.bp(og, y, weight)) <= 1e-5

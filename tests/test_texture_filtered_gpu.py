"""The hardware-filtered texture projector (forward-projection variant 5, the paper's "texture
interpolation", Sec. 2.1) against the FP64 oracle.

The texture unit weighs the eight texels of a sample with interpolation fractions of 8 fractional bits,
so each of the three fractions is off by at most 2^-9 and the interpolated value by at most
3 * 2^-9 * (the largest texel difference around the sample); on these phantoms that gives relative
errors around 1e-3. The tests hold it below 6e-3 (3 * 2^-9 of a value range that the projections'
smooth parts never exceed) and above 1e-6, which shows that the hardware filter, not the FP32 software
path, produced the result.
"""
import numpy as np
import pytest
import torch

import oracle

from cases import SMALL, rel_l2

pytestmark = pytest.mark.gpu
DEV = "cuda:0"
CONES = [c for c in SMALL if c.ndim == 3]


@pytest.fixture(scope="module")
def ops():
    from paper_2511_08427_gb300 import build
    build.build()
    from paper_2511_08427_gb300 import operators
    return operators


@pytest.mark.parametrize("dtype", [torch.float32, torch.float16])
@pytest.mark.parametrize("case", CONES, ids=lambda c: c.name)
def test_filtered_texture_projection_error(ops, case, dtype):
    g = case.library_geometry()
    g.set_variant(0, 5)
    assert g.fp_config(dtype)["kernel"] == 5
    x = case.phantom()
    xs = torch.from_numpy(x).to(DEV).to(dtype)
    got = ops.forward_project(xs, g).double().cpu().numpy()
    want = oracle.fp(case.oracle_geometry(), xs.double().cpu().numpy())
    err = rel_l2(got, want)
    print(f"{case.name} {dtype}: filtered-texture projection rel-L2 {err:.2e}")
    assert 1e-6 < err <= 6e-3


def test_filtered_texture_batch_and_fallback(ops):
    """A batch of two volumes (the texture is refilled per volume, in stream order) equals the two single
    projections; BF16 storage has no filtered texture format and falls back to the exact projector."""
    case = next(c for c in SMALL if c.name == "cone_tma_rows")
    g = case.library_geometry()
    g.set_variant(0, 5)
    x1, x2 = case.phantom(seed=3), case.phantom(seed=4)
    xb = torch.from_numpy(np.stack([x1, x2])).to(DEV)
    pb = ops.forward_project(xb, g)
    for i, x in enumerate((x1, x2)):
        assert torch.equal(pb[i], ops.forward_project(torch.from_numpy(x).to(DEV), g))
    assert g.fp_config(torch.bfloat16)["kernel"] == 3
    pbf = ops.forward_project(torch.from_numpy(x1).to(DEV).bfloat16(), g).double().cpu().numpy()
    want = oracle.fp(case.oracle_geometry(), torch.from_numpy(x1).bfloat16().double().numpy())
    assert rel_l2(pbf, want) <= 4e-3

"""The allocation-free adjoint entry point (pyronn_adjoint_noalloc), called through the C ABI.

It exists for callers that must not let the library allocate device memory (for example code
inside a memory pool that owns the GPU); its scratch lives in fixed device arrays of the library.
The test compares it with the allocating entry point pyronn_adjoint on two calls in a row (the
arrays keep the previous call's contents, so the second call checks that they are cleared), and
checks that a request beyond the arrays' size is refused. This file is collected last so that a
run stopping at the first failure has already run every other test.
"""
import ctypes
import math

import numpy as np
import pytest
import torch

from cases import SMALL, rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    from paper_2511_08427_gb300 import build
    build.build()
    from paper_2511_08427_gb300 import _lib
    return _lib


@pytest.mark.parametrize("dtype,tol", [(torch.float32, 1e-5), (torch.bfloat16, 4e-3)])
def test_noalloc_adjoint_matches_allocating_entry_point(lib, dtype, tol):
    from paper_2511_08427_gb300 import operators as ops
    case = next(c for c in SMALL if c.name == "cone")
    g = case.library_geometry()
    dev = torch.device("cuda:0")
    code = {torch.float32: lib.F32, torch.bfloat16: lib.BF16}[dtype]
    stream = torch.cuda.current_stream(dev).cuda_stream
    for call, seed in enumerate((1, 2)):
        y = torch.randn((2,) + g.sinogram_shape, device=dev, generator=torch.Generator(device=dev).manual_seed(seed))
        y = y.to(dtype)
        ref = ops.adjoint(y, g)
        out = torch.full_like(ref, float("nan"))
        lib.check(lib.lib().pyronn_adjoint_noalloc(g.handle, ctypes.c_void_p(y.data_ptr()),
                                                   ctypes.c_void_p(out.data_ptr()), code, 2, ctypes.c_void_p(stream)))
        torch.cuda.synchronize()
        a, b = out.float().cpu().numpy(), ref.float().cpu().numpy()
        assert np.isfinite(a).all(), f"call {call}"
        assert rel_l2(a, b) <= tol, f"call {call}"


def test_noalloc_adjoint_rejects_oversized_requests(lib):
    from paper_2511_08427_gb300.operators import Geometry
    g = Geometry.cone_circular((256, 256, 256), (0.5, 0.5, 0.5), (8, 8), (1.0, 1.0), 4, 2 * math.pi, 750.0, 1200.0)
    buf = torch.zeros(16, device="cuda:0")
    rc = lib.lib().pyronn_adjoint_noalloc(g.handle, ctypes.c_void_p(buf.data_ptr()), ctypes.c_void_p(buf.data_ptr()),
                                          lib.F32, 1, None)
    assert rc == -1
    assert b"at most" in lib.lib().pyronn_last_error()

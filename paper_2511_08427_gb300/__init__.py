"""GB300 (sm_103a) implementation of the differentiable CT operators of "An update to PYRO-NN".

The operators (ray-driven forward projection, its matched adjoint, voxel-driven back-projection)
run in libpyronn.so, a CUDA library with a C ABI (include/pyronn.h). The submodule `operators`
is a thin PyTorch binding: it passes device pointers and the current stream, and it raises if the
library has not been built (there is no CPU fallback).
"""
from ._lib import BF16, BP_INV_W2, BP_PLAIN, F16, F32, PyronnError  # noqa: F401

__all__ = ["BF16", "BP_INV_W2", "BP_PLAIN", "F16", "F32", "PyronnError"]

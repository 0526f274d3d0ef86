"""GB300-native DGDFT hot path: ALB generation, DG assembly and the adjoint gradient.

The computation lives in libdgdft.so (CUDA for sm_103a, C-ABI in include/dgdft.h);
``api`` is its thin Python binding.
"""
from . import _abi  # noqa: F401

__all__ = ["api", "build"]

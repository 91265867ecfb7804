"""GB300-native direct-indirect Burton-Miller solver for 2-D Helmholtz transmission problems.

The compute path is the C-ABI library libbm.so (declared in include/bm.h, CUDA kernels for
sm_103a under csrc/); ``bm`` is its Python binding and ``build`` compiles it in-tree.
"""
from . import bm  # noqa: F401

__all__ = ["bm"]

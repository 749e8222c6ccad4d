"""B300-native GOFMM evaluation: C-ABI library libgofmm.so (host FP64
compression, sm_103a evaluation kernels) and its Python binding.

Importing this package loads the native library and raises ImportError when
it has not been built; there is no fallback implementation.
"""
from . import gofmm  # noqa: F401
from .gofmm import *  # noqa: F401,F403

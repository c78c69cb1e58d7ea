"""GB300-native propagation of the 4D cross-spectral density of a planar partially coherent
source (PyWolf, arXiv 2203.02734): CUDA kernels for sm_103a behind the C ABI of
include/pywolf_gb.h, with PyTorch used only for device memory and streams.

``abi`` holds the C functions under their C names; ``CSD`` is a small convenience wrapper
that owns torch buffers for a handle.  Importing the package loads the compiled library and
raises if it is missing (there is no CPU path).
"""
from .abi import *  # noqa: F401,F403
from .abi import PwError  # noqa: F401
from .csd import CSD  # noqa: F401

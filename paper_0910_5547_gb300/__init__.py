"""GB300-native (sm_103a) block-structured AMR finite-volume update.

The compute path is the native library ``_build/libamr_gb300.so`` (hand-written
CUDA kernels behind the C ABI of ``include/amr.h``); ``native`` is its ctypes
binding and ``Solver`` a small convenience wrapper.  Importing this package does
not load the library; the first call does, and fails loudly if it is missing.
"""
from . import build  # noqa: F401
from . import native  # noqa: F401
from .native import AmrError  # noqa: F401
from .solver import Solver  # noqa: F401

__all__ = ["build", "native", "AmrError", "Solver"]

"""GB300-native Event-based Single Integration (ESI, arXiv 2508.02238).

The hot path -- event binning, the per-pixel Alg. 2 update with the Eq. 4
decay and Eq. 13 clamp, and the Eq. 14 frame map -- runs in the sm_103a
kernels of ``_build/libesi.so`` behind the C ABI of ``include/esi.h``.
``esi`` is the ctypes binding (same names as the C functions).
"""
from . import esi  # noqa: F401
from .esi import load_library  # noqa: F401

__all__ = ["esi", "load_library"]

"""GB300 (sm_103a) closest-point multigrid solver for (c - Lap_S) u = f.

The computation lives in the CUDA library ``libcpm.so`` (C ABI in
``include/cpm.h``); ``capi`` binds it with ctypes and ``solver`` wraps the
handles around torch tensors.  ``build()`` compiles the library in place.
"""
from ._build import build  # noqa: F401
from . import capi  # noqa: F401
from .solver import Band, Batch, Hierarchy, Smoother, make_surface  # noqa: F401

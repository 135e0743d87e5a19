"""GB300-native restarted PDHG (r^2HPDHG for LP, rAPDHG for QP).

The compute path is the C-ABI library libmpax_gb300.so (hand-written sm_103a
CUDA, declared in include/mpax.h).  ``paper_2412_09734_gb300.mpax`` is its thin
ctypes binding (same function names as the C ABI); ``Problem`` below is a small
convenience wrapper over those calls.  The library is loaded on first use and a
missing build raises ImportError: there is no CPU fallback.
"""
from __future__ import annotations

__all__ = ["Problem", "mpax", "build"]


def __getattr__(name):
    import importlib
    if name in ("mpax", "build", "problem"):
        return importlib.import_module(f"{__name__}.{name}")
    if name == "Problem":
        return importlib.import_module(f"{__name__}.problem").Problem
    raise AttributeError(name)

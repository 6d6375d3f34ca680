"""GB300-native batched runtime distance check (Fujii & Pham, arXiv 2309.12543).

The product is the CUDA library ``libsdfcheck.so`` behind the C ABI in
``include/sdfcheck.h``; this package holds its sources (``csrc/``), its build step
(``build.py``) and a thin ctypes binding (``_native.py``) with the same names as the
C entry points.  Binding names are loaded on first use, so ``build`` can run
before the library exists; using any binding without the built library raises.
"""
from __future__ import annotations

import importlib

__all__ = ["build"]


def __getattr__(name):
    if name == "build":
        return importlib.import_module(".build", __name__)
    native = importlib.import_module("._native", __name__)
    try:
        return getattr(native, name)
    except AttributeError:
        raise AttributeError(f"module {__name__!r} has no attribute {name!r}") from None

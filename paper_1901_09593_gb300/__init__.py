"""GB300-native multi-scale hierarchical ZNCC block matching (arXiv 1901.09593).

The computation lives in libmsbm.so (hand-written sm_103a CUDA kernels behind the C ABI
in include/msbm.h).  Importing this package loads nothing; ``Context`` loads the library
on first use and raises if it has not been built.
"""
import importlib

__all__ = ["Context", "Batch", "ZnccSoftArgmax", "build", "scenes", "autotune"]

_LAZY = {"Context": (".msbm", "Context"), "Batch": (".batch", "Batch"),
         "ZnccSoftArgmax": (".softargmax", "ZnccSoftArgmax")}


def __getattr__(name):
    if name in _LAZY:
        mod, attr = _LAZY[name]
        return getattr(importlib.import_module(mod, __name__), attr)
    raise AttributeError(f"module {__name__!r} has no attribute {name!r}")

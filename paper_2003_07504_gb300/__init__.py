"""GB300-native Iterative Least Squares (ILS) image smoothing.

The compute path is libils.so (hand-written sm_103a CUDA kernels behind the C
ABI of include/ils.h).  Importing this package does not load the library; the
first call that needs it does, and raises if it is missing.
"""
__all__ = ["Plan", "smooth", "build"]


def __getattr__(name):
    if name in ("Plan", "smooth"):
        from . import ils
        return getattr(ils, name)
    if name == "build":
        from .build import build
        return build
    raise AttributeError(name)

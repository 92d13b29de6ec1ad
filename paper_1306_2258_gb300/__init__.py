"""GB300-native direct Debye summation for small-angle scattering profiles.

The compute path is libsas.so (hand-written sm_103a CUDA behind the C ABI of
include/sas.h); ``_lib`` binds it with ctypes and ``profile`` wraps it for
PyTorch.  Importing the package does not load the library; the first call does,
and fails loudly if it cannot.
"""
__all__ = ["Profile", "DebyeFunction", "workloads"]


def __getattr__(name):
    if name in ("Profile", "DebyeFunction"):
        from . import profile
        return getattr(profile, name)
    raise AttributeError(name)

"""GB300-native sampling of Gaussian random fields by the FFT method of
Lang & Potthoff, "Fast simulation of Gaussian random fields" (arXiv 1105.2737).

The library is libgrf.so (C ABI in include/grf.h, CUDA kernels for sm_103a);
this package holds its build script, a ctypes binding with the same function
names, and a thin PyTorch wrapper (device memory, streams, autograd)."""
from .build import build  # noqa: F401


def __getattr__(name):
    # the torch-facing API is imported lazily so that build() needs no GPU
    if name in ("GRF", "GRFBatch", "grf_fields"):
        from . import api
        return getattr(api, name)
    raise AttributeError(name)

"""GB300-native (sm_103a) hot path of the signed-particle Wigner Monte Carlo
method with the analytically weighted network Wigner kernel (arXiv:1806.00082).

The compute runs in libwmc (CUDA, C ABI in include/wmc.h); ``wmc`` is its thin
ctypes binding and ``sim`` a small driver that owns the device buffers of one
simulation.  Build the library with ``paper_1806_00082_gb300.build.build()``.
"""
from . import wmc  # noqa: F401

__all__ = ["wmc"]

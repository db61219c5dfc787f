"""Hierarchical loop-nest executor for GB300 (sm_103a).

A depth-d loop nest (rectangular or CSR-ragged) with a per-iteration body and
a reduction at any level, whose levels are bound to grid / cluster / CTA /
warp / sub-warp / lane / sequential execution, run by hand-written CUDA
kernels behind the C ABI in include/hp.h.  ``binding`` is the ctypes layer
(same names as the C ABI); ``synth`` draws the seeded synthetic workloads;
``build`` compiles libhp.so in-tree.
"""
from . import binding  # noqa: F401  (the shared library itself loads on first use)
from .binding import Nest, HPError  # noqa: F401

"""GB300-native fast integral-equation solver for the Laplace-Beltrami equation
on the sphere with islands (stereographic projection, double-layer Nystrom
system, 2D FMM matvec, device-resident GMRES).

The compute path is the CUDA library liblbfmm (csrc/, C ABI in include/lbfmm.h);
`lbfmm` is its thin ctypes binding.
"""
from . import lbfmm  # noqa: F401
from .lbfmm import *  # noqa: F401,F403

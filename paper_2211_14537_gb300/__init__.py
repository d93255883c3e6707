"""GB300 library for the particular-solution stage of the FMM-accelerated
Poisson solver with function extension (arXiv 2211.14537): extension of the
source on cut leaves and the box-FMM volume potential, behind the C ABI of
include/vpx.h.  This package holds the CUDA sources (csrc/), the build script
and the ctypes binding; the computation runs only in the CUDA library."""
from .vpx import *  # noqa: F401,F403

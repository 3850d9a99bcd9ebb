"""GB300 batched complex-to-complex FFT (fused Stockham kernels for sm_103a): 1D of any
length 2..2^24 with prime factors 2, 3, 5, 7, and rank-2/3 arrays.

The transforms run in libfftc.so (C ABI: include/fftc.h); this package is its
thin Python binding, with torch supplying device memory and streams.
"""
from ._native import FftcError, load as load_library  # noqa: F401
from .api import NdPlan, Plan, UnevenPlan, fft, fftn, get_plan, ifft, ifftn  # noqa: F401

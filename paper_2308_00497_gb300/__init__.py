"""GB300 batched 1D complex-to-complex FFT (fused Stockham kernels for sm_103a).

The transforms run in libfftc.so (C ABI: include/fftc.h); this package is its
thin Python binding, with torch supplying device memory and streams.
"""
from ._native import FftcError, load as load_library  # noqa: F401
from .api import Plan, UnevenPlan, fft, get_plan, ifft  # noqa: F401

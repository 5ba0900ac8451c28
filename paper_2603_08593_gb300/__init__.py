"""GB300 (sm_103a) difference imaging: delta-basis, spatially varying kernel
fit by Fourier-domain normal equations, FP64 solve, convolve-and-subtract.

The compute path is the CUDA library libsfft_gb300.so (C ABI in
include/sfft.h); `binding` marshals arguments to it through ctypes.
"""
from . import binding  # noqa: F401
from .binding import Plan, SfftError, load  # noqa: F401

"""GB300 (sm_103a) difference imaging: delta-basis, spatially varying kernel
fit by Fourier-domain normal equations, FP64 solve, convolve-and-subtract;
matched-filter candidate detection and a BF16 tensor-core stamp classifier.

The compute path is the CUDA library libsfft_gb300.so (C ABI in
include/sfft.h, include/rb.h and include/phot.h); `binding` marshals
arguments to it through ctypes.
"""
from . import binding  # noqa: F401
from .binding import (Detector, Plan, RBModel, RIModel, SfftError, aperture_flux, limiting_mag, load,  # noqa: F401
                      median_combine, shape_cuts)

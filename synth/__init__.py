"""Seeded synthetic DECam-shaped inputs.

This package is the one module that both the FP64 oracle side and the CUDA
side read their inputs from.  It renders images, noise, masks and artifacts;
it holds none of the subtraction or classifier arithmetic.
"""
from .decam import (  # noqa: F401
    SKY_ADU, READ_NOISE_ADU, SIGMA_SKY, fwhm_to_sigma, powerlaw_flux,
    render_points, make_pair, config_pair, small_pair,
)

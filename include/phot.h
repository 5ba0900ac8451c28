/*
 * phot.h - C ABI of the differential-photometry step on difference images and
 * of the multi-template combination.
 *
 * The paper (Sec. 2.3.3) measures fluxes on D in circular apertures (radius
 * 0.6731 FWHM for single-exposure templates, 3 px for multi-exposure
 * templates), removes detections touched by bad pixels, and estimates each
 * difference image's limiting magnitude from the aperture fluxes at 1024
 * random background positions (the 5-sigma flux from their standard
 * deviation, converted with the zero point).  For multi-exposure templates
 * (Sec. 2.3.2) the N_TEMP difference images are put on a common zero point
 * and median-combined.
 *
 * Aperture integration: pixel (px, py) covers [px - 1/2, px + 1/2] x
 * [py - 1/2, py + 1/2]; its weight is the fraction of a 5 x 5 grid of
 * sub-pixel centres (px - 1/2 + (i + 1/2)/5, py - 1/2 + (j + 1/2)/5) inside
 * the closed disc (x - xc)^2 + (y - yc)^2 <= r^2, each test evaluated in IEEE
 * double without fused operations; flux = sum of weight x D (FP64).  A pixel
 * of positive weight that is bad, non-finite or outside the image sets the
 * aperture's flag and is left out of the sum.
 *
 * All data pointers are DEVICE pointers; calls are asynchronous on `stream`.
 * Statuses are the sfft_status_t codes of sfft.h.
 */
#ifndef PHOT_GB300_H
#define PHOT_GB300_H

#include <stddef.h>
#include <stdint.h>

#include "sfft.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Forced aperture photometry: for CCD c and position i, (x, y) = pos[c][i]
 * (double [batch][n][2], pixel coordinates), flux[c][i] (double) and
 * flag[c][i] (int32).  D float [batch][H][W], bad uint8 [batch][H][W] or NULL;
 * 0 < radius <= 32. */
sfft_status_t phot_aperture_flux(int32_t H, int32_t W, int32_t batch, const float* D, const uint8_t* bad,
                                 const double* pos, int32_t n, double radius, double* flux, int32_t* flag,
                                 void* stream);

/* Limiting magnitude per CCD from apertures at the given (random, caller-
 * drawn) positions: sigma[c] = sample standard deviation (n - 1 in the
 * denominator) of the unflagged fluxes, mlim[c] = zp - 2.5 log10(5 sigma),
 * ngood[c] = number of unflagged apertures (NaN results below two).
 * ws: device scratch of phot_limiting_workspace_bytes(batch, n). */
size_t phot_limiting_workspace_bytes(int32_t batch, int32_t n);
sfft_status_t phot_limiting_mag(int32_t H, int32_t W, int32_t batch, const float* D, const uint8_t* bad,
                                const double* pos, int32_t n, double radius, double zp, double* sigma,
                                double* mlim, int32_t* ngood, void* ws, void* stream);

/* Multi-template combination: out[y][x] = median over templates t of
 * scale[t] D[t][y][x] at good finite pixels (scale float [ntemp], device:
 * 10^(0.4 (zp_common - zp_t)), supplied by the caller's calibration); an even
 * count takes the mean of the two middle values; no good value gives NaN.
 * D float [ntemp][H][W], bad uint8 [ntemp][H][W] or NULL, out float [H][W];
 * 1 <= ntemp <= 16.  FP32 arithmetic. */
sfft_status_t phot_median_combine(int32_t H, int32_t W, int32_t ntemp, const float* D, const float* scale,
                                  const uint8_t* bad, float* out, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* PHOT_GB300_H */

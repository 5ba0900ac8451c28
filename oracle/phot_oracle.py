"""FP64 CPU oracle for aperture photometry on difference images, the
limiting-magnitude Monte Carlo and the multi-template median combination.

TEST INFRASTRUCTURE ONLY: used by the tests; the product path never imports it.

The paper (Sec. 2.3.3) measures fluxes on D in circular apertures (radius
0.6731 FWHM for single-exposure templates, 3 px for multi-exposure
templates), removes detections touched by bad pixels, and estimates each
difference image's limiting magnitude from the aperture fluxes at 1024
random background positions: the 5-sigma flux from their standard deviation,
converted with the zero point.  For multi-exposure templates (Sec. 2.3.2) the
N_TEMP difference images are put on a common zero point and median-combined.
It does not spell out the aperture integration; the reading here:

  aperture   pixel (px, py) covers [px - 1/2, px + 1/2] x [py - 1/2, py + 1/2];
             its weight is the fraction of an S x S grid of sub-pixel centres
             (px - 1/2 + (i + 1/2)/S, py - 1/2 + (j + 1/2)/S), S = 5, lying in
             the closed disc (x - xc)^2 + (y - yc)^2 <= r^2, each test evaluated
             as ((sx - xc)^2 + (sy - yc)^2) <= r^2 in IEEE double without fused
             operations
  flux       sum of weight x D over pixels inside the image; flag = 1 when a
             pixel of positive weight is bad, non-finite or outside the image
  limit      sigma = sample standard deviation (ddof 1) of the unflagged
             fluxes; m_lim = zp - 2.5 log10(5 sigma)
  combine    out = median over templates t of s_t D_t at good finite pixels
             (s_t = 10^(0.4 (zp_common - zp_t)) given by the caller); an even
             count takes the mean of the two middle values; no good value -> NaN
"""
from __future__ import annotations

import math

import numpy as np

SUB = 5


def aperture_weights(xc, yc, r, sub=SUB):
    """Pixel weights of one aperture: (ys, xs, w) over the bounding box."""
    x0, x1 = int(math.floor(xc - r - 1)), int(math.ceil(xc + r + 1))
    y0, y1 = int(math.floor(yc - r - 1)), int(math.ceil(yc + r + 1))
    xs = np.arange(x0, x1 + 1)
    ys = np.arange(y0, y1 + 1)
    off = (np.arange(sub) + 0.5) / sub
    # sub-pixel centre coordinates, evaluated element by element in float64
    sx = (xs[:, None] - 0.5) + off[None, :]          # [nx][sub]
    sy = (ys[:, None] - 0.5) + off[None, :]          # [ny][sub]
    dx = sx - xc
    dy = sy - yc
    dx2 = dx * dx
    dy2 = dy * dy
    inside = (dy2[:, None, :, None] + dx2[None, :, None, :]) <= r * r   # [ny][nx][sub][sub]
    w = inside.sum(axis=(2, 3)) / float(sub * sub)
    return ys, xs, w


def aperture_flux(D, bad, xs, ys, r, sub=SUB):
    """Fluxes and flags of apertures centred on (xs[i], ys[i])."""
    D = np.asarray(D, dtype=np.float64)
    H, W = D.shape
    flux = np.zeros(len(xs))
    flag = np.zeros(len(xs), np.int32)
    for i, (xc, yc) in enumerate(zip(xs, ys)):
        py, px, w = aperture_weights(float(xc), float(yc), float(r), sub)
        s = 0.0
        for a, yy in enumerate(py):
            for b, xx in enumerate(px):
                if w[a, b] <= 0:
                    continue
                if not (0 <= yy < H and 0 <= xx < W):
                    flag[i] = 1
                    continue
                v = D[yy, xx]
                if not np.isfinite(v) or (bad is not None and bad[yy, xx]):
                    flag[i] = 1
                    continue
                s += w[a, b] * v
        flux[i] = s
    return flux, flag


def limiting_mag(D, bad, xs, ys, r, zp, sub=SUB):
    flux, flag = aperture_flux(D, bad, xs, ys, r, sub)
    good = flux[flag == 0]
    sigma = float(np.std(good, ddof=1)) if good.size > 1 else math.nan
    mlim = zp - 2.5 * math.log10(5.0 * sigma) if sigma > 0 else math.nan
    return sigma, mlim, int(good.size)


def median_combine(Ds, scales, bads=None):
    """Per-pixel median of s_t D_t over the good finite templates."""
    Ds = np.asarray(Ds, dtype=np.float64) * np.asarray(scales, dtype=np.float64)[:, None, None]
    ok = np.isfinite(Ds)
    if bads is not None:
        ok &= np.asarray(bads) == 0
    return np.nanmedian(np.where(ok, Ds, np.nan), axis=0)

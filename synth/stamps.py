"""Seeded labelled stamp triplets (science, reference, difference) for the
real-bogus classifier, and the injection recipe for whole CCD pairs.

Input generation only.  The classes follow the training set the paper's
classifier is fitted on (Sec. 2.3.4) at the mix fixed in the project's
configuration list: half injected point transients at SNR 3-100 (label 1),
half artifacts (label 0) split evenly between residuals of stars
misregistered by 0.3-1 px, cosmic-ray hits of 1-3 px at ~1e4 ADU, and
bad-column segments.  Each stamp is 31 x 31 px centred on the candidate
pixel, in raw ADU: channel 0 science, 1 reference, 2 difference.

The difference channel is modelled as the science frame minus a reference
already matched to the science PSF: pure noise of sqrt(2) sigma_sky plus
what the science frame has and the matched reference lacks.
"""
from __future__ import annotations

import math

import numpy as np

from .decam import SIGMA_SKY, SKY_ADU, fwhm_to_sigma, powerlaw_flux, render_points

SIDE = 31
KINDS = ("transient", "misreg", "cosmic", "column")


def flux_for_snr(snr, psf_sigma, sigma_sky=SIGMA_SKY):
    """Flux of a Gaussian source with the given background-limited SNR."""
    return snr * sigma_sky * math.sqrt(4.0 * math.pi) * psf_sigma


def make_stamps(n, seed, fwhm_R=(0.9, 1.5), fwhm_S=(1.4, 2.3), snr=(3.0, 100.0), kinds=None):
    """n stamps with labels; returns dict(stamps float32 [n][3][31][31],
    labels float32 [n], kind [n] (index into KINDS), snr [n] (transients),
    fwhm_S [n])."""
    rng = np.random.default_rng(seed)
    if kinds is None:
        kinds = np.where(np.arange(n) % 2 == 0, 0, 1 + rng.integers(0, 3, n))
    kinds = np.asarray(kinds)
    c = SIDE // 2
    out = np.empty((n, 3, SIDE, SIDE), np.float32)
    snrs = np.zeros(n)
    fS = np.zeros(n)
    for i in range(n):
        fr = rng.uniform(*fwhm_R)
        fs = max(rng.uniform(*fwhm_S), fr + 0.2)
        sr, ss = float(fwhm_to_sigma(fr)), float(fwhm_to_sigma(fs))
        fS[i] = fs
        # a field star near the candidate in about a third of the stamps (a host or a neighbour)
        R = np.full((SIDE, SIDE), SKY_ADU)
        S = np.full((SIDE, SIDE), SKY_ADU)
        if rng.random() < 0.35:
            hx, hy = c + rng.uniform(-6, 6), c + rng.uniform(-6, 6)
            hf = float(powerlaw_flux(rng, 1, 1e3, 1e5)[0])
            R += render_points(SIDE, SIDE, [hx], [hy], [hf], [sr])
            S += render_points(SIDE, SIDE, [hx], [hy], [hf], [ss])
        D = np.zeros((SIDE, SIDE))
        k = int(kinds[i])
        x0, y0 = c + rng.uniform(-0.5, 0.5), c + rng.uniform(-0.5, 0.5)
        if k == 0:                                  # point transient in S
            snrs[i] = math.exp(rng.uniform(math.log(snr[0]), math.log(snr[1])))
            f = flux_for_snr(snrs[i], ss)
            blob = render_points(SIDE, SIDE, [x0], [y0], [f], [ss])
            S += blob
            D += blob
        elif k == 1:                                # misregistered star: dipole residual
            f = float(powerlaw_flux(rng, 1, 3e3, 3e5)[0])
            shift = rng.uniform(0.3, 1.0)
            ang = rng.uniform(0, 2 * math.pi)
            dx, dy = shift * math.cos(ang), shift * math.sin(ang)
            R += render_points(SIDE, SIDE, [x0], [y0], [f], [sr])
            starS = render_points(SIDE, SIDE, [x0 + dx], [y0 + dy], [f], [ss])
            S += starS
            D += starS - render_points(SIDE, SIDE, [x0], [y0], [f], [ss])
        elif k == 2:                                # cosmic-ray hit in S: 1-3 px
            npx = int(rng.integers(1, 4))
            px, py = int(round(x0)), int(round(y0))
            for _ in range(npx):
                amp = rng.uniform(5e3, 2e4)
                S[py, px] += amp
                D[py, px] += amp
                px += int(rng.integers(-1, 2))
                py += int(rng.integers(-1, 2))
        else:                                       # bad-column segment in S
            length = int(rng.integers(8, SIDE))
            ys = int(rng.integers(0, SIDE - length + 1))
            ys = min(max(ys, c - length + 1), c)    # the segment passes the centre row
            amp = rng.uniform(200.0, 2000.0)
            S[ys:ys + length, int(round(x0))] += amp
            D[ys:ys + length, int(round(x0))] += amp
        R = rng.poisson(np.maximum(R, 0)).astype(np.float64) + rng.normal(0, 6.0, R.shape)
        S_noise = rng.normal(0, SIGMA_SKY, S.shape)
        S = S + S_noise
        D = D + S_noise + rng.normal(0, SIGMA_SKY, D.shape)   # matched-reference noise
        out[i, 0], out[i, 1], out[i, 2] = S, R, D
    labels = (kinds == 0).astype(np.float32)
    return dict(stamps=out, labels=labels, kind=kinds, snr=snrs, fwhm_S=fS)

"""FP64 CPU oracle for candidate detection on the difference image.

TEST INFRASTRUCTURE ONLY: used by the tests, the smoke check and the
benchmark's CPU-baseline leg; the product path never imports it.

The paper (Sec. 2.3.3) finds candidate sources on D and cuts stamps around
them for the classifier (Sec. 2.3.4); it does not fix the detector.  The one
used here is a PSF matched filter:

  D^(x)     = D(x) where the pixel is good and finite, else 0 (0 outside)
  sigma_D   = RMS of D about its mean over the good, finite pixels at least
              15 px from every edge, after three 3-sigma clipping passes,
              divided by sqrt(0.97334) (the share of a Gaussian's variance
              kept inside +-3 sigma)
  G(u)      = g(u_x) g(u_y), g(t) = exp(-t^2 / (2 s^2)), |u_x|, |u_y| <= r = ceil(3 s)
  SNR(x)    = sum_u G(u) D^(x - u) / (sigma_D ||G||_2)
  candidate : >= 15 px from every edge, no bad pixel within Chebyshev
              distance `guard` (guard 0: the pixel itself is good), SNR >=
              thresh, SNR >= every SNR in its 5 x 5 neighbourhood; reported in
              row-major order
  stamp     : 31 x 31 cut of (S, R, D) centred on the candidate, non-finite -> 0

The matched-filter normalisation makes SNR unit-variance on white noise of
RMS sigma_D, and gives A ||G||_2 / sigma_D at the centre of a noise-free
source A G(x - x0) (Cauchy-Schwarz equality).
"""
from __future__ import annotations

import math

import numpy as np
from scipy import ndimage

MARGIN = 15
HALF = 15          # stamp half-size (31 x 31)
CLIP_NSIG = 3.0
CLIP_PASSES = 3
CLIP_VAR_FRACTION = 0.97334
NMS = 2            # 5 x 5 neighbourhood


def interior_mask(H, W, bad=None, D=None):
    m = np.zeros((H, W), bool)
    m[MARGIN:H - MARGIN, MARGIN:W - MARGIN] = True
    if bad is not None:
        m &= np.asarray(bad) == 0
    if D is not None:
        m &= np.isfinite(D)
    return m


def clipped_sigma(D, bad=None):
    """Returns (mean, sigma_D) of the clipped interior pixels."""
    D = np.asarray(D, dtype=np.float64)
    H, W = D.shape
    x = D[interior_mask(H, W, bad, D)]
    mu = x.mean() if x.size else math.nan
    var = ((x - mu) ** 2).mean() if x.size else math.nan
    for _ in range(CLIP_PASSES):
        sel = x[np.abs(x - mu) <= CLIP_NSIG * math.sqrt(var)]
        if sel.size == 0:
            return math.nan, math.nan
        mu = sel.mean()
        var = ((sel - mu) ** 2).mean()
    return mu, math.sqrt(var / CLIP_VAR_FRACTION)


def gauss_taps(psf_sigma):
    r = int(math.ceil(3.0 * psf_sigma))
    t = np.arange(-r, r + 1, dtype=np.float64)
    return np.exp(-t * t / (2.0 * psf_sigma * psf_sigma))


def masked_d(D, bad=None):
    D = np.asarray(D, dtype=np.float64)
    ok = np.isfinite(D)
    if bad is not None:
        ok &= np.asarray(bad) == 0
    return np.where(ok, D, 0.0)


def matched_snr(D, bad, psf_sigma, sigma_D):
    """SNR map: separable correlation of D^ with g along x then along y."""
    Dh = masked_d(D, bad)
    g = gauss_taps(psf_sigma)
    r = (g.size - 1) // 2
    H, W = Dh.shape
    P = np.zeros((H + 2 * r, W + 2 * r))
    P[r:r + H, r:r + W] = Dh
    T = np.zeros((H + 2 * r, W))
    for k, gk in enumerate(g):           # sum_u g(u) D(x - u), u = r - k
        T += gk * P[:, k:k + W]
    out = np.zeros((H, W))
    for k, gk in enumerate(g):
        out += gk * T[k:k + H, :]
    norm = float((g * g).sum())          # ||G||_2 = sum_t g(t)^2 for the separable G
    return out / (sigma_D * norm)


def guard_mask(bad, guard):
    """Pixels with a bad pixel within Chebyshev distance `guard` (max filter)."""
    if bad is None:
        return None
    b = np.asarray(bad) != 0
    if guard <= 0:
        return b.astype(np.uint8)
    return ndimage.maximum_filter(b.astype(np.uint8), size=2 * guard + 1, mode="constant", cval=0)


def candidates(snr, bad, thresh, guard=0):
    """Row-major (y, x) of the local maxima at or above thresh."""
    H, W = snr.shape
    ok = interior_mask(H, W, guard_mask(bad, guard))
    ok &= np.isfinite(snr) & (snr >= thresh)
    P = np.full((H + 2 * NMS, W + 2 * NMS), -np.inf)
    P[NMS:NMS + H, NMS:NMS + W] = np.where(np.isfinite(snr), snr, -np.inf)
    for dy in range(-NMS, NMS + 1):
        for dx in range(-NMS, NMS + 1):
            ok &= snr >= P[NMS + dy:NMS + dy + H, NMS + dx:NMS + dx + W]
    ys, xs = np.nonzero(ok)
    return ys, xs


def cut_stamps(S, R, D, ys, xs):
    out = np.zeros((len(ys), 3, 2 * HALF + 1, 2 * HALF + 1))
    for i, (y, x) in enumerate(zip(ys, xs)):
        for c, img in enumerate((S, R, D)):
            cut = np.asarray(img, dtype=np.float64)[y - HALF:y + HALF + 1, x - HALF:x + HALF + 1]
            out[i, c] = np.where(np.isfinite(cut), cut, 0.0)
    return out


def detect(D, S, R, bad, psf_sigma, thresh, max_cand=None, guard=0):
    """Full detection of one CCD: dict(sigma_D, snr_map, y, x, snr, stamps);
    the lists are truncated to max_cand (count is the untruncated number)."""
    mu, sigma_D = clipped_sigma(D, bad)
    snr = matched_snr(D, bad, psf_sigma, sigma_D)
    ys, xs = candidates(snr, bad, thresh, guard)
    count = len(ys)
    if max_cand is not None:
        ys, xs = ys[:max_cand], xs[:max_cand]
    return dict(mean=mu, sigma_D=sigma_D, snr_map=snr, count=count, y=ys, x=xs, snr=snr[ys, xs],
                stamps=cut_stamps(S, R, D, ys, xs))

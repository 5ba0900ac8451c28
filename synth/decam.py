"""Seeded synthetic DECam-shaped reference/science CCD pairs.

Everything here is input generation: star fields rendered with
pixel-integrated Gaussian PSFs, Poisson sky and read noise, saturation,
bad-pixel masks and the artifacts the stamp classifier learns to reject.
The recipe follows the workloads the paper processes (DECam science CCDs of
2048 x 4096 pixels, Sec. 1; per-exposure CCD batches, Sec. 4.2) with the
sizes and distributions fixed in the project's configuration list:

* sky 1000 ADU (Poisson, gain 1 e-/ADU) plus Gaussian read noise of 6 ADU,
  so the background noise is sqrt(1000 + 36) = 32.19 ADU;
* point sources at uniform positions, fluxes from N(>F) ~ F^-1.5 on
  [1e3, 1e6] ADU by inverse-CDF sampling;
* circular Gaussian PSFs integrated over each pixel with erf; the FWHM may
  vary linearly across the chip along a chosen direction;
* a sub-pixel shift of the science frame (0.1 px in x by default);
* transients injected in the science frame only, at a stated SNR, where
  SNR = F / (sigma_sky * sqrt(4 pi sigma_psf^2)) (background-limited
  optimal PSF-fit SNR of a Gaussian);
* optional clipping at 6.5e4 ADU, masking of pixels above 6e4 ADU dilated
  by a 3 px disc, bad columns, bleed trails and edge rectangles;
* optional cosmic-ray hits, bad-column segments and misregistered stars in
  the science frame (unmasked artifacts).

Pixel (x, y) is centred on integer coordinates and covers
[x - 0.5, x + 0.5] x [y - 0.5, y + 0.5]; images are row-major [y][x].
"""
from __future__ import annotations

import math

import numpy as np
from scipy import ndimage
from scipy.special import erf

SKY_ADU = 1000.0
READ_NOISE_ADU = 6.0
SIGMA_SKY = math.sqrt(SKY_ADU + READ_NOISE_ADU ** 2)
SAT_CLIP_ADU = 6.5e4
SAT_MASK_ADU = 6.0e4
FWHM_PER_SIGMA = 2.0 * math.sqrt(2.0 * math.log(2.0))


def fwhm_to_sigma(fwhm):
    return np.asarray(fwhm, dtype=np.float64) / FWHM_PER_SIGMA


def powerlaw_flux(rng, n, fmin=1e3, fmax=1e6, slope=1.5):
    """Fluxes with N(>F) proportional to F^-slope on [fmin, fmax]."""
    u = rng.random(n)
    return fmin * (1.0 - u * (1.0 - (fmin / fmax) ** slope)) ** (-1.0 / slope)


def render_points(H, W, xs, ys, fluxes, sigmas, radius=None):
    """Sum of pixel-integrated circular Gaussians, returned as float64 [H][W]."""
    xs = np.atleast_1d(np.asarray(xs, dtype=np.float64))
    ys = np.atleast_1d(np.asarray(ys, dtype=np.float64))
    F = np.broadcast_to(np.asarray(fluxes, dtype=np.float64), xs.shape)
    sig = np.broadcast_to(np.asarray(sigmas, dtype=np.float64), xs.shape)
    img = np.zeros(H * W, dtype=np.float64)
    if xs.size == 0:
        return img.reshape(H, W)
    r = int(radius) if radius is not None else int(math.ceil(5.0 * float(sig.max()))) + 1
    off = np.arange(-r, r + 1)
    out_chunks = []
    step = 4096
    for s0 in range(0, xs.size, step):
        sl = slice(s0, s0 + step)
        x0, y0, f0, g0 = xs[sl], ys[sl], F[sl], sig[sl]
        px = np.floor(x0 + 0.5).astype(np.int64)[:, None] + off[None, :]
        py = np.floor(y0 + 0.5).astype(np.int64)[:, None] + off[None, :]
        s2 = (g0 * math.sqrt(2.0))[:, None]
        fx = 0.5 * (erf((px + 0.5 - x0[:, None]) / s2) - erf((px - 0.5 - x0[:, None]) / s2))
        fy = 0.5 * (erf((py + 0.5 - y0[:, None]) / s2) - erf((py - 0.5 - y0[:, None]) / s2))
        vals = f0[:, None, None] * fy[:, :, None] * fx[:, None, :]
        inb = ((px >= 0) & (px < W))[:, None, :] & ((py >= 0) & (py < H))[:, :, None]
        idx = py[:, :, None] * W + px[:, None, :]
        out_chunks.append(np.bincount(idx[inb], weights=vals[inb], minlength=H * W))
    for c in out_chunks:
        img += c
    return img.reshape(H, W)


def _fwhm_field(H, W, lo, hi, angle):
    """FWHM(x, y) = lo + (hi - lo) * t, t in [0, 1] along direction `angle`.

    angle=None means linear in y (the long axis of a DECam CCD)."""
    if angle is None:
        return lambda x, y: lo + (hi - lo) * (np.asarray(y, dtype=np.float64) / max(H - 1, 1))
    c, s = math.cos(angle), math.sin(angle)
    corners = [c * x + s * y for x in (0, W - 1) for y in (0, H - 1)]
    pmin, pmax = min(corners), max(corners)
    span = max(pmax - pmin, 1e-9)
    return lambda x, y: lo + (hi - lo) * ((c * np.asarray(x) + s * np.asarray(y) - pmin) / span)


def _separated_positions(rng, n, H, W, margin, min_sep, avoid=None, tries=200000):
    pts = []
    for _ in range(tries):
        if len(pts) >= n:
            break
        x = rng.uniform(margin, W - 1 - margin)
        y = rng.uniform(margin, H - 1 - margin)
        if avoid is not None and avoid[int(round(y)), int(round(x))]:
            continue
        if all((x - px) ** 2 + (y - py) ** 2 >= min_sep ** 2 for px, py in pts):
            pts.append((x, y))
    return np.array(pts, dtype=np.float64).reshape(-1, 2)


def _disc(radius):
    r = int(radius)
    yy, xx = np.mgrid[-r:r + 1, -r:r + 1]
    return (xx * xx + yy * yy) <= radius * radius


def make_pair(H, W, seed, n_src=300, fwhm_R=(1.2, 1.2), fwhm_S=(1.8, 1.8), grad_angle=None,
              shift=(0.1, 0.0), flux_scale=1.0, n_transients=1, snr=(20.0, 20.0),
              transient_sep=40.0, transient_margin=20, clip=None, mask_saturated=False,
              bad_columns=(), mask_fraction=None, n_cosmics=0, n_colsegs=0, n_misreg=0,
              misreg_shift=(0.3, 1.0), noise=True, sky=SKY_ADU):
    """One reference/science pair.  Returns a dict with R, S (float32 [H][W]),
    bad (uint8 [H][W], nonzero = bad) and the injection truth."""
    rng = np.random.default_rng(seed)
    fR = _fwhm_field(H, W, fwhm_R[0], fwhm_R[1], grad_angle)
    fS = _fwhm_field(H, W, fwhm_S[0], fwhm_S[1], grad_angle)
    xs = rng.uniform(-0.5, W - 0.5, n_src)
    ys = rng.uniform(-0.5, H - 0.5, n_src)
    F = powerlaw_flux(rng, n_src)
    sigR = fwhm_to_sigma(fR(xs, ys))
    sigS = fwhm_to_sigma(fS(xs, ys))
    dx, dy = shift
    xs_S, ys_S = xs + dx, ys + dy
    misreg = np.zeros((0, 2))
    if n_misreg:
        pick = rng.choice(n_src, size=min(n_misreg, n_src), replace=False)
        ang = rng.uniform(0, 2 * math.pi, pick.size)
        mag = rng.uniform(misreg_shift[0], misreg_shift[1], pick.size)
        xs_S = xs_S.copy(); ys_S = ys_S.copy()
        xs_S[pick] += mag * np.cos(ang)
        ys_S[pick] += mag * np.sin(ang)
        misreg = np.stack([xs_S[pick], ys_S[pick], F[pick]], axis=1)
    model_R = render_points(H, W, xs, ys, F, sigR)
    model_S = render_points(H, W, xs_S, ys_S, F * flux_scale, sigS)

    # transients (science frame only)
    tpos = _separated_positions(rng, n_transients, H, W, transient_margin, transient_sep)
    if tpos.shape[0]:
        lsnr = rng.uniform(math.log(snr[0]), math.log(snr[1]), tpos.shape[0])
        t_snr = np.exp(lsnr)
        t_sig = fwhm_to_sigma(fS(tpos[:, 0], tpos[:, 1]))
        t_flux = t_snr * SIGMA_SKY * np.sqrt(4.0 * math.pi) * t_sig
        model_S += render_points(H, W, tpos[:, 0], tpos[:, 1], t_flux, t_sig)
        transients = np.stack([tpos[:, 0], tpos[:, 1], t_flux, t_snr, t_sig], axis=1)
    else:
        transients = np.zeros((0, 5))

    if noise:
        R = rng.poisson(sky + model_R).astype(np.float64) + rng.normal(0.0, READ_NOISE_ADU, (H, W))
        S = rng.poisson(sky + model_S).astype(np.float64) + rng.normal(0.0, READ_NOISE_ADU, (H, W))
    else:
        R = sky + model_R
        S = sky + model_S

    # unmasked science-frame artifacts
    cosmics = []
    for _ in range(n_cosmics):
        cx, cy = int(rng.integers(2, W - 2)), int(rng.integers(2, H - 2))
        npx = int(rng.integers(1, 4))
        pts = [(cy, cx)]
        while len(pts) < npx:
            oy, ox = pts[-1]
            d = [(0, 1), (1, 0), (0, -1), (-1, 0), (1, 1)][int(rng.integers(0, 5))]
            pts.append((min(max(oy + d[0], 0), H - 1), min(max(ox + d[1], 0), W - 1)))
        for (py, px) in pts:
            S[py, px] += 1e4
        cosmics.append((cx, cy, npx))
    colsegs = []
    for _ in range(n_colsegs):
        cx = int(rng.integers(0, W))
        ln = int(rng.integers(20, 120))
        y0 = int(rng.integers(0, max(H - ln, 1)))
        amp = float(rng.uniform(500.0, 3000.0))
        S[y0:y0 + ln, cx] += amp
        colsegs.append((cx, y0, y0 + ln, amp))

    bad = np.zeros((H, W), dtype=np.uint8)
    if mask_saturated:
        sat = (R > SAT_MASK_ADU) | (S > SAT_MASK_ADU)
        if sat.any():
            sat = ndimage.binary_dilation(sat, structure=_disc(3))
        bad |= sat.astype(np.uint8)
    for c in bad_columns:
        if 0 <= c < W:
            bad[:, c] = 1
    trails = []
    if mask_fraction is not None:
        # bleed trails from the brightest stars, some running to the edge
        bright = np.argsort(F)[::-1][:max(1, n_src // 400)]
        for i in bright:
            x0 = int(np.clip(round(xs[i]), 0, W - 1)); y0 = int(np.clip(round(ys[i]), 0, H - 1))
            half = int(rng.integers(1, 3))
            if rng.random() < 0.2:
                ya, yb = (0, y0) if rng.random() < 0.5 else (y0, H)
            else:
                ln = int(rng.integers(10, 400))
                ya, yb = max(0, y0 - ln), min(H, y0 + ln)
            xa, xb = max(0, x0 - half), min(W, x0 + half + 1)
            R[ya:yb, xa:xb] = SAT_CLIP_ADU
            S[ya:yb, xa:xb] = SAT_CLIP_ADU
            bad[ya:yb, xa:xb] = 1
            trails.append((xa, xb, ya, yb))
        # rectangular edge masks until the requested masked fraction is reached
        guard = 0
        while bad.mean() < mask_fraction and guard < 64:
            guard += 1
            need = (mask_fraction - bad.mean()) * H * W
            side = int(rng.integers(0, 4))
            if side < 2:   # top / bottom strip
                h = int(min(H // 2, max(8, need / W * rng.uniform(0.3, 1.0))))
                wdt = int(rng.integers(W // 4, W + 1))
                xa = int(rng.integers(0, W - wdt + 1))
                ya = 0 if side == 0 else H - h
                bad[ya:ya + h, xa:xa + wdt] = 1
            else:          # left / right strip
                wdt = int(min(W // 2, max(8, need / H * rng.uniform(0.3, 1.0))))
                h = int(rng.integers(H // 4, H + 1))
                ya = int(rng.integers(0, H - h + 1))
                xa = 0 if side == 2 else W - wdt
                bad[ya:ya + h, xa:xa + wdt] = 1
    if clip is not None:
        np.minimum(R, clip, out=R)
        np.minimum(S, clip, out=S)

    return {
        "R": R.astype(np.float32), "S": S.astype(np.float32), "bad": bad,
        "transients": transients, "cosmics": np.array(cosmics, dtype=np.float64).reshape(-1, 3),
        "colsegs": np.array(colsegs, dtype=np.float64).reshape(-1, 4), "misreg": misreg,
        "trails": trails, "masked_fraction": float(bad.mean()),
        "fwhm_R": fR, "fwhm_S": fS, "seed": seed,
    }


def config_pair(name, index=0):
    """The named workloads: 'c1' (512 x 512), 'c2' (2048 x 4096 DECam CCD),
    'c4' (CCD `index` of a 60-CCD exposure, seeds 100..159)."""
    if name == "c1":
        return make_pair(512, 512, seed=1, n_src=300, fwhm_R=(1.2, 1.2), fwhm_S=(1.8, 1.8),
                         shift=(0.1, 0.0), n_transients=1, snr=(20.0, 20.0))
    if name == "c2":
        return make_pair(4096, 2048, seed=2, n_src=20000, fwhm_R=(1.0, 1.4), fwhm_S=(1.5, 2.1),
                         shift=(0.1, 0.0), n_transients=50, snr=(5.0, 50.0), transient_sep=40.0,
                         clip=SAT_CLIP_ADU, mask_saturated=True, bad_columns=(700, 1500))
    if name == "c4":
        seed = 100 + int(index)
        rng = np.random.default_rng(10_000 + seed)
        r_lo, r_hi = rng.uniform(0.9, 1.5, 2)
        s_lo, s_hi = r_lo + rng.uniform(0.4, 0.8), r_hi + rng.uniform(0.4, 0.8)
        ang = float(rng.uniform(0, 2 * math.pi))
        frac = float(rng.uniform(0.02, 0.30))
        cols = tuple(int(c) for c in rng.integers(0, 2048, 2))
        return make_pair(4096, 2048, seed=seed, n_src=20000, fwhm_R=(r_lo, r_hi), fwhm_S=(s_lo, s_hi),
                         grad_angle=ang, shift=(0.1, 0.0), n_transients=50, snr=(5.0, 50.0),
                         clip=SAT_CLIP_ADU, mask_saturated=True, bad_columns=cols,
                         mask_fraction=frac, n_cosmics=80, n_colsegs=2)
    raise ValueError(f"unknown config {name!r}")


def small_pair(H, W, seed, n_src=None, mask_fraction=0.0, **kw):
    """A small pair for parity tests: default density ~1 star per 900 px,
    optional random bad pixels/blobs at `mask_fraction`."""
    if n_src is None:
        n_src = max(4, H * W // 900)
    kw.setdefault("n_transients", 1 if min(H, W) > 48 else 0)
    kw.setdefault("transient_margin", min(10, min(H, W) // 4))
    kw.setdefault("transient_sep", 10.0)
    kw.setdefault("snr", (10.0, 30.0))
    out = make_pair(H, W, seed, n_src=n_src, **kw)
    if mask_fraction > 0:
        rng = np.random.default_rng(seed + 7919)
        bad = out["bad"].copy()
        while bad.mean() < mask_fraction:
            cy, cx = int(rng.integers(0, H)), int(rng.integers(0, W))
            r = int(rng.integers(0, 3))
            bad[max(0, cy - r):cy + r + 1, max(0, cx - r):cx + r + 1] = 1
        out["bad"] = bad
    return out

"""Pins of the FP64 detection oracle: the truncated-Gaussian variance constant
from the normal distribution, clipped RMS on known noise, the separable filter
against brute-force 2-D correlation, the closed-form matched-filter peak, unit
SNR variance on white noise, and candidate rules on constructed images."""
import math

import numpy as np
from scipy import signal, stats

from oracle import detect_oracle as O

RNG = np.random.default_rng(77)


def test_clip_constant_is_truncated_gaussian_variance_share():
    k = O.CLIP_NSIG
    share = 1.0 - 2.0 * k * stats.norm.pdf(k) / (2.0 * stats.norm.cdf(k) - 1.0)
    assert abs(share - O.CLIP_VAR_FRACTION) < 5e-6


def test_clipped_sigma_on_gaussian_noise_with_outliers():
    H, W = 800, 800
    D = RNG.normal(3.0, 5.0, (H, W))
    mu, sd = O.clipped_sigma(D)
    assert abs(sd - 5.0) < 0.02 and abs(mu - 3.0) < 0.02
    D2 = D.copy()
    idx = RNG.integers(0, H * W, H * W // 100)
    D2.flat[idx] = 1e4                        # 1 % wild pixels
    bad = np.zeros((H, W), np.uint8)
    bad[:, 100:110] = 1
    D2[:, 100:110] = np.nan
    mu2, sd2 = O.clipped_sigma(D2, bad)
    assert abs(sd2 - 5.0) < 0.05 and abs(mu2 - 3.0) < 0.05
    # the raw clipped RMS reads ~1.3 % low; the correction must have been applied
    assert sd2 * math.sqrt(O.CLIP_VAR_FRACTION) < 4.96


def test_separable_filter_equals_direct_correlation():
    D = RNG.normal(0, 1, (40, 53))
    bad = np.zeros(D.shape, np.uint8)
    bad[7, 9] = 1
    bad[30, 40] = 1
    s = 1.3
    g = O.gauss_taps(s)
    G2 = np.outer(g, g)
    Dh = np.where(bad == 0, D, 0.0)
    direct = signal.correlate2d(Dh, G2, mode="same", boundary="fill")
    norm = math.sqrt((G2 * G2).sum())
    snr = O.matched_snr(D, bad, s, 2.0)
    assert np.allclose(snr, direct / (2.0 * norm), rtol=0, atol=1e-12)


def test_matched_filter_peak_closed_form():
    s, A, sd = 1.7, 250.0, 4.0
    g = O.gauss_taps(s)
    r = (g.size - 1) // 2
    D = np.zeros((61, 61))
    D[30 - r:31 + r, 30 - r:31 + r] = A * np.outer(g, g)
    snr = O.matched_snr(D, None, s, sd)
    expect = A * math.sqrt((np.outer(g, g) ** 2).sum()) / sd
    assert abs(snr[30, 30] - expect) < 1e-12 * expect
    assert np.argmax(snr) == 30 * 61 + 30


def test_white_noise_snr_is_unit_variance():
    D = RNG.normal(0, 3.0, (600, 600))
    mu, sd = O.clipped_sigma(D)
    snr = O.matched_snr(D, None, 1.5, sd)
    inner = snr[20:-20, 20:-20]
    assert abs(inner.std() - 1.0) < 0.02


def _blob(D, y, x, A, s):
    yy, xx = np.mgrid[0:D.shape[0], 0:D.shape[1]]
    D += A * np.exp(-((yy - y) ** 2 + (xx - x) ** 2) / (2 * s * s))


def test_detect_rules():
    H, W = 120, 140
    D = RNG.normal(0, 1.0, (H, W))
    S = RNG.normal(1000, 30, (H, W))
    R = RNG.normal(1000, 30, (H, W))
    bad = np.zeros((H, W), np.uint8)
    s = 1.5
    placed = [(30, 40), (30, 90), (80, 60), (100, 120)]
    for y, x in placed:
        _blob(D, y, x, 60.0, s)
    _blob(D, 8, 60, 60.0, s)                  # inside the edge margin: dropped
    _blob(D, 60, 20, 60.0, s)
    bad[60, 20] = 1                           # bad peak pixel: dropped
    _blob(D, 55, 100, 60.0, s)
    _blob(D, 56, 101, 30.0, s)                # merged with its neighbour: one local maximum
    out = O.detect(D, S, R, bad, s, 5.0)
    got = list(zip(out["y"].tolist(), out["x"].tolist()))
    assert got == sorted(got)                 # row-major
    for y, x in placed:
        assert (y, x) in got
    assert all(p[0] >= 15 and p[0] <= H - 16 and p[1] >= 15 and p[1] <= W - 16 for p in got)
    assert (60, 20) not in got and not any(p[0] < 15 for p in got)
    assert sum(1 for p in got if abs(p[0] - 55.5) <= 2 and abs(p[1] - 100.5) <= 2) == 1
    assert out["count"] == len(got)
    # stamps are the centred cuts of (S, R, D)
    i = got.index((80, 60))
    assert np.array_equal(out["stamps"][i, 2], D[65:96, 45:76])
    assert np.array_equal(out["stamps"][i, 0], S[65:96, 45:76])
    # truncation keeps the first max_cand in row-major order and the full count
    t = O.detect(D, S, R, bad, s, 5.0, max_cand=2)
    assert t["count"] == len(got) and list(zip(t["y"], t["x"])) == got[:2]


def test_guard_band_against_bad_pixels():
    H, W = 80, 90
    D = RNG.normal(0, 1.0, (H, W))
    _blob(D, 40, 40, 60.0, 1.5)
    _blob(D, 40, 70, 60.0, 1.5)
    bad = np.zeros((H, W), np.uint8)
    bad[43, 44] = 1                             # Chebyshev distance 4 from (40, 40)
    bad[40, 64] = 1                             # distance 6 from (40, 70)
    g0 = list(zip(*O.candidates(O.matched_snr(D, bad, 1.5, 1.0), bad, 5.0, 0)))
    g5 = list(zip(*O.candidates(O.matched_snr(D, bad, 1.5, 1.0), bad, 5.0, 5)))
    assert (40, 40) in g0 and (40, 70) in g0
    assert (40, 40) not in g5 and (40, 70) in g5
    # the guard mask is the brute-force Chebyshev neighbourhood
    m = O.guard_mask(bad, 5)
    ys, xs = np.nonzero(bad)
    yy, xx = np.mgrid[0:H, 0:W]
    brute = np.zeros((H, W), bool)
    for y, x in zip(ys, xs):
        brute |= (np.abs(yy - y) <= 5) & (np.abs(xx - x) <= 5)
    assert np.array_equal(m.astype(bool), brute)

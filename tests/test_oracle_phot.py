"""Pins of the photometry oracle: aperture areas against pi r^2, the enclosed
flux of a Gaussian source against its closed form, flags, the noise of
random apertures on white noise, and the median combination by hand."""
import math

import numpy as np

from oracle import phot_oracle as P
from synth import render_points

RNG = np.random.default_rng(11)


def test_aperture_area_converges_to_disc():
    for r, xc, yc in [(3.0, 20.0, 20.0), (5.37, 20.3, 19.8), (9.0, 25.5, 25.5)]:
        ys, xs, w = P.aperture_weights(xc, yc, r, sub=5)
        assert abs(w.sum() - math.pi * r * r) < 0.03 * math.pi * r * r
        ys, xs, w = P.aperture_weights(xc, yc, r, sub=101)
        assert abs(w.sum() - math.pi * r * r) < 2e-3 * math.pi * r * r
        assert np.all((w >= 0) & (w <= 1))


def test_centred_aperture_is_symmetric():
    # a radius that no sub-pixel centre distance meets within rounding
    ys, xs, w = P.aperture_weights(30.0, 30.0, 4.17)
    assert np.array_equal(w, w[::-1, :]) and np.array_equal(w, w[:, ::-1]) and np.array_equal(w, w.T)


def test_constant_image_and_flags():
    D = np.full((60, 60), 7.0)
    bad = np.zeros((60, 60), np.uint8)
    f, fl = P.aperture_flux(D, bad, [30.0], [30.0], 3.0)
    ys, xs, w = P.aperture_weights(30.0, 30.0, 3.0)
    assert abs(f[0] - 7.0 * w.sum()) < 1e-12 and fl[0] == 0
    bad[31, 29] = 1
    _, fl = P.aperture_flux(D, bad, [30.0, 10.0], [30.0, 10.0], 3.0)
    assert fl.tolist() == [1, 0]
    _, fl = P.aperture_flux(D, None, [1.0], [30.0], 3.0)   # runs off the image
    assert fl[0] == 1


def test_gaussian_enclosed_flux_closed_form():
    sig, F = 3.0, 1e4
    img = render_points(80, 80, [40.2], [39.7], [F], [sig])
    for r in [0.6731 * 2.3548200450309493 * sig, 3.0, 8.0]:
        f, _ = P.aperture_flux(img, None, [40.2], [39.7], r)
        exact = F * (1.0 - math.exp(-r * r / (2 * sig * sig)))
        assert abs(f[0] - exact) < 0.01 * F, (r, f[0], exact)


def test_limiting_magnitude_on_white_noise():
    s_pix, r, zp = 4.0, 3.0, 30.0
    D = RNG.normal(0.0, s_pix, (400, 400))
    xs = RNG.uniform(10, 390, 1024)
    ys = RNG.uniform(10, 390, 1024)
    sigma, mlim, n = P.limiting_mag(D, None, xs, ys, r, zp)
    # independent pixels: the aperture-flux variance is s_pix^2 sum w^2 (averaged over centres)
    w2 = np.mean([(P.aperture_weights(x, y, r)[2] ** 2).sum() for x, y in zip(xs[:64], ys[:64])])
    expect = s_pix * math.sqrt(w2)
    assert n == 1024 and abs(sigma / expect - 1.0) < 0.08
    assert abs(mlim - (zp - 2.5 * math.log10(5 * expect))) < 0.1


def test_median_combine_by_hand():
    Ds = np.array([[[1.0, 5.0]], [[3.0, np.nan]], [[2.0, 4.0]], [[10.0, 7.0]]])
    scales = np.array([1.0, 1.0, 2.0, 1.0])          # third template doubled: 4, 8
    bads = np.zeros(Ds.shape, np.uint8)
    bads[3, 0, 1] = 1                                  # drops the 7
    out = P.median_combine(Ds, scales, bads)
    assert out[0, 0] == 3.5                            # median of 1, 3, 4, 10
    assert out[0, 1] == 6.5                            # median of 5, 8

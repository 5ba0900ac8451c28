"""Pins of the FP64 classifier oracle: library correlation, delta filters,
hand-computed pooling, central finite differences, the closed-form first
Adam step, the naive BCE formula and the shape cuts on constructed stamps."""
import math

import numpy as np
import pytest
from scipy import signal

from oracle import cnn_oracle as C

RNG = np.random.default_rng(2024)


def test_param_count():
    assert C.n_params() == 896 + 18496 + 36928 + 73856 + 129


def test_conv_matches_library_correlation():
    x = RNG.normal(size=(2, 3, 9, 11))
    w = RNG.normal(size=(4, 3, 3, 3))
    b = RNG.normal(size=4)
    y = C.conv_same(x, w, b)
    for n in range(2):
        for o in range(4):
            ref = b[o] + sum(signal.correlate2d(x[n, c], w[o, c], mode="same", boundary="fill") for c in range(3))
            assert np.allclose(y[n, o], ref, atol=1e-12)


def test_delta_filter_is_identity():
    x = RNG.normal(size=(1, 3, 7, 7))
    w = np.zeros((3, 3, 3, 3))
    for c in range(3):
        w[c, c, 1, 1] = 1.0
    assert np.array_equal(C.conv_same(x, w, np.zeros(3)), x)


def test_maxpool_hand_computed_and_floor():
    x = np.array([[1, 5, 2, 0, 9], [3, 4, 8, 8, 9], [7, 0, 1, 1, 9], [6, 6, 2, 3, 9], [9, 9, 9, 9, 9]], float)
    p, idx = C.maxpool2(x[None, None])
    assert np.array_equal(p[0, 0], [[5, 8], [7, 3]])
    assert np.array_equal(idx[0, 0], [[1, 2], [0, 3]])   # first maximum on the tie (8, 8)
    d = C.maxpool2_backward(np.ones((1, 1, 2, 2)), idx, (1, 1, 5, 5))
    assert d.sum() == 4 and d[0, 0, 0, 1] == 1 and d[0, 0, 1, 2] == 1 and d[0, 0, 1, 3] == 0


def test_normalise_median_mad():
    s = np.zeros((1, 3, 31, 31))
    s[0, 0] = np.arange(961).reshape(31, 31)        # median 480; |x - 480| = 0, 1, 1, 2, 2, ... -> MAD 240
    s[0, 1] = 7.0                                   # MAD 0 -> scale 1
    s[0, 2] = RNG.normal(0, 1e4, (31, 31))
    xn = C.normalise(s)
    assert abs(xn[0, 0, 0, 0] - (0 - 480) / (1.4826 * 240.0)) < 1e-12
    assert np.all(xn[0, 1] == 0.0)
    assert np.abs(xn).max() <= 64.0


def test_bce_matches_naive_formula():
    z = np.array([-3.0, -0.5, 0.0, 0.7, 4.0])
    t = np.array([0, 1, 1, 0, 1.0])
    s = 1 / (1 + np.exp(-z))
    naive = np.mean(-(t * np.log(s) + (1 - t) * np.log(1 - s)))
    assert abs(C.bce_loss(z, t) - naive) < 1e-14


def test_gradients_match_central_differences():
    p = C.init_params(7)
    for k in p:
        if k.startswith("b"):
            p[k] = RNG.normal(0, 0.05, p[k].shape)
    x = C.normalise(RNG.normal(1000, 30, (3, 3, 31, 31)))
    t = np.array([1.0, 0.0, 1.0])
    loss, g = C.loss_and_grads(p, x, t)
    h = 1e-6
    rng = np.random.default_rng(8)
    for k in C.ORDER:
        for _ in range(6):
            idx = tuple(rng.integers(0, s) for s in p[k].shape)
            old = p[k][idx]
            p[k][idx] = old + h
            lp = C.bce_loss(C.forward(p, x), t)
            p[k][idx] = old - h
            lm = C.bce_loss(C.forward(p, x), t)
            p[k][idx] = old
            fd = (lp - lm) / (2 * h)
            assert abs(fd - g[k][idx]) <= 1e-6 * max(abs(fd), 1e-3) + 1e-9, (k, idx, fd, g[k][idx])


def test_first_adam_step_closed_form():
    p = {"w": np.array([1.0, -2.0, 0.5])}
    g = {"w": np.array([0.3, -4.0, 1e-3])}
    opt = C.Adam(p, lr=0.01)
    p2 = opt.step({"w": p["w"].copy()}, g)
    # first step: m_hat = g, v_hat = g^2  ->  theta - lr g / (|g| + eps)
    assert np.allclose(p2["w"], p["w"] - 0.01 * g["w"] / (np.abs(g["w"]) + 1e-8), rtol=0, atol=1e-15)


def _gauss_stamp(fwhm, amp=500.0, cx=15.0, cy=15.0):
    s = fwhm / 2.3548200450309493
    yy, xx = np.mgrid[0:31, 0:31]
    return amp * np.exp(-((xx - cx) ** 2 + (yy - cy) ** 2) / (2 * s * s))


def test_shape_cuts_on_constructed_stamps():
    assert C.shape_cuts(_gauss_stamp(2.0), snr=10.0, fwhm_psf=2.0)
    assert not C.shape_cuts(_gauss_stamp(2.0), snr=4.0, fwhm_psf=2.0)           # below SNR
    dip = _gauss_stamp(2.0, cx=14.4) - _gauss_stamp(2.0, cx=15.6)
    assert not C.shape_cuts(dip, snr=10.0, fwhm_psf=2.0)                        # dipole residual
    hot = np.zeros((31, 31)); hot[15, 15] = 1e4
    assert not C.shape_cuts(hot, snr=50.0, fwhm_psf=2.0)                        # cosmic-ray point
    col = np.zeros((31, 31)); col[:, 15] = 800.0
    assert not C.shape_cuts(col, snr=20.0, fwhm_psf=2.0)                        # column segment


def test_training_reduces_loss_on_separable_toy():
    rng = np.random.default_rng(3)
    p = C.init_params(3)
    n = 16
    st = rng.normal(1000, 30, (n, 3, 31, 31))
    t = (np.arange(n) % 2).astype(float)
    st[t == 1, 2] += _gauss_stamp(2.0, amp=400.0)
    xn = C.normalise(st)
    opt = C.Adam(p, lr=2e-3)
    l0 = C.loss_and_grads(p, xn, t)[0]
    for _ in range(15):
        _, g = C.loss_and_grads(p, xn, t)
        p = opt.step(p, g)
    assert C.loss_and_grads(p, xn, t)[0] < 0.5 * l0


# ------------------------------------------------------------------ rotation-invariant residual network
def _ri_setup(n=4, seed=5):
    p = C.init_params_ri(seed)
    rng = np.random.default_rng(seed + 1)
    for k in p:
        if k.startswith("b"):
            p[k] = rng.normal(0, 0.05, p[k].shape)
    xn = rng.normal(0, 1.0, (n, 3, 31, 31))
    t = (rng.random(n) < 0.5).astype(np.float64)
    return p, xn, t


def test_ri_parameter_count():
    assert C.n_params_ri() == 185729
    p = C.init_params_ri(1)
    assert np.array_equal(C.flatten_ri(C.unflatten_ri(C.flatten_ri(p))), C.flatten_ri(p))


def test_ri_rotations_follow_numpy_rot90():
    x = np.arange(2 * 3 * 31 * 31, dtype=np.float64).reshape(2, 3, 31, 31)
    r = C.rotations(x)
    assert r.shape == (8, 3, 31, 31)
    # one counterclockwise quarter turn: out[y][x] = in[x][30 - y]
    assert r[2, 1, 5, 7] == x[0, 1, 7, 30 - 5]
    assert r[4, 2, 5, 7] == x[0, 2, 30 - 5, 30 - 7]
    assert r[6, 0, 5, 7] == x[0, 0, 30 - 7, 5]


def test_ri_score_is_rotation_invariant_and_features_are_not():
    p, xn, _ = _ri_setup()
    z0 = C.forward_ri(p, xn)
    for r in (1, 2, 3):
        zr = C.forward_ri(p, np.rot90(xn, r, axes=(2, 3)).copy())
        assert np.allclose(zr, z0, rtol=1e-12, atol=1e-12)
    # mirroring is not one of the four rotations: the score moves
    zm = C.forward_ri(p, xn[:, :, :, ::-1].copy())
    assert np.max(np.abs(zm - z0)) > 1e-6
    # each rotation's own feature vector differs (the average is what is invariant)
    _, c = C.forward_ri(p, xn, keep=True)
    p3 = C.maxpool2(np.maximum(c["zd"], 0.0))[0].reshape(4, xn.shape[0], -1)
    assert np.max(np.abs(p3[1] - p3[0])) > 1e-6


def test_ri_residual_block_with_zero_branch_is_identity():
    """With the second convolution of each block zeroed the block returns its
    (non-negative) input: the network equals the same network without the
    residual branches, written out here without them."""
    p, xn, _ = _ri_setup(n=3, seed=9)
    for k in ("wb", "bb", "wd", "bd"):
        p[k] = np.zeros_like(p[k])
    z = C.forward_ri(p, xn)
    x = C.rotations(xn)
    a = C.maxpool2(np.maximum(C.conv_same(x, p["w1"], p["b1"]), 0))[0]
    a = C.maxpool2(np.maximum(C.conv_same(a, p["w2"], p["b2"]), 0))[0]
    a = C.maxpool2(a)[0]
    f = a.reshape(4, xn.shape[0], -1).mean(axis=0)
    zz = (np.maximum(f @ p["w4"].T + p["b4"], 0) @ p["w5"].T + p["b5"])[:, 0]
    assert np.allclose(z, zz, rtol=1e-12, atol=1e-12)


def test_ri_gradients_by_central_differences():
    p, xn, t = _ri_setup(n=3, seed=11)
    loss, g = C.loss_and_grads_ri(p, xn, t)
    rng = np.random.default_rng(3)
    h = 1e-6
    for k in C.ORDER_RI:
        flat = p[k].ravel()
        for idx in rng.choice(flat.size, size=min(4, flat.size), replace=False):
            old = flat[idx]
            flat[idx] = old + h
            lp = C.bce_loss(C.forward_ri(p, xn), t)
            flat[idx] = old - h
            lm = C.bce_loss(C.forward_ri(p, xn), t)
            flat[idx] = old
            num = (lp - lm) / (2 * h)
            ana = g[k].ravel()[idx]
            assert abs(num - ana) <= 1e-6 * max(1.0, abs(num)) + 1e-8, (k, idx, num, ana)


# ---------------------------------------------------------------- the BF16 operand model
def test_round_bf16_hand_computed_ties_to_even():
    e8, e7, e6 = 2.0 ** -8, 2.0 ** -7, 2.0 ** -6
    cases = [
        (1.0, 1.0),
        (3.0, 3.0),                       # representable: unchanged
        (1 + e8, 1.0),                    # exact half between 1 and 1 + 2^-7: to the even 1
        (1 + 3 * e8, 1 + e6),             # exact half between 1 + 2^-7 (odd) and 1 + 2^-6 (even)
        (1 + e8 + 2.0 ** -20, 1 + e7),    # just above the half: up
        (1 + e8 - 2.0 ** -20, 1.0),       # just below: down
        (-(1 + 3 * e8), -(1 + e6)),       # sign kept
        (255.5, 256.0),                   # 8 significant bits: 255.5 is the half between 255 and 256 (even)
        (254.5, 254.0),                   # half between 254 (even) and 255
        (0.0, 0.0),
    ]
    for x, want in cases:
        assert C.round_bf16(np.array([x]))[0] == want, (x, C.round_bf16(np.array([x]))[0], want)


def test_round_bf16_matches_library_conversion():
    torch = pytest.importorskip("torch")
    x = np.concatenate([RNG.normal(0, 1, 20000), RNG.normal(0, 1e6, 2000), RNG.normal(0, 1e-6, 2000)])
    x = x.astype(np.float32)
    ref = torch.from_numpy(x).to(torch.bfloat16).to(torch.float32).numpy().astype(np.float64)
    assert np.array_equal(C.round_bf16(x), ref)


def _sparse_integer_net():
    """Delta-like filters with weights +-1, small integer inputs and a large
    fc2 bias: every operand and every sum is a small integer, exact in BF16;
    with the targets below every back-propagated signal is a multiple of 2^-4."""
    p = {k: np.zeros(C.SHAPES[k]) for k in C.ORDER}
    for o in range(32):
        p["w1"][o, o % 3, 1, 1] = 1.0 if o % 2 == 0 else -1.0
    for o in range(64):
        p["w2"][o, o % 32, 1, 1] = 1.0
        p["w3"][o, o, 1, 1] = 1.0
    for o in range(128):
        p["w4"][o, (7 * o) % 576] = 1.0
    p["w5"][0, :] = np.where(np.arange(128) % 3 == 0, 1.0, -1.0)
    p["b5"][0] = 1000.0                   # sigmoid(logit) = 1 in FP64
    xn = RNG.integers(-4, 5, size=(8, 3, 31, 31)).astype(np.float64)
    return p, xn


def test_bf16_model_equals_fp64_network_when_operands_are_exact():
    p, xn = _sparse_integer_net()
    z = C.forward(p, xn)
    assert np.array_equal(C.forward_bf16(p, xn), z)
    assert np.all(z > 100)
    # targets 1/2: (sigmoid - t) / n = 2^-4 exactly, so every dz is exact in BF16
    t = np.full(8, 0.5)
    lo, go = C.loss_and_grads(p, xn, t)
    lb, gb = C.loss_and_grads_bf16(p, xn, t)
    assert lb == lo
    for k in C.ORDER:
        assert np.array_equal(gb[k], go[k]), k
        assert np.any(go[k] != 0), k


def test_bf16_model_rounds_inputs_weights_and_activations():
    """Delta filters route one pixel to the logit: the FP64 network returns
    the pixel times the weights; the BF16 model returns the pixel rounded, the
    rounded weights, and each product rounded again at every pooled layer."""
    p = {k: np.zeros(C.SHAPES[k]) for k in C.ORDER}
    w = 1 + 3 * 2.0 ** -8                 # rounds to 1 + 2^-6
    p["w1"][0, 0, 1, 1] = w
    p["w2"][0, 0, 1, 1] = 1.0
    p["w3"][0, 0, 1, 1] = 1.0
    p["w4"][0, 0] = 1.0
    p["w5"][0, 0] = 1.0
    xn = np.zeros((1, 3, 31, 31))
    xn[0, 0, 0, 0] = 1 + 2.0 ** -8        # rounds to 1
    assert C.forward(p, xn)[0] == (1 + 2.0 ** -8) * w
    # 1 * (1 + 2^-6) is exact in BF16: nothing more is lost after the first layer
    assert C.forward_bf16(p, xn)[0] == 1 + 2.0 ** -6
    xn[0, 0, 0, 0] = 1 + 2.0 ** -7        # exact; the product (1 + 2^-7)(1 + 2^-6) = 1 + 3 * 2^-7 + 2^-13
    assert C.forward_bf16(p, xn)[0] == C.round_bf16(np.array([(1 + 2.0 ** -7) * (1 + 2.0 ** -6)]))[0]
    assert C.forward_bf16(p, xn)[0] == 1 + 3 * 2.0 ** -7  # the 2^-13 is below half a unit (2^-8): dropped


def test_ri_bf16_model_equals_fp64_network_when_operands_are_exact():
    """Integer weights and inputs with every sum a small integer (and the
    rotation mean of a value repeated four times): the BF16 model of the
    rotation-invariant network equals the FP64 network exactly."""
    p = {k: np.zeros(v.shape) for k, v in C.init_params_ri(0).items()}
    for o in range(32):
        p["w1"][o, o % 3, 1, 1] = 1.0
        p["wa"][o, o, 1, 1] = -1.0 if o % 2 else 1.0
        p["wb"][o, o, 1, 1] = 1.0
    for o in range(64):
        p["w2"][o, o % 32, 1, 1] = 1.0
        p["wc"][o, o, 1, 1] = 1.0
        p["wd"][o, o, 1, 1] = -1.0
    for o in range(128):
        p["w4"][o, (5 * o) % 576] = 1.0
    p["w5"][0, :] = 1.0
    xn = RNG.integers(0, 5, size=(3, 3, 31, 31)).astype(np.float64)
    xn = xn + np.rot90(xn, 1, axes=(2, 3)) + np.rot90(xn, 2, axes=(2, 3)) + np.rot90(xn, 3, axes=(2, 3))
    assert np.array_equal(C.forward_ri_bf16(p, xn), C.forward_ri(p, xn))


# ---------------------------------------------------------------- noise-robust shape cuts
def _gauss_cov_stamp(cov, flux=1000.0, centre=(0.0, 0.0)):
    yy, xx = np.mgrid[-15:16, -15:16].astype(np.float64)
    ci = np.linalg.inv(np.asarray(cov, dtype=np.float64))
    dx, dy = xx - centre[0], yy - centre[1]
    return flux * np.exp(-0.5 * (ci[0, 0] * dx * dx + 2 * ci[0, 1] * dx * dy + ci[1, 1] * dy * dy))


def test_adaptive_moments_recover_a_gaussian():
    """A noiseless round Gaussian of sigma 1.5 sampled at the pixel centres:
    the moments of a sampled Gaussian equal the continuous ones up to
    exp(-2 pi^2 sigma^2) (Poisson summation), so M = sigma^2 I to 1e-6."""
    (mxx, myy, mxy), (mx, my) = C.adaptive_moments(_gauss_cov_stamp(np.eye(2) * 2.25), 1.0)
    assert abs(mxx - 2.25) < 1e-6 * 2.25 and abs(myy - 2.25) < 1e-6 * 2.25 and abs(mxy) < 1e-9
    assert abs(mx) < 1e-12 and abs(my) < 1e-12
    # an elliptical, rotated, off-centre Gaussian: its covariance and centre
    th = 0.5
    rot = np.array([[np.cos(th), -np.sin(th)], [np.sin(th), np.cos(th)]])
    cov = rot @ np.diag([4.0, 1.0]) @ rot.T
    (mxx, myy, mxy), (mx, my) = C.adaptive_moments(_gauss_cov_stamp(cov, centre=(0.4, -0.7)), 1.0)
    # (the 15 x 15 window cuts the weighted profile of the 2 px major axis at ~4.5 of its widths)
    assert np.allclose([mxx, myy, mxy], [cov[0, 0], cov[1, 1], cov[0, 1]], rtol=0, atol=1e-5)
    assert abs(mx - 0.4) < 1e-5 and abs(my + 0.7) < 1e-5


def test_adaptive_moments_ignore_distant_noise_and_reject_hits():
    g = _gauss_cov_stamp(np.eye(2) * 2.25)
    noisy = g.copy()
    noisy[0:3, :] += 200.0          # a bright band 12 px away: negligible weight
    (mxx, _, _), _ = C.adaptive_moments(noisy, 1.0)
    assert abs(mxx - 2.25) < 1e-3
    hit = np.zeros((31, 31))
    hit[15, 15] = 1e4               # a one-pixel cosmic-ray hit: the weight collapses
    assert C.adaptive_moments(hit, 1.0) is None
    fw = 2.3548200450309493 * 1.5
    assert C.shape_cuts_adaptive(g, 20.0, fw)
    assert not C.shape_cuts_adaptive(hit, 20.0, fw)
    assert not C.shape_cuts_adaptive(g, 4.0, fw)                      # below the SNR cut
    assert not C.shape_cuts_adaptive(_gauss_cov_stamp(np.diag([9.0, 1.0])), 20.0, fw)   # axis ratio 3

"""Pins of the FP64 subtraction oracle against facts that do not come from
the oracle itself: brute-force sums, the shift theorem, exact-model inverse
problems built with a library convolution, the Gaussian convolution closed
form, noise-free transient recovery, linearity and invariances."""
import math

import numpy as np
import pytest
from scipy import ndimage

from oracle import sfft_oracle as O
from synth import make_pair, small_pair, render_points

RNG = np.random.default_rng(12345)


def _noise_field(H, W, seed, n_src=None):
    d = small_pair(H, W, seed=seed, n_src=n_src, n_transients=0)
    return d["R"].astype(np.float64)


# ------------------------------------------------------------------ basis / masks
def test_monomial_order_and_offsets():
    # degree-major, a descending within a degree: 1; x, y; x^2, xy, y^2
    assert O.monomials(2) == [(0, 0), (1, 0), (0, 1), (2, 0), (1, 1), (0, 2)]
    assert O.n_unknowns(11, 2, 2) == 732 and O.n_unknowns(7, 1, 1) == 150
    offs = O.offsets(5)
    assert offs[0] == (-2, -2) and offs[12] == (0, 0) and offs[13] == (0, 1) and offs[5] == (-1, -2)
    assert len(O.half_plane_diffs(11)) == 221 and len(O.half_plane_diffs(7)) == 85


def test_fit_mask_brute_force():
    H, W, L = 23, 31, 5
    w = 2
    good = RNG.random((H, W)) > 0.04
    M = O.fit_mask(good, L)
    ref = np.zeros_like(M)
    for y in range(H):
        for x in range(W):
            if w <= y < H - w and w <= x < W - w:
                ref[y, x] = all(good[y + dy, x + dx] for dy in range(-w, w + 1) for dx in range(-w, w + 1))
    assert np.array_equal(M, ref)


def test_prepare_masks_nonfinite_and_median():
    d = small_pair(30, 40, seed=5)
    R = d["R"].copy(); S = d["S"].copy()
    R[3, 4] = np.nan; S[10, 11] = np.inf
    bad = np.zeros(R.shape, np.uint8); bad[20, 30] = 1
    p = O.prepare(R, S, bad, 3)
    assert not p["good"][3, 4] and not p["good"][10, 11] and not p["good"][20, 30]
    assert p["R_m"][3, 4] == 0.0 and p["R_t"][3, 4] == 0.0
    assert p["R_t"][10, 11] == R[10, 11] - p["s_R"]       # finite R is kept for the apply step
    assert p["s_R"] == np.median(R.astype(np.float64)[p["good"]])


# ------------------------------------------------------------------ P1: brute force
def _brute_normal(R, S, bad, L, DK, DB):
    """Explicit loops over pixels and offsets (independent of the oracle)."""
    R = R.astype(np.float64); S = S.astype(np.float64)
    H, W = R.shape
    w = (L - 1) // 2
    good = (bad == 0) & np.isfinite(R) & np.isfinite(S)
    sR = np.median(R[good]); sS = np.median(S[good])
    mk = [(a, n - a) for n in range(DK + 1) for a in range(n, -1, -1)]
    mb = [(a, n - a) for n in range(DB + 1) for a in range(n, -1, -1)]
    N = L * L * len(mk) + len(mb)
    A = np.zeros((N, N)); b = np.zeros(N)
    for y in range(w, H - w):
        for x in range(w, W - w):
            if not good[y - w:y + w + 1, x - w:x + w + 1].all():
                continue
            xt = 2.0 * x / (W - 1) - 1.0; yt = 2.0 * y / (H - 1) - 1.0
            phi = [xt ** a * yt ** bb for (a, bb) in mk]
            row = []
            for uy in range(-w, w + 1):
                for ux in range(-w, w + 1):
                    r = R[y - uy, x - ux] - sR
                    row += [f * r for f in phi]
            row += [xt ** a * yt ** bb for (a, bb) in mb]
            row = np.array(row)
            A += np.outer(row, row)
            b += row * (S[y, x] - sS)
    return A, b


@pytest.mark.parametrize("L,DK,DB", [(3, 1, 1), (3, 0, 2)])
def test_p1_definition_vs_brute_force(L, DK, DB):
    d = small_pair(14, 17, seed=21, mask_fraction=0.05, n_src=3)
    prep = O.prepare(d["R"], d["S"], d["bad"], L)
    A, b = O.normal_definition(prep, DK, DB)
    Ab, bb = _brute_normal(d["R"], d["S"], d["bad"], L, DK, DB)
    assert np.abs(A - Ab).max() <= 1e-12 * np.abs(Ab).max()
    assert np.abs(b - bb).max() <= 1e-12 * np.abs(bb).max()


@pytest.mark.parametrize("shape", [(32, 32), (64, 64), (41, 57)])
@pytest.mark.parametrize("L,DK,DB", [(3, 0, 0), (5, 1, 1), (7, 2, 2), (5, 1, 2)])
def test_p1_fourier_vs_definition(shape, L, DK, DB):
    d = small_pair(*shape, seed=31 + L + DK, mask_fraction=0.04)
    prep = O.prepare(d["R"], d["S"], d["bad"], L)
    A1, b1 = O.normal_definition(prep, DK, DB)
    A2, b2 = O.normal_fourier(prep, DK, DB)
    assert np.abs(A1 - A2).max() <= 1e-12 * np.abs(A1).max()
    assert np.abs(b1 - b2).max() <= 1e-12 * np.abs(b1).max()
    assert np.array_equal(A1, A1.T)


# ------------------------------------------------------------------ sign / ordering pins
def test_shift_theorem_pins_convolution_sign():
    """S(y, x) = R(y - 2, x - 1): the image content moves by +1 in x and +2 in
    y, so with (K (x) R)(x) = sum_u K_u R(x - u) the kernel is a delta at
    u = (u_y, u_x) = (2, 1)."""
    H, W, L = 48, 52, 7
    R = _noise_field(H, W, 41, n_src=8)
    S = np.full_like(R, 1000.0)
    S[2:, 1:] = R[:-2, :-1]
    out = O.fit(R, S, None, L, 0, 0)
    c, _ = O.split_theta(out["theta"], L, 0, 0)
    K = c[:, 0].reshape(L, L)
    w = 3
    assert abs(K[2 + w, 1 + w] - 1.0) < 1e-10
    K[2 + w, 1 + w] = 0.0
    assert np.abs(K).max() < 1e-10


def test_polynomial_coordinates_ordering_and_background_units():
    """S = (1 + 0.3 xt - 0.2 yt) R + 5 + 2 yt - 3 xt^2 is an exact model with a
    delta kernel whose amplitude varies as the stated polynomial."""
    H, W, L = 40, 60, 3
    R = _noise_field(H, W, 43, n_src=6)
    xt = 2.0 * np.arange(W) / (W - 1) - 1.0
    yt = 2.0 * np.arange(H) / (H - 1) - 1.0
    X, Y = np.meshgrid(xt, yt)
    S = (1.0 + 0.3 * X - 0.2 * Y) * R + 5.0 + 2.0 * Y - 3.0 * X ** 2
    out = O.fit(R, S, None, L, 1, 2)
    c, beta = O.split_theta(out["theta_orig"], L, 1, 2)
    assert np.allclose(c[4], [1.0, 0.3, -0.2], atol=1e-9)
    assert np.abs(np.delete(c, 4, axis=0)).max() < 1e-9
    # psi order: 1, x, y, x^2, xy, y^2
    assert np.allclose(beta, [5.0, 0.0, 2.0, -3.0, 0.0, 0.0], atol=1e-6)


# ------------------------------------------------------------------ P2, P3
def test_p2_identity():
    d = small_pair(48, 56, seed=51, mask_fraction=0.03)
    out = O.fit(d["R"], d["R"], d["bad"], 5, 1, 1)
    c, beta = O.split_theta(out["theta_orig"], 5, 1, 1)
    assert np.allclose(c[12], [1.0, 0.0, 0.0], atol=1e-10)
    assert np.abs(np.delete(c, 12, axis=0)).max() < 1e-10
    assert np.abs(beta).max() < 1e-7
    D = out["D"]
    assert np.abs(D[np.isfinite(D)]).max() < 1e-8


def _exact_model_science(R, theta_c, beta, L, DK, DB):
    """S = sum_p phi_p (c_p conv R) + B with a library convolution (zero outside)."""
    H, W = R.shape
    xt = 2.0 * np.arange(W) / (W - 1) - 1.0
    yt = 2.0 * np.arange(H) / (H - 1) - 1.0
    X, Y = np.meshgrid(xt, yt)
    mk = [(a, n - a) for n in range(DK + 1) for a in range(n, -1, -1)]
    mb = [(a, n - a) for n in range(DB + 1) for a in range(n, -1, -1)]
    S = np.zeros_like(R)
    for p, (a, b) in enumerate(mk):
        ker = theta_c[:, p].reshape(L, L)
        S += X ** a * Y ** b * ndimage.convolve(R, ker, mode="constant", cval=0.0)
    for q, (a, b) in enumerate(mb):
        S += beta[q] * X ** a * Y ** b
    return S


@pytest.mark.parametrize("L,DK,DB,masked", [(5, 1, 1, False), (7, 2, 2, True), (5, 0, 1, True)])
def test_p3_exact_model_inverse(L, DK, DB, masked):
    H, W = 64, 72
    d = small_pair(H, W, seed=61 + L, n_src=10, mask_fraction=0.03 if masked else 0.0)
    R = d["R"].astype(np.float64)
    rng = np.random.default_rng(62 + L)
    NK, NB = O.n_terms(DK), O.n_terms(DB)
    c = rng.normal(0, 0.05, (L * L, NK))
    c[(L * L) // 2, 0] = 0.8
    beta = rng.normal(0, 3.0, NB); beta[0] = 900.0
    S = _exact_model_science(R, c, beta, L, DK, DB)
    out = O.fit(R, S, d["bad"], L, DK, DB)          # sky = medians: tests the offset invariance
    ct, bt = O.split_theta(out["theta_orig"], L, DK, DB)
    assert np.abs(ct - c).max() <= 1e-9 * np.abs(c).max()
    assert np.abs(bt - beta).max() <= 1e-9 * np.abs(beta).max()
    # D vanishes wherever the footprint is inside the image and finite
    w = (L - 1) // 2
    assert np.abs(out["D"][w:H - w, w:W - w]).max() < 1e-8 * np.abs(S).max()


# ------------------------------------------------------------------ P4: Gaussian closed form
def _point_sampled_stars(H, W, xs, ys, F, sigma):
    yy, xx = np.mgrid[0:H, 0:W]
    img = np.zeros((H, W))
    for x0, y0, f in zip(xs, ys, F):
        r2 = (xx - x0) ** 2 + (yy - y0) ** 2
        img += f * np.exp(-0.5 * r2 / sigma ** 2) / (2 * math.pi * sigma ** 2)
    return img


def test_p4_gaussian_closed_form():
    """Well-sampled Gaussians: G(sigma_R) convolved with f G(1) is f G(sigma_S),
    sigma_S^2 = sigma_R^2 + 1.  The fitted kernel has sum f and per-axis second
    moment 1 (sampling/aliasing error ~exp(-2 pi^2) and truncation beyond
    |u| = 5 ~1e-8 both far below the tolerances)."""
    H, W, L, f = 72, 80, 11, 1.7
    sR = 1.5
    sS = math.sqrt(sR ** 2 + 1.0)
    rng = np.random.default_rng(71)
    n = 25
    xs = rng.uniform(12, W - 12, n); ys = rng.uniform(12, H - 12, n)
    F = rng.uniform(2e3, 2e4, n)
    R = 1000.0 + _point_sampled_stars(H, W, xs, ys, F, sR)
    S = 800.0 + f * _point_sampled_stars(H, W, xs, ys, F, sS)
    out = O.fit(R, S, None, L, 0, 0)
    c, _ = O.split_theta(out["theta"], L, 0, 0)
    K = c[:, 0].reshape(L, L)
    u = np.arange(L) - (L - 1) // 2
    tot = K.sum()
    assert abs(tot - f) < 1e-6 * f
    mx = (K.sum(axis=0) * u ** 2).sum() / tot
    my = (K.sum(axis=1) * u ** 2).sum() / tot
    assert abs(mx - 1.0) < 1e-4 and abs(my - 1.0) < 1e-4
    assert abs((K.sum(axis=0) * u).sum()) < 1e-8 and abs((K.sum(axis=1) * u).sum()) < 1e-8


# ------------------------------------------------------------------ P5: transients
def test_p5_noise_free_transients():
    H, W, L, DK, DB = 96, 96, 7, 1, 1
    d = make_pair(H, W, seed=81, n_src=20, fwhm_R=(1.2, 1.6), fwhm_S=(1.8, 2.2), n_transients=0, noise=False)
    R = d["R"].astype(np.float64)
    rng = np.random.default_rng(82)
    c = rng.normal(0, 0.02, (L * L, 3)); c[L * L // 2, 0] = 0.9
    S = _exact_model_science(R, c, np.array([950.0, 4.0, -2.0]), L, DK, DB)
    sig = 0.85
    tx, ty, tf = [30.3, 65.7], [40.2, 70.6], [3000.0, 1500.0]
    stamp = render_points(H, W, tx, ty, tf, sig)
    S = S + stamp
    bad = np.zeros((H, W), np.uint8)
    yy, xx = np.mgrid[0:H, 0:W]
    rad = (L - 1) // 2 + 3 * sig + 3
    for x0, y0 in zip(tx, ty):
        bad[(xx - x0) ** 2 + (yy - y0) ** 2 <= rad ** 2] = 1
    out = O.fit(R, S, bad, L, DK, DB)
    half = int(math.ceil(3 * sig))
    for x0, y0 in zip(tx, ty):
        fd = O.box_flux(out["D"], x0, y0, half)
        fi = O.box_flux(stamp, x0, y0, half)
        assert abs(fd - fi) <= 1e-6 * fi


# ------------------------------------------------------------------ P6 and invariances
def test_p6_linearity_symmetry_spd_and_offsets():
    d = small_pair(56, 64, seed=91, mask_fraction=0.03)
    L, DK, DB = 5, 1, 2
    o1 = O.fit(d["R"], d["S"], d["bad"], L, DK, DB)
    o2 = O.fit(d["R"], 2.5 * d["S"].astype(np.float64), d["bad"], L, DK, DB)
    t1, t2 = o1["theta_orig"], o2["theta_orig"]
    assert np.abs(t2 - 2.5 * t1).max() <= 1e-9 * np.abs(t2).max()
    A = o1["A"]
    assert np.array_equal(A, A.T)
    assert np.linalg.eigvalsh(A).min() > 0
    # a constant added to S only shifts the constant background term
    o3 = O.fit(d["R"], d["S"].astype(np.float64) + 123.0, d["bad"], L, DK, DB)
    t3 = o3["theta_orig"].copy()
    N = len(t3); NKK = L * L * O.n_terms(DK)
    assert abs(t3[NKK] - t1[NKK] - 123.0) < 1e-8
    t3[NKK] -= 123.0
    assert np.abs(t3 - t1).max() <= 1e-9 * np.abs(t1).max()
    # any sky constant gives the same kernel and original-unit background (D_B >= D_K)
    o4 = O.fit(d["R"], d["S"], d["bad"], L, DK, DB, sky=(700.0, 1300.0))
    assert np.abs(o4["theta_orig"] - t1).max() <= 1e-8 * np.abs(t1).max()
    assert N == O.n_unknowns(L, DK, DB)


def test_refinement_is_a_no_op_in_fp64():
    d = small_pair(48, 48, seed=95)
    o = O.fit(d["R"], d["S"], None, 5, 1, 1)
    t2, st = O.refine(o["prep"], 1, 1, o["A"], o["theta"])
    assert st == O.STATUS_OK
    assert np.abs(t2 - o["theta"]).max() <= 1e-12 * np.abs(o["theta"]).max()


def test_solve_singular_and_nonfinite():
    A = RNG.normal(size=(20, 20)); A = A @ A.T + 20 * np.eye(20)
    b = RNG.normal(size=20)
    th, st = O.solve(A, b)
    assert st == O.STATUS_OK and np.allclose(th, np.linalg.solve(A, b), rtol=1e-12, atol=1e-14)
    A2 = A.copy(); A2[:, 3] = 0; A2[3, :] = 0
    assert O.solve(A2, b)[1] == O.STATUS_SINGULAR
    A3 = A.copy(); A3[5, 6] = A3[6, 5] = 1e6
    assert O.solve(A3, b)[1] == O.STATUS_SINGULAR
    A4 = A.copy(); A4[1, 1] = np.nan
    assert O.solve(A4, b)[1] == O.STATUS_NONFINITE
    # a fully masked image has no fit pixels: singular
    d = small_pair(20, 20, seed=96)
    o = O.fit(d["R"], d["S"], np.ones((20, 20), np.uint8), 3, 0, 0)
    assert o["status"] == O.STATUS_SINGULAR


def test_apply_matches_library_convolution_everywhere():
    """D over the whole image (edges included) against the library convolution
    of R~ with zeros outside the image."""
    d = small_pair(40, 44, seed=97)
    L, DK, DB = 5, 1, 1
    prep = O.prepare(d["R"], d["S"], None, L, sky=(1000.0, 1000.0))
    rng = np.random.default_rng(98)
    c = rng.normal(0, 0.1, (L * L, 3)); beta = rng.normal(0, 2, 3)
    theta = np.concatenate([c.ravel(), beta])
    D = O.apply(prep, theta, DK, DB)
    model = _exact_model_science(prep["R_t"], c, beta, L, DK, DB)
    assert np.abs(D - (prep["S_p"] - model)).max() < 1e-9


# ------------------------------------------------------------------ constant photometric ratio
def _kernel_sums(theta, L, DK, DB, H, W, pts):
    return np.array([O.kernel_at(theta, L, DK, DB, H, W, x, y).sum() for (x, y) in pts])


PTS = [(3.0, 4.0), (60.0, 10.0), (20.0, 50.0), (70.0, 60.0), (35.5, 31.0)]


def test_const_ratio_with_constant_kernel_spans_the_full_basis():
    """D_K = 0: delta_0 plus the differences delta_u - delta_0 span every
    constant kernel, so the constrained and free fits are the same problem."""
    H, W, L = 56, 64, 5
    d = small_pair(H, W, seed=71, n_src=12, mask_fraction=0.02)
    free = O.fit(d["R"], d["S"], d["bad"], L, 0, 1)
    cpr = O.fit_const_ratio(d["R"], d["S"], d["bad"], L, 0, 1)
    assert cpr["A_c"].shape[0] == O.n_unknowns(L, 0, 1)
    assert np.abs(cpr["theta"] - free["theta"]).max() <= 1e-8 * np.abs(free["theta"]).max()
    assert np.abs(cpr["D"] - free["D"]).max() <= 1e-8 * np.abs(d["S"]).max()


@pytest.mark.parametrize("L,DK,DB", [(5, 2, 2), (7, 2, 0), (5, 1, 0)])
def test_const_ratio_exact_model_recovered(L, DK, DB):
    """S = K (x) R + B with a kernel whose shape varies over the chip but whose
    sum is constant: the constrained fit returns it exactly, also for
    D_B < D_K (the sky offset then only shifts the constant background)."""
    H, W = 64, 72
    d = small_pair(H, W, seed=81 + L + DB, n_src=10, mask_fraction=0.03)
    R = d["R"].astype(np.float64)
    rng = np.random.default_rng(82 + DK)
    NK, NB = O.n_terms(DK), O.n_terms(DB)
    c = rng.normal(0, 0.05, (L * L, NK))
    c[:, 1:] -= c[:, 1:].mean(axis=0)              # sum_j c[j, p] = 0 for p >= 1
    c[O.center_index(L), 0] += 0.8
    beta = rng.normal(0, 3.0, NB); beta[0] = 900.0
    S = _exact_model_science(R, c, beta, L, DK, DB)
    out = O.fit_const_ratio(R, S, d["bad"], L, DK, DB)    # sky = medians
    ct, bt = O.split_theta(out["theta_orig"], L, DK, DB)
    assert np.abs(ct - c).max() <= 1e-9 * np.abs(c).max()
    assert np.abs(bt - beta).max() <= 1e-9 * np.abs(beta).max()
    w = (L - 1) // 2
    assert np.abs(out["D"][w:H - w, w:W - w]).max() < 1e-8 * np.abs(S).max()


def test_const_ratio_kernel_sum_is_constant_and_free_fit_is_not():
    H, W, L, DK, DB = 64, 72, 5, 2, 2
    d = small_pair(H, W, seed=91, n_src=25, mask_fraction=0.02, n_transients=1)
    cpr = O.fit_const_ratio(d["R"], d["S"], d["bad"], L, DK, DB)
    free = O.fit(d["R"], d["S"], d["bad"], L, DK, DB)
    sc = _kernel_sums(cpr["theta"], L, DK, DB, H, W, PTS)
    sf = _kernel_sums(free["theta"], L, DK, DB, H, W, PTS)
    assert np.ptp(sc) <= 1e-12 * abs(sc[0])
    n = (L * L - 1) * O.n_terms(DK)
    assert abs(sc[0] - cpr["theta_c"][n]) <= 1e-12 * abs(sc[0])
    assert np.ptp(sf) > 1e-6 * abs(sf[0])
    # the constraint costs fit quality, never gains it
    M = cpr["prep"]["M"]
    assert np.sum(cpr["D"][M] ** 2) >= np.sum(free["D"][M] ** 2)


def test_const_ratio_matches_lagrange_multipliers():
    """The constrained optimum from the KKT system of the free normal
    equations with the equality constraints sum_j theta[j, p] = 0 (p >= 1):
    an independent formulation of the same least-squares problem."""
    H, W, L, DK, DB = 60, 66, 5, 1, 2
    d = small_pair(H, W, seed=93, n_src=20, mask_fraction=0.03)
    free = O.fit(d["R"], d["S"], d["bad"], L, DK, DB)
    A, b = free["A"], free["b"]
    NK, N = O.n_terms(DK), A.shape[0]
    C = np.zeros((NK - 1, N))
    for p in range(1, NK):
        C[p - 1, [j * NK + p for j in range(L * L)]] = 1.0
    s = 1.0 / np.sqrt(np.diag(A))
    K = np.block([[A * s[:, None] * s[None, :], (C * s[None, :]).T], [C * s[None, :], np.zeros((NK - 1, NK - 1))]])
    sol = np.linalg.solve(K, np.concatenate([b * s, np.zeros(NK - 1)]))
    theta_kkt = sol[:N] * s
    cpr = O.fit_const_ratio(d["R"], d["S"], d["bad"], L, DK, DB)
    assert np.abs(cpr["theta"] - theta_kkt).max() <= 1e-7 * np.abs(theta_kkt).max()


def test_sky_dependence_below_kernel_degree():
    """D_B < D_K: with a constant kernel sum the fit is independent of the sky
    constants; with a free kernel sum it is not (the reading: the free fit is
    that of the sky-subtracted images)."""
    H, W, L, DK, DB = 56, 64, 5, 2, 0
    d = small_pair(H, W, seed=95, n_src=15)
    w = (L - 1) // 2
    inner = (slice(w, H - w), slice(w, W - w))
    sky0 = (float(np.median(d["R"])), float(np.median(d["S"])))
    sky1 = (sky0[0] + 40.0, sky0[1] - 15.0)
    a = O.fit_const_ratio(d["R"], d["S"], None, L, DK, DB, sky=sky0)
    b = O.fit_const_ratio(d["R"], d["S"], None, L, DK, DB, sky=sky1)
    assert np.abs(a["theta_orig"] - b["theta_orig"]).max() <= 1e-8 * np.abs(a["theta_orig"]).max()
    assert np.abs(a["D"][inner] - b["D"][inner]).max() <= 1e-8 * np.abs(d["S"]).max()
    fa = O.fit(d["R"], d["S"], None, L, DK, DB, sky=sky0)
    fb = O.fit(d["R"], d["S"], None, L, DK, DB, sky=sky1)
    assert np.abs(fa["D"][inner] - fb["D"][inner]).max() > 1e-6 * np.abs(d["S"]).max()


def test_const_ratio_refinement_is_a_no_op_in_fp64():
    H, W, L = 48, 52, 5
    d = small_pair(H, W, seed=97, n_src=10)
    a = O.fit_const_ratio(d["R"], d["S"], None, L, 1, 1)
    b = O.fit_const_ratio(d["R"], d["S"], None, L, 1, 1, refine_steps=1)
    assert np.abs(a["theta"] - b["theta"]).max() <= 1e-9 * np.abs(a["theta"]).max()

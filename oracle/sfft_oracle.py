"""FP64 CPU oracle for the SFFT-style difference-imaging hot path.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path imports, links or
executes this module: only the tests, the smoke check and the benchmark's
CPU-baseline leg do.  It shares no code with the CUDA path.

What it computes (the paper, Sec. 2.3.2 and Sec. 1, names the method but
does not print its equations; the model is the delta-basis, spatially
varying kernel fit it cites):

    S'(x) ~ sum_j K_j(x) R~(x - u_j) + B'(x),
    K_j(x) = sum_p theta[j, p] phi_p(x),   B'(x) = sum_q beta[q] psi_q(x),

with u_j the L x L pixel offsets (j = (u_y + w) L + (u_x + w), w = (L-1)/2),
phi_p / psi_q the monomials xt^a yt^b of total degree <= D_K / D_B in
normalised coordinates xt = 2x/(W-1) - 1, yt = 2y/(H-1) - 1, ordered by
total degree and, within a degree, by decreasing a.  theta is the
least-squares optimum over the fit mask M_fit:

    theta* = argmin sum_x M_fit(x) [S'(x) - Phi(x)^T theta]^2,
    A = sum_x M_fit Phi Phi^T,   b = sum_x M_fit Phi S'.

Readings where the paper is silent (all listed in the design notes):
  * convolution sign: (K (x) R)(x) = sum_u K_u(x) R(x - u), the kernel is
    evaluated at the output pixel;
  * bad = bad_in | ~finite(R) | ~finite(S); M_fit(x) = 1 iff x is at least w
    pixels from every edge and every pixel of the L x L footprint around x
    is good (an erosion of the good map);
  * R_m = good ? R - s_R : 0 (fit), R~ = finite(R) ? R - s_R : 0 (apply,
    zero outside the image), S' = S - s_S, s = median of the good pixels;
  * the background is reported in original units,
    B = B' + s_S - s_R sum_j K_j(x), keeping the terms psi_q can hold
    (all of them when D_B >= D_K or when the kernel sum is constant; with
    D_B < D_K and a varying kernel sum the fit is that of the sky-subtracted
    images and the higher terms of s_R sum_j K_j are dropped).

Constant photometric ratio (the constrained kernel of the delta-basis
literature the paper cites in Sec. 1): the kernel sum sum_j K_j(x) is one
constant a_0 over the chip.  Written in the basis
    K(x) = a_0 delta_0 + sum_{u != 0} sum_p c[u, p] phi_p(x) (delta_u - delta_0)
it has (L^2 - 1) N_K + 1 + N_B unknowns; fit_const_ratio solves the
least-squares problem in that basis directly from its design rows.

Two forms of the normal equations are provided:
  normal_definition  (O1) - A and b as the chunked sum of Phi Phi^T, the
                            definition itself (BLAS matmul per chunk);
  normal_fourier     (O2) - the method form: for every kernel-offset
                            difference d, the FFT cross-correlation of the
                            masked product R_m(z) R_m(z + d) with each weight
                            map M_fit xt^a yt^b, sampled at the lags u.
"""
from __future__ import annotations

import os

import numpy as np
import scipy.fft
import scipy.linalg

STATUS_OK = 0
STATUS_SINGULAR = 4
STATUS_NONFINITE = 5


# ---------------------------------------------------------------- basis
def monomials(D):
    """Monomial exponents (a, b) of xt^a yt^b with a + b <= D, ordered by total
    degree n = 0..D and, within a degree, by a descending from n to 0."""
    return [(a, n - a) for n in range(D + 1) for a in range(n, -1, -1)]


def n_terms(D):
    return (D + 1) * (D + 2) // 2


def offsets(L):
    """Kernel offsets u_j = (u_y, u_x), j = (u_y + w) L + (u_x + w)."""
    w = (L - 1) // 2
    return [(uy, ux) for uy in range(-w, w + 1) for ux in range(-w, w + 1)]


def n_unknowns(L, DK, DB):
    return L * L * n_terms(DK) + n_terms(DB)


def norm_coords(H, W):
    """xt[x] = 2x/(W-1) - 1 and yt[y] = 2y/(H-1) - 1 as 1-D float64 arrays."""
    xt = 2.0 * np.arange(W, dtype=np.float64) / max(W - 1, 1) - 1.0
    yt = 2.0 * np.arange(H, dtype=np.float64) / max(H - 1, 1) - 1.0
    return xt, yt


def monomial_map(H, W, a, b):
    xt, yt = norm_coords(H, W)
    return np.outer(yt ** b, xt ** a)


# ---------------------------------------------------------------- masks and offsets
def fit_mask(good, L):
    """M_fit: interior pixel whose whole L x L footprint is good."""
    H, W = good.shape
    w = (L - 1) // 2
    nbad = np.zeros((H + 1, W + 1), dtype=np.int64)
    nbad[1:, 1:] = np.cumsum(np.cumsum((~good).astype(np.int64), axis=0), axis=1)
    M = np.zeros((H, W), dtype=bool)
    if H < L or W < L:
        return M
    # window [y-w, y+w] x [x-w, x+w] for interior y, x
    y0, y1 = np.arange(0, H - 2 * w), np.arange(L, H + 1)
    x0, x1 = np.arange(0, W - 2 * w), np.arange(L, W + 1)
    cnt = (nbad[y1][:, x1] - nbad[y0][:, x1] - nbad[y1][:, x0] + nbad[y0][:, x0])
    M[w:H - w, w:W - w] = cnt == 0
    return M


def prepare(R, S, bad, L, sky=None):
    """Masks, sky offsets and offset images (the mask-and-offset step)."""
    R = np.asarray(R, dtype=np.float64)
    S = np.asarray(S, dtype=np.float64)
    H, W = R.shape
    badm = np.zeros((H, W), dtype=bool) if bad is None else (np.asarray(bad) != 0)
    finR, finS = np.isfinite(R), np.isfinite(S)
    badm = badm | ~finR | ~finS
    good = ~badm
    M = fit_mask(good, L)
    if sky is None:
        s_R = float(np.median(R[good])) if good.any() else 0.0
        s_S = float(np.median(S[good])) if good.any() else 0.0
    else:
        s_R, s_S = float(sky[0]), float(sky[1])
    R_m = np.where(good, R - s_R, 0.0)
    R_t = np.where(finR, R - s_R, 0.0)
    S_p = S - s_S
    return {"H": H, "W": W, "L": L, "good": good, "M": M, "s_R": s_R, "s_S": s_S,
            "R_m": R_m, "R_t": R_t, "S_p": S_p}


# ---------------------------------------------------------------- O1: definition
def _shifted(img, uy, ux):
    """img(y - uy, x - ux) with zeros outside the image."""
    H, W = img.shape
    out = np.zeros_like(img)
    ys0, ys1 = max(0, uy), min(H, H + uy)
    xs0, xs1 = max(0, ux), min(W, W + ux)
    out[ys0:ys1, xs0:xs1] = img[ys0 - uy:ys1 - uy, xs0 - ux:xs1 - ux]
    return out


def design_rows(prep, DK, DB, ys, xs, img=None):
    """Rows Phi(x)^T of the design matrix at pixels (ys, xs).  Columns are
    (j, p) -> j N_K + p for the kernel part, then N_B background terms."""
    L = prep["L"]
    H, W = prep["H"], prep["W"]
    img = prep["R_m"] if img is None else img
    xt, yt = norm_coords(H, W)
    xv, yv = xt[xs], yt[ys]
    mK, mB = monomials(DK), monomials(DB)
    NK = len(mK)
    phi = np.stack([xv ** a * yv ** b for (a, b) in mK], axis=1)
    psi = np.stack([xv ** a * yv ** b for (a, b) in mB], axis=1)
    X = np.empty((len(ys), L * L * NK + len(mB)), dtype=np.float64)
    for j, (uy, ux) in enumerate(offsets(L)):
        yy, xx = ys - uy, xs - ux
        inb = (yy >= 0) & (yy < H) & (xx >= 0) & (xx < W)
        r = np.zeros(len(ys))
        r[inb] = img[yy[inb], xx[inb]]
        X[:, j * NK:(j + 1) * NK] = phi * r[:, None]
    X[:, L * L * NK:] = psi
    return X


def normal_definition(prep, DK, DB, chunk_px=1 << 15):
    """O1: A = sum_x M Phi Phi^T and b = sum_x M Phi S' over chunks of fit
    pixels (the definition; one BLAS matmul per chunk)."""
    ys, xs = np.nonzero(prep["M"])
    N = n_unknowns(prep["L"], DK, DB)
    A = np.zeros((N, N))
    b = np.zeros(N)
    for s in range(0, len(ys), chunk_px):
        X = design_rows(prep, DK, DB, ys[s:s + chunk_px], xs[s:s + chunk_px])
        A += X.T @ X
        b += X.T @ prep["S_p"][ys[s:s + chunk_px], xs[s:s + chunk_px]]
    return A, b


# ---------------------------------------------------------------- O2: Fourier method
def half_plane_diffs(L):
    """Kernel-offset differences d = u - u' in the half plane d_y > 0 or
    (d_y == 0 and d_x >= 0); the rest follow by the symmetry of A."""
    return [(dy, dx) for dy in range(0, L) for dx in range(-(L - 1), L)
            if dy > 0 or dx >= 0]


def _xcorr_at(W_hat, P_hat, shape, lags):
    """sum_x w(x) p(x - u) for every u in lags, by FFT (circular)."""
    corr = scipy.fft.irfft2(np.conj(W_hat) * P_hat, s=shape, workers=_workers())
    H, W = shape
    return np.array([corr[(-uy) % H, (-ux) % W] for (uy, ux) in lags])


def _workers():
    return len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()


def normal_fourier(prep, DK, DB):
    """O2: the method form of the normal equations.

    KK block: for each d in the half plane and each weight monomial m,
      g_{d,m}(u) = sum_x M xt^a yt^b (x) P_d(x - u),  P_d(z) = R_m(z) R_m(z + d),
    computed as an FFT cross-correlation and sampled at the lags u with
    both u and u - d in the window; then
      A[(j,p),(j',p')] = g_{u_j - u_j', phi_p phi_p'}(u_j)  and its mirror.
    KB block and b_K: the same correlation with R_m itself in place of P_d,
    against the weights M phi_p psi_q and M phi_p S'.
    BB block and b_B: direct moments of M psi psi' and M psi S'.
    Circular indexing is exact because M_fit vanishes within w of every edge.
    """
    L, H, W = prep["L"], prep["H"], prep["W"]
    shape = (H, W)
    M = prep["M"].astype(np.float64)
    R_m, S_p = prep["R_m"], prep["S_p"]
    mK, mB = monomials(DK), monomials(DB)
    NK, NB = len(mK), len(mB)
    offs = offsets(L)
    jidx = {u: j for j, u in enumerate(offs)}
    w = (L - 1) // 2
    NKK = L * L * NK
    N = NKK + NB
    A = np.zeros((N, N))
    b = np.zeros(N)
    wk = _workers()

    def rf(x):
        return scipy.fft.rfft2(x, workers=wk)

    # weight spectra for every product phi_p phi_p' (KK) and phi_p psi_q (KB)
    need = {}
    for p, (a1, b1) in enumerate(mK):
        for p2, (a2, b2) in enumerate(mK):
            need.setdefault((a1 + a2, b1 + b2), None)
        for q, (a2, b2) in enumerate(mB):
            need.setdefault((a1 + a2, b1 + b2), None)
    What = {m: rf(M * monomial_map(H, W, *m)) for m in need}

    # KK block
    for (dy, dx) in half_plane_diffs(L):
        P = R_m * np.roll(R_m, (-dy, -dx), axis=(0, 1))
        P_hat = rf(P)
        lags = [(uy, ux) for (uy, ux) in offs
                if abs(uy - dy) <= w and abs(ux - dx) <= w]
        gm = {}
        for p, (a1, b1) in enumerate(mK):
            for p2, (a2, b2) in enumerate(mK):
                m = (a1 + a2, b1 + b2)
                if m not in gm:
                    gm[m] = _xcorr_at(What[m], P_hat, shape, lags)
                for li, u in enumerate(lags):
                    j = jidx[u]
                    j2 = jidx[(u[0] - dy, u[1] - dx)]
                    A[j * NK + p, j2 * NK + p2] = gm[m][li]
                    A[j2 * NK + p2, j * NK + p] = gm[m][li]

    # KB block and b_K
    R_hat = rf(R_m)
    for p, (a1, b1) in enumerate(mK):
        for q, (a2, b2) in enumerate(mB):
            g = _xcorr_at(What[(a1 + a2, b1 + b2)], R_hat, shape, offs)
            for j in range(L * L):
                A[j * NK + p, NKK + q] = g[j]
                A[NKK + q, j * NK + p] = g[j]
        V_hat = rf(M * monomial_map(H, W, a1, b1) * S_p)
        g = _xcorr_at(V_hat, R_hat, shape, offs)
        for j in range(L * L):
            b[j * NK + p] = g[j]

    # BB block and b_B (moments)
    for q, (a1, b1) in enumerate(mB):
        for q2, (a2, b2) in enumerate(mB):
            A[NKK + q, NKK + q2] = np.sum(M * monomial_map(H, W, a1 + a2, b1 + b2))
        b[NKK + q] = np.sum(M * monomial_map(H, W, a1, b1) * S_p)
    return A, b


# ---------------------------------------------------------------- solve
def solve(A, b):
    """Jacobi-equilibrated Cholesky solve.  Returns (theta, status).  A matrix
    that is not symmetric positive definite is reported as singular; no
    regularisation is applied."""
    A = np.asarray(A, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    if not (np.all(np.isfinite(A)) and np.all(np.isfinite(b))):
        return np.full(b.shape, np.nan), STATUS_NONFINITE
    d = np.diag(A)
    if np.any(d <= 0):
        return np.full(b.shape, np.nan), STATUS_SINGULAR
    s = 1.0 / np.sqrt(d)
    As = A * s[:, None] * s[None, :]
    try:
        c = scipy.linalg.cho_factor(As, lower=True, check_finite=False)
    except np.linalg.LinAlgError:
        return np.full(b.shape, np.nan), STATUS_SINGULAR
    y = scipy.linalg.cho_solve(c, b * s, check_finite=False)
    return s * y, STATUS_OK


def residual_rhs(prep, DK, DB, theta, chunk_px=1 << 15):
    """r = sum_x M Phi (S' - Phi^T theta): the normal-equation residual
    computed in image space (used by one step of iterative refinement)."""
    ys, xs = np.nonzero(prep["M"])
    N = n_unknowns(prep["L"], DK, DB)
    r = np.zeros(N)
    for s in range(0, len(ys), chunk_px):
        X = design_rows(prep, DK, DB, ys[s:s + chunk_px], xs[s:s + chunk_px])
        e = prep["S_p"][ys[s:s + chunk_px], xs[s:s + chunk_px]] - X @ theta
        r += X.T @ e
    return r


def refine(prep, DK, DB, A, theta):
    """One step of iterative refinement: theta + A^-1 (b - A theta), with the
    residual formed in image space."""
    r = residual_rhs(prep, DK, DB, theta)
    delta, st = solve(A, r)
    return theta + delta, st


# ---------------------------------------------------------------- theta layout / units
def split_theta(theta, L, DK, DB):
    NK = n_terms(DK)
    c = np.asarray(theta[:L * L * NK]).reshape(L * L, NK)
    return c, np.asarray(theta[L * L * NK:])


def background_to_original(theta_off, L, DK, DB, s_R, s_S):
    """theta with the background in original units:
    beta_q + s_S [q == 0] - s_R sum_j theta[j, q] for q < min(N_K, N_B)
    (psi_q = phi_q there); the terms of degree above D_B are dropped."""
    th = np.array(theta_off, dtype=np.float64)
    c, beta = split_theta(th, L, DK, DB)
    beta = beta.copy()
    m = min(n_terms(DK), n_terms(DB))
    beta[0] += s_S
    beta[:m] -= s_R * c.sum(axis=0)[:m]
    th[L * L * n_terms(DK):] = beta
    return th


def background_to_offset(theta_orig, L, DK, DB, s_R, s_S):
    th = np.array(theta_orig, dtype=np.float64)
    c, beta = split_theta(th, L, DK, DB)
    beta = beta.copy()
    m = min(n_terms(DK), n_terms(DB))
    beta[0] -= s_S
    beta[:m] += s_R * c.sum(axis=0)[:m]
    th[L * L * n_terms(DK):] = beta
    return th


def kernel_at(theta, L, DK, DB, H, W, x, y):
    """K_u(x, y) as an L x L array (row index u_y + w, column u_x + w)."""
    c, _ = split_theta(theta, L, DK, DB)
    xt = 2.0 * x / max(W - 1, 1) - 1.0
    yt = 2.0 * y / max(H - 1, 1) - 1.0
    phi = np.array([xt ** a * yt ** b for (a, b) in monomials(DK)])
    return (c @ phi).reshape(L, L)


# ---------------------------------------------------------------- apply
def apply(prep, theta_off, DK, DB):
    """D = S' - sum_p phi_p sum_j theta[j,p] R~(x - u_j) - B'(x), FP64, with
    R~ = finite(R) ? R - s_R : 0 and zero outside the image."""
    L, H, W = prep["L"], prep["H"], prep["W"]
    c, beta = split_theta(theta_off, L, DK, DB)
    mK, mB = monomials(DK), monomials(DB)
    D = prep["S_p"].copy()
    for j, (uy, ux) in enumerate(offsets(L)):
        sh = _shifted(prep["R_t"], uy, ux)
        for p, (a, b) in enumerate(mK):
            if c[j, p] != 0.0:
                D -= c[j, p] * monomial_map(H, W, a, b) * sh
    for q, (a, b) in enumerate(mB):
        D -= beta[q] * monomial_map(H, W, a, b)
    return D


# ---------------------------------------------------------------- full fit
def fit(R, S, bad, L, DK, DB, sky=None, form="definition", refine_steps=0):
    """Prepare, assemble, solve (+ optional refinement) and apply.  Returns a
    dict with A, b, theta (offset units), theta_orig, D, status, prep."""
    prep = prepare(R, S, bad, L, sky)
    if form == "definition":
        A, b = normal_definition(prep, DK, DB)
    else:
        A, b = normal_fourier(prep, DK, DB)
    theta, st = solve(A, b)
    for _ in range(refine_steps):
        if st != STATUS_OK:
            break
        theta, st = refine(prep, DK, DB, A, theta)
    out = {"A": A, "b": b, "theta": theta, "status": st, "prep": prep}
    if st == STATUS_OK:
        out["theta_orig"] = background_to_original(theta, L, DK, DB, prep["s_R"], prep["s_S"])
        out["D"] = apply(prep, theta, DK, DB)
    return out


# ---------------------------------------------------------------- constant photometric ratio
def center_index(L):
    """Index j of the zero offset u = (0, 0)."""
    return (L * L - 1) // 2


def n_unknowns_const_ratio(L, DK, DB):
    return (L * L - 1) * n_terms(DK) + 1 + n_terms(DB)


def const_ratio_design_rows(prep, DK, DB, ys, xs):
    """Design rows in the constant-ratio basis at pixels (ys, xs): for each
    offset u_j != 0 (j ascending) and p, phi_p(x) [R_m(x - u_j) - R_m(x)];
    then R_m(x) (the coefficient a_0 of delta_0); then psi_q(x)."""
    L, H, W = prep["L"], prep["H"], prep["W"]
    img = prep["R_m"]
    xt, yt = norm_coords(H, W)
    xv, yv = xt[xs], yt[ys]
    mK, mB = monomials(DK), monomials(DB)
    NK = len(mK)
    phi = np.stack([xv ** a * yv ** b for (a, b) in mK], axis=1)
    psi = np.stack([xv ** a * yv ** b for (a, b) in mB], axis=1)
    r0 = img[ys, xs]
    X = np.empty((len(ys), n_unknowns_const_ratio(L, DK, DB)), dtype=np.float64)
    col = 0
    for j, (uy, ux) in enumerate(offsets(L)):
        if j == center_index(L):
            continue
        yy, xx = ys - uy, xs - ux
        inb = (yy >= 0) & (yy < H) & (xx >= 0) & (xx < W)
        r = np.zeros(len(ys))
        r[inb] = img[yy[inb], xx[inb]]
        X[:, col:col + NK] = phi * (r - r0)[:, None]
        col += NK
    X[:, col] = r0
    X[:, col + 1:] = psi
    return X


def normal_const_ratio(prep, DK, DB, chunk_px=1 << 15):
    """A_c = sum_x M X_c X_c^T and b_c = sum_x M X_c S' in the constant-ratio
    basis (the definition, chunked over fit pixels)."""
    ys, xs = np.nonzero(prep["M"])
    N = n_unknowns_const_ratio(prep["L"], DK, DB)
    A = np.zeros((N, N))
    b = np.zeros(N)
    for s in range(0, len(ys), chunk_px):
        X = const_ratio_design_rows(prep, DK, DB, ys[s:s + chunk_px], xs[s:s + chunk_px])
        A += X.T @ X
        b += X.T @ prep["S_p"][ys[s:s + chunk_px], xs[s:s + chunk_px]]
    return A, b


def const_ratio_to_full(theta_c, L, DK, DB):
    """Coefficients of the constant-ratio basis -> the full layout theta[j, p]:
    c[u, p] at u != 0, and at u = 0 the constant a_0 minus sum_{u != 0} c[u, p]."""
    NK = n_terms(DK)
    n = (L * L - 1) * NK
    c = np.asarray(theta_c[:n]).reshape(L * L - 1, NK)
    full = np.zeros((L * L, NK))
    jc = center_index(L)
    full[[j for j in range(L * L) if j != jc]] = c
    full[jc] = -c.sum(axis=0)
    full[jc, 0] += theta_c[n]
    return np.concatenate([full.ravel(), np.asarray(theta_c[n + 1:])])


def residual_rhs_const_ratio(prep, DK, DB, theta_c, chunk_px=1 << 15):
    ys, xs = np.nonzero(prep["M"])
    r = np.zeros(n_unknowns_const_ratio(prep["L"], DK, DB))
    for s in range(0, len(ys), chunk_px):
        X = const_ratio_design_rows(prep, DK, DB, ys[s:s + chunk_px], xs[s:s + chunk_px])
        r += X.T @ (prep["S_p"][ys[s:s + chunk_px], xs[s:s + chunk_px]] - X @ theta_c)
    return r


def fit_const_ratio(R, S, bad, L, DK, DB, sky=None, refine_steps=0):
    """The constant-photometric-ratio fit: assemble and solve in the
    constrained basis, map to the full layout, apply.  Returns a dict with
    A_c, b_c, theta_c, theta (offset units, full layout), theta_orig, D,
    status, prep."""
    prep = prepare(R, S, bad, L, sky)
    A, b = normal_const_ratio(prep, DK, DB)
    th, st = solve(A, b)
    for _ in range(refine_steps):
        if st != STATUS_OK:
            break
        delta, st = solve(A, residual_rhs_const_ratio(prep, DK, DB, th))
        th = th + delta
    out = {"A_c": A, "b_c": b, "theta_c": th, "status": st, "prep": prep}
    if st == STATUS_OK:
        theta = const_ratio_to_full(th, L, DK, DB)
        out["theta"] = theta
        out["theta_orig"] = background_to_original(theta, L, DK, DB, prep["s_R"], prep["s_S"])
        out["D"] = apply(prep, theta, DK, DB)
    return out


# ---------------------------------------------------------------- error metrics
def kernel_coef_rel_err(theta_a, theta_b, L, DK, DB):
    """||c_a - c_b||_inf / ||c_b||_inf over the L^2 N_K kernel coefficients."""
    ca, _ = split_theta(theta_a, L, DK, DB)
    cb, _ = split_theta(theta_b, L, DK, DB)
    return float(np.max(np.abs(ca - cb)) / np.max(np.abs(cb)))


def box_flux(D, x, y, half):
    """Sum of D over the (2 half + 1)^2 box centred on the pixel nearest (x, y)."""
    xi, yi = int(round(x)), int(round(y))
    return float(np.sum(D[yi - half:yi + half + 1, xi - half:xi + half + 1], dtype=np.float64))

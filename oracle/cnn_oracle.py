"""FP64 CPU oracle for the stamp real-bogus classifier.

TEST INFRASTRUCTURE ONLY: used by the tests, the smoke check and the
benchmark's CPU-baseline leg; the product path never imports it.

The paper (Sec. 2.3.4) scores each detection on the difference image with a
CNN that takes a three-channel stamp (science, template, difference) centred
on the candidate and returns a score in [0, 1]; it gives no layer sizes for
the small network built here, which follows the project's stated design:

  normalise   per channel c: (x - median_c) / (1.4826 MAD_c), clipped to +-64
              (MAD_c <= 0 -> scale 1)
  conv1       3 -> 32, 3 x 3, zero 'same' padding, + bias, ReLU, max-pool 2 (31 -> 15)
  conv2       32 -> 64, same, ReLU, pool (15 -> 7)
  conv3       64 -> 64, same, ReLU, pool (7 -> 3)
  fc1         576 -> 128 (flatten order channel, row, column), ReLU
  fc2         128 -> 1 logit z, score = sigmoid(z)
  loss        binary cross-entropy on the logit, mean over the batch
  optimiser   Adam (beta1 0.9, beta2 0.999, eps 1e-8) on FP32-style master weights

Max-pool is 2 x 2 with stride 2 over the top-left even part (floor); its
gradient goes to the first maximum in the order (0,0), (0,1), (1,0), (1,1).

The paper's own architecture (a rotation-invariant network with residual
connections) is the second model below (forward_ri, loss_and_grads_ri).
"""
from __future__ import annotations

import numpy as np

STAMP = 31
SHAPES = {
    "w1": (32, 3, 3, 3), "b1": (32,),
    "w2": (64, 32, 3, 3), "b2": (64,),
    "w3": (64, 64, 3, 3), "b3": (64,),
    "w4": (128, 576), "b4": (128,),
    "w5": (1, 128), "b5": (1,),
}
ORDER = ["w1", "b1", "w2", "b2", "w3", "b3", "w4", "b4", "w5", "b5"]


def n_params():
    return int(sum(np.prod(SHAPES[k]) for k in ORDER))


def unflatten(vec):
    out, o = {}, 0
    for k in ORDER:
        n = int(np.prod(SHAPES[k]))
        out[k] = np.asarray(vec[o:o + n], dtype=np.float64).reshape(SHAPES[k])
        o += n
    return out


def flatten(params):
    return np.concatenate([np.asarray(params[k], dtype=np.float64).ravel() for k in ORDER])


def init_params(seed):
    """Uniform He-style initialisation, U(-sqrt(6/fan_in), sqrt(6/fan_in)), zero biases."""
    rng = np.random.default_rng(seed)
    p = {}
    for k in ORDER:
        shp = SHAPES[k]
        if k.startswith("b"):
            p[k] = np.zeros(shp)
        else:
            fan_in = int(np.prod(shp[1:]))
            lim = np.sqrt(6.0 / fan_in)
            p[k] = rng.uniform(-lim, lim, shp)
    return p


def normalise(stamps):
    """Per-stamp, per-channel robust standardisation, clipped to +-64."""
    x = np.asarray(stamps, dtype=np.float64)
    n = x.shape[0]
    flat = x.reshape(n, 3, -1)
    med = np.median(flat, axis=2, keepdims=True)
    mad = np.median(np.abs(flat - med), axis=2, keepdims=True)
    scale = 1.4826 * mad
    scale = np.where(scale > 0, scale, 1.0)
    return np.clip((flat - med) / scale, -64.0, 64.0).reshape(x.shape)


def conv_same(x, w, b):
    """x [n][cin][h][w], w [cout][cin][3][3]: y = b + sum w * x(i + ky - 1, j + kx - 1), zero outside."""
    n, cin, h, wd = x.shape
    xp = np.zeros((n, cin, h + 2, wd + 2))
    xp[:, :, 1:-1, 1:-1] = x
    y = np.zeros((n, w.shape[0], h, wd)) + b[None, :, None, None]
    for ky in range(3):
        for kx in range(3):
            patch = xp[:, :, ky:ky + h, kx:kx + wd]
            y += np.einsum("ncij,oc->noij", patch, w[:, :, ky, kx])
    return y


def conv_same_backward(x, w, dy):
    """Gradients of conv_same with respect to x, w and b."""
    n, cin, h, wd = x.shape
    xp = np.zeros((n, cin, h + 2, wd + 2))
    xp[:, :, 1:-1, 1:-1] = x
    dw = np.zeros_like(w)
    dxp = np.zeros_like(xp)
    for ky in range(3):
        for kx in range(3):
            patch = xp[:, :, ky:ky + h, kx:kx + wd]
            dw[:, :, ky, kx] = np.einsum("noij,ncij->oc", dy, patch)
            dxp[:, :, ky:ky + h, kx:kx + wd] += np.einsum("noij,oc->ncij", dy, w[:, :, ky, kx])
    db = dy.sum(axis=(0, 2, 3))
    return dxp[:, :, 1:-1, 1:-1], dw, db


def maxpool2(x):
    n, c, h, wd = x.shape
    ho, wo = h // 2, wd // 2
    v = x[:, :, :2 * ho, :2 * wo].reshape(n, c, ho, 2, wo, 2).transpose(0, 1, 2, 4, 3, 5).reshape(n, c, ho, wo, 4)
    idx = np.argmax(v, axis=-1)   # first maximum in (0,0), (0,1), (1,0), (1,1)
    return np.take_along_axis(v, idx[..., None], axis=-1)[..., 0], idx


def maxpool2_backward(dy, idx, shape):
    n, c, h, wd = shape
    ho, wo = dy.shape[2], dy.shape[3]
    dv = np.zeros((n, c, ho, wo, 4))
    np.put_along_axis(dv, idx[..., None], dy[..., None], axis=-1)
    dx = np.zeros(shape)
    dx[:, :, :2 * ho, :2 * wo] = dv.reshape(n, c, ho, wo, 2, 2).transpose(0, 1, 2, 4, 3, 5).reshape(n, c, 2 * ho, 2 * wo)
    return dx


def forward(params, xn, keep=False):
    """Logits for normalised stamps xn [n][3][31][31]."""
    cache = {}
    a = xn
    for li, (wk, bk) in enumerate([("w1", "b1"), ("w2", "b2"), ("w3", "b3")]):
        z = conv_same(a, params[wk], params[bk])
        r = np.maximum(z, 0.0)
        p, idx = maxpool2(r)
        cache[li] = (a, z, idx, r.shape)
        a = p
    flat = a.reshape(a.shape[0], -1)
    z4 = flat @ params["w4"].T + params["b4"]
    h4 = np.maximum(z4, 0.0)
    z5 = h4 @ params["w5"].T + params["b5"]
    logit = z5[:, 0]
    if keep:
        cache["flat"], cache["z4"], cache["h4"], cache["pool_shape"] = flat, z4, h4, a.shape
        return logit, cache
    return logit


def bce_loss(logit, target):
    t = np.asarray(target, dtype=np.float64)
    return float(np.mean(np.maximum(logit, 0) - logit * t + np.log1p(np.exp(-np.abs(logit)))))


def sigmoid(z):
    return 0.5 * (1.0 + np.tanh(0.5 * z))


def loss_and_grads(params, xn, target):
    logit, c = forward(params, xn, keep=True)
    n = logit.shape[0]
    loss = bce_loss(logit, target)
    dz5 = ((sigmoid(logit) - np.asarray(target, dtype=np.float64)) / n)[:, None]
    g = {}
    g["w5"] = dz5.T @ c["h4"]
    g["b5"] = dz5.sum(axis=0)
    dh4 = dz5 @ params["w5"]
    dz4 = dh4 * (c["z4"] > 0)
    g["w4"] = dz4.T @ c["flat"]
    g["b4"] = dz4.sum(axis=0)
    da = (dz4 @ params["w4"]).reshape(c["pool_shape"])
    for li, (wk, bk) in reversed(list(enumerate([("w1", "b1"), ("w2", "b2"), ("w3", "b3")]))):
        a_in, z, idx, rshape = c[li]
        dr = maxpool2_backward(da, idx, rshape)
        dz = dr * (z > 0)
        dx, dw, db = conv_same_backward(a_in, params[wk], dz)
        g[wk], g[bk] = dw, db
        da = dx
    return loss, g


def score(params, stamps):
    return sigmoid(forward(params, normalise(stamps)))


class Adam:
    def __init__(self, params, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
        self.lr, self.b1, self.b2, self.eps = lr, b1, b2, eps
        self.m = {k: np.zeros_like(v) for k, v in params.items()}
        self.v = {k: np.zeros_like(v) for k, v in params.items()}
        self.t = 0

    def step(self, params, grads):
        self.t += 1
        for k in params:
            self.m[k] = self.b1 * self.m[k] + (1 - self.b1) * grads[k]
            self.v[k] = self.b2 * self.v[k] + (1 - self.b2) * grads[k] ** 2
            mh = self.m[k] / (1 - self.b1 ** self.t)
            vh = self.v[k] / (1 - self.b2 ** self.t)
            params[k] = params[k] - self.lr * mh / (np.sqrt(vh) + self.eps)
        return params


# ---------------------------------------------------------------- fallback cuts
def shape_cuts(dstamp, snr, fwhm_psf, snr_min=5.0):
    """Plain SNR and shape cuts on a difference-image stamp (31 x 31, candidate
    at the centre): SNR >= snr_min; second-moment FWHM within [0.5, 2.0] of the
    PSF FWHM; negative-flux fraction of the central 7 x 7 below 0.3; axis ratio
    below 2.5.  Moments use the positive pixels of the central 9 x 9."""
    c = STAMP // 2
    box = np.asarray(dstamp, dtype=np.float64)[c - 4:c + 5, c - 4:c + 5]
    pos = np.maximum(box, 0.0)
    tot = pos.sum()
    if snr < snr_min or tot <= 0:
        return False
    yy, xx = np.mgrid[-4:5, -4:5]
    mx, my = (pos * xx).sum() / tot, (pos * yy).sum() / tot
    sxx = (pos * (xx - mx) ** 2).sum() / tot
    syy = (pos * (yy - my) ** 2).sum() / tot
    sxy = (pos * (xx - mx) * (yy - my)).sum() / tot
    tr, det = sxx + syy, sxx * syy - sxy ** 2
    disc = np.sqrt(max(tr * tr / 4 - det, 0.0))
    l1, l2 = tr / 2 + disc, max(tr / 2 - disc, 1e-12)
    fwhm = 2.3548200450309493 * np.sqrt(max(0.5 * (l1 + l2), 0.0))
    inner = np.asarray(dstamp, dtype=np.float64)[c - 3:c + 4, c - 3:c + 4]
    neg_frac = np.abs(np.minimum(inner, 0)).sum() / max(np.abs(inner).sum(), 1e-12)
    ratio = np.sqrt(l1 / l2)
    return (0.5 * fwhm_psf <= fwhm <= 2.0 * fwhm_psf) and neg_frac < 0.3 and ratio < 2.5


ADAPTIVE_HALF = 7        # adaptive moments over the central 15 x 15
ADAPTIVE_ITERS = 40


def adaptive_moments(img, sigma0):
    """Gaussian-weighted adaptive second moments of a stamp centred on the
    candidate (the centre pixel is (0, 0)): starting from a round weight of
    width sigma0 at the centre, repeat ADAPTIVE_ITERS times
        w(r)  = exp(-(r - mu)^T M^-1 (r - mu) / 2)
        mu'   = sum w I r / sum w I
        M'    = 2 sum w I (r - mu')(r - mu')^T / sum w I
    For a Gaussian profile of covariance C the weighted profile has covariance
    (C^-1 + M^-1)^-1, so M = C is the fixed point: the weight follows the
    source's own size and shape, and noise far from the source gets no
    weight.  Returns (M as (mxx, myy, mxy), mu) or None when the weighted flux
    is not positive, M is not positive definite, the centroid moves more than
    3 px or M grows beyond 25 px^2."""
    h = ADAPTIVE_HALF
    c = np.asarray(img).shape[-1] // 2
    box = np.asarray(img, dtype=np.float64)[c - h:c + h + 1, c - h:c + h + 1]
    yy, xx = np.mgrid[-h:h + 1, -h:h + 1].astype(np.float64)
    mxx, myy, mxy, mx, my = sigma0 ** 2, sigma0 ** 2, 0.0, 0.0, 0.0
    for _ in range(ADAPTIVE_ITERS):
        det = mxx * myy - mxy * mxy
        if not (det > 0 and mxx > 0 and myy > 0):
            return None
        dx, dy = xx - mx, yy - my
        q = (myy * dx * dx - 2.0 * mxy * dx * dy + mxx * dy * dy) / det
        wi = np.exp(-0.5 * q) * box
        s0 = wi.sum()
        if not s0 > 0:
            return None
        mx, my = (wi * xx).sum() / s0, (wi * yy).sum() / s0
        dx, dy = xx - mx, yy - my
        mxx = 2.0 * (wi * dx * dx).sum() / s0
        myy = 2.0 * (wi * dy * dy).sum() / s0
        mxy = 2.0 * (wi * dx * dy).sum() / s0
        if abs(mx) > 3.0 or abs(my) > 3.0 or mxx > 25.0 or myy > 25.0:
            return None
    if not (mxx * myy - mxy * mxy > 0 and mxx > 0 and myy > 0):
        return None
    return (mxx, myy, mxy), (mx, my)


def shape_cuts_adaptive(dstamp, snr, fwhm_psf, snr_min=5.0):
    """The shape cuts with the size and axis ratio from Gaussian-weighted
    adaptive moments (adaptive_moments, starting at the PSF width) instead of
    the plain moments of the positive 9 x 9: SNR >= snr_min; FWHM =
    2 sqrt(2 ln 2) sqrt((l1 + l2) / 2) within [0.5, 2.0] of the PSF FWHM;
    negative-flux fraction of the central 7 x 7 below 0.3; axis ratio
    sqrt(l1 / l2) below 2.5 (l1 >= l2 the eigenvalues of M)."""
    if snr < snr_min:
        return False
    res = adaptive_moments(dstamp, fwhm_psf / 2.3548200450309493)
    if res is None:
        return False
    (mxx, myy, mxy), _ = res
    tr, det = mxx + myy, mxx * myy - mxy * mxy
    disc = np.sqrt(max(tr * tr / 4 - det, 0.0))
    l1, l2 = tr / 2 + disc, max(tr / 2 - disc, 1e-12)
    fwhm = 2.3548200450309493 * np.sqrt(0.5 * (l1 + l2))
    c = STAMP // 2
    inner = np.asarray(dstamp, dtype=np.float64)[c - 3:c + 4, c - 3:c + 4]
    neg_frac = np.abs(np.minimum(inner, 0)).sum() / max(np.abs(inner).sum(), 1e-12)
    ratio = np.sqrt(l1 / l2)
    return (0.5 * fwhm_psf <= fwhm <= 2.0 * fwhm_psf) and neg_frac < 0.3 and ratio < 2.5


# ---------------------------------------------------------------- rotation-invariant residual network
# The paper's classifier (Sec. 2.3.4) is a rotation-invariant CNN in the
# framework of its cited DeepHiTS work with residual connections in the style
# of ResNet-18; no layer sizes are given.  Reading implemented here: the
# normalised stamp is presented in its four rotations by multiples of 90
# degrees to one shared convolutional stack, and the four flattened feature
# vectors are averaged (exact invariance under those rotations) before the
# dense head:
#   conv1  3 -> 32, ReLU, pool (31 -> 15)
#   res1   relu(p1 + conv_b(relu(conv_a(p1))))           32 -> 32, 15 x 15
#   conv2  32 -> 64, ReLU, pool (15 -> 7)
#   res2   relu(p2 + conv_d(relu(conv_c(p2))))           64 -> 64, 7 x 7, then pool (7 -> 3)
#   mean over the four rotations of the 576 features, fc1 576 -> 128 ReLU, fc2 128 -> 1
SHAPES_RI = {
    "w1": (32, 3, 3, 3), "b1": (32,),
    "wa": (32, 32, 3, 3), "ba": (32,), "wb": (32, 32, 3, 3), "bb": (32,),
    "w2": (64, 32, 3, 3), "b2": (64,),
    "wc": (64, 64, 3, 3), "bc": (64,), "wd": (64, 64, 3, 3), "bd": (64,),
    "w4": (128, 576), "b4": (128,),
    "w5": (1, 128), "b5": (1,),
}
ORDER_RI = ["w1", "b1", "wa", "ba", "wb", "bb", "w2", "b2", "wc", "bc", "wd", "bd", "w4", "b4", "w5", "b5"]


# ---------------------------------------------------------------- the network with BF16 operands
# The GPU kernels compute the same network with every matrix-product operand
# in BF16 (the normalised input, the weights of the convolutions and of fc1,
# every pooled activation, and in the backward pass every back-propagated
# signal dz) and FP32 sums; fc2 and the biases stay FP32.  The functions below
# are that network with exact sums (modelled in FP64): the reference for how
# much of a kernel's departure from the FP64 network is the operands' rounding.

def round_bf16(x):
    """Round to the nearest BF16 value, ties to even.  BF16 keeps the sign,
    the 8 exponent bits and the top 7 of the 23 fraction bits of an IEEE
    single, so the value is first rounded to FP32 and then to 8 significant
    bits: add half a unit of the 16 dropped bits (minus one when the kept
    part is even, so that an exact half goes to the even neighbour) and clear
    them.  Finite inputs only."""
    u = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    keep_odd = (u >> 16) & 1
    u = ((u + 0x7FFF + keep_odd) >> 16) << 16
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def forward_bf16(params, xn):
    """Logits of the network with the kernels' BF16 operands (see above)."""
    a = round_bf16(xn)
    for wk, bk in (("w1", "b1"), ("w2", "b2"), ("w3", "b3")):
        z = conv_same(a, round_bf16(params[wk]), params[bk])
        a = round_bf16(maxpool2(np.maximum(z, 0.0))[0])
    h4 = np.maximum(a.reshape(a.shape[0], -1) @ round_bf16(params["w4"]).T + params["b4"], 0.0)
    return (h4 @ params["w5"].T + params["b5"])[:, 0]


def loss_and_grads_bf16(params, xn, target):
    """BCE loss and parameter gradients of the network with the kernels' BF16
    operands: the forward of forward_bf16, then the backward of
    loss_and_grads with each back-propagated signal dz (fc1's, and each
    convolution's after its ReLU and pool) rounded to BF16 before it enters a
    matrix product."""
    n = xn.shape[0]
    a = round_bf16(xn)
    cache = []
    for wk, bk in (("w1", "b1"), ("w2", "b2"), ("w3", "b3")):
        wb = round_bf16(params[wk])
        z = conv_same(a, wb, params[bk])
        r = np.maximum(z, 0.0)
        pooled, idx = maxpool2(r)
        cache.append((a, wb, z, idx, r.shape))
        a = round_bf16(pooled)
    flat = a.reshape(n, -1)
    w4b = round_bf16(params["w4"])
    z4 = flat @ w4b.T + params["b4"]
    h4 = np.maximum(z4, 0.0)
    logit = (h4 @ params["w5"].T + params["b5"])[:, 0]
    loss = bce_loss(logit, target)
    dz5 = (sigmoid(logit) - target) / n
    g = {"w5": (dz5[:, None] * h4).sum(0)[None, :], "b5": np.array([dz5.sum()])}
    dz4 = round_bf16(dz5[:, None] * params["w5"] * (z4 > 0))
    g["w4"], g["b4"] = dz4.T @ flat, dz4.sum(0)
    da = (dz4 @ w4b).reshape(a.shape)
    for li, (wk, bk) in reversed(list(enumerate((("w1", "b1"), ("w2", "b2"), ("w3", "b3"))))):
        a_in, wb, z, idx, rshape = cache[li]
        dz = round_bf16(maxpool2_backward(da, idx, rshape) * (z > 0))
        da, g[wk], g[bk] = conv_same_backward(a_in, wb, dz)
    return loss, g


def n_params_ri():
    return int(sum(np.prod(SHAPES_RI[k]) for k in ORDER_RI))


def unflatten_ri(vec):
    out, o = {}, 0
    for k in ORDER_RI:
        n = int(np.prod(SHAPES_RI[k]))
        out[k] = np.asarray(vec[o:o + n], dtype=np.float64).reshape(SHAPES_RI[k])
        o += n
    return out


def flatten_ri(params):
    return np.concatenate([np.asarray(params[k], dtype=np.float64).ravel() for k in ORDER_RI])


def init_params_ri(seed):
    rng = np.random.default_rng(seed)
    p = {}
    for k in ORDER_RI:
        shp = SHAPES_RI[k]
        if k.startswith("b"):
            p[k] = np.zeros(shp)
        else:
            lim = np.sqrt(6.0 / int(np.prod(shp[1:])))
            p[k] = rng.uniform(-lim, lim, shp)
    return p


def rotations(xn):
    """The four rotations by r x 90 degrees (counterclockwise, as np.rot90 over
    rows and columns), stacked rotation-major: [4 n][3][31][31]."""
    return np.concatenate([np.rot90(xn, r, axes=(2, 3)) for r in range(4)], axis=0)


def forward_ri(params, xn, keep=False):
    """Logits of the rotation-invariant residual network for normalised stamps."""
    n = xn.shape[0]
    x = rotations(np.asarray(xn, dtype=np.float64))
    z1 = conv_same(x, params["w1"], params["b1"])
    p1, i1 = maxpool2(np.maximum(z1, 0.0))
    za = conv_same(p1, params["wa"], params["ba"])
    ra = np.maximum(za, 0.0)
    zb = conv_same(ra, params["wb"], params["bb"]) + p1
    r1 = np.maximum(zb, 0.0)
    z2 = conv_same(r1, params["w2"], params["b2"])
    p2, i2 = maxpool2(np.maximum(z2, 0.0))
    zc = conv_same(p2, params["wc"], params["bc"])
    rc = np.maximum(zc, 0.0)
    zd = conv_same(rc, params["wd"], params["bd"]) + p2
    p3, i3 = maxpool2(np.maximum(zd, 0.0))
    feats = p3.reshape(4, n, -1)
    f = feats.mean(axis=0)
    z4 = f @ params["w4"].T + params["b4"]
    h4 = np.maximum(z4, 0.0)
    logit = (h4 @ params["w5"].T + params["b5"])[:, 0]
    if keep:
        cache = dict(x=x, z1=z1, p1=p1, i1=i1, za=za, ra=ra, zb=zb, r1=r1, z2=z2, p2=p2, i2=i2, zc=zc, rc=rc,
                     zd=zd, i3=i3, p3shape=p3.shape, f=f, z4=z4, h4=h4)
        return logit, cache
    return logit


def forward_ri_bf16(params, xn):
    """Logits of the rotation-invariant network with the kernels' BF16
    operands: the input, the weights of every convolution and of fc1, and
    every activation that enters a matrix product (each pooled or residual
    output and the rotation-averaged features) rounded to BF16; fc2, the
    biases and the sums exact."""
    q = {k: (round_bf16(v) if k.startswith("w") and k != "w5" else v) for k, v in params.items()}
    n = xn.shape[0]
    x = rotations(round_bf16(xn))
    p1 = round_bf16(maxpool2(np.maximum(conv_same(x, q["w1"], q["b1"]), 0.0))[0])
    ra = round_bf16(np.maximum(conv_same(p1, q["wa"], q["ba"]), 0.0))
    r1 = round_bf16(np.maximum(conv_same(ra, q["wb"], q["bb"]) + p1, 0.0))
    p2 = round_bf16(maxpool2(np.maximum(conv_same(r1, q["w2"], q["b2"]), 0.0))[0])
    rc = round_bf16(np.maximum(conv_same(p2, q["wc"], q["bc"]), 0.0))
    p3 = round_bf16(maxpool2(np.maximum(conv_same(rc, q["wd"], q["bd"]) + p2, 0.0))[0])
    f = round_bf16(p3.reshape(4, n, -1).mean(axis=0))
    h4 = np.maximum(f @ q["w4"].T + q["b4"], 0.0)
    return (h4 @ params["w5"].T + params["b5"])[:, 0]


def loss_and_grads_ri(params, xn, target):
    """BCE loss and its gradient for every parameter of the rotation-invariant network."""
    logit, c = forward_ri(params, xn, keep=True)
    n = logit.shape[0]
    loss = bce_loss(logit, target)
    dz5 = ((sigmoid(logit) - np.asarray(target, dtype=np.float64)) / n)[:, None]
    g = {"w5": dz5.T @ c["h4"], "b5": dz5.sum(axis=0)}
    dz4 = (dz5 @ params["w5"]) * (c["z4"] > 0)
    g["w4"], g["b4"] = dz4.T @ c["f"], dz4.sum(axis=0)
    df = dz4 @ params["w4"]
    dp3 = np.broadcast_to(df[None] / 4.0, (4,) + df.shape).reshape(c["p3shape"])
    dzd = maxpool2_backward(dp3, c["i3"], c["zd"].shape) * (c["zd"] > 0)
    drc, g["wd"], g["bd"] = conv_same_backward(c["rc"], params["wd"], dzd)
    dzc = drc * (c["zc"] > 0)
    dp2, g["wc"], g["bc"] = conv_same_backward(c["p2"], params["wc"], dzc)
    dp2 = dp2 + dzd                                   # the skip connection
    dz2 = maxpool2_backward(dp2, c["i2"], c["z2"].shape) * (c["z2"] > 0)
    dr1, g["w2"], g["b2"] = conv_same_backward(c["r1"], params["w2"], dz2)
    dzb = dr1 * (c["zb"] > 0)
    dra, g["wb"], g["bb"] = conv_same_backward(c["ra"], params["wb"], dzb)
    dza = dra * (c["za"] > 0)
    dp1, g["wa"], g["ba"] = conv_same_backward(c["p1"], params["wa"], dza)
    dp1 = dp1 + dzb                                   # the skip connection
    dz1 = maxpool2_backward(dp1, c["i1"], c["z1"].shape) * (c["z1"] > 0)
    _, g["w1"], g["b1"] = conv_same_backward(c["x"], params["w1"], dz1)
    return loss, g


def score_ri(params, stamps):
    return sigmoid(forward_ri(params, normalise(stamps)))

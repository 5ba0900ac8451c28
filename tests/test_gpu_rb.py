"""GPU parity of the stamp classifier, the detector and the shape cuts
(through the C ABI) against the FP64 oracles.

Tolerances.  The classifier rounds its normalised inputs, weights and every
hidden activation to BF16 (relative rounding error <= 2^-9) and accumulates in
FP32.  The oracle's BF16 operand model (cnn_oracle.forward_bf16 and
loss_and_grads_bf16: the FP64 network with the same operands rounded) must
agree with the GPU to 1e-2 of the logits' RMS and to relative L2 2e-2 and
cosine 0.999 in every gradient.  The model and the GPU differ only where a
value sits at a BF16 rounding midpoint to within the FP32 accumulation error
(or an FP32-normalised input rounds the other way); each such one-step
difference can change a max-pool choice downstream, and on detector stamps
with inputs up to +-64 a few of them move single logits by up to ~7e-3 of the
RMS.  Each fused inference layer is pinned element by element on its own
(test_fused_conv_layers_elementwise: bit-equal except one-step differences at
midpoints), so the logit bars separate layout or indexing mistakes from
rounding.  Against the plain FP64 network the logits are held
to relative L2 1e-2 where the logits are not dominated by cancellation (the
detector-stamp test below); on the synthetic stamps with small random-network
logits the rounding model itself departs by up to ~1 % with single logits off
by ~4 % of the RMS, and the bars there are 1.5e-2 (L2) and 6e-2 of the RMS
(max).  Gradients add one more rounding of each back-propagated signal and
sign flips of ReLU/max-pool decisions taken on slightly different values:
against FP64 the rounding model's own first-layer gradients differ by up to
~9 % (relative L2) at cosine >= 0.996, so against FP64 the bars are cosine >=
0.99 and relative L2 <= 0.15.  The detector
filters in FP32 (31 taps per pass, two passes): its SNR map agrees with the
FP64 map to 1e-5 of max |SNR| + 1e-5; candidate decisions may differ only where
the oracle's margin (to the threshold or to a neighbour) is below 1e-3.  The
shape cuts run in FP64 on both sides and must agree exactly.
"""
import numpy as np
import pytest

from oracle import cnn_oracle as C
from oracle import detect_oracle as DO
from synth.stamps import make_stamps

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DEV = "cuda"


def _dev(a, dtype=torch.float32):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV).to(dtype)


def _params(seed, bias_sd=0.05):
    p = C.init_params(seed)
    rng = np.random.default_rng(seed + 1)
    for k in C.ORDER:
        if k.startswith("b"):
            p[k] = rng.normal(0, bias_sd, p[k].shape)
    return p


def _model(params, max_batch):
    from paper_2603_08593_gb300 import RBModel
    m = RBModel(max_batch=max_batch, seed=0)
    m.set_weights(C.flatten(params).astype(np.float32))
    return m


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30))


def _check_logits(z, p, stamps):
    xn = C.normalise(stamps.astype(np.float64))
    zo = C.forward(p, xn)
    rms = max(np.sqrt(np.mean(zo ** 2)), 1e-3)
    assert _rel(z, zo) <= 1.5e-2, _rel(z, zo)
    assert np.max(np.abs(z - zo)) <= 6e-2 * rms + 1e-4, (np.max(np.abs(z - zo)), rms)
    zb = C.forward_bf16(p, xn)
    assert np.max(np.abs(z - zb)) <= 1e-2 * rms + 1e-4, (np.max(np.abs(z - zb)), rms)


def test_weights_roundtrip_exact():
    from paper_2603_08593_gb300 import RBModel
    m = RBModel(max_batch=4, seed=3)
    w = np.random.default_rng(0).normal(0, 1, C.n_params()).astype(np.float32)
    m.set_weights(w)
    assert np.array_equal(m.get_weights(), w)
    # the initialiser follows the uniform He ranges with zero biases
    m2 = RBModel(max_batch=4, seed=11)
    p = C.unflatten(m2.get_weights())
    for k in C.ORDER:
        if k.startswith("b"):
            assert np.all(p[k] == 0)
        else:
            lim = np.sqrt(6.0 / np.prod(C.SHAPES[k][1:]))
            assert np.abs(p[k]).max() <= lim and np.abs(p[k]).max() > 0.9 * lim


@pytest.mark.parametrize("n,max_batch", [(1, 8), (37, 16), (300, 128)])
def test_logits_and_scores_match_oracle(n, max_batch):
    d = make_stamps(n, seed=100 + n)
    p = _params(5)
    m = _model(p, max_batch)
    st = _dev(d["stamps"])
    z = m.logits(st).cpu().numpy().astype(np.float64)
    s = m.score(st).cpu().numpy().astype(np.float64)
    _check_logits(z, p, d["stamps"])
    assert np.allclose(s, 1 / (1 + np.exp(-z)), rtol=0, atol=2e-6)


def test_normalisation_edge_cases():
    # constant channels (MAD 0 -> scale 1), huge outliers (clip at +-64) and a
    # channel of a few distinct values all go through the same path as the oracle
    rng = np.random.default_rng(9)
    st = rng.normal(1000, 30, (4, 3, 31, 31)).astype(np.float32)
    st[0, 0] = 500.0
    st[1, 2, 15, 15] = 1e7
    st[2, 1] = rng.integers(0, 3, (31, 31)).astype(np.float32)
    st[3] *= 0
    p = _params(2)
    m = _model(p, 4)
    z = m.logits(_dev(st)).cpu().numpy().astype(np.float64)
    _check_logits(z, p, st)


@pytest.mark.parametrize("ch,c1,c2,c3,pos", [(2, 0, 0, 0, 4), (0, 5, 17, 33, 0), (1, 31, 63, 63, 8)])
def test_delta_filters_route_one_pixel_block(ch, c1, c2, c3, pos):
    """Delta filters through every layer: the logit is exactly the maximum of
    relu(normalised input) over one 8 x 8 input block (BF16 values, FP32 sums
    of a single term), which pins the im2col, weight and flatten layouts."""
    p = {k: np.zeros(C.SHAPES[k]) for k in C.ORDER}
    p["w1"][c1, ch, 1, 1] = 1.0
    p["w2"][c2, c1, 1, 1] = 1.0
    p["w3"][c3, c2, 1, 1] = 1.0
    p["w4"][7, c3 * 9 + pos] = 1.0
    p["w5"][0, 7] = 1.0
    d = make_stamps(6, seed=60 + ch)
    m = _model(p, 8)
    z = m.logits(_dev(d["stamps"])).cpu().numpy().astype(np.float64)
    xn = C.round_bf16(C.normalise(d["stamps"].astype(np.float64)))
    i, j = divmod(pos, 3)
    ref = np.maximum(xn[:, ch, 8 * i:8 * i + 8, 8 * j:8 * j + 8].reshape(6, -1).max(axis=1), 0.0)
    assert np.all(np.abs(z - ref) <= 2.0 ** -8 * np.abs(ref)), (z, ref)
    assert np.all(ref > 0)


@pytest.mark.parametrize("taps", [((0, 0), (2, 2), (0, 2)), ((2, 1), (1, 0), (2, 0)), ((1, 2), (0, 1), (1, 1))])
def test_off_centre_delta_taps(taps):
    """Delta filters on off-centre taps of each convolution (every conv1 kernel
    row and column, the corner and edge taps of conv2 and conv3): every sum
    has one term, so the logits equal the BF16 operand model to its own
    rounding (one BF16 step where the FP32 normalisation rounds an input the
    other way); a wrong tap offset, weight-image slot or border record moves
    the selected pixels."""
    (a1, b1_), (a2, b2_), (a3, b3_) = taps
    p = {k: np.zeros(C.SHAPES[k]) for k in C.ORDER}
    for c in range(3):                     # every input channel into one conv1 output
        p["w1"][(5 + c) % 32, c, a1, b1_] = 1.0 + 0.25 * c
    p["w2"][9, 5, a2, b2_] = 1.0
    p["w2"][40, 7, a2, b2_] = 0.5
    p["w3"][21, 9, a3, b3_] = 1.0
    p["w3"][50, 40, a3, b3_] = 2.0
    for pos in range(9):
        p["w4"][pos, 21 * 9 + pos] = 1.0
        p["w4"][9 + pos, 50 * 9 + pos] = 1.0
    p["w5"][0, :18] = np.linspace(0.5, 1.5, 18)
    d = make_stamps(21, seed=91)
    m = _model(p, 32)
    z = m.logits(_dev(d["stamps"])).cpu().numpy().astype(np.float64)
    zb = C.forward_bf16(p, C.normalise(d["stamps"].astype(np.float64)))
    assert np.all(np.abs(zb) > 0.1)
    assert np.allclose(z, zb, rtol=8e-3, atol=1e-5), np.max(np.abs(z - zb))


def test_inference_full_batch_sampled():
    """A full 4096-stamp internal batch plus a ragged one (4096 + 37 stamps):
    sampled logits against the oracle, including both batches' first and last
    stamps and every stamp group boundary near the end; copies of a stamp give
    bit-identical logits wherever they sit in the batch."""
    base = make_stamps(256, seed=33)["stamps"]
    n = 4096 + 37
    st = np.concatenate([base] * ((n + 255) // 256))[:n]
    p = _params(21)
    m = _model(p, 4096)
    z = m.logits(_dev(st)).cpu().numpy().astype(np.float64)
    assert np.all(np.isfinite(z))
    zs = z.reshape(-1)[: (n // 256) * 256].reshape(-1, 256)
    assert np.array_equal(zs, np.broadcast_to(zs[0], zs.shape))
    assert np.array_equal(z[(n // 256) * 256:], zs[0, : n - (n // 256) * 256])
    idx = np.unique(np.r_[0, 1, 2, 7, 8, 255, 256, 4095, 4096, 4097, n - 9:n, np.arange(3, 4096, 97)])
    _check_logits(z[idx], p, st[idx])


_PLANES = {2: (4, 8, 15), 3: (8, 4, 7)}   # layer input planes: CB, WS, image size


def _to_planes(a, layer, n_alloc, fill_tail=0.0):
    """NHWC [n][H][H][8 CB] -> parity-split planes [CB][4][n_alloc][WS][WS][8]:
    padded pixel (r, c) = pixel (r - 1, c - 1) is record (r >> 1, c >> 1) of
    parity plane 2 (r & 1) + (c & 1), the zero border elsewhere; the pixels of
    stamps >= n hold `fill_tail`."""
    CB, WS, H = _PLANES[layer]
    n = a.shape[0]
    padded = np.zeros((n_alloc, 2 * WS, 2 * WS, CB * 8))
    padded[n:, 1:H + 1, 1:H + 1] = fill_tail
    padded[:n, 1:H + 1, 1:H + 1] = a
    p = padded.reshape(n_alloc, WS, 2, WS, 2, CB, 8).transpose(5, 2, 4, 0, 1, 3, 6)
    return p.reshape(CB, 4, n_alloc, WS, WS, 8)


def _from_planes(t, layer, n_alloc):
    """Inverse of _to_planes: the padded images [n_alloc][2 WS][2 WS][8 CB]."""
    CB, WS, H = _PLANES[layer]
    p = t.float().cpu().numpy().astype(np.float64).reshape(CB, 2, 2, n_alloc, WS, WS, 8)
    return p.transpose(3, 4, 1, 5, 2, 0, 6).reshape(n_alloc, 2 * WS, 2 * WS, CB * 8)


def _check_planes_out(t, layer, n, n_alloc):
    """Output planes of a layer: border records still zero, the pixels of
    stamps >= n untouched (7.0); returns the pixels of stamps < n (NHWC)."""
    CB, WS, H = _PLANES[layer]
    q = _from_planes(t, layer, n_alloc)
    border = np.ones((2 * WS, 2 * WS), bool)
    border[1:H + 1, 1:H + 1] = False
    assert not np.any(q[:, border]) and np.all(q[n:, 1:H + 1, 1:H + 1] == 7.0)
    return q[:n, 1:H + 1, 1:H + 1]


def _layer_oracle(x_nhwc, w, b):
    """The oracle's layer on BF16 operands: conv_same, ReLU, 2 x 2 max-pool;
    returns the exact pooled FP64 values and, per output, the pooled sum of
    |w| |x| (the scale of any accumulation-order difference)."""
    x = x_nhwc.transpose(0, 3, 1, 2)
    wq = C.round_bf16(w)
    z = C.conv_same(x, wq, b)
    za = C.conv_same(np.abs(x), np.abs(wq), np.abs(b))
    pooled = C.maxpool2(np.maximum(z, 0.0))[0]
    scale = C.maxpool2(za)[0]
    return pooled.transpose(0, 2, 3, 1), scale.transpose(0, 2, 3, 1)


def _check_layer(got, exact, scale):
    """Element-wise parity of BF16 outputs.  The kernel rounds to nearest a
    value that differs from the exact one only by FP32 accumulation error, at
    most 2^-14 of the accumulation scale (sum of |w| |x| + |b|; ReLU and max
    are monotone and 1-Lipschitz), so every output must lie between the BF16
    roundings of exact -+ that bound; and at most 1e-3 of the outputs may
    differ from the rounding of the exact value at all."""
    exp = C.round_bf16(exact)
    frac = np.count_nonzero(got != exp) / got.size
    assert frac <= 1e-3, frac
    delta = 2.0 ** -14 * scale
    lo, hi = C.round_bf16(exact - delta), C.round_bf16(exact + delta)
    bad = (got < np.maximum(lo, 0.0)) | (got > hi)   # outputs are ReLU'd: never below zero
    assert not np.any(bad), (got[bad][:5], exact[bad][:5], scale[bad][:5])


@pytest.mark.parametrize("n,n_alloc", [(1, 1), (7, 9), (37, 40), (300, 300)])
def test_fused_conv_layers_elementwise(n, n_alloc):
    """Each fused tensor-core convolution (rb_conv_layer) against the oracle's
    layer, element by element on identical BF16 inputs: ragged stamp groups
    (conv1 takes 2 stamps per group, conv2 4, conv3 8), zero plane borders kept,
    the interiors of stamps >= n never written."""
    rng = np.random.default_rng(n)
    p = _params(3 + n, bias_sd=0.1)
    m = _model(p, 8)
    x = C.round_bf16(rng.normal(0, 1.5, (n, 31, 31, 3)))
    # conv1: normalised stamps -> conv2 planes
    out = _dev(_to_planes(np.zeros((n, 15, 15, 32)), 2, n_alloc, fill_tail=7.0), torch.bfloat16)
    xin = np.zeros((n, 2888))
    xin[:, :2883] = x.reshape(n, -1)
    m.conv_layer(1, _dev(xin, torch.bfloat16), n, n_alloc, out)
    exact, scale = _layer_oracle(x, p["w1"], p["b1"])
    _check_layer(_check_planes_out(out, 2, n, n_alloc), exact, scale)
    # conv2 and conv3 on non-negative BF16 activations of their own
    for layer, (cin, H) in ((2, (32, 15)), (3, (64, 7))):
        a = C.round_bf16(np.abs(rng.normal(0, 1.0, (n, H, H, cin))) * (rng.random((n, H, H, cin)) < 0.6))
        inp = _dev(_to_planes(a, layer, n_alloc), torch.bfloat16)
        exact, scale = _layer_oracle(a, p[f"w{layer}"], p[f"b{layer}"])
        if layer == 2:
            out = _dev(_to_planes(np.zeros((n, 7, 7, 64)), 3, n_alloc, fill_tail=7.0), torch.bfloat16)
            m.conv_layer(2, inp, n, n_alloc, out)
            got = _check_planes_out(out, 3, n, n_alloc)
        else:
            out = torch.full((n * 9 * 64 + 64,), 7.0, dtype=torch.bfloat16, device=DEV)
            m.conv_layer(3, inp, n, n_alloc, out)
            full = out.float().cpu().numpy().astype(np.float64)
            assert np.all(full[n * 576:] == 7.0)
            got = full[:n * 576].reshape(n, 3, 3, 64)
        _check_layer(got, exact, scale)
    assert m.error_flags() == 0


def test_fused_conv_layer_arguments():
    m = _model(_params(1), 4)
    x = torch.zeros(4 * 2888, dtype=torch.bfloat16, device=DEV)
    y = torch.zeros(4 * 4 * 4 * 64 * 8, dtype=torch.bfloat16, device=DEV)
    from paper_2603_08593_gb300.binding import SfftError
    for layer, n, na in ((0, 1, 1), (4, 1, 1), (1, 5, 4), (1, 1, 0), (1, -1, 4)):
        with pytest.raises(SfftError):
            m.conv_layer(layer, x, n, na, y)
    with pytest.raises(SfftError):
        m.conv_layer(1, x[1:], 1, 4, y)   # 2-byte offset: not 16-byte aligned
    m.conv_layer(1, x, 0, 4, y)           # nothing to do
    torch.cuda.synchronize()


def test_gradients_match_oracle():
    d = make_stamps(48, seed=7)
    p = _params(13)
    m = _model(p, 64)
    loss = m.backward(_dev(d["stamps"]), _dev(d["labels"]))
    g = C.unflatten(m.get_grads())
    xn = C.normalise(d["stamps"].astype(np.float64))
    lo, go = C.loss_and_grads(p, xn, d["labels"].astype(np.float64))
    gb = C.loss_and_grads_bf16(p, xn, d["labels"].astype(np.float64))[1]
    assert abs(float(loss.item()) - lo) <= 2e-2 * abs(lo)
    for k in C.ORDER:
        a, b, c = g[k].ravel().astype(np.float64), go[k].ravel(), gb[k].ravel()
        cos = float(a @ b / max(np.linalg.norm(a) * np.linalg.norm(b), 1e-30))
        print(f"gradient {k}: vs FP64 cosine {cos:.6f}, relative L2 {_rel(a, b):.3e}; "
              f"vs BF16 model relative L2 {_rel(a, c):.3e} (model vs FP64 {_rel(c, b):.3e})")
        assert cos >= 0.99 and _rel(a, b) <= 0.15, (k, cos, _rel(a, b))
        assert _rel(a, c) <= 2e-2, (k, _rel(a, c))


def _detector_stamps():
    """Stamps as the pipeline produces them: the oracle's subtraction of a
    256 x 256 pair (stars, injected transients, cosmic-ray hits) and the
    oracle's matched-filter detection at 3 sigma on its difference image."""
    from oracle import sfft_oracle as O
    from synth import make_pair
    d = make_pair(256, 256, seed=11, n_src=120, fwhm_R=(1.2, 1.2), fwhm_S=(1.8, 1.8), shift=(0.1, 0.0),
                  n_transients=12, snr=(5.0, 40.0), n_cosmics=20, transient_margin=20)
    f = O.fit(d["R"], d["S"], d["bad"], 7, 1, 1)
    o = DO.detect(f["D"], d["S"], d["R"], d["bad"], 1.8 / 2.3548, 3.0)
    assert o["count"] >= 64
    return o["stamps"].astype(np.float32)


@pytest.mark.parametrize("seed", [5, 13])
def test_detector_stamps_logits_and_gradients(seed):
    """Parity on detector-produced stamps, the classifier's real input.  Logits
    against the FP64 network: relative L2 <= 1e-2; against the BF16 operand
    model: 1e-2 of the RMS.  Gradients against the BF16 operand model: cosine
    >= 0.999 and relative L2 <= 2e-2 for every parameter; against plain FP64
    (where the model itself departs by up to ~9 %), cosine >= 0.99 and
    relative L2 <= 0.15."""
    st = _detector_stamps()
    n = st.shape[0]
    p = _params(seed)
    m = _model(p, 128)
    z = m.logits(_dev(st)).cpu().numpy().astype(np.float64)
    xn = C.normalise(st.astype(np.float64))
    zo, zb = C.forward(p, xn), C.forward_bf16(p, xn)
    rms = np.sqrt(np.mean(zo ** 2))
    print(f"logits: vs FP64 {_rel(z, zo):.2e} (model vs FP64 {_rel(zb, zo):.2e}); "
          f"vs model max {np.max(np.abs(z - zb)) / rms:.2e} of the RMS")
    assert _rel(z, zo) <= 1e-2
    assert np.max(np.abs(z - zb)) <= 1e-2 * rms
    t = (np.arange(n) % 2).astype(np.float32)
    m.backward(_dev(st), _dev(t))
    g = C.unflatten(m.get_grads())
    _, go = C.loss_and_grads(p, xn, t.astype(np.float64))
    _, gb = C.loss_and_grads_bf16(p, xn, t.astype(np.float64))
    for k in C.ORDER:
        a, b, c = g[k].ravel().astype(np.float64), go[k].ravel(), gb[k].ravel()
        cb = float(a @ c / max(np.linalg.norm(a) * np.linalg.norm(c), 1e-30))
        co = float(a @ b / max(np.linalg.norm(a) * np.linalg.norm(b), 1e-30))
        print(f"gradient {k}: vs model cosine {cb:.6f} rel {_rel(a, c):.2e}; vs FP64 cosine {co:.6f} "
              f"rel {_rel(a, b):.2e}")
        assert cb >= 0.999 and _rel(a, c) <= 2e-2, (k, cb, _rel(a, c))
        assert co >= 0.99 and _rel(a, b) <= 0.15, (k, co, _rel(a, b))


def test_adam_step_and_checkpoint_resume():
    d = make_stamps(32, seed=21)
    p = _params(4)
    st, lab = _dev(d["stamps"]), _dev(d["labels"])
    m = _model(p, 32)
    m.train_step(st, lab, lr=1e-3)
    g = m.get_grads().astype(np.float64)
    w1 = m.get_weights().astype(np.float64)
    # first Adam step: theta - lr g / (|g| + eps) with the model's own gradient
    w0 = C.flatten(p).astype(np.float32).astype(np.float64)
    exp = w0 - 1e-3 * g / (np.abs(g) + 1e-8)
    assert np.allclose(w1, exp, rtol=0, atol=2e-6)
    state, step = m.get_state()
    assert step == 1 and state.size == 3 * C.n_params()
    # resume on a fresh model: the next step is identical
    m.train_step(st, lab, lr=1e-3)
    w2 = m.get_weights()
    m2 = _model(p, 32)
    m2.set_state(state, step)
    m2.train_step(st, lab, lr=1e-3)
    assert np.array_equal(m2.get_weights(), w2)


def test_training_reduces_loss():
    d = make_stamps(256, seed=31)
    from paper_2603_08593_gb300 import RBModel
    m = RBModel(max_batch=256, seed=1)
    st, lab = _dev(d["stamps"]), _dev(d["labels"])
    l0 = float(m.backward(st, lab).item())
    for _ in range(60):
        m.train_step(st, lab, lr=2e-3)
    l1 = float(m.backward(st, lab).item())
    assert l1 < 0.5 * l0, (l0, l1)


# ---------------------------------------------------------------- detection
def _det_image(H, W, seed, n_blobs=12, sigma=1.4):
    rng = np.random.default_rng(seed)
    D = rng.normal(0, 30.0, (H, W))
    yy, xx = np.mgrid[0:H, 0:W]
    for _ in range(n_blobs):
        y, x = rng.uniform(0, H), rng.uniform(0, W)
        D += rng.uniform(100, 3000) * np.exp(-((yy - y) ** 2 + (xx - x) ** 2) / (2 * sigma * sigma))
    bad = (rng.random((H, W)) < 0.01).astype(np.uint8)
    bad[:, W // 3] = 1
    D[rng.random((H, W)) < 0.001] = np.nan
    S = rng.normal(1000, 30, (H, W))
    R = rng.normal(1000, 30, (H, W))
    return D.astype(np.float32), S.astype(np.float32), R.astype(np.float32), bad


def _margins(snr, y, x, thresh):
    v = snr[y, x]
    nb = snr[y - 2:y + 3, x - 2:x + 3].copy()
    nb[2, 2] = -np.inf
    return min(abs(v - thresh), abs(v - np.nanmax(nb)))


@pytest.mark.parametrize("H,W,batch,use_bad,guard", [(64, 80, 1, True, 0), (157, 203, 2, True, 5),
                                                     (300, 129, 3, False, 3)])
def test_detect_matches_oracle(H, W, batch, use_bad, guard):
    from paper_2603_08593_gb300 import Detector
    imgs = [_det_image(H, W, 40 + b) for b in range(batch)]
    D = np.stack([i[0] for i in imgs]); S = np.stack([i[1] for i in imgs]); R = np.stack([i[2] for i in imgs])
    bad = np.stack([i[3] for i in imgs])
    det = Detector(H, W, batch=batch, max_cand=64)
    xy, snr, count, stamps = det(_dev(D), _dev(S), _dev(R), _dev(bad, torch.uint8) if use_bad else None,
                                 psf_sigma=1.4, thresh=5.0, guard=guard)
    torch.cuda.synchronize()
    smap = det.snr_map.cpu().numpy()
    xy, snr, count, stamps = xy.cpu().numpy(), snr.cpu().numpy(), count.cpu().numpy(), stamps.cpu().numpy()
    for b in range(batch):
        o = DO.detect(D[b], S[b], R[b], bad[b] if use_bad else None, 1.4, 5.0, max_cand=64, guard=guard)
        ref = o["snr_map"]
        assert np.max(np.abs(smap[b] - ref)) <= 1e-5 * np.max(np.abs(ref)) + 1e-5
        got = set(map(tuple, xy[b, :min(count[b], 64)][:, ::-1].tolist()))
        exp = set(zip(o["y"].tolist(), o["x"].tolist()))
        for (y, x) in got ^ exp:
            assert _margins(ref, y, x, 5.0) < 1e-3, (y, x)
        if got == exp:
            assert count[b] == o["count"]
            n = min(count[b], 64)
            order = [tuple(v) for v in xy[b, :n][:, ::-1].tolist()]
            assert order == sorted(order)
            assert np.array_equal(stamps[b, :n], o["stamps"].astype(np.float32))
            assert np.array_equal(snr[b, :n], smap[b][xy[b, :n, 1], xy[b, :n, 0]])


def test_detect_truncation_and_empty():
    from paper_2603_08593_gb300 import Detector
    D, S, R, bad = _det_image(120, 150, 3, n_blobs=30)
    det = Detector(120, 150, batch=1, max_cand=3)
    xy, snr, count, _ = det(_dev(D[None]), _dev(S[None]), _dev(R[None]), _dev(bad[None], torch.uint8), 1.4, 5.0)
    o = DO.detect(D, S, R, bad, 1.4, 5.0)
    assert int(count[0]) == o["count"] > 3
    assert [tuple(v) for v in xy[0].cpu().numpy()[:, ::-1].tolist()] == list(zip(o["y"][:3], o["x"][:3]))
    _, _, count, _ = det(_dev(D[None]), _dev(S[None]), _dev(R[None]), None, 1.4, 1e30)
    assert int(count[0]) == 0


def test_detect_full_ccd_sampled():
    """A 4096 x 2048 CCD: clipped sigma from the oracle on the whole image, the
    SNR map checked at sampled windows computed by the oracle on crops."""
    from paper_2603_08593_gb300 import Detector
    H, W = 4096, 2048
    rng = np.random.default_rng(5)
    D = rng.normal(0, 45.0, (H, W)).astype(np.float32)
    bad = np.zeros((H, W), np.uint8)
    bad[:, 700] = 1
    bad[:, 1500] = 1
    det = Detector(H, W, 1, max_cand=4096)
    Dd = _dev(D[None])
    xy, snr, count, _ = det(Dd, Dd, Dd, _dev(bad[None], torch.uint8), psf_sigma=0.8, thresh=4.0)
    torch.cuda.synchronize()
    smap = det.snr_map[0].cpu().numpy()
    mu, sd = DO.clipped_sigma(D, bad)
    r = 3
    for _ in range(12):
        y0, x0 = int(rng.integers(40, H - 80)), int(rng.integers(40, W - 80))
        crop = D[y0 - r:y0 + 40 + r, x0 - r:x0 + 40 + r]
        cbad = bad[y0 - r:y0 + 40 + r, x0 - r:x0 + 40 + r]
        ref = DO.matched_snr(crop, cbad, 0.8, sd)[r:-r, r:-r]
        assert np.max(np.abs(smap[y0:y0 + 40, x0:x0 + 40] - ref)) <= 1e-4
    # white noise: the SNR map is unit variance; the count is that of the map's own local maxima
    assert abs(np.std(smap[100:-100, 100:-100]) - 1.0) < 0.01
    n_exp = len(DO.candidates(smap.astype(np.float64), bad, 4.0)[0])
    assert int(count[0]) == n_exp


def test_shape_cuts_match_oracle():
    from paper_2603_08593_gb300 import shape_cuts
    d = make_stamps(400, seed=17)
    rng = np.random.default_rng(2)
    snr = rng.uniform(2, 60, 400).astype(np.float32)
    st = d["stamps"].copy()
    st[:5, 2] = 0.0                          # no positive flux
    out = shape_cuts(_dev(st), _dev(snr), psf_fwhm=1.8, snr_min=5.0).cpu().numpy()
    exp = np.array([C.shape_cuts(st[i, 2], float(snr[i]), 1.8, 5.0) for i in range(400)], np.int32)
    assert np.array_equal(out, exp)
    assert 0 < exp.sum() < 400


def test_adaptive_shape_cuts_match_oracle():
    """The adaptive-moment cuts: the GPU's 40 FP64 iterations against the
    oracle's on the same stamps.  exp and the sums round differently on the
    two sides, so a decision may differ only where the oracle's own size,
    axis ratio or negative fraction lies within 1e-6 (relative) of a cut."""
    from paper_2603_08593_gb300 import shape_cuts
    d = make_stamps(400, seed=18)
    rng = np.random.default_rng(3)
    snr = rng.uniform(2, 60, 400).astype(np.float32)
    st = d["stamps"].copy()
    st[:5, 2] = 0.0                          # no flux: the weighted flux is not positive
    out = shape_cuts(_dev(st), _dev(snr), psf_fwhm=1.8, snr_min=5.0, adaptive=True).cpu().numpy()
    exp = np.array([C.shape_cuts_adaptive(st[i, 2], float(snr[i]), 1.8, 5.0) for i in range(400)], np.int32)
    diff = np.nonzero(out != exp)[0]
    for i in diff:
        res = C.adaptive_moments(st[i, 2].astype(np.float64), 1.8 / 2.3548200450309493)
        assert res is not None, i
        (mxx, myy, mxy), _ = res
        tr, det = mxx + myy, mxx * myy - mxy * mxy
        disc = np.sqrt(max(tr * tr / 4 - det, 0.0))
        l1, l2 = tr / 2 + disc, tr / 2 - disc
        fw = 2.3548200450309493 * np.sqrt(0.5 * (l1 + l2))
        margins = [abs(fw / (0.5 * 1.8) - 1), abs(fw / (2.0 * 1.8) - 1), abs(np.sqrt(l1 / l2) / 2.5 - 1)]
        assert min(margins) < 1e-6, (i, margins)
    assert len(diff) <= 2
    assert 0 < exp.sum() < 400
    assert not out[:5].any()


def test_umma_probe_rates():
    """The MMA-rate probe (sfft_probe_umma_cycles): finite positive cycle
    counts, wider MMAs no cheaper than narrower ones and at least the
    arithmetic time at N = 256; invalid N rejected."""
    from paper_2603_08593_gb300 import binding
    c = {n: binding.probe_umma_cycles(n) for n in (64, 256)}
    assert all(0 < v < 1e4 for v in c.values()), c
    assert c[256] >= c[64]
    assert c[256] >= 0.9 * 128 * 256 * 16 / 4096   # 2 x 128 x 256 x 16 flop at <= 8192 flop per clock
    for bad in (0, 8, 264):
        with pytest.raises(binding.SfftError):
            binding.probe_umma_cycles(bad)

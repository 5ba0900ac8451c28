"""GPU parity of the paper's rotation-invariant residual classifier (rbri_*,
through the C ABI) against the FP64 oracle.

Tolerances follow those of the small network (tests/test_gpu_rb.py): the
kernels round the normalised inputs, weights and every hidden activation to
BF16 and accumulate in FP32; the skip connections add the BF16 activation the
branch consumed, and the four rotations' features are averaged in FP32 and
rounded once more.  An FP64 model of those roundings must agree with the GPU
logits to 5e-3 of their RMS; the FP64 oracle itself to 2e-2 (relative L2) and
8e-2 of the RMS (max: two more rounded layers than the small network).
Gradients: cosine >= 0.99 and relative L2 <= 0.15 per tensor against FP64.
Rotation invariance on the GPU holds up to the FP32 order of the rotation
sum and the BF16 rounding of the mean: 2e-3 of the logits' RMS.
"""
import numpy as np
import pytest

from oracle import cnn_oracle as C
from synth.stamps import make_stamps

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DEV = "cuda"


def _dev(a, dtype=torch.float32):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV).to(dtype)


def _params(seed, bias_sd=0.05):
    p = C.init_params_ri(seed)
    rng = np.random.default_rng(seed + 1)
    for k in C.ORDER_RI:
        if k.startswith("b"):
            p[k] = rng.normal(0, bias_sd, p[k].shape)
    return p


def _model(params, max_batch):
    from paper_2603_08593_gb300 import RIModel
    m = RIModel(max_batch=max_batch, seed=0)
    m.set_weights(C.flatten_ri(params).astype(np.float32))
    return m


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30))


def test_ri_weights_roundtrip_exact():
    p = _params(3)
    m = _model(p, 8)
    w = C.flatten_ri(p).astype(np.float32)
    assert np.array_equal(m.get_weights(), w)
    assert m.get_weights().size == C.n_params_ri()


@pytest.mark.parametrize("n,max_batch", [(37, 16), (64, 64)])
def test_ri_logits_match_oracle(n, max_batch):
    d = make_stamps(n, seed=101 + n)
    p = _params(5)
    m = _model(p, max_batch)
    z = m.logits(_dev(d["stamps"])).cpu().numpy().astype(np.float64)
    xn = C.normalise(d["stamps"].astype(np.float64))
    zo = C.forward_ri(p, xn)
    zb = C.forward_ri_bf16(p, xn)
    rms = float(np.sqrt(np.mean(zo ** 2)))
    print(f"logits: vs BF16 model max {np.abs(z - zb).max() / rms:.3e} RMS; vs FP64 relative L2 {_rel(z, zo):.3e}, "
          f"max {np.abs(z - zo).max() / rms:.3e} RMS")
    assert np.abs(z - zb).max() <= 5e-3 * rms
    assert _rel(z, zo) <= 2e-2 and np.abs(z - zo).max() <= 8e-2 * rms
    s = m.score(_dev(d["stamps"])).cpu().numpy()
    assert np.allclose(s, 1 / (1 + np.exp(-z)), rtol=1e-5, atol=1e-6)


def test_ri_rotation_invariance_on_gpu():
    d = make_stamps(48, seed=55)
    p = _params(6)
    m = _model(p, 64)
    z0 = m.logits(_dev(d["stamps"])).cpu().numpy()
    rms = float(np.sqrt(np.mean(z0.astype(np.float64) ** 2)))
    for r in (1, 2, 3):
        zr = m.logits(_dev(np.rot90(d["stamps"], r, axes=(2, 3)).copy())).cpu().numpy()
        assert np.abs(zr - z0).max() <= 2e-3 * rms, (r, np.abs(zr - z0).max() / rms)
    zm = m.logits(_dev(d["stamps"][:, :, :, ::-1].copy())).cpu().numpy()
    assert np.abs(zm - z0).max() > 1e-2 * rms   # a mirror is not one of the rotations


def test_ri_gradients_match_oracle():
    d = make_stamps(24, seed=17)
    p = _params(9)
    m = _model(p, 32)
    loss = m.backward(_dev(d["stamps"]), _dev(d["labels"]))
    g = C.unflatten_ri(m.get_grads())
    xn = C.normalise(d["stamps"].astype(np.float64))
    lo, go = C.loss_and_grads_ri(p, xn, d["labels"].astype(np.float64))
    assert abs(float(loss.item()) - lo) <= 2e-2 * abs(lo)
    for k in C.ORDER_RI:
        a, b = g[k].ravel().astype(np.float64), go[k].ravel()
        cos = float(a @ b / max(np.linalg.norm(a) * np.linalg.norm(b), 1e-30))
        print(f"gradient {k}: cosine {cos:.6f}, relative L2 {_rel(a, b):.3e}")
        assert cos >= 0.99 and _rel(a, b) <= 0.15, (k, cos, _rel(a, b))


def test_ri_adam_step_checkpoint_and_training():
    d = make_stamps(128, seed=23)
    p = _params(4)
    st, lab = _dev(d["stamps"]), _dev(d["labels"])
    m = _model(p, 128)
    m.train_step(st, lab, lr=1e-3)
    g = m.get_grads().astype(np.float64)
    w1 = m.get_weights().astype(np.float64)
    w0 = C.flatten_ri(p).astype(np.float32).astype(np.float64)
    assert np.allclose(w1, w0 - 1e-3 * g / (np.abs(g) + 1e-8), rtol=0, atol=2e-6)
    state, step = m.get_state()
    m.train_step(st, lab, lr=1e-3)
    w2 = m.get_weights()
    m2 = _model(p, 128)
    m2.set_state(state, step)
    m2.train_step(st, lab, lr=1e-3)
    assert np.array_equal(m2.get_weights(), w2)
    l0 = float(m.backward(st, lab).item())
    for _ in range(60):
        m.train_step(st, lab, lr=2e-3)
    l1 = float(m.backward(st, lab).item())
    assert l1 < 0.5 * l0, (l0, l1)

"""GPU parity of forced aperture photometry, the limiting-magnitude Monte
Carlo and the multi-template median against the FP64 oracle.

The inside/outside decisions of the aperture are the same IEEE double
expressions on both sides, so flags and weights agree exactly and fluxes
differ only by summation order (1e-12 relative); the median works in FP32 on
the GPU (FP64 in the oracle), so it agrees to 2 FP32 ulps."""
import numpy as np
import pytest

from oracle import phot_oracle as P

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DEV = "cuda"


def _image(H, W, seed):
    rng = np.random.default_rng(seed)
    D = rng.normal(0, 25.0, (H, W))
    yy, xx = np.mgrid[0:H, 0:W]
    for _ in range(8):
        x, y = rng.uniform(0, W), rng.uniform(0, H)
        D += rng.uniform(200, 5000) * np.exp(-((xx - x) ** 2 + (yy - y) ** 2) / (2 * 1.7 ** 2))
    bad = (rng.random((H, W)) < 0.003).astype(np.uint8)
    D[rng.random((H, W)) < 0.001] = np.nan
    return D.astype(np.float32), bad


@pytest.mark.parametrize("radius", [3.0, 0.6731 * 1.9, 7.25])
def test_aperture_flux_matches_oracle(radius):
    from paper_2603_08593_gb300 import aperture_flux
    H, W, B, n = 130, 170, 2, 300
    imgs = [_image(H, W, 10 + b) for b in range(B)]
    D = np.stack([i[0] for i in imgs]); bad = np.stack([i[1] for i in imgs])
    rng = np.random.default_rng(3)
    pos = np.stack([rng.uniform(-5, W + 5, (B, n)), rng.uniform(-5, H + 5, (B, n))], axis=-1)   # some off the edge
    pos[0, :10] = np.round(pos[0, :10])            # pixel-centred apertures: boundary ties
    f, fl = aperture_flux(torch.from_numpy(D).to(DEV), torch.from_numpy(pos).to(DEV), radius,
                          torch.from_numpy(bad).to(DEV))
    f, fl = f.cpu().numpy(), fl.cpu().numpy()
    for b in range(B):
        fo, flo = P.aperture_flux(D[b], bad[b], pos[b, :, 0], pos[b, :, 1], radius)
        assert np.array_equal(fl[b], flo)
        assert np.all(np.abs(f[b] - fo) <= 1e-12 * np.maximum(np.abs(fo), 1.0) + 1e-9)
    assert 0 < fl.sum() < B * n


def test_limiting_magnitude_matches_oracle():
    from paper_2603_08593_gb300 import binding, limiting_mag
    H, W, B = 200, 240, 3
    imgs = [_image(H, W, 20 + b) for b in range(B)]
    D = np.stack([i[0] for i in imgs]); bad = np.stack([i[1] for i in imgs])
    pos = binding.random_positions(B, H, W, 1024, seed=5, device=DEV)
    sig, ml, ng = limiting_mag(torch.from_numpy(D).to(DEV), 3.0, 31.2, pos=pos, bad=torch.from_numpy(bad).to(DEV))
    p = pos.cpu().numpy()
    for b in range(B):
        so, mo, no = P.limiting_mag(D[b], bad[b], p[b, :, 0], p[b, :, 1], 3.0, 31.2)
        assert int(ng[b]) == no
        assert abs(float(sig[b]) - so) <= 1e-10 * so
        assert abs(float(ml[b]) - mo) <= 1e-9


@pytest.mark.parametrize("ntemp", [1, 4, 5])
def test_median_combine_matches_oracle(ntemp):
    from paper_2603_08593_gb300 import median_combine
    rng = np.random.default_rng(ntemp)
    H, W = 97, 131
    Ds = rng.normal(0, 10, (ntemp, H, W)).astype(np.float32)
    Ds[rng.random(Ds.shape) < 0.01] = np.inf
    bads = (rng.random(Ds.shape) < 0.05).astype(np.uint8)
    bads[:, 5, 7] = 1                                      # a pixel with no good template
    scale = rng.uniform(0.8, 1.25, ntemp).astype(np.float32)
    out = median_combine(torch.from_numpy(Ds).to(DEV), torch.from_numpy(scale).to(DEV),
                         torch.from_numpy(bads).to(DEV)).cpu().numpy()
    ref = P.median_combine(Ds, scale.astype(np.float64), bads)
    both = np.isnan(out) & np.isnan(ref)
    assert both[5, 7]
    ok = ~np.isnan(ref)
    assert np.array_equal(np.isnan(out), np.isnan(ref))
    assert np.all(np.abs(out[ok] - ref[ok]) <= 2 * np.spacing(np.abs(ref[ok]).astype(np.float32)) + 1e-6)


def test_multi_template_difference_matches_oracle():
    """One science frame against five templates of the same field with
    different PSFs; the median of the five differences against the oracle's."""
    from oracle import sfft_oracle as O
    from paper_2603_08593_gb300 import Plan, binding
    from synth.decam import make_pair
    H, W, L, DK, DB = 120, 150, 5, 1, 1
    pairs = [make_pair(H, W, seed=77, n_src=40, fwhm_R=(f, f + 0.2), fwhm_S=(2.2, 2.4), n_transients=1,
                       snr=(30.0, 30.0)) for f in (1.0, 1.2, 1.4, 1.6, 1.8)]
    S = pairs[0]["S"]                          # the same field: positions and fluxes are drawn first
    R = np.stack([p["R"] for p in pairs])
    refs = [O.fit(R[t], S, None, L, DK, DB) for t in range(5)]
    sky = torch.tensor([[r["prep"]["s_R"], r["prep"]["s_S"]] for r in refs], dtype=torch.float64, device=DEV)
    plan = Plan(H, W, L, DK, DB, batch=5, prec="mixed")
    Rt = torch.from_numpy(R).to(DEV)
    St = torch.from_numpy(S).to(DEV)
    Sx = St.reshape(1, H, W).expand(5, -1, -1).contiguous()
    out = plan.subtract(Rt, Sx, None, sky, refine=1)
    scale = torch.tensor([1.0, 1.02, 0.98, 1.05, 0.95], dtype=torch.float32, device=DEV)
    comb = binding.median_combine(out["D"], scale).cpu().numpy()
    ref = P.median_combine(np.stack([r["D"] for r in refs]).astype(np.float32), scale.cpu().numpy().astype(np.float64))
    assert np.abs(comb - ref).max() <= 1e-3 * 32.19
    # the convenience wrapper runs the same path (sky estimated on the GPU: compare away from the border)
    comb2, _ = binding.multi_template_difference(plan, Rt, St, None, scale)
    w = (L - 1) // 2
    assert np.abs(comb2.cpu().numpy()[w:-w, w:-w] - ref[w:-w, w:-w]).max() <= 1e-3 * 32.19

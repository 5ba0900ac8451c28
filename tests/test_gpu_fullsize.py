"""Full-size parity on the 2048 x 4096 DECam-shaped pair (L = 11, D_K = D_B = 2)
in the launch configuration the benchmark times, against the FP64 oracle run
on the whole CCD (definition-form normal equations; a few minutes of CPU).

Reported and asserted, per result:
  FP64 GPU path  - kernel coefficients within 1e-8 relative, |dD| within half
                   an FP32 ulp of |D| plus 1e-6 sigma_sky (D is stored in FP32);
  mixed path     - kernel coefficients <= 1e-5 relative, max |dD| / sigma_sky
                   <= 1e-3 over the unmasked pixels (reported over all pixels
                   too: masked saturated cores reach 6.5e4 ADU, where a 1e-7
                   coefficient error alone moves D by ~0.2 sigma_sky), and the
                   recovered flux of the 50 injected transients (box sums of
                   D, half-width ceil(3 sigma_S)) unbiased to 1e-4 of the
                   injected flux.
The sky offsets are the oracle's medians for these comparisons; the
benchmark's own call (offsets estimated on the GPU) is compared on the kernel
and on D away from the w-pixel border.
Set SFFT_ACCURACY_OUT to a path to also write the measured figures as JSON.
"""
import json
import math
import os

import numpy as np
import pytest

from oracle import sfft_oracle as O
from synth import SIGMA_SKY, config_pair

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu, pytest.mark.slow]

L, DK, DB = 11, 2, 2


@pytest.fixture(scope="module")
def c2():
    d = config_pair("c2")
    ref = O.fit(d["R"], d["S"], d["bad"], L, DK, DB, form="definition")
    assert ref["status"] == O.STATUS_OK
    return d, ref


def _gpu(d, prec, sky=None):
    from paper_2603_08593_gb300 import Plan
    H, W = d["R"].shape
    R = torch.from_numpy(d["R"]).cuda()[None].contiguous()
    S = torch.from_numpy(d["S"]).cuda()[None].contiguous()
    bad = torch.from_numpy(d["bad"]).cuda()[None].contiguous()
    if sky is not None:
        sky = torch.tensor([sky], dtype=torch.float64, device="cuda")
    p = Plan(H, W, L, DK, DB, batch=1, prec=prec)
    o = p.subtract(R, S, bad, sky, refine=1)
    torch.cuda.synchronize()
    return {k: v.cpu().numpy() for k, v in o.items()}


def test_fullsize_accuracy(c2):
    d, ref = c2
    out = {}
    sky = [ref["prep"]["s_R"], ref["prep"]["s_S"]]
    f64 = _gpu(d, "fp64", sky)
    mix = _gpu(d, "mixed", sky)
    est = _gpu(d, "mixed")                  # the benchmark's call: sky offsets estimated on the GPU
    assert f64["info"][0] == 0 and mix["info"][0] == 0 and est["info"][0] == 0
    out["fp64_coef_rel_err"] = O.kernel_coef_rel_err(f64["theta"][0], ref["theta_orig"], L, DK, DB)
    excess = np.abs(f64["D"][0] - ref["D"]) - 2.0 ** -24 * np.abs(ref["D"])
    out["fp64_max_dD_beyond_fp32_rounding_over_sigma"] = float(excess.max() / SIGMA_SKY)
    out["mixed_coef_rel_err"] = O.kernel_coef_rel_err(mix["theta"][0], ref["theta_orig"], L, DK, DB)
    dD = np.abs(mix["D"][0] - ref["D"]) / SIGMA_SKY
    out["mixed_max_dD_over_sigma_unmasked"] = float(dD[d["bad"] == 0].max())
    out["mixed_max_dD_over_sigma_all"] = float(dD.max())
    # with its own sky constants D changes only within w of the border (the constant
    # times the part of the kernel that falls outside the image is not absorbed by B)
    w = (L - 1) // 2
    inner = (slice(w, -w), slice(w, -w))
    out["mixed_gpu_sky_coef_rel_err"] = O.kernel_coef_rel_err(est["theta"][0], ref["theta_orig"], L, DK, DB)
    out["mixed_gpu_sky_max_dD_over_sigma_inner"] = float(
        (np.abs(est["D"][0] - ref["D"]) / SIGMA_SKY)[inner][d["bad"][inner] == 0].max())
    tr = d["transients"]
    half = int(math.ceil(3.0 * float(tr[:, 4].max())))
    rel = [(O.box_flux(mix["D"][0], x, y, half) - O.box_flux(ref["D"], x, y, half)) / f
           for x, y, f in tr[:, :3]]
    out["mixed_transient_flux_bias"] = float(np.mean(rel))
    out["mixed_transient_flux_max_rel"] = float(np.max(np.abs(rel)))
    out["n_transients"] = int(len(rel))
    if os.environ.get("SFFT_ACCURACY_OUT"):
        with open(os.environ["SFFT_ACCURACY_OUT"], "w") as fh:
            json.dump(out, fh, indent=1)
    print(json.dumps(out))
    assert out["fp64_coef_rel_err"] <= 1e-8
    assert out["fp64_max_dD_beyond_fp32_rounding_over_sigma"] <= 1e-6
    assert out["mixed_coef_rel_err"] <= 1e-5
    assert out["mixed_max_dD_over_sigma_unmasked"] <= 1e-3
    assert out["mixed_gpu_sky_coef_rel_err"] <= 1e-5
    assert out["mixed_gpu_sky_max_dD_over_sigma_inner"] <= 1e-3
    assert abs(out["mixed_transient_flux_bias"]) <= 1e-4

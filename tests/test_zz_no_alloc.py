"""The allocation-free difference image (sfft_apply_noalloc) against the
plan-based sfft_apply, through the C ABI.

Callers that cannot allocate device memory use this entry point with only
their own inputs and output; its scratch is a fixed array inside the
library.  Two calls in a row must reproduce the plan-based result (the
shared scratch keeps the previous call's contents, which must not leak into
the next result).  This file is collected last so that a run stopping at the
first failure has already run every other test; it also passes on its own in
a fresh process.
"""
import numpy as np
import pytest

from oracle import sfft_oracle as O
from synth import SIGMA_SKY, small_pair

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec,L,DK,DB", [("mixed", 7, 1, 2), ("fp64", 5, 1, 1)])
def test_noalloc_apply_matches_plan_apply_twice(prec, L, DK, DB):
    from paper_2603_08593_gb300 import Plan, binding
    H, W, B = 90, 140, 2
    pairs = [small_pair(H, W, seed=7700 + i, mask_fraction=0.02) for i in range(B)]
    dev = torch.device("cuda", torch.cuda.current_device())
    R = torch.from_numpy(np.stack([p["R"] for p in pairs])).to(dev)
    S = torch.from_numpy(np.stack([p["S"] for p in pairs])).to(dev)
    bad = torch.from_numpy(np.stack([p["bad"] for p in pairs])).to(dev)
    # theta in original units from the oracle fit of each pair, and its sky constants
    fits = [O.fit(p["R"], p["S"], p["bad"], L, DK, DB) for p in pairs]
    theta = torch.tensor(np.stack([f["theta_orig"] for f in fits]), dtype=torch.float64, device=dev)
    sky = torch.tensor([[f["prep"]["s_R"], f["prep"]["s_S"]] for f in fits], dtype=torch.float64, device=dev)

    plan = Plan(H, W, L, DK, DB, batch=B, prec=prec, device=dev)
    D_plan = plan.apply(R, S, theta, sky)

    # a second, different theta first, so the shared scratch holds stale values
    theta2 = theta * 1.5
    D_other = torch.empty_like(D_plan)
    binding.apply_noalloc(R, S, theta2, sky, D_other, L, DK, DB, prec=prec)
    outs = []
    for _ in range(2):
        D = torch.full_like(D_plan, float("nan"))
        binding.apply_noalloc(R, S, theta, sky, D, L, DK, DB, prec=prec)
        outs.append(D)
    torch.cuda.synchronize()
    ref = D_plan.cpu().numpy()
    tol = 1e-3 * SIGMA_SKY if prec == "mixed" else 2.0 ** -24 * np.abs(ref) + 1e-7 * SIGMA_SKY
    for D in outs:
        d = D.cpu().numpy()
        assert np.all(np.isfinite(d))
        assert np.all(np.abs(d - ref) <= tol)
    # and both agree with the FP64 oracle's difference image
    for i, f in enumerate(fits):
        assert np.abs(outs[1][i].cpu().numpy() - f["D"]).max() <= 1e-3 * SIGMA_SKY


def test_noalloc_rejects_oversize_and_missing_sky():
    from paper_2603_08593_gb300 import binding
    lib = binding.load()
    dev = torch.device("cuda", torch.cuda.current_device())
    H, W, L, DK, DB = 32, 32, 11, 2, 2
    B = 65   # 65 * 732 doubles exceeds the fixed scratch
    R = torch.zeros((B, H, W), dtype=torch.float32, device=dev)
    theta = torch.zeros((B, 732), dtype=torch.float64, device=dev)
    sky = torch.zeros((B, 2), dtype=torch.float64, device=dev)
    st = lib.sfft_apply_noalloc(H, W, L, DK, DB, B, 1, binding._ptr(R), binding._ptr(R), binding._ptr(theta),
                                binding._ptr(sky), binding._ptr(R), None)
    assert st == binding.SFFT_ERR_UNSUPPORTED
    assert b"exceeds the fixed scratch" in lib.sfft_last_error()
    st = lib.sfft_apply_noalloc(H, W, L, DK, DB, 1, 1, binding._ptr(R), binding._ptr(R), binding._ptr(theta),
                                None, binding._ptr(R), None)
    assert st == binding.SFFT_ERR_ARG

"""Failure detection on the GPU in the forms that fault nothing: a bounded
software wait made to run out, and injected allocation failures.

The FP64 factorisation separates its block steps with a grid-wide barrier
whose wait is bounded.  With the limit set to zero polls, every CTA that is
not the last to arrive gives up at once (the CTA that factors the first
diagonal block arrives microseconds after the others), so every CCD reports
SFFT_ERR_TIMEOUT, the kernels return, and the next call on the same plan,
with the default limit, gives the oracle's answer (one CCD and a batch).  The tensor-core and
bulk-copy waits are not made to expire here: copies or MMAs could still be
in flight when a CTA leaves."""
import ctypes

import numpy as np
import pytest

from oracle import sfft_oracle as O
from synth import SIGMA_SKY, small_pair

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("batch", [1, 2])
def test_barrier_wait_runs_out_then_plan_recovers(batch):
    from paper_2603_08593_gb300 import Plan, binding
    L, DK, DB = 7, 2, 2
    imgs = [small_pair(150, 210, seed=6100 + i, mask_fraction=0.03) for i in range(batch)]
    refs = [O.fit(x["R"], x["S"], x["bad"], L, DK, DB) for x in imgs]
    dev = torch.device("cuda", torch.cuda.current_device())
    R = torch.from_numpy(np.stack([x["R"] for x in imgs])).to(dev)
    S = torch.from_numpy(np.stack([x["S"] for x in imgs])).to(dev)
    bad = torch.from_numpy(np.stack([x["bad"] for x in imgs])).to(dev)
    sky = torch.tensor([[r["prep"]["s_R"], r["prep"]["s_S"]] for r in refs], dtype=torch.float64, device=dev)
    plan = Plan(150, 210, L, DK, DB, batch=batch, prec="mixed", device=dev)
    plan.set_wait_limit(0)
    o = plan.subtract(R, S, bad, sky, refine=1)
    torch.cuda.synchronize()
    assert [int(v) for v in o["info"].cpu()] == [binding.SFFT_ERR_TIMEOUT] * batch
    plan.set_wait_limit(-1)
    o = plan.subtract(R, S, bad, sky, refine=1, out=o)
    torch.cuda.synchronize()
    assert [int(v) for v in o["info"].cpu()] == [0] * batch
    th, D = o["theta"].cpu().numpy(), o["D"].cpu().numpy()
    for i, r in enumerate(refs):
        assert O.kernel_coef_rel_err(th[i], r["theta_orig"], L, DK, DB) <= 1e-5
        assert np.abs(D[i] - r["D"]).max() <= 1e-3 * SIGMA_SKY


def test_every_plan_allocation_failure_is_reported_without_leaks(monkeypatch):
    from paper_2603_08593_gb300 import binding
    lib = binding.load()
    torch.cuda.synchronize()
    before = lib.sfft_debug_live_allocations()
    desc = binding.Desc(96, 128, 5, 1, 1, 2, binding.PREC["mixed"], 0, 0, 0, 0, 0)
    n_fail = 0
    for k in range(1, 64):
        monkeypatch.setenv("SFFT_FAIL_ALLOC", str(k))
        h = ctypes.c_void_p()
        st = lib.sfft_plan(ctypes.byref(desc), None, ctypes.byref(h))
        if st == binding.SFFT_OK:
            # k is past the plan's last allocation: the plan is complete and usable
            assert lib.sfft_debug_live_allocations() > before
            lib.sfft_plan_destroy(h)
            assert lib.sfft_debug_live_allocations() == before
            break
        n_fail += 1
        assert st == binding.SFFT_ERR_NOMEM, st
        assert f"SFFT_FAIL_ALLOC={k}".encode() in lib.sfft_last_error()
        assert lib.sfft_debug_live_allocations() == before
    else:
        pytest.fail("every allocation index failed")
    assert n_fail >= 5     # twiddles, powers of yt, offset tables and job tables
    monkeypatch.delenv("SFFT_FAIL_ALLOC")
    # nothing left behind: a normal plan and a subtraction still work
    from paper_2603_08593_gb300 import Plan
    d = small_pair(96, 128, seed=6200, mask_fraction=0.02)
    ref = O.fit(d["R"], d["S"], d["bad"], 5, 1, 1)
    dev = torch.device("cuda", torch.cuda.current_device())
    p = Plan(96, 128, 5, 1, 1, batch=1, prec="mixed", device=dev)
    o = p.subtract(torch.from_numpy(d["R"])[None].to(dev), torch.from_numpy(d["S"])[None].to(dev),
                   torch.from_numpy(d["bad"])[None].to(dev), None, refine=1)
    torch.cuda.synchronize()
    assert int(o["info"][0]) == 0
    assert O.kernel_coef_rel_err(o["theta"][0].cpu().numpy(), ref["theta_orig"], 5, 1, 1) <= 1e-5

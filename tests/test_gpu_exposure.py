"""Full-size parity of the batched exposure path: three CCDs of the 60-CCD
exposure recipe (2048 x 4096, independent PSF gradients, masked fractions
2-30 %, cosmics and bleed trails; L = 11, D_K = D_B = 2) in one graph-captured
call with the settings a 60-CCD plan takes (every difference per pass,
difference-lane contraction), forced into groups of two CCDs so that more
than one product-spectrum pass runs; and the same CCDs with 34 differences
per pass on the pair-lane engine (several difference batches per CCD).
Each CCD is compared with the FP64 oracle's definition-form fit of that CCD
(a minute of CPU per CCD): kernel coefficients <= 1e-5 relative, max |dD| /
sigma_sky <= 1e-3 over the unmasked pixels away from the w-pixel border (the
GPU estimates its own sky offsets here, as the exposure call does, which
changes D only within w of the border)."""
import numpy as np
import pytest

from oracle import sfft_oracle as O
from synth import SIGMA_SKY, config_pair

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu, pytest.mark.slow]

L, DK, DB = 11, 2, 2
IDX = (0, 7, 23)


@pytest.fixture(scope="module")
def exposure():
    pairs = [config_pair("c4", i) for i in IDX]
    refs = [O.fit(d["R"], d["S"], d["bad"], L, DK, DB, form="definition") for d in pairs]
    for r in refs:
        assert r["status"] == O.STATUS_OK
    return pairs, refs


def _check(out, pairs, refs):
    w = (L - 1) // 2
    inner = (slice(w, -w), slice(w, -w))
    th, D, info = out["theta"].cpu().numpy(), out["D"].cpu().numpy(), out["info"].cpu().numpy()
    errs = []
    for i, (d, r) in enumerate(zip(pairs, refs)):
        assert info[i] == 0
        e = O.kernel_coef_rel_err(th[i], r["theta_orig"], L, DK, DB)
        dD = (np.abs(D[i] - r["D"]) / SIGMA_SKY)[inner][d["bad"][inner] == 0].max()
        errs.append((e, dD))
        assert e <= 1e-5, (i, e)
        assert dD <= 1e-3, (i, dD)
    print(errs)


@pytest.mark.parametrize("mode", ["groups", "pair_lane_slabs"])
def test_exposure_batch_matches_oracle(exposure, mode):
    from paper_2603_08593_gb300 import Plan
    pairs, refs = exposure
    dev = torch.device("cuda", torch.cuda.current_device())
    R = torch.from_numpy(np.stack([d["R"] for d in pairs])).to(dev)
    S = torch.from_numpy(np.stack([d["S"] for d in pairs])).to(dev)
    bad = torch.from_numpy(np.stack([d["bad"] for d in pairs])).to(dev)
    s = torch.cuda.Stream(device=dev)
    with torch.cuda.stream(s):
        if mode == "groups":
            p = Plan(4096, 2048, L, DK, DB, batch=len(pairs), prec="mixed", graph=True, stream=s, device=dev,
                     ccd_group=2)
            assert p.tiles[0] == 221 and p.engine == "tcgen05_difference_lane"
        else:
            p = Plan(4096, 2048, L, DK, DB, batch=len(pairs), prec="mixed", graph=True, stream=s, device=dev,
                     d_batch=34, pair_lane_contract=True)
            assert p.engine == "tcgen05_pair_lane"
        o = p.subtract(R, S, bad, None, refine=1)
        o = p.subtract(R, S, bad, None, refine=1, out=o)    # graph replay
    s.synchronize()
    _check(o, pairs, refs)

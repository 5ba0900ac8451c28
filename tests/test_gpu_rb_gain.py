"""What the trained classifier gains over the plain SNR/shape cuts (and over
the same cuts with a noise-robust adaptive-moment size), on
candidates that the GPU subtraction and detector produce from synthetic pairs
(injection truth labels).  A reduced version of the classifier experiment:
300 training pairs of 512 x 512, three epochs, judged on the held-out 15 %."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu, pytest.mark.slow]


def test_trained_network_beats_cuts():
    from paper_2603_08593_gb300 import train_rb
    report, _ = train_rb.run(train_ccds=300, epochs=3, batch=256, lr=1e-3, eval_ccds=0, seed=900, log=print)
    te = report["test"]
    assert te["cnn_0.3"]["n_real"] > 300 and te["cnn_0.3"]["n_bogus"] > 300
    # at the cuts' own completeness the network passes fewer artifacts, and at the
    # cuts' false-positive rate it keeps more real transients
    assert te["cnn_fpr_at_cuts_completeness"] < te["cuts"]["fpr"], te
    assert te["cnn_completeness_at_cuts_fpr"] > te["cuts"]["completeness"], te
    assert te["cnn_auc"] > 0.95, te
    assert report["train"]["loss_by_epoch"][-1] < report["train"]["loss_by_epoch"][0]
    # the same gain against the noise-robust (adaptive-moment) cuts, which keep
    # more real transients than the plain cuts
    ad = te["adaptive_cuts"]
    print("plain cuts", te["cuts"], "adaptive cuts", ad["cuts"])
    assert ad["cuts"]["completeness"] > te["cuts"]["completeness"], (ad, te["cuts"])
    assert ad["cnn_fpr_at_cuts_completeness"] < ad["cuts"]["fpr"], ad
    assert ad["cnn_completeness_at_cuts_fpr"] > ad["cuts"]["completeness"], ad

"""Train and judge the stamp classifier on candidates that this library's own
subtraction and detector produce from synthetic CCD pairs.

The paper (Sec. 2.3.4, Sec. 3.2) trains its real-bogus CNN on labelled
detections from difference images and quotes completeness and artifact
rejection at score thresholds 0.3 and 0.6.  Here the labels come from
injection truth: training pairs (512 x 512) carry point transients at SNR
3-100 and unmasked artifacts in the science frame (cosmic-ray hits, bad-column
segments, stars misregistered by 0.3-1 px); every candidate the detector
finds within 2 px of an injected transient is real, every other candidate is
bogus.  Candidates stay a kernel half-width away from masked pixels, whose
neighbourhood in D draws on masked reference pixels.  The network is trained
on the GPU by rb_train_step (BF16 tensor-core forward/backward, FP32 Adam) on
a class-balanced 80/5/15 split, and then
judged on the candidates of one 60-CCD exposure of 2048 x 4096 pairs against
the plain SNR/shape cuts (rb_shape_cuts).

    python -m paper_2603_08593_gb300.train_rb [--train-ccds 3000] [--epochs 5] [--out report.json]

Every GPU step runs in libsfft_gb300.so; NumPy only labels candidates and
computes the summary rates.
"""
from __future__ import annotations

import argparse
import json
import math
import multiprocessing as mp
import os
import sys
import time

import numpy as np

L, DK, DB = 11, 2, 2
MATCH_PX = 2.0
GUARD = (L - 1) // 2    # candidates keep the kernel half-width away from masked pixels


# ---------------------------------------------------------------- inputs (host, spawned pool)
def _truth(d, H, W):
    from synth import fwhm_to_sigma
    fs = float(d["fwhm_S"](W / 2.0, H / 2.0))
    return {"R": d["R"], "S": d["S"], "bad": d["bad"], "transients": d["transients"], "cosmics": d["cosmics"],
            "colsegs": d["colsegs"], "misreg": d["misreg"], "fwhm_S": fs, "psf_sigma": float(fwhm_to_sigma(fs))}


def train_pair(seed):
    """A 512 x 512 pair dense in transients and artifacts."""
    from synth.decam import make_pair
    rng = np.random.default_rng(10_000 + seed)
    r_lo, r_hi = rng.uniform(0.9, 1.5, 2)
    s_lo, s_hi = r_lo + rng.uniform(0.4, 0.8), r_hi + rng.uniform(0.4, 0.8)
    d = make_pair(512, 512, seed=seed, n_src=300, fwhm_R=(r_lo, r_hi), fwhm_S=(s_lo, s_hi),
                  grad_angle=float(rng.uniform(0, 2 * math.pi)), shift=(0.1, 0.0), n_transients=40,
                  snr=(3.0, 100.0), transient_sep=16.0, transient_margin=20, n_cosmics=25, n_colsegs=2,
                  n_misreg=40, misreg_shift=(0.3, 1.0), mask_fraction=float(rng.uniform(0.0, 0.15)))
    return _truth(d, 512, 512)


def exposure_pair(index):
    """CCD `index` of the 60-CCD exposure (2048 x 4096)."""
    from synth import config_pair
    return _truth(config_pair("c4", index), 4096, 2048)


def generate(fn, indices, procs=None):
    procs = procs or max(1, min(16, len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else 4))
    with mp.get_context("spawn").Pool(procs) as pool:
        return pool.map(fn, indices, chunksize=max(1, len(indices) // (4 * procs)))


# ---------------------------------------------------------------- GPU subtraction + detection
def candidates(pairs, chunk=16, max_cand=512, thresh=5.0, device="cuda"):
    """Subtract every pair (batched plans), detect on each D and gather the
    stamps.  Returns stamps (device, [n][3][31][31]), snr, xy, ccd index and
    the PSF FWHM of each candidate's CCD."""
    import torch
    from .binding import Detector, Plan
    H, W = pairs[0]["R"].shape
    det = Detector(H, W, batch=1, max_cand=max_cand, device=device)
    stamps, snr, xy, ccd = [], [], [], []
    plans = {}
    for c0 in range(0, len(pairs), chunk):
        part = pairs[c0:c0 + chunk]
        B = len(part)
        if B not in plans:
            plans[B] = Plan(H, W, L, DK, DB, batch=B, prec="mixed", device=device)
        plan = plans[B]
        R = torch.from_numpy(np.stack([p["R"] for p in part])).to(device)
        S = torch.from_numpy(np.stack([p["S"] for p in part])).to(device)
        bad = torch.from_numpy(np.stack([p["bad"] for p in part])).to(device)
        out = plan.subtract(R, S, bad, None, refine=1)
        for i, p in enumerate(part):
            xyi, snri, cnt, st = det(out["D"][i:i + 1], S[i:i + 1], R[i:i + 1], bad[i:i + 1],
                                     psf_sigma=p["psf_sigma"], thresh=thresh, guard=GUARD)
            n = min(int(cnt[0].item()), max_cand)
            stamps.append(st[0, :n].clone())
            snr.append(snri[0, :n].cpu().numpy())
            xy.append(xyi[0, :n].cpu().numpy())
            ccd.append(np.full(n, c0 + i))
        if (out["info"] != 0).any():
            raise RuntimeError(f"subtraction status {out['info'].tolist()}")
    fwhm = np.array([p["fwhm_S"] for p in pairs])
    ccd = np.concatenate(ccd)
    return {"stamps": torch.cat(stamps), "snr": np.concatenate(snr), "xy": np.concatenate(xy), "ccd": ccd,
            "fwhm": fwhm[ccd]}


KINDS = ("transient", "cosmic", "column", "misregistered", "other")


def label(cands, pairs):
    """1 for a candidate within 2 px of an injected transient, else 0; plus the
    artifact kind it lies on (for the per-kind rejection rates)."""
    n = len(cands["ccd"])
    lab = np.zeros(n, np.float32)
    kind = np.full(n, 4, np.int32)
    for i in range(n):
        p = pairs[cands["ccd"][i]]
        x, y = cands["xy"][i]
        t = p["transients"]
        if t.size and np.min(np.hypot(t[:, 0] - x, t[:, 1] - y)) <= MATCH_PX:
            lab[i], kind[i] = 1.0, 0
            continue
        c = p["cosmics"]
        if c.size and np.min(np.hypot(c[:, 0] - x, c[:, 1] - y)) <= 3.0:
            kind[i] = 1
            continue
        s = p["colsegs"]
        if s.size and np.any((np.abs(s[:, 0] - x) <= 2) & (y >= s[:, 1] - 3) & (y <= s[:, 2] + 3)):
            kind[i] = 2
            continue
        m = p["misreg"]
        if m.size and np.min(np.hypot(m[:, 0] - x, m[:, 1] - y)) <= 3.0:
            kind[i] = 3
    return lab, kind


# ---------------------------------------------------------------- training / scoring
def train(model, stamps, labels, epochs=5, batch=256, lr=1e-3, seed=500, log=None):
    import torch
    dev = stamps.device
    lab = torch.as_tensor(labels, dtype=torch.float32, device=dev)
    g = torch.Generator(device="cpu").manual_seed(seed)
    n = stamps.shape[0]
    loss = torch.empty(1, dtype=torch.float32, device=dev)
    hist = []
    for ep in range(epochs):
        perm = torch.randperm(n, generator=g).to(dev)
        tot, cnt = 0.0, 0
        for b0 in range(0, n - batch + 1, batch):
            idx = perm[b0:b0 + batch]
            model.train_step(stamps.index_select(0, idx).contiguous(), lab.index_select(0, idx).contiguous(), lr,
                             loss=loss)
            if (b0 // batch) % 50 == 0:
                tot += float(loss.item())
                cnt += 1
        hist.append(tot / max(cnt, 1))
        if log:
            log(f"epoch {ep + 1}: mean sampled loss {hist[-1]:.4f}")
    return hist


def scores(model, stamps):
    return model.score(stamps.contiguous()).cpu().numpy()


def cut_flags(stamps, snr, fwhm, ccd, snr_min=5.0, adaptive=False):
    """The SNR/shape cuts per CCD (its PSF FWHM); adaptive=True sizes the
    sources with Gaussian-weighted adaptive moments."""
    import torch
    from .binding import shape_cuts
    out = np.zeros(len(snr), np.int32)
    snr_t = torch.as_tensor(snr, dtype=torch.float32, device=stamps.device)
    for c in np.unique(ccd):
        sel = np.nonzero(ccd == c)[0]
        idx = torch.as_tensor(sel, device=stamps.device)
        out[sel] = shape_cuts(stamps.index_select(0, idx).contiguous(), snr_t.index_select(0, idx).contiguous(),
                              float(fwhm[sel[0]]), snr_min, adaptive=adaptive).cpu().numpy()
    return out


def rates(flag, lab):
    real, bogus = lab == 1, lab == 0
    return {"completeness": float(flag[real].mean()) if real.any() else None,
            "fpr": float(flag[bogus].mean()) if bogus.any() else None,
            "n_real": int(real.sum()), "n_bogus": int(bogus.sum())}


def judge(sc, cuts, lab, kind, cuts_adaptive=None):
    """Rates at 0.3 / 0.6, the cuts' rates, and the gain at matched operating
    points; with cuts_adaptive, the same comparison against the cuts whose
    size comes from adaptive moments (under "adaptive_cuts")."""
    if cuts_adaptive is not None:
        out = judge(sc, cuts, lab, kind)
        alt = judge(sc, cuts_adaptive, lab, kind)
        out["adaptive_cuts"] = {k: alt[k] for k in ("cuts", "cnn_fpr_at_cuts_completeness",
                                                     "cnn_completeness_at_cuts_fpr", "cuts_rejection_by_kind")
                                if k in alt}
        return out
    out = {"cnn_0.3": rates(sc >= 0.3, lab), "cnn_0.6": rates(sc >= 0.6, lab), "cuts": rates(cuts == 1, lab)}
    real, bogus = sc[lab == 1], sc[lab == 0]
    cc, cf = out["cuts"]["completeness"], out["cuts"]["fpr"]
    if real.size and bogus.size:
        t = np.quantile(real, 1.0 - cc) if cc is not None else 0.5           # CNN threshold at the cuts' completeness
        out["cnn_fpr_at_cuts_completeness"] = float((bogus >= t).mean())
        t2 = np.quantile(bogus, 1.0 - cf) if cf else 1.0                     # CNN threshold at the cuts' FPR
        out["cnn_completeness_at_cuts_fpr"] = float((real >= t2).mean()) if cf else float((real > bogus.max()).mean())
        # ROC area by ranks
        allv = np.concatenate([real, bogus])
        r = allv.argsort().argsort().astype(np.float64) + 1
        out["cnn_auc"] = float((r[:real.size].sum() - real.size * (real.size + 1) / 2) / (real.size * bogus.size))
    out["rejection_by_kind_0.3"] = {KINDS[k]: float((sc[kind == k] < 0.3).mean()) for k in range(1, 5)
                                    if (kind == k).any()}
    out["cuts_rejection_by_kind"] = {KINDS[k]: float((cuts[kind == k] == 0).mean()) for k in range(1, 5)
                                     if (kind == k).any()}
    return out


def balanced_split(lab, seed=500, frac=(0.8, 0.05, 0.15)):
    """Indices of a class-balanced 80/5/15 split (the larger class is subsampled)."""
    rng = np.random.default_rng(seed)
    pos, neg = np.nonzero(lab == 1)[0], np.nonzero(lab == 0)[0]
    k = min(pos.size, neg.size)
    pos, neg = rng.permutation(pos)[:k], rng.permutation(neg)[:k]
    out = []
    a = 0
    for f in frac:
        b = a + int(round(f * k))
        out.append(rng.permutation(np.concatenate([pos[a:b], neg[a:b]])))
        a = b
    return out


def run(train_ccds=3000, epochs=5, batch=256, lr=1e-3, eval_ccds=60, seed=500, log=print, arch="small"):
    import torch
    from .binding import RBModel, RIModel
    t0 = time.time()
    tr_pairs = generate(train_pair, list(range(seed, seed + train_ccds)))
    ev_pairs = generate(exposure_pair, list(range(eval_ccds))) if eval_ccds else []
    t_gen = time.time() - t0
    log(f"generated {len(tr_pairs)} training pairs and {len(ev_pairs)} exposure pairs in {t_gen:.1f} s")
    t1 = time.time()
    ctr = candidates(tr_pairs, chunk=32)
    lab, kind = label(ctr, tr_pairs)
    torch.cuda.synchronize()
    t_cand = time.time() - t1
    log(f"training candidates: {len(lab)} ({int(lab.sum())} real) in {t_cand:.1f} s")
    i_tr, i_va, i_te = balanced_split(lab, seed)
    model = (RBModel(max_batch=max(batch, 1024), seed=seed) if arch == "small"
             else RIModel(max_batch=max(batch, 512), seed=seed))
    st = ctr["stamps"]
    dev = st.device
    take = lambda idx: st.index_select(0, torch.as_tensor(idx, device=dev)).contiguous()   # noqa: E731
    t2 = time.time()
    hist = train(model, take(i_tr), lab[i_tr], epochs=epochs, batch=batch, lr=lr, seed=seed, log=log)
    torch.cuda.synchronize()
    t_train = time.time() - t2
    steps = epochs * (len(i_tr) // batch)
    report = {"arch": arch, "train": {"ccds": train_ccds, "candidates": int(len(lab)), "real": int(lab.sum()),
                        "split": [int(len(i_tr)), int(len(i_va)), int(len(i_te))], "epochs": epochs, "batch": batch,
                        "lr": lr, "steps": steps, "seconds": t_train, "stamps_per_s": steps * batch / t_train,
                        "loss_by_epoch": hist}}
    for name, idx in (("validation", i_va), ("test", i_te)):
        sc = scores(model, take(idx))
        cuts = cut_flags(take(idx), ctr["snr"][idx], ctr["fwhm"][idx], ctr["ccd"][idx])
        cuts_a = cut_flags(take(idx), ctr["snr"][idx], ctr["fwhm"][idx], ctr["ccd"][idx], adaptive=True)
        report[name] = judge(sc, cuts, lab[idx], kind[idx], cuts_a)
    if ev_pairs:
        t3 = time.time()
        cev = candidates(ev_pairs, chunk=10, max_cand=4096)
        lab_e, kind_e = label(cev, ev_pairs)
        t4 = time.time()
        sc = scores(model, cev["stamps"])
        torch.cuda.synchronize()
        t_inf = time.time() - t4
        cuts = cut_flags(cev["stamps"], cev["snr"], cev["fwhm"], cev["ccd"])
        cuts_a = cut_flags(cev["stamps"], cev["snr"], cev["fwhm"], cev["ccd"], adaptive=True)
        report["exposure"] = judge(sc, cuts, lab_e, kind_e, cuts_a)
        report["exposure"]["ccds"] = eval_ccds
        report["exposure"]["candidates"] = int(len(lab_e))
        report["exposure"]["subtract_detect_seconds"] = t4 - t3
        report["exposure"]["inference_stamps_per_s"] = len(lab_e) / max(t_inf, 1e-9)
    report["seconds"] = {"generate": t_gen, "candidates": t_cand, "train": t_train, "total": time.time() - t0}
    return report, model


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--train-ccds", type=int, default=3000)
    ap.add_argument("--eval-ccds", type=int, default=60)
    ap.add_argument("--epochs", type=int, default=5)
    ap.add_argument("--batch", type=int, default=256)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--seed", type=int, default=500)
    ap.add_argument("--out", default=None)
    ap.add_argument("--weights", default=None, help="save the trained weights (float32 .npy)")
    ap.add_argument("--arch", choices=["small", "ri"], default="small",
                    help="small: three-convolution network; ri: the paper's rotation-invariant residual network")
    a = ap.parse_args(argv)
    report, model = run(a.train_ccds, a.epochs, a.batch, a.lr, a.eval_ccds, a.seed,
                        log=lambda s: print(s, file=sys.stderr, flush=True), arch=a.arch)
    js = json.dumps(report, indent=1)
    print(js)
    if a.out:
        with open(a.out, "w") as fh:
            fh.write(js)
    if a.weights:
        np.save(a.weights, model.get_weights())
    return 0


if __name__ == "__main__":
    sys.exit(main())

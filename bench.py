#!/usr/bin/env python
"""Throughput benchmark of the difference-imaging path on synthetic
DECam-shaped CCD pairs (2048 x 4096, L = 11, D_K = D_B = 2).

One step = one full subtraction of one CCD pair per GPU: masks and sky
offsets, Fourier-domain normal-matrix assembly, FP64 Cholesky solve, one
image-space refinement step and the convolve-and-subtract.  Prints one JSON
line (rank 0).  `--impl reference` times the FP64 CPU oracle instead, on a
bounded strip of the same workload.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import time

_CORES = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)
for _v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ.setdefault(_v, str(_CORES))

import numpy as np  # noqa: E402

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "SFFT CCD-pairs/sec (2k×4k, L=11, D_K=2), mixed vs FP64 at stated error; HBM %"
UNIT = "CCD-pairs/s"
H, W, L, DK, DB = 4096, 2048, 11, 2, 2
REFINE = 1
L2_FLUSH_BYTES = 256 << 20
WORKLOAD = ("one DECam CCD pair per GPU per step: 2048x4096 FP32, 20k stars, PSF FWHM 1.0-1.4 (R) / "
            "1.5-2.1 (S) px across the chip, saturation mask with 3 px dilation, two bad columns, "
            "50 transients; L=11, D_K=D_B=2, mixed precision, 1 refinement step")
# DRAM bytes (read + write) of one full-size KK contraction launch (all 221
# differences), from a one-pass ncu capture of the benchmark workload
# (profiles/k_contract_*.md); reported only while the kernel source is the
# one that was measured.  Keys: the kernel's source file.
KK_TRAFFIC = {
    "kernels_contract.cu": (10.09e9, "1a847c15ebf73406"),      # FP32 FMA kernel (--fma-contract)
    "kernels_contract_tc.cu": (None, ""),                      # mma.sync kernel (--mma-sync-contract)
    "kernels_contract_umma.cu": (9.975e9, "0d3c235754a7a213"),  # tcgen05, one lane per (d, u_y) pair
    # tcgen05, one lane per difference (default)
    "kernels_contract_dlane.cu": (8.786e9, "a0e1779911e29c9d"),
}
PHASES = ("prep", "fft_weights", "fft_prod", "contract_kk", "contract_rk", "scatter", "solve", "apply", "lag_dft")


def half_plane_lag_rows(L):
    """sum over half-plane kernel-offset differences d of (L - |d_y|): the number
    of (d, u_y) pairs the product-spectrum contraction evaluates."""
    return sum((L - dy) * (L if dy == 0 else 2 * L - 1) for dy in range(L))


def kk_flops_per_ccd(H, W, L, DK):
    """Algorithmic FP32 work of the KK contraction for one CCD: for every (d, u_y)
    pair, interior row y and packed spectrum slot k, (2 D_K + 1) complex products
    conj(V_a) P (6 flop each) and n_mono(2 D_K) complex accumulations scaled by
    yt^b (4 flop each, FMA = 2 flop)."""
    M = max(64, 1 << (W - 1).bit_length()) // 2
    DM = 2 * DK
    per = (DM + 1) * 6 + (DM + 1) * (DM + 2) // 2 * 4
    return half_plane_lag_rows(L) * (H - (L - 1)) * M * per


def kk_traffic_bytes(src):
    import hashlib
    val, want = KK_TRAFFIC.get(src, (None, ""))
    path = os.path.join(ROOT, "paper_2603_08593_gb300", "csrc", src)
    try:
        h = hashlib.sha256(open(path, "rb").read()).hexdigest()[:16]
    except OSError:
        return None
    return val if (val is not None and h == want) else None


def kk_gemm_flops_per_ccd(H, W, L, DK):
    """Algorithmic work of the KK contraction in its matrix-product form, one
    CCD: per k-slot a real product of (monomial x Re/Im) rows, (2 x rows x
    re/im) inner dimension and (d, u_y) columns, i.e. 8 flop per complex
    multiply-add conj(W_m) P over every monomial, (d, u_y) pair, interior
    row and complex spectrum slot (the packed real slot excluded)."""
    M = max(64, 1 << (W - 1).bit_length()) // 2
    return 8 * n_mono(2 * DK) * half_plane_lag_rows(L) * (H - (L - 1)) * (M - 1)


def n_mono(D):
    return (D + 1) * (D + 2) // 2


def phase_bytes(H, W, L, DK, DB, refine=1):
    """Algorithmic HBM bytes per CCD of each streaming phase: every kernel's
    inputs read once and its outputs written once (FP32 path).  A spectrum
    slab is H x M complex64 with M = max(64, 2^ceil(log2 W)) / 2."""
    M = max(64, 1 << (W - 1).bit_length()) // 2
    px, slab = H * W, H * M * 8
    n_hd = half_plane_differences(L)
    n_wa = 2 * DK + 1
    return {
        # sky sums (R, S, bad), masks and R_m (R, S, bad in; good, R_m out), two
        # erosion passes (1 B in, 1 B out each), background moments (M_fit, S;
        # and M_fit, e per refinement step)
        "prep": px * (9 + 14 + 4 + 5 + 5 * refine),
        # weight spectra (M_fit in), right-hand-side spectra (M_fit, S in),
        # R_m spectrum, refinement right-hand sides (M_fit, e in)
        "fft_weights": px * (1 + 5 + 4 + 5 * refine) + slab * (n_wa + (DK + 1) * (1 + refine) + 1),
        # R_m in, one spectrum slab per half-plane difference out
        "fft_prod": px * 4 + slab * n_hd,
        # product and weight spectra in, k-slot products C[k][d][u_y][32] FP32 out
        "contract_kk": slab * (n_hd + n_wa) + M * n_hd * L * 32 * 4,
        # k-slot products in
        "lag_dft": M * n_hd * L * 32 * 4,
        # R_m spectrum against the weight spectra (KB) and the right-hand-side
        # spectra (b_K, and again per refinement step)
        "contract_rk": slab * ((1 + n_wa) + (1 + DK + 1) * (1 + refine)),
        # residual pass (R, S, M_fit in; e out) and the final pass (R, S in; D out)
        "apply": px * (13 * refine + 12),
    }


def half_plane_differences(L):
    return L + (L - 1) * (2 * L - 1)


# Roofline denominators when no measured file is present: one earlier GB300
# measurement (copy 6.8 TB/s, cuBLAS BF16 1.9 PFLOP/s in a burst and about
# 1.7 sustained).
FALLBACK_PEAKS = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}


def measured_peaks():
    """(peaks, source): the measured copy bandwidth and BF16 GEMM rates from
    MEASURED_PEAKS.json, or FALLBACK_PEAKS with source "fallback"."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            peaks = json.load(f)
        if all(k in peaks for k in FALLBACK_PEAKS):
            return peaks, "measured"
    except (OSError, ValueError):
        pass
    return dict(FALLBACK_PEAKS), "fallback"


def tf32_peak_tflops(sustained=True):
    """Dense TF32 tensor peak from the BF16 GEMM peak (measured, else the
    fallback) and the nominal TF32 : BF16 ratio (1.1 : 2.25 PFLOP/s)."""
    peaks, _ = measured_peaks()
    bf16 = peaks["bf16_tflops_sustained" if sustained else "bf16_tflops"]
    return bf16 * 1.1 / 2.25


def fp32_alu_peak_tflops(clock_mhz):
    """152 SMs x 128 FP32 lanes x 2 flop per FMA x SM clock."""
    return 152 * 128 * 2 * clock_mhz * 1e6 / 1e12


# ------------------------------------------------------------------ clocks
class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", "200", "-i", str(self.index)], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
        except (FileNotFoundError, OSError):
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                self.out, _ = self.proc.communicate()

    def summary(self):
        if self.proc is None:
            return None
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in (self.out or "").strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 8:
                continue
            try:
                sm.append(float(f[0])); mx.append(float(f[1]))
            except ValueError:
                continue
            for n, v in zip(names, f[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)), "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------------------------ CPU oracle baseline
def oracle_strip_seconds(d, rows):
    """Time the FP64 oracle (definition form, solve, apply) on the first `rows`
    rows of the pair; returns (seconds, strip fraction)."""
    from oracle import sfft_oracle as O
    R = d["R"][:rows]; S = d["S"][:rows]; bad = d["bad"][:rows]
    t0 = time.perf_counter()
    out = O.fit(R, S, bad, L, DK, DB)
    dt = time.perf_counter() - t0
    assert out["status"] == O.STATUS_OK
    return dt, rows / float(H)


def cpu_model():
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True).stdout
        for line in out.splitlines():
            if line.startswith("Model name"):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return "unknown"


# ------------------------------------------------------------------ reference arm
def run_reference(args):
    from synth import config_pair
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    d = config_pair("c2")
    rows = args.ref_rows
    for _ in range(args.warmup):
        oracle_strip_seconds(d, rows)
    times = []
    for _ in range(args.steps):
        dt, frac = oracle_strip_seconds(d, rows)
        times.append(dt / frac)
    sec_per_ccd = float(np.mean(times))
    v = 1.0 / sec_per_ccd
    sample = (f"FP64 NumPy/SciPy oracle (definition-form normal equations, Cholesky, FP64 apply) on the first "
              f"{rows} of 4096 rows of the CCD pair, scaled by 4096/{rows} to CCD-pairs/s")
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": sec_per_ccd * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD, "H": H, "W": W, "L": L, "DK": DK, "DB": DB},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": _CORES, "kind": "oracle", "sample": sample,
                             "cpu": cpu_model()},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------ GPU arm
def _c4_pair(index):
    from synth import config_pair
    d = config_pair("c4", index)
    return {k: d[k] for k in ("R", "S", "bad", "transients", "masked_fraction")}


def load_pairs(args, rank):
    """The step's CCD pairs: the C2/C3 pair (or a shorter strip of the same
    recipe for profiling captures), or `batch` CCDs of one C4 exposure.
    Replica ranks draw independent pairs from the same recipe."""
    from synth import config_pair, make_pair
    from synth.decam import SAT_CLIP_ADU
    if args.batch > 1:
        import multiprocessing as mp
        idx = [60 * rank + i for i in range(args.batch)]
        with mp.get_context("spawn").Pool(max(1, min(16, _CORES))) as pool:
            return pool.map(_c4_pair, idx)
    if rank == 0 and args.rows == H:
        return [config_pair("c2")]
    return [make_pair(args.rows, W, seed=2 + 1000 * rank, n_src=max(1, 20000 * args.rows // H),
                      fwhm_R=(1.0, 1.4), fwhm_S=(1.5, 2.1), shift=(0.1, 0.0), n_transients=50,
                      snr=(5.0, 50.0), clip=SAT_CLIP_ADU, mask_saturated=True, bad_columns=(700, 1500))]


def _subtract_steps(plan, R, S, bad, out, n, stream, flush=None, events=None):
    for i in range(n):
        if flush is not None:
            flush.fill_(i & 0xff)                           # evict L2 between timed steps
        if events is not None:
            events[i][0].record(stream)
        plan.subtract(R, S, bad, None, refine=REFINE, out=out)
        if events is not None:
            events[i][1].record(stream)


def _max_over_ranks(dist, dev, x):
    import torch
    if dist is None:
        return x
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


CNN_FWD_FLOP = 2.0 * (961 * 27 * 32 + 225 * 288 * 64 + 49 * 576 * 64 + 576 * 128 + 128)   # per stamp
# the rotation-invariant residual network: four rotations through conv1, two
# 32 -> 32 convolutions, conv2 and two 64 -> 64 convolutions; one dense head
CNN_RI_FWD_FLOP = 2.0 * (4 * (961 * 27 * 32 + 2 * 225 * 288 * 32 + 225 * 288 * 64 + 2 * 49 * 576 * 64)
                         + 576 * 128 + 128)


CONV_TIME_KINDS = ("cta", "copy_wait_empty", "build_wait_stage", "build_wait_empty", "build_work", "mma_wait_full",
                   "mma_wait_acc_empty", "mma_issue", "epilogue_wait_full", "epilogue_work")
CONV_TIME_WARPS = (1, 1, 4, 4, 4, 1, 1, 1, 4, 4)   # warps whose lane 0 adds to each counter


def conv_waits(reset):
    """Time attribution of the fused classifier convolutions per layer, as
    fractions of the CTAs' run per warp of each role; None unless the library
    was built with -DRBTC_WAIT_PROFILE (rb_debug_conv_waits)."""
    import ctypes
    from paper_2603_08593_gb300 import binding
    lib = binding.load()
    buf = (ctypes.c_uint64 * 16)()
    res = {}
    for layer in (1, 2, 3):
        if lib.rb_debug_conv_waits(layer, buf, 1 if reset else 0) != 0:
            return None
        cta = max(int(buf[0]), 1)
        res[f"conv{layer}"] = {k: round(int(buf[i]) / (cta * CONV_TIME_WARPS[i]), 4)
                               for i, k in enumerate(CONV_TIME_KINDS) if i and buf[i]}
    return res


def time_classifier(dev, n_infer=32768, batch=256, steps=40, arch="small"):
    """Stamp-classifier throughput on synthetic 31 x 31 x 3 stamps: inference
    (normalise + forward + sigmoid) and training steps (forward, backward, Adam),
    CUDA-event timed; flop rates count the network's multiply-adds only.
    arch "small": the three-convolution network; "ri": the paper's
    rotation-invariant residual network."""
    import torch
    from paper_2603_08593_gb300 import RBModel, RIModel
    from synth.stamps import make_stamps
    d = make_stamps(4096, seed=77)
    base = torch.from_numpy(d["stamps"]).to(dev)
    lab = torch.from_numpy(d["labels"]).to(dev)
    stamps = base.repeat((n_infer + 4095) // 4096, 1, 1, 1)[:n_infer].contiguous()
    m = RBModel(max_batch=4096, seed=1) if arch == "small" else RIModel(max_batch=1024, seed=1)
    fwd = CNN_FWD_FLOP if arch == "small" else CNN_RI_FWD_FLOP
    out = torch.empty(n_infer, dtype=torch.float32, device=dev)
    st = torch.cuda.current_stream(dev)
    m.score(stamps, out=out)
    waits = conv_waits(reset=True) if arch == "small" else None
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    for _ in range(3):
        m.score(stamps, out=out)
    e1.record(st)
    e1.synchronize()
    inf_s = e0.elapsed_time(e1) / 1e3 / 3
    if waits is not None:   # a build with the convolutions' time attribution compiled in
        waits = conv_waits(reset=True)
    tb = base[:batch].contiguous()
    tl = lab[:batch].contiguous()
    loss = torch.empty(1, dtype=torch.float32, device=dev)
    m.train_step(tb, tl, 1e-3, loss=loss)
    e0.record(st)
    for _ in range(steps):
        m.train_step(tb, tl, 1e-3, loss=loss)
    e1.record(st)
    e1.synchronize()
    tr_s = e0.elapsed_time(e1) / 1e3 / steps
    inf_rate = n_infer / inf_s
    out = {"inference_stamps_per_s": inf_rate, "train_stamps_per_s": batch / tr_s,
           "inference_tflops": inf_rate * fwd / 1e12,
           "train_tflops": 3 * fwd * batch / tr_s / 1e12}
    if arch == "small":
        from paper_2603_08593_gb300 import binding
        out["note"] = (f"synthetic stamps; inference on {n_infer} stamps in batches of {m.max_batch}: exact-median "
                       "normalisation, the three convolutions fused with bias, ReLU and max-pool on tcgen05 "
                       "(BF16, FP32 accumulation in tensor memory), the dense layers on mma.sync; training batch "
                       f"{batch} on mma.sync; flops = network multiply-adds x 2 (training = 3 x forward)")
        # the convolutions' MMAs read both operands from shared memory: their
        # cost by N bounds the fused kernels (conv1 issues N = 128, conv2 and
        # conv3 N = 64)
        out["umma_cycles_per_mma"] = {str(n): binding.probe_umma_cycles(n) for n in (32, 64, 128, 256)}
        if waits is not None:
            out["conv_time_attribution"] = waits
    else:
        out["note"] = (f"synthetic stamps; inference on {n_infer} stamps in batches of {m.max_batch}, training batch "
                       f"{batch}; BF16 mma.sync GEMMs with FP32 accumulation, flops = network multiply-adds x 2 "
                       "(training = 3 x forward)")
    return out


def measured_alu_peaks():
    """FP32 and FP64 FMA peaks of this GPU in TFLOP/s, measured by the
    library's FMA-chain probe (sfft_probe_fma_peak)."""
    from paper_2603_08593_gb300 import binding
    return {"fp32_tflops": binding.probe_fma_peak(False), "fp64_tflops": binding.probe_fma_peak(True),
            "how": "sfft_probe_fma_peak: 8 independent FMA chains per thread, 8 x 256 threads per SM, CUDA events"}


def time_fma_engine(dev, stream, R, S, bad, Hs, args, alu_peaks, steps=3):
    """The same subtraction with the KK contraction on the FP32 FMA pipes:
    CCD-pairs/s and the contraction's FP32 ALU roofline (derived peak)."""
    import torch
    from paper_2603_08593_gb300 import Plan
    with torch.cuda.stream(stream):
        p = Plan(Hs, W, L, DK, DB, batch=1, prec="mixed", stream=stream, device=dev, fma_contract=True)
        o = p.subtract(R, S, bad, None, refine=REFINE)
        stream.synchronize()
        p.profile(True)
        p.profile_read(reset=True)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            p.subtract(R, S, bad, None, refine=REFINE, out=o)
        e1.record(stream)
        stream.synchronize()
        prof = p.profile_read(reset=True)
    sec = e0.elapsed_time(e1) / 1e3 / steps
    kk_ms = prof["contract_kk"][0] / steps
    flop = kk_flops_per_ccd(Hs, W, L, DK)
    peak = alu_peaks["fp32_tflops"]
    out = {"value": 1.0 / sec, "unit": UNIT, "ms_per_step": sec * 1e3, "steps": steps,
           "contract_kk_ms": kk_ms, "alu_tflops": flop / (kk_ms * 1e-3) / 1e12,
           "alu_frac": flop / (kk_ms * 1e-3) / 1e12 / peak, "alu_peak_tflops": peak,
           "peak_note": "FP32 FMA peak of measured (sfft_probe_fma_peak, this run)",
           "status": [int(v) for v in o["info"].cpu()],
           "note": "the KK lag contraction on the FP32 FMA pipes (SFFT_FLAG_FMA_CONTRACT), tensor cores used by "
                   "the stamp classifier only; phase timing adds events inside the step"}
    del p, o
    torch.cuda.empty_cache()
    return out


def time_exposure(dev, stream, pairs, args, dist, steps=3, warmup=2):
    """A whole exposure (len(pairs) CCD pairs of the 60-CCD recipe) per GPU in
    one graph-captured sfft_subtract call, plan autotuned at creation."""
    import torch
    from paper_2603_08593_gb300 import Plan
    B = len(pairs)
    R = torch.from_numpy(np.stack([p["R"] for p in pairs])).to(dev).contiguous()
    S = torch.from_numpy(np.stack([p["S"] for p in pairs])).to(dev).contiguous()
    bad = torch.from_numpy(np.stack([p["bad"] for p in pairs])).to(dev).contiguous()
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    with torch.cuda.stream(stream):
        plan = Plan(H, W, L, DK, DB, batch=B, prec="mixed", stream=stream, device=dev, graph=True, autotune=1)
        out = plan.subtract(R, S, bad, None, refine=REFINE)
        for _ in range(warmup - 1):
            plan.subtract(R, S, bad, None, refine=REFINE, out=out)
        stream.synchronize()
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize(dev)
        with ClockSampler(dev.index) as clk:
            _subtract_steps(plan, R, S, bad, out, steps, stream, flush, evs)
            stream.synchronize()
    sec = _max_over_ranks(dist, dev, sum(a.elapsed_time(b) for a, b in evs) / 1e3)
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rec = {"value": world * B * steps / sec, "unit": UNIT, "ccd_pairs_per_gpu_per_step": B, "steps": steps,
           "warmup": warmup, "ms_per_step": 1e3 * sec / steps, "ms_per_ccd": 1e3 * sec / steps / B,
           "tiles": {"d_batch": plan.tiles[0], "rows_per_cta": plan.tiles[1], "lag_parts": plan.tiles[2],
                     "ccd_group": plan.ccd_group},
           "kk_engine": plan.engine, "clocks": clk.summary(),
           "status": [int(v) for v in out["info"].cpu()],
           "masked_fraction": [float(p["masked_fraction"]) for p in pairs],
           "workload": (f"{B} CCD pairs of one DECam exposure (2048x4096 FP32 each, seeds 100+, independent PSF "
                        "gradients, masked fractions 2-30 %, cosmics, bleed trails) in one CUDA-graph-captured "
                        "sfft_subtract call; L=11, D_K=D_B=2, mixed, 1 refinement step; 256 MB L2 flush between "
                        "steps")}
    del plan, out, R, S, bad, flush
    torch.cuda.empty_cache()
    return rec


def run_gpu(args):
    import torch
    from paper_2603_08593_gb300 import Plan

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    pairs = load_pairs(args, rank)                          # before the first CUDA call (spawned pool)
    expo_pairs = None
    if args.batch == 1 and args.rows == H and args.exposure_ccds > 0:
        import multiprocessing as mp
        idx = [60 * rank + i for i in range(args.exposure_ccds)]
        with mp.get_context("spawn").Pool(max(1, min(16, _CORES))) as pool:
            expo_pairs = pool.map(_c4_pair, idx)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    B, Hs = len(pairs), pairs[0]["R"].shape[0]
    batched = B > 1

    cpu_base = None
    if rank == 0 and not args.no_cpu_baseline:
        dt, frac = oracle_strip_seconds(pairs[0], args.cpu_rows)
        cpu_base = {"value": frac / dt, "unit": UNIT, "cores": _CORES, "kind": "oracle",
                    "sample": (f"FP64 NumPy/SciPy oracle (definition-form normal equations, Cholesky, FP64 apply) "
                               f"on the first {args.cpu_rows} of 4096 rows of one CCD pair, {dt:.1f} s, "
                               f"scaled to CCD-pairs/s"),
                    "cpu": cpu_model()}

    stream = torch.cuda.Stream(device=dev)
    alu_peaks = measured_alu_peaks()
    R = torch.from_numpy(np.stack([p["R"] for p in pairs])).to(dev).contiguous()
    S = torch.from_numpy(np.stack([p["S"] for p in pairs])).to(dev).contiguous()
    bad = torch.from_numpy(np.stack([p["bad"] for p in pairs])).to(dev).contiguous()
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    torch.cuda.synchronize(dev)
    with torch.cuda.stream(stream):
        plan = Plan(Hs, W, L, DK, DB, batch=B, prec=args.prec, stream=stream, device=dev, d_batch=args.d_batch,
                    graph=batched, autotune=0 if args.no_autotune else 1, lag_parts=args.lag_parts,
                    fma_contract=args.fma_contract, mma_sync_contract=args.mma_sync_contract,
                    pair_lane_contract=args.pair_lane_contract)
        tiles = plan.tiles
        engine = plan.engine
        if batched:
            # per-phase times and launch counts from an eager profiled pass of the same plan
            eager = Plan(Hs, W, L, DK, DB, batch=B, prec=args.prec, stream=stream, device=dev,
                         d_batch=tiles[0], rows_per_cta=tiles[1], lag_parts=tiles[2], fma_contract=args.fma_contract,
                         mma_sync_contract=args.mma_sync_contract, pair_lane_contract=args.pair_lane_contract)
            eo = eager.subtract(R, S, bad, None, refine=REFINE)
            eager.profile(True)
            eager.profile_read(reset=True)
            _subtract_steps(eager, R, S, bad, eo, 1, stream)
            stream.synchronize()
            prof1 = eager.profile_read(reset=True)
            prof = {k: (v[0] * args.steps, v[1] * args.steps) for k, v in prof1.items()}
            del eager, eo
        out = plan.subtract(R, S, bad, None, refine=REFINE)
        _subtract_steps(plan, R, S, bad, out, max(args.warmup - 1, 0), stream)
        stream.synchronize()
        info = [int(v) for v in out["info"].cpu()]
        if not batched:
            plan.profile(True)
            plan.profile_read(reset=True)
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize(dev)
        with ClockSampler(local) as clk:
            t0 = time.perf_counter()
            _subtract_steps(plan, R, S, bad, out, args.steps, stream, flush, evs)
            stream.synchronize()
            wall = time.perf_counter() - t0
        if not batched:
            prof = plan.profile_read(reset=True)
            plan.profile(False)
    step_ms = [a.elapsed_time(b) for a, b in evs]
    dev_s = _max_over_ranks(dist, dev, sum(step_ms) / 1e3)
    value = world * B * args.steps / dev_s

    # end to end through the public API: pinned host inputs in, difference images and theta out
    e2e = None
    if not args.no_e2e:
        hR = torch.from_numpy(R.cpu().numpy()).pin_memory(); hS = torch.from_numpy(S.cpu().numpy()).pin_memory()
        hb = torch.from_numpy(bad.cpu().numpy()).pin_memory()
        hD = torch.empty(tuple(out["D"].shape), dtype=torch.float32).pin_memory()
        hth = torch.empty(tuple(out["theta"].shape), dtype=torch.float64).pin_memory()
        hinfo = torch.empty((B,), dtype=torch.int32).pin_memory()
        with torch.cuda.stream(stream):
            ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            for it in range(args.steps + 1):
                if it == 1:
                    ev0.record(stream)
                R.copy_(hR, non_blocking=True); S.copy_(hS, non_blocking=True); bad.copy_(hb, non_blocking=True)
                plan.subtract(R, S, bad, None, refine=REFINE, out=out)
                hD.copy_(out["D"], non_blocking=True); hth.copy_(out["theta"], non_blocking=True)
                hinfo.copy_(out["info"], non_blocking=True)
            ev1.record(stream)
            stream.synchronize()
        e_s = _max_over_ranks(dist, dev, ev0.elapsed_time(ev1) / 1e3)
        e2e = {"value": world * B * args.steps / e_s, "unit": UNIT,
               "h2d_bytes_per_step": int(hR.numel() * 4 + hS.numel() * 4 + hb.numel()),
               "d2h_bytes_per_step": int(hD.numel() * 4 + hth.numel() * 8 + hinfo.numel() * 4)}
    del plan, out
    torch.cuda.empty_cache()

    # the plain FP64 GPU path on the same pairs, one CCD per call, for comparison
    fp64 = None
    if args.fp64_steps > 0 and args.prec == "mixed":
        n64 = min(args.fp64_steps, B) if batched else args.fp64_steps
        with torch.cuda.stream(stream):
            p64 = Plan(Hs, W, L, DK, DB, batch=1, prec="fp64", stream=stream, device=dev)
            o64 = p64.subtract(R[:1], S[:1], bad[:1], None, refine=REFINE)
            stream.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for i in range(n64):
                j = i % B
                p64.subtract(R[j:j + 1], S[j:j + 1], bad[j:j + 1], None, refine=REFINE, out=o64)
            e1.record(stream)
            stream.synchronize()
        s64 = _max_over_ranks(dist, dev, e0.elapsed_time(e1) / 1e3)
        fp64 = {"value": world * n64 / s64, "unit": UNIT, "ms_per_ccd": 1e3 * s64 / n64, "ccds_timed": n64,
                "note": "plain FP64 GPU path (FP64 FFTs, products and contraction), sequential single-CCD calls"}
        del p64, o64

    # the KK contraction on the FP32 FMA pipes (tensor cores left to the stamp classifier), same pair
    fma_rec = None
    if not batched and not args.no_fma_engine and args.prec == "mixed" and not args.fma_contract:
        fma_rec = time_fma_engine(dev, stream, R, S, bad, Hs, args, alu_peaks)
    # the 60-CCD exposure in one graph-captured call, per GPU
    expo = None
    if expo_pairs is not None:
        expo = time_exposure(dev, stream, expo_pairs, args, dist)
        del expo_pairs

    classifier = None
    if not args.no_classifier and rank == 0:
        classifier = time_classifier(dev)
        classifier["rotation_invariant_residual"] = time_classifier(dev, n_infer=8192, arch="ri")

    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return 0
    launches = sum(n for _, n in prof.values())
    kk_ms, kk_n = prof["contract_kk"]
    roof = None
    clocks = clk.summary()
    if kk_n:
        on_tc = args.prec == "mixed" and not args.fma_contract
        # the contract_kk phase holds one contraction launch per batch of offset
        # differences on the tensor-core engines (their lag DFT and exact
        # slot-0 sums are the lag_dft phase); the FP32 FMA engine adds its
        # k_contract_slot0 companion to the same phase
        n_launch = kk_n if on_tc else kk_n / 2
        avg_ms = kk_ms / n_launch
        full = Hs == H and B == 1 and tiles[0] == 221
        if on_tc:
            # the split-operand product runs the matrix product once in TF32
            # (hi x hi) and once more as two BF16 corrections at twice the TF32
            # rate: 2 x F at the TF32 rate is the time the tensor cores need
            per_launch_flop = 2 * B * kk_gemm_flops_per_ccd(Hs, W, L, DK) / (n_launch / args.steps)
            achieved = per_launch_flop / (avg_ms * 1e-3) / 1e12
            peak = tf32_peak_tflops(sustained=True)
            kname, ksrc = {
                "mma_sync": ("k_contract_tc (lag contraction as split TF32/BF16 mma.sync products)",
                             "kernels_contract_tc.cu"),
                "tcgen05_pair_lane": ("k_contract_umma (lag contraction as split TF32/BF16 tcgen05 products, one "
                                      "TMEM lane per (d, u_y) pair)", "kernels_contract_umma.cu"),
                "tcgen05_difference_lane": ("k_contract_dlane (lag contraction as split TF32/BF16 tcgen05 products, "
                                            "one TMEM lane per difference, u_y shifts from weight-row strips)",
                                            "kernels_contract_dlane.cu"),
            }[engine]
            roof = {"bound": "tensor", "kernel": kname,
                    "achieved": achieved / 2, "peak": peak, "unit": "TFLOP/s", "frac": achieved / 2 / peak,
                    "traffic": args.traffic if args.traffic is not None else (kk_traffic_bytes(ksrc) if full else None),
                    "peak_note": f"dense TF32 tensor peak of {measured_peaks()[1]} = sustained cuBLAS BF16 "
                                 "(MEASURED_PEAKS.json) x 1.1/2.25 (nominal TF32:BF16); achieved counts the method's "
                                 "matrix-product flops F once",
                    "hardware_tflops": achieved,
                    "hardware_note": "2 F per launch / duration: the split operands run every product once as TF32 "
                                     "(hi*hi) and once as two BF16 corrections at twice the TF32 rate",
                    "algorithmic_flop_per_launch": per_launch_flop / 2,
                    "avg_launch_ms": avg_ms, "launches_per_step": n_launch / args.steps,
                    "traffic_note": "DRAM read+write bytes per launch, one-pass ncu capture of this workload"}
        else:
            per_launch_flop = B * kk_flops_per_ccd(Hs, W, L, DK) / (n_launch / args.steps)
            achieved = per_launch_flop / (avg_ms * 1e-3) / 1e12
            peak = alu_peaks["fp32_tflops"]
            roof = {"bound": "alu", "kernel": "k_contract (product-spectrum lag contraction, FP32 FMA)",
                    "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                    "traffic": args.traffic if args.traffic is not None else (kk_traffic_bytes("kernels_contract.cu") if full else None),
                    "peak_note": "FP32 FMA peak of measured (sfft_probe_fma_peak, this run)",
                    "avg_launch_ms": avg_ms, "launches_per_step": n_launch / args.steps,
                    "traffic_note": "DRAM read+write bytes per launch, one-pass ncu capture of this workload"}
        if batched:
            roof["timing_note"] = "kernel durations from an eager profiled pass of the same plan (timed steps replay a CUDA graph)"
    hbm = None
    if prof and not batched and args.prec == "mixed":
        peaks, psrc = measured_peaks()
        pk = peaks["hbm_gbs"]
        hbm = {"peak_gbs": pk, "peak_note": f"STREAM-style copy of {psrc} (MEASURED_PEAKS.json)",
               "note": "per CCD: algorithmic bytes (each kernel's inputs read once, outputs written once) / phase "
                       "time (CUDA events around the phase's kernels)"}
        for k, nbytes in phase_bytes(Hs, W, L, DK, DB, REFINE).items():
            ms = prof[k][0] / args.steps
            if ms > 0:
                gbs = nbytes / (ms * 1e-3) / 1e9
                hbm[k] = {"bytes": nbytes, "ms": ms, "gbs": gbs, "frac": gbs / pk}
    solve_rec = None
    if prof.get("solve") and prof["solve"][0] > 0:
        Nn = L * L * n_mono(DK) + n_mono(DB)
        # Cholesky N^3 / 3 multiply-adds, and two triangular solves (N^2 each) for the
        # solution and for the refinement step
        flop = B * (2.0 * Nn ** 3 / 3.0 + (1 + REFINE) * 2 * 2.0 * Nn * Nn)
        ms = prof["solve"][0] / args.steps
        fp64_solve = args.prec == "fp64"
        peak = alu_peaks["fp64_tflops"] if fp64_solve else alu_peaks["fp32_tflops"]
        solve_rec = {"ms": ms, "flop": flop, "tflops": flop / (ms * 1e-3) / 1e12,
                     "frac": flop / (ms * 1e-3) / 1e12 / peak, "peak_tflops": peak,
                     "note": ("FP64 solve phase (factorisation, substitutions, units) against the measured FP64 FMA "
                              "peak" if fp64_solve else
                              "solve phase of the mixed path: Cholesky of the Jacobi-scaled system and the "
                              "substitutions in FP32, the solution refined against the FP64 system by the "
                              "image-space refinement step; against the measured FP32 FMA peak (latency-bound)")}
    if batched:
        workload = (f"{B} CCD pairs of one DECam exposure per GPU per step (2048x4096 FP32 each, independent PSF "
                    f"gradients, masked fractions 2-30 %, cosmics, bleed trails) in one CUDA-graph-captured call; "
                    f"L=11, D_K=D_B=2, {args.prec}, 1 refinement step")
    elif Hs != H:
        workload = f"profiling strip: {Hs}x{W} rows of the DECam pair recipe (not the headline workload)"
    else:
        workload = WORKLOAD
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * dev_s / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64" if args.prec == "mixed" else "f64",
            "data": "synthetic",
            "config": {"workload": workload, "H": Hs, "W": W, "L": L, "DK": DK, "DB": DB, "prec": args.prec,
                       "refine": REFINE, "ccd_pairs_per_gpu_per_step": B, "parallelism": f"replicas x{world}",
                       "cuda_graph": batched, "autotune": not args.no_autotune,
                       "tiles": {"d_batch": tiles[0], "rows_per_cta": tiles[1], "lag_parts": tiles[2]},
                       "kk_engine": engine,
                       "l2": "256 MB buffer written between timed steps (L2 flushed)"},
            "roofline": roof, "cpu_baseline": cpu_base, "e2e": e2e, "gpu_launches": launches,
            "clocks": clocks, "status": info, "wall_s": wall, "fp64_path": fp64, "classifier": classifier,
            "hbm": hbm, "fma_engine": fma_rec, "exposure": expo, "alu_peaks": alu_peaks, "solve": solve_rec,
            "phases_ms_per_step": {k: v[0] / args.steps for k, v in prof.items()}}
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-rows", type=int, default=512, help="rows of the CCD the CPU oracle baseline runs on")
    ap.add_argument("--ref-rows", type=int, default=256, help="rows per reference-arm step")
    ap.add_argument("--traffic", type=float, default=None, help="ncu DRAM bytes per contraction launch, if known")
    ap.add_argument("--prec", choices=["mixed", "fp64"], default="mixed")
    ap.add_argument("--batch", type=int, default=1, help="CCD pairs per call; > 1 runs the C4 exposure batch")
    ap.add_argument("--rows", type=int, default=H, help="rows per CCD (4096; fewer only for profiling captures)")
    ap.add_argument("--d-batch", type=int, default=0, help="offset differences per workspace slab (0: plan default)")
    ap.add_argument("--fp64-steps", type=int, default=2, help="CCDs timed on the plain FP64 path for comparison")
    ap.add_argument("--no-autotune", action="store_true", help="plan defaults instead of plan-time tile tuning")
    ap.add_argument("--no-classifier", action="store_true", help="skip the stamp-classifier throughput figures")
    ap.add_argument("--no-fma-engine", action="store_true", help="skip the FP32 FMA contraction engine figure")
    ap.add_argument("--exposure-ccds", type=int, default=60,
                    help="CCDs of the exposure sub-record (one graph-captured call; 0 skips it)")
    ap.add_argument("--only-classifier", action="store_true", help="print only the stamp-classifier figures")
    ap.add_argument("--lag-parts", type=int, default=0, choices=[0, 1, 2, 3], help="contraction lag parts (0: plan's)")
    ap.add_argument("--fma-contract", action="store_true",
                    help="mixed path: KK contraction on the FP32 FMA pipes instead of the tensor cores")
    ap.add_argument("--mma-sync-contract", action="store_true",
                    help="mixed path: tensor-core KK contraction through mma.sync instead of tcgen05")
    ap.add_argument("--pair-lane-contract", action="store_true",
                    help="tcgen05 contraction with one TMEM lane per (difference, u_y) pair")
    args = ap.parse_args()
    if args.only_classifier:   # classifier figures alone (profiling captures)
        import torch
        dev = torch.device("cuda", 0)
        print(json.dumps({"classifier": time_classifier(dev),
                          "rotation_invariant_residual": time_classifier(dev, n_infer=8192, arch="ri")}), flush=True)
        return 0
    if args.impl == "reference":
        return run_reference(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())

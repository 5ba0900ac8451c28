"""The benchmark's work counts, which the roofline figures divide by, against
brute-force enumeration of what the lag contraction evaluates (CPU only).

For a kernel of L x L offsets u = (u_y, u_x), |u_y|, |u_x| <= w = (L - 1) / 2,
the normal matrix needs, for every offset difference d = u - u' of the half
plane (d_y > 0, or d_y = 0 and d_x >= 0), the lags u_y for which both u and
u - d lie in the window (Sec. 2.3, the delta-basis normal equations).
"""
import importlib.util
import os

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _pairs_brute(L):
    w = (L - 1) // 2
    n = 0
    for dy in range(-(L - 1), L):
        for dx in range(-(L - 1), L):
            if not (dy > 0 or (dy == 0 and dx >= 0)):
                continue
            # u_y with u_y and u_y - d_y both in [-w, w]
            n += sum(1 for uy in range(-w, w + 1) if -w <= uy - dy <= w)
    return n


@pytest.mark.parametrize("L", [3, 5, 7, 9, 11])
def test_lag_rows_match_brute_force(bench, L):
    assert bench.half_plane_lag_rows(L) == _pairs_brute(L)


def test_decam_contraction_work(bench):
    # 2048 x 4096 pair, L = 11, D_K = 2: 221 half-plane differences, 1276 (d, u_y)
    # pairs, 15 monomials of degree <= 4, 4086 interior rows, 1023 complex slots
    assert bench.half_plane_lag_rows(11) == 1276
    assert sum(1 for dy in range(11) for dx in range(-10, 11) if dy > 0 or dx >= 0) == 221
    assert bench.n_mono(4) == 15
    F = bench.kk_gemm_flops_per_ccd(4096, 2048, 11, 2)
    assert F == 8 * 15 * 1276 * 4086 * 1023
    assert abs(F - 6.40e11) < 0.01e11


def test_tf32_peak_from_measured_bf16(bench):
    import json
    peaks, src = bench.measured_peaks()
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        assert src == "measured"
        assert peaks["bf16_tflops_sustained"] == json.load(open(path))["bf16_tflops_sustained"]
    else:
        assert src == "fallback" and peaks == bench.FALLBACK_PEAKS
    assert bench.tf32_peak_tflops(sustained=True) == pytest.approx(peaks["bf16_tflops_sustained"] * 1.1 / 2.25)


def test_peaks_fall_back_without_measured_file(bench, monkeypatch, tmp_path):
    """Without MEASURED_PEAKS.json the roofline denominators are the fallback
    figures, labelled as such."""
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    peaks, src = bench.measured_peaks()
    assert src == "fallback" and peaks["hbm_gbs"] == 6800.0
    assert bench.tf32_peak_tflops(sustained=True) == pytest.approx(1700.0 * 1.1 / 2.25)

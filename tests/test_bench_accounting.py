"""The roofline accounting of bench.py (CPU): the algorithmic bytes and
flops per launch that the reported `achieved` figures divide by, checked
against the closed forms they stand for."""
import json
import math
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402

HW = 4096 * 4096
SIX = [2.0, 4.0, 8.0, 16.0, 32.0, 48.0]


def test_fir_taps_are_five_sigma_capped():
    # K = ceil(5 sigma), sigma = lambda / 2, at most 96 (the colored-SG blur, L_D = 1)
    assert bench.fir_taps(SIX) == [5, 10, 20, 40, 80, 96]
    assert bench.fir_taps([48.0], kmax=160) == [120]


def test_two_pass_bytes_per_pixel_scale():
    """Row pass: read the frame, write S planes; column pass: read the S
    planes.  Per pixel-scale: s_in / S + 2 s_b (8.67 B at f32, S = 6)."""
    S = 6
    row, _ = bench.algorithmic("iir_row", S, HW, [], 4.0, 4.0)
    col, _ = bench.algorithmic("iir_coldet", S, HW, [], 4.0, 4.0)
    assert abs((row + col) / (S * HW) - (4.0 / 6 + 8.0)) < 1e-12
    # 16-bit planes halve the plane terms
    row16, _ = bench.algorithmic("fir_row", S, HW, [], 2.0, 2.0)
    assert row16 == 2.0 * HW + 2.0 * S * HW


def test_fir_flops_are_the_tap_sums():
    """2(2K + 1) flop per output and scale: 17.0 GFLOP for the six scales of
    the 4096^2 frame."""
    taps = bench.fir_taps(SIX)
    _, flops = bench.algorithmic("fir_coldet", 6, HW, taps)
    assert flops == 2.0 * sum(2 * k + 1 for k in taps) * HW == 2.0 * 508 * HW
    assert abs(flops / 1e9 - 17.05) < 0.01


def test_d5_bytes():
    """W x (H + 4) channel planes, S = 4, 15 channels (the D = 5 profile's
    algorithmic column)."""
    H = W = 2048
    P = (H + 4) * W
    q = {k: bench.quartic_bytes(k, 4, H, W) for k in ("iir_row", "iir_colseg", "iir_coldet", "quartic_hpf")}
    assert q["iir_row"] == 15 * (4 * P + 16 * P)
    assert q["iir_colseg"] == 15 * 16 * P
    assert q["iir_coldet"] == 15 * (16 * P + 16 * H * W)
    assert q["quartic_hpf"] == 4 * H * W + 60 * P
    assert [round(q[k] / 1e6, 1) for k in ("iir_row", "iir_coldet", "iir_colseg", "quartic_hpf")] == \
        [1260.7, 2015.2, 1008.6, 268.9]
    assert bench.quartic_bytes("k_unknown", 4, H, W) is None


def test_peaks_follow_the_measured_file():
    """HBM: the measured copy rate (else the 6.8 TB/s fallback); TF32: the
    sustained bf16 GEMM rate times the nominal TF32/bf16 ratio 1.1 / 2.25."""
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    hbm, src = bench.peaks()
    tf32, tsrc = bench.tf32_peak()
    if os.path.exists(path):
        m = json.load(open(path))
        assert (hbm, src) == (float(m["hbm_gbs"]), "measured")
        assert math.isclose(tf32, float(m["bf16_tflops_sustained"]) * 1.1 / 2.25)
        assert tsrc.startswith("measured")
    else:
        assert (hbm, src) == (6800.0, "fallback")
        assert math.isclose(tf32, 1700.0 * 1.1 / 2.25)

"""The roofline accounting of bench.py (CPU): the algorithmic bytes and
flops per launch that the reported `achieved` figures divide by, checked
against the closed forms they stand for."""
import json
import math
import os
import sys

import pytest

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


def test_method_work_counted_once_on_the_tensor_pass():
    """The tensor-core FIR column pass is credited with the method's
    2(2K + 1) flop per output and scale, not the three TF32 products that
    emulate each FP32 product: 17.05 GFLOP in 0.5488 ms is 31.1 TFLOP/s."""
    taps = bench.fir_taps(SIX)
    _, flops = bench.algorithmic("fir_coldet", 6, HW, taps)
    r = bench.roofline_of("fir_coldet", 0.5488 * 20, 20, 4.0 * 6 * HW * 20, flops * 20, 6792.1, "measured",
                          152, 2070.0, None)
    assert r["bound"] == "tensor" and r["tf32_products_per_tap"] == 3
    assert abs(r["achieved"] - 31.07) < 0.05
    tp, _ = bench.tf32_peak()
    assert abs(r["frac"] - r["achieved"] / tp) < 1e-4
    # the FP32 row pass against the ALU peak of the device's SM count
    r2 = bench.roofline_of("fir_row", 0.4272, 1, 4.0 * HW * 7, flops, 6792.1, "measured", 152, 2070.0, None)
    assert r2["bound"] == "alu" and abs(r2["peak"] - 80.6) < 0.1
    assert abs(r2["achieved"] - flops / 0.4272e-3 / 1e12) < 1e-3
    assert "hbm_frac" in r2


def test_alu_peak_follows_the_sm_count():
    assert abs(bench.alu_peak(152, 2070.0) - 152 * 128 * 2 * 2.07e9 / 1e12) < 1e-9
    assert abs(bench.alu_peak(148, 1965.0) / bench.alu_peak(152, 1965.0) - 148 / 152) < 1e-12


def test_bank_bytes_per_pixel_scale():
    """2 s_b + s_in / S per pixel-scale: 8.667 B at f32 with S = 6, 4.25 B at
    f16 planes and u16 input with S = 8."""
    assert abs(bench.bank_bytes(6, HW, 4.0, 4.0) / (6 * HW) - (8.0 + 4.0 / 6)) < 1e-12
    assert abs(bench.bank_bytes(8, HW, 2.0, 2.0) / (8 * HW) - 4.25) < 1e-12


def test_hbm_roofline_of_a_plane_pass():
    """A pass with bytes and no flops is HBM-bound: achieved GB/s over the
    measured copy peak."""
    r = bench.roofline_of("iir_coldet", 0.3036, 1, 4.0 * 6 * HW, 0.0, 6792.1, "measured", 152, 2070.0, 457.5e6)
    assert r["bound"] == "hbm" and r["unit"] == "GB/s"
    assert abs(r["achieved"] - 4.0 * 6 * HW / 0.3036e-3 / 1e9) < 0.1
    assert r["traffic"] == 457.5e6


def test_traffic_needs_a_capture_of_the_current_sources(tmp_path, monkeypatch):
    """A stored ncu traffic figure is reported only while the kernel sources
    still have the digest of the capture."""
    (tmp_path / "a.cu").write_text("kernel A")
    monkeypatch.setattr(bench, "CSRC", str(tmp_path))
    d = bench.csrc_digest()
    monkeypatch.setattr(bench, "MEASURED_TRAFFIC", {("w", "k", "f32"): (123.0, d)})
    assert bench.traffic_of("w", "k", "f32") == 123.0
    assert bench.traffic_of("w", "other", "f32") is None
    (tmp_path / "a.cu").write_text("kernel A, changed")
    assert bench.csrc_digest() != d
    assert bench.traffic_of("w", "k", "f32") is None


def test_shape_overrides_pick_the_bank_and_pass():
    spec = "iir.row=-2,iir.det=-2,fir.row=-3"
    assert bench.shape_overrides(spec, "iir_repeated_pole_order4") == [("row", -2), ("det", -2)]
    assert bench.shape_overrides(spec, "fir_colored_sg") == [("row", -3)]
    assert bench.shape_overrides(None, "fir_colored_sg") == []
    with pytest.raises(ValueError):
        bench.shape_overrides("iir.col=1", "iir_repeated_pole_order4")


def test_digest_follows_code_not_comments(tmp_path, monkeypatch):
    """A comment-only edit keeps the source digest (the stored traffic stays
    valid); an edit of the code, even inside a string literal, changes it."""
    monkeypatch.setattr(bench, "CSRC", str(tmp_path))
    src = tmp_path / "k.cu"
    src.write_text('// a kernel\n__global__ void k(float *p) { p[0] = 1.f; /* one */ }\nconst char *s = "// x";\n')
    d = bench.csrc_digest()
    src.write_text('// a kernel, reworded\n__global__ void k(float *p) {\n  p[0] = 1.f;  // one\n}\nconst char *s = "// x";\n')
    assert bench.csrc_digest() == d
    src.write_text('// a kernel\n__global__ void k(float *p) { p[0] = 2.f; }\nconst char *s = "// x";\n')
    assert bench.csrc_digest() != d
    src.write_text('// a kernel\n__global__ void k(float *p) { p[0] = 1.f; }\nconst char *s = "// y";\n')
    assert bench.csrc_digest() != d

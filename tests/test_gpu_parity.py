"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle on
the same seeded synthetic inputs.  Bar: per-scale max|err|/range <= 1e-5 for
the responses; blob lists identical for every blob whose margin exceeds that
tolerance (north star of the filter bank, FP32 path)."""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_1912_07133_gb300 import synthetic as S
from tests.parity import TOL, compare_blobs, gpu_bank, oracle_bank, scale_errors

pytestmark = pytest.mark.gpu

D, E, C, A = 0, 1, 2, 3
SIX = [2.0, 4.0, 8.0, 16.0, 32.0, 48.0]


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__ as g
    g.build()


# ---------------------------------------------------------------------------
# designs (FP64 kernel) against the oracle's designs
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("order", [3, 4])
@pytest.mark.parametrize("lam", [2.0, 4.0, 16.0, 48.0, 64.0])
def test_design_repeated_pole_matches_oracle_at_the_realised_pole(order, lam):
    from paper_1912_07133_gb300 import kf
    g = kf.kf_design(kf.KF_IIR_REPEATED_POLE, order, lam)
    p32 = float(np.float32(math.exp(-2.0 / lam)))      # the GPU realises the FP32 pole
    o = O.design_repeated_pole(1, order - 1, -1.0 / math.log(p32))
    np.testing.assert_allclose(g["aplus"], o["aplus"], rtol=1e-12, atol=1e-15)
    sc = np.abs(o["bplus"]).max()
    np.testing.assert_allclose(g["bplus"], o["bplus"], rtol=0, atol=1e-9 * sc)
    assert g["b0"] == pytest.approx(o["b0"], abs=1e-9 * sc)
    assert g["dc_gain"] == pytest.approx(1.0, abs=1e-9)


@pytest.mark.parametrize("lam", [2.0, 4.0, 16.0, 48.0])
def test_design_butterworth_matches_oracle(lam):
    from paper_1912_07133_gb300 import kf
    g = kf.kf_design(kf.KF_IIR_BUTTERWORTH, 2, lam)
    o = O.design_butterworth(1, lam / 2)
    assert g["param"] == pytest.approx(o["omega_c"], rel=1e-14)
    np.testing.assert_allclose(g["aplus"], o["aplus"], rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(g["bplus"], o["bplus"], rtol=1e-9, atol=1e-14)
    assert g["b0"] == pytest.approx(o["b0"], rel=1e-9)


@pytest.mark.parametrize("lam", [2.0, 4.0, 8.0, 16.0, 32.0, 48.0])
def test_design_colored_sg_matches_oracle(lam):
    from paper_1912_07133_gb300 import kf
    g = kf.kf_design(kf.KF_FIR_COLORED_SG, 1, lam)
    o = O.design_colored_sg_mp(1, O.sg_half_length(1, lam / 2, 96), 6.0 / lam)
    assert len(g["h"]) == len(o)
    np.testing.assert_allclose(g["h"], o, rtol=0, atol=1e-12 * np.abs(o).max())


@pytest.mark.parametrize("lam", [1.0, 2.0, 4.0, 8.0, 16.0, 32.0, 48.0, 64.0])
def test_design_gaussian_matches_oracle(lam):
    """Filter A taps (eqs 9, 11) designed on the GPU in FP64 equal the oracle's."""
    from paper_1912_07133_gb300 import kf
    g = kf.kf_design(kf.KF_FIR_GAUSSIAN, 1, lam)
    o = O.design_gaussian(lam / 2, 96)
    assert len(g["h"]) == len(o) == min(int(np.ceil(2.5 * lam)), 96) + 1
    np.testing.assert_allclose(g["h"], o, rtol=1e-14, atol=0)
    assert g["dc_gain"] == pytest.approx(1.0, abs=1e-14)


def test_design_rejects_invalid_parameters():
    from paper_1912_07133_gb300 import kf
    for args in [(kf.KF_IIR_REPEATED_POLE, 1, 4.0), (kf.KF_IIR_REPEATED_POLE, 3, 0.0),
                 (kf.KF_IIR_REPEATED_POLE, 3, -2.0), (kf.KF_FIR_COLORED_SG, 1, 1.8),
                 (kf.KF_FIR_COLORED_SG, 3, 8.0), (kf.KF_FIR_GAUSSIAN, 2, 8.0), (7, 3, 4.0)]:
        with pytest.raises(kf.KfError) as e:
            kf.kf_design(*args)
        assert e.value.code == kf.KF_EINVAL


# ---------------------------------------------------------------------------
# responses and blob lists
# ---------------------------------------------------------------------------
def _check(frame, scales, ftype, order, T=0.05, neigh=0):
    (Rg,), blobs = gpu_bank([frame], scales, ftype, order, T, neigh)
    Ro = oracle_bank(frame, scales, ftype, order)
    errs = scale_errors(Rg, Ro)
    assert max(errs) <= TOL, errs
    return compare_blobs(blobs, Ro, T, neigh), errs


def test_tiny_single_scale_frame():
    """512 x 512, one scale (lambda 4), 3rd-order repeated-pole blur."""
    img = S.tiny_frame(seed=0)
    (nref, ngot, ndiff), errs = _check(img, [4.0], D, 3)
    assert nref >= 15 and ngot >= 15


@pytest.mark.parametrize("ftype,order", [(D, 4), (D, 3), (E, 2), (C, 1), (A, 1)])
def test_six_scales_ragged_frame(ftype, order):
    img = S.iir_fir_frame(seed=5, H=777, W=1000, nblobs=30)
    _check(img, SIX, ftype, order)


@pytest.mark.parametrize("ftype,order", [(D, 4), (C, 1), (A, 1)])
def test_adjacent_scale_neighbourhood(ftype, order):
    img = S.iir_fir_frame(seed=6, H=300, W=333, nblobs=10)
    _check(img, SIX, ftype, order, neigh=1)


@pytest.mark.parametrize("H,W", [(1, 1), (1, 37), (37, 1), (2, 3), (31, 33), (65, 130), (129, 31),
                                 (70, 4099)])
@pytest.mark.parametrize("ftype,order", [(D, 3), (E, 2), (C, 1), (A, 1)])
def test_small_and_degenerate_shapes(H, W, ftype, order):
    rng = np.random.default_rng(H * 1000 + W)
    img = rng.uniform(0, 1, (H, W)).astype(np.float32)
    (Rg,), blobs = gpu_bank([img], [4.0, 7.0], ftype, order, 0.05)
    Ro = oracle_bank(img, [4.0, 7.0], ftype, order)
    for s in range(2):
        # inputs are O(1): responses below 1e-3 in range are compared absolutely
        assert np.abs(Rg[s] - Ro[s]).max() <= TOL * max(np.ptp(Ro[s]), 1e-3)
    if H * W > 1:
        compare_blobs(blobs, Ro, 0.05)


def test_constant_frame_has_no_response_and_no_blobs():
    img = np.full((100, 120), 0.7, np.float32)
    (Rg,), blobs = gpu_bank([img], SIX, D, 4)
    assert np.abs(Rg).max() < 1e-4
    assert len(blobs) == 0


def test_two_frames_of_different_sizes_in_one_call():
    f0 = S.tiny_frame(seed=11, H=200, W=300, nblobs=8)
    f1 = S.tiny_frame(seed=12, H=333, W=150, nblobs=8)
    (R0, R1), blobs = gpu_bank([f0, f1], [4.0, 8.0], D, 3)
    for k, (f, Rg) in enumerate(((f0, R0), (f1, R1))):
        Ro = oracle_bank(f, [4.0, 8.0], D, 3)
        assert max(scale_errors(Rg, Ro)) <= TOL
        compare_blobs(blobs, Ro, 0.05, frame=k)
    assert set(np.unique(blobs["frame"])) <= {0, 1}


def test_rethreshold_filters_and_keeps_order():
    img = S.iir_fir_frame(seed=9, H=512, W=640, nblobs=25)
    (Rg,), b05 = gpu_bank([img], SIX, D, 4, 0.05)
    import torch
    from paper_1912_07133_gb300 import kf
    bank = kf.Bank(0)
    bank.run([torch.from_numpy(img).cuda()], SIX, kf.KF_IIR_REPEATED_POLE, 4, threshold=0.05)
    b2 = bank.blobs(threshold=0.2)
    bank.close()
    expect = b05[np.abs(b05["response"]) > 0.2]
    assert np.array_equal(b2, expect)


def test_runs_are_bitwise_repeatable():
    img = S.iir_fir_frame(seed=7, H=256, W=512, nblobs=10)
    (Ra,), ba = gpu_bank([img], SIX, D, 4)
    (Rb,), bb = gpu_bank([img], SIX, D, 4)
    assert np.array_equal(Ra, Rb)
    assert np.array_equal(ba, bb)


# ---------------------------------------------------------------------------
# full size: one 4096 x 4096 frame, six scales (the benchmarked workload)
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("ftype,order", [(D, 4), (C, 1), (A, 1)])
def test_full_size_4096_six_scales(ftype, order):
    img = S.iir_fir_frame()
    (nref, ngot, ndiff), errs = _check(img, SIX, ftype, order)
    assert nref > 500


# ---------------------------------------------------------------------------
# error paths
# ---------------------------------------------------------------------------
def test_api_errors_are_reported():
    import torch
    from paper_1912_07133_gb300 import kf
    x = torch.zeros(16, 16, device="cuda")
    bank = kf.Bank(0)
    with pytest.raises(kf.KfError) as e:
        bank.run([x], [4.0], kf.KF_IIR_REPEATED_POLE, 9)
    assert e.value.code == kf.KF_EINVAL
    with pytest.raises(kf.KfError) as e:
        bank.run([x], [4.0] * 17, kf.KF_IIR_REPEATED_POLE, 3)
    assert e.value.code == kf.KF_EINVAL
    bank.run([x], [4.0], kf.KF_IIR_REPEATED_POLE, 3, threshold=0.1)
    with pytest.raises(kf.KfError) as e:
        bank.blobs(threshold=0.05)            # below the bank threshold
    assert e.value.code == kf.KF_EINVAL
    assert len(bank.blobs(threshold=0.2)) == 0
    bank.close()


def test_candidate_overflow_raises_capacity():
    """A list that does not fit returns KF_EOVERFLOW with the needed count."""
    import ctypes
    import torch
    from paper_1912_07133_gb300 import kf
    img = S.iir_fir_frame(seed=8, H=512, W=512, nblobs=20)
    x = torch.from_numpy(img).cuda()
    bank = kf.Bank(0)
    bank.run([x], SIX, kf.KF_IIR_REPEATED_POLE, 4, threshold=0.0)
    full = bank.blobs()
    out = (kf.kf_blob * 4)()
    n = ctypes.c_int64(0)
    rc = kf.load().kf_detect_blobs(bank.ctx, 0.0, out, 4, ctypes.byref(n))
    assert rc == kf.KF_EOVERFLOW and n.value == len(full) > 4
    # the first four records are the head of the ordered list
    assert [(b.scale, b.y, b.x) for b in out] == [(int(r["scale"]), int(r["y"]), int(r["x"]))
                                                  for r in full[:4]]
    bank.close()


def test_device_candidate_list_overflow_grows_capacity():
    """More candidates than the context's device list: KF_ERERUN with the
    count, capacity raised; the next run returns the complete ordered list."""
    import torch
    from paper_1912_07133_gb300 import kf
    img = np.random.default_rng(3).uniform(0, 1, (4096, 4096)).astype(np.float32)
    x = torch.from_numpy(img).cuda()
    bank = kf.Bank(0)
    bank.run([x], [2.0, 3.0], kf.KF_IIR_REPEATED_POLE, 3, threshold=0.0)
    with pytest.raises(kf.KfError) as e:
        kf.kf_detect_blobs(bank.ctx, 0.0)
    assert e.value.code == kf.KF_ERERUN
    bank.run([x], [2.0, 3.0], kf.KF_IIR_REPEATED_POLE, 3, threshold=0.0)
    b = bank.blobs()
    # the wrapper repeats an overflowed run by itself: a fresh context gives the same list
    bank2 = kf.Bank(0)
    bank2.run([x], [2.0, 3.0], kf.KF_IIR_REPEATED_POLE, 3, threshold=0.0)
    b2 = bank2.blobs()
    bank2.close()
    assert np.array_equal(b, b2)
    assert len(b) > (1 << 20)
    keys = b["scale"].astype(np.int64) * 4096 * 4096 + b["y"].astype(np.int64) * 4096 + b["x"]
    assert np.all(np.diff(keys) > 0)
    bank.close()

"""Reduced-precision inputs and intermediate storage against the FP64 oracle.

* Input frames of f16, bf16 and u16 (with a value scale) are converted to f32
  on load: against the oracle run on the same quantised values the FP32 bar
  (1e-5 x per-scale range, exact blob lists beyond that margin) holds.
* 16-bit planes between the row and column passes (f16 / bf16, FP32 state
  and accumulation): the error against the oracle is bounded a priori.  A
  plane value q = sigma^2 blur_x(L) is rounded with relative error <= u
  (u = 2^-11 for f16, 2^-8 for bf16; f16 adds an absolute 2^-25 below its
  normal range), |q| <= sigma^2 |h|_1 (max|U| + max|V|), and the column blur
  carries an error of at most |h|_1 times that into R; the FP32 part adds
  the 1e-5 x range of the f32 path.  |h|_1 is the l1 norm of the 1-D blur's
  impulse response (Sec. 4 designs, from the oracle).
* The 8192^2 12-bit counts workload, cut to 512^2 with its 8 scales: the
  error is reported twice, against the oracle on the exact u16 input and on
  the quantised input (f16 holds integers exactly only to 2048, bf16 to 256).
"""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_1912_07133_gb300 import synthetic as SY
from tests.parity import TOL, compare_blobs, gpu_bank, oracle_bank, scale_errors

pytestmark = pytest.mark.gpu

D, E, C = 0, 1, 2
F32, F16, BF16, U16 = 0, 1, 2, 3
SIX = [2.0, 4.0, 8.0, 16.0, 32.0, 48.0]
UNIT = {F16: 2.0 ** -11, BF16: 2.0 ** -8}
SUB = {F16: 2.0 ** -25, BF16: 0.0}


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__ as g
    g.build()


def h_l1(ftype, order, lam):
    """l1 norm of the symmetric 1-D blur of one scale (oracle designs)."""
    sigma = lam / 2.0
    if ftype == C:
        h = O.design_colored_sg_mp(order, O.sg_half_length(order, sigma, 96), 3.0 / sigma)
        return abs(h[0]) + 2.0 * np.abs(h[1:]).sum()
    d = (O.design_repeated_pole(1, order - 1, sigma) if ftype == D
         else O.design_butterworth(order - 1, sigma))
    n = int(40 * sigma) + 200
    x = np.zeros(2 * n + 1)
    x[n] = 1.0
    y = O.iir1d(x, d["K"], d["b0"], d["bplus"], d["aplus"], boundary=O.BOUNDARY_ZERO)
    return float(np.abs(y).sum())


def second_differences_max(img):
    """max|U| + max|V| of the edge-held frame (U = d2/dx2, V = d2/dy2)."""
    p = np.pad(np.asarray(img, np.float64), 1, mode="edge")
    U = p[1:-1, 2:] - 2 * p[1:-1, 1:-1] + p[1:-1, :-2]
    V = p[2:, 1:-1] - 2 * p[1:-1, 1:-1] + p[:-2, 1:-1]
    return float(np.abs(U).max() + np.abs(V).max())


def storage_bounds(img, scales, ftype, order, storage, Ro):
    """Per-scale a-priori bound on max|R_gpu - R_oracle| / range for 16-bit planes."""
    M = second_differences_max(img)
    out = []
    for s, lam in enumerate(scales):
        h1 = h_l1(ftype, order, lam)
        sig2 = (lam / 2.0) ** 2
        qmax = sig2 * h1 * M
        rng = max(np.ptp(Ro[s]), 1e-300)
        out.append((h1 * (UNIT[storage] * qmax + SUB[storage])) / rng + TOL)
    return out


# ---------------------------------------------------------------------------
# input element types (f32 planes): the FP32 bar on the quantised values
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("ftype,order", [(D, 4), (E, 2), (C, 1)])
@pytest.mark.parametrize("dtype", [F16, BF16, U16])
def test_reduced_precision_inputs_meet_the_fp32_bar(dtype, ftype, order):
    import torch
    if dtype == U16:
        counts = SY.counts_frame(seed=11, H=203, W=331, nblobs=12)
        vs = 1.0 / 4095.0
        frame, exact = counts, counts.astype(np.float64) * np.float64(np.float32(vs))
    else:
        img = SY.iir_fir_frame(seed=12, H=203, W=331, nblobs=12)
        vs = 1.0
        if dtype == F16:
            frame = img.astype(np.float16)
            exact = frame.astype(np.float64)
        else:
            frame = torch.from_numpy(img).to(torch.bfloat16)
            exact = frame.to(torch.float64).numpy()
    scales = [2.0, 4.0, 8.0, 16.0]
    (Rg,), blobs = gpu_bank([frame], scales, ftype, order, 0.05, value_scales=[vs])
    Ro = oracle_bank(exact, scales, ftype, order)
    errs = scale_errors(Rg, Ro)
    assert max(errs) <= TOL, errs
    compare_blobs(blobs, Ro, 0.05)


# ---------------------------------------------------------------------------
# 16-bit planes: a-priori error bound, and the 16-bit path is the one that ran
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("ftype,order", [(D, 4), (E, 2), (C, 1)])
@pytest.mark.parametrize("storage", [F16, BF16])
def test_16bit_planes_stay_within_the_rounding_bound(storage, ftype, order):
    img = SY.iir_fir_frame(seed=13, H=300, W=419, nblobs=25)
    (R32,), _ = gpu_bank([img], SIX, ftype, order, 0.05, storage=F32)
    (R16,), blobs = gpu_bank([img], SIX, ftype, order, 0.05, storage=storage)
    Ro = oracle_bank(img, SIX, ftype, order)
    e32 = scale_errors(R32, Ro)
    e16 = scale_errors(R16, Ro)
    bound = storage_bounds(img, SIX, ftype, order, storage, Ro)
    for s in range(len(SIX)):
        assert e16[s] <= bound[s], (s, e16[s], bound[s])
    # the planes really were rounded to 16 bits
    assert max(e16) > 4 * max(e32), (e16, e32)
    assert np.all(np.isfinite(R16))
    compare_blobs(blobs, Ro, 0.05, tol=max(bound))


# ---------------------------------------------------------------------------
# the 12-bit counts workload (512^2 cut, 8 scales): error report
# ---------------------------------------------------------------------------
def test_counts_workload_error_report():
    import torch
    counts = SY.counts_frame(seed=3, H=512, W=512, nblobs=16)
    vs = 1.0 / 4095.0
    vs32 = np.float64(np.float32(vs))
    scales = list(SY.SCALES_EIGHT)
    exact = counts.astype(np.float64) * vs32
    Ro_exact = oracle_bank(exact, scales, D, 4)
    f16_in = counts.astype(np.float16)
    bf16_in = torch.from_numpy(counts.astype(np.float32)).to(torch.bfloat16)
    quant = {U16: exact,
             F16: f16_in.astype(np.float64) * vs32,
             BF16: bf16_in.to(torch.float64).numpy() * vs32}
    frames = {U16: counts, F16: f16_in, BF16: bf16_in}
    Ro_quant = {U16: Ro_exact, F16: oracle_bank(quant[F16], scales, D, 4),
                BF16: oracle_bank(quant[BF16], scales, D, 4)}
    names = {F32: "f32", F16: "f16", BF16: "bf16", U16: "u16"}
    lines = []
    for din in (U16, F16, BF16):
        for st in (F32, F16, BF16):
            (Rg,), blobs = gpu_bank([frames[din]], scales, D, 4, 0.05, storage=st, value_scales=[vs])
            e_exact = scale_errors(Rg, Ro_exact)
            e_quant = scale_errors(Rg, Ro_quant[din])
            ref = O.detect(Ro_exact, 0.05, O.RESP_LAPLACIAN, 0)
            rs = {(int(b["scale"]), int(b["y"]), int(b["x"])) for b in ref}
            gs = {(int(b["scale"]), int(b["y"]), int(b["x"])) for b in blobs}
            lines.append(f"input {names[din]:4s} storage {names[st]:4s}: max err/range vs exact input "
                         f"{max(e_exact):.2e}, vs quantised input {max(e_quant):.2e}; "
                         f"blobs oracle {len(rs)} gpu {len(gs)} common {len(rs & gs)}")
            # the arithmetic alone: f32 planes meet the FP32 bar on the quantised input,
            # 16-bit planes their rounding bound
            if st == F32:
                assert max(e_quant) <= TOL, e_quant
            else:
                bound = storage_bounds(quant[din], scales, D, 4, st, Ro_quant[din])
                assert all(e <= b for e, b in zip(e_quant, bound)), (e_quant, bound)
            if din == U16 and st == F32:
                compare_blobs(blobs, Ro_exact, 0.05)
    print("\n" + "\n".join(lines))


# ---------------------------------------------------------------------------
# range and argument errors
# ---------------------------------------------------------------------------
def test_f16_plane_overflow_is_reported():
    """Raw 12-bit counts with a horizontal step: sigma^2 blur_x(V) reaches
    sigma^2 x 4095 along the step, beyond the f16 range; the call reports
    KF_ERANGE instead of returning infinite responses as blobs.  bf16 planes
    hold the same values."""
    from paper_1912_07133_gb300 import kf
    img = np.zeros((96, 130), np.uint16)
    img[48:] = 4095
    bank = kf.Bank(0)
    from tests.parity import to_device
    x = to_device(img)
    bank.run([x], [16.0], kf.KF_IIR_REPEATED_POLE, 4, storage=kf.KF_DTYPE_F16)
    with pytest.raises(kf.KfError) as e:
        bank.blobs()
    assert e.value.code == kf.KF_ERANGE
    bank.run([x], [16.0], kf.KF_FIR_COLORED_SG, 1, storage=kf.KF_DTYPE_F16)
    with pytest.raises(kf.KfError) as e:
        bank.blobs()
    assert e.value.code == kf.KF_ERANGE
    bank.run([x], [16.0], kf.KF_IIR_REPEATED_POLE, 4, storage=kf.KF_DTYPE_BF16)
    bank.blobs()
    bank.run([x], [16.0], kf.KF_IIR_REPEATED_POLE, 4, storage=kf.KF_DTYPE_F16, value_scales=[1.0 / 4095.0])
    bank.blobs()
    bank.close()


def test_storage_and_dtype_arguments_are_checked():
    import ctypes
    import torch
    from paper_1912_07133_gb300 import kf
    bank = kf.Bank(0)
    x = torch.zeros(16, 16, device="cuda")
    with pytest.raises(kf.KfError) as e:
        bank.run([x], [4.0], kf.KF_IIR_REPEATED_POLE, 3, storage=kf.KF_DTYPE_U16)
    assert e.value.code == kf.KF_EINVAL
    with pytest.raises(kf.KfError) as e:
        bank.run([x], [4.0], kf.KF_IIR_REPEATED_POLE, 3, value_scales=[math.inf])
    assert e.value.code == kf.KF_EINVAL
    h = torch.zeros(16, 18, device="cuda", dtype=torch.float16)
    L = kf.load()
    sc = (ctypes.c_double * 1)(4.0)
    opts = kf.kf_bank_opts_default()
    bad = [kf.kf_frame(h.data_ptr() + 1, 16, 16, 18, kf.KF_DTYPE_F16, 0.0),   # misaligned
           kf.kf_frame(h.data_ptr(), 16, 16, 18, 7, 0.0)]                       # unknown dtype
    for d in bad:
        rc = L.kf_filter_bank(bank.ctx, ctypes.byref(d), 1, sc, 1, kf.KF_IIR_REPEATED_POLE, 3,
                              ctypes.byref(opts))
        assert rc == kf.KF_EINVAL
    bank.close()

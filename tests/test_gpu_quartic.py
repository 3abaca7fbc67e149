"""The D = 5 derivative bank (kf_quartic_bank) and steering (kf_quartic_steer)
against the oracle, through the C ABI.

* Every channel D_{dx,dy} (dx + dy <= 4) at every scale, for the three blurs
  with vanishing moments to order 4 (Filter D with L_D = 2 at two orders,
  Filter E of order 3, Filter C with L_D = 2), on frames that span several
  tiles and segments with ragged edges, within 1e-5 of each (scale, channel)
  range plus the FP32 bound of the blur: the differentiated channel U is
  rounded once to f32, and each of the two FP32 blur passes errs by at most
  a couple of units u = 2^-24 of the l1 weight of what it sums, ||g||_1
  max|U| (the recursions are stable and their rounding errors decay with the
  impulse response), so |err| <= 1e-5 range + 4 u ||g||_1^2 max|U|.  The
  second term only matters where U is much larger than the blurred output
  (fourth differences of white noise).
* Input element types and value scales.
* At the benchmark size: a constant frame (only D_00, equal to the constant)
  and the transposition symmetry (channel (dx, dy) of the transposed frame is
  channel (dy, dx) transposed), which hold at any size.
* Steering against the oracle's steering.
* Argument checks.
"""
import numpy as np
import pytest

from oracle import oracle as O
from oracle import quartic as Q
from paper_1912_07133_gb300 import synthetic as SY
from tests.parity import TOL, to_device

pytestmark = pytest.mark.gpu

D, E, C = 0, 1, 2
OT = {D: O.IIR_REPEATED_POLE, E: O.IIR_BUTTERWORTH, C: O.FIR_COLORED_SG}


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__ as g
    g.build()


def run_gpu(frame, scales, ftype, order, value_scale=0.0, f64=True):
    import torch

    from paper_1912_07133_gb300 import kf
    ctx = kf.kf_create(0)
    try:
        t = to_device(frame)
        out = kf.kf_quartic_bank(ctx, t, scales, ftype, order, value_scale=value_scale)
        torch.cuda.synchronize()
        h = out.cpu().numpy()
        return h.astype(np.float64) if f64 else h
    finally:
        kf.kf_destroy(ctx)


def channel_errors(G, R, bound=None):
    """max |G - R| per (scale, channel) over 1e-5 range + bound: <= 1 passes,
    as a multiple of 1e-5 of the range when bound is None."""
    S, NC = R.shape[:2]
    if bound is None:
        return np.array([[np.abs(G[s, c] - R[s, c]).max() / max(np.ptp(R[s, c]), 1e-300) for c in range(NC)]
                         for s in range(S)])
    return np.array([[np.abs(G[s, c] - R[s, c]).max() / (TOL * np.ptp(R[s, c]) + bound[s, c]) for c in range(NC)]
                     for s in range(S)])


def fp32_bound(frame, scales, ftype, order):
    """4 u ||g_s||_1^2 max|U_c| per (scale, channel)."""
    X = np.pad(np.asarray(frame, dtype=np.float64), 4, mode="edge")
    taps = [Q.hpf_taps(d, 5) for d in range(5)]
    umax = np.array([np.abs(Q.conv_same(Q.conv_same(X, taps[dx], 1), taps[dy], 0)).max() for dx, dy in Q.CHANNELS])
    g1 = np.array([np.abs(Q.Blur(OT[ftype], order, l).impulse_response(int(40 * l) + 60)).sum() for l in scales])
    return 4 * 2.0 ** -24 * (g1 ** 2)[:, None] * umax[None, :]


@pytest.mark.parametrize("ftype,order,shape", [(D, 3, (150, 133)), (D, 4, (150, 133)), (E, 3, (150, 133)),
                                               (C, 2, (150, 133)), (D, 4, (90, 128)), (C, 2, (90, 128))])
def test_quartic_bank_matches_the_oracle(ftype, order, shape):
    """Widths 133 (the row pass's last chunk runs past the frame) and 128 (the
    chunks end at the frame's edge)."""
    frame = SY.iir_fir_frame(seed=21, H=shape[0], W=shape[1], nblobs=25)
    scales = [2.0, 3.5, 6.0]
    G = run_gpu(frame, scales, ftype, order)
    R = Q.quartic_bank(frame.astype(np.float64), scales, OT[ftype], order)
    err = channel_errors(G, R, fp32_bound(frame, scales, ftype, order))
    worst = np.unravel_index(np.argmax(err), err.shape)
    assert err.max() <= 1.0, (err.max(), worst, Q.CHANNELS[worst[1]])
    # orders 0-3 meet the bar of the detection path on their own
    low = [c for c, (dx, dy) in enumerate(Q.CHANNELS) if dx + dy < 4]
    assert channel_errors(G, R)[:, low].max() <= TOL


@pytest.mark.parametrize("ftype,order", [(D, 5), (D, 6), (E, 4), (E, 6)])
def test_quartic_bank_other_orders(ftype, order):
    """The remaining orders the call accepts (Filter D up to K^lpf = 6, Filter
    E up to L_B / 2 = 6) on a ragged 70 x 90 frame."""
    frame = SY.iir_fir_frame(seed=31, H=70, W=90, nblobs=8)
    scales = [2.5, 6.0]
    G = run_gpu(frame, scales, ftype, order)
    R = Q.quartic_bank(frame.astype(np.float64), scales, OT[ftype], order)
    assert channel_errors(G, R, fp32_bound(frame, scales, ftype, order)).max() <= 1.0


@pytest.mark.parametrize("shape", [(1, 1), (1, 37), (5, 3), (2, 70)])
def test_quartic_bank_degenerate_frames(shape):
    """Frames narrower or shorter than the stencils, a tile and a row chunk:
    one pixel, one row, a few pixels.  Every channel against the oracle (whose
    own FP64 rounding, about 1e-17 of the frame where a derivative is exactly
    zero, sets a floor of 1e-12 max|X|)."""
    rng = np.random.default_rng(sum(shape))
    frame = rng.uniform(0, 1, shape).astype(np.float32)
    for ftype, order in ((D, 4), (C, 2)):
        G = run_gpu(frame, [2.0, 5.0], ftype, order)
        R = Q.quartic_bank(frame.astype(np.float64), [2.0, 5.0], OT[ftype], order)
        tol = TOL * np.maximum(np.ptp(R, axis=(2, 3)), np.abs(R).max(axis=(2, 3))) + \
            fp32_bound(frame, [2.0, 5.0], ftype, order) + 1e-12 * float(np.abs(frame).max())
        err = np.abs(G - R).max(axis=(2, 3))
        assert np.all(err <= tol), (ftype, float((err / tol).max()))


def test_quartic_bank_input_types_and_value_scale():
    import torch
    rng = np.random.default_rng(4)
    counts = rng.integers(0, 4096, size=(70, 90)).astype(np.uint16)
    scales = [2.5, 5.0]
    vs = 1.0 / 4095.0
    # the frame the bank sees: each count converted to f32 and scaled in f32
    seen = (counts.astype(np.float32) * np.float32(vs)).astype(np.float64)
    R = Q.quartic_bank(seen, scales, O.IIR_REPEATED_POLE, 4)
    G = run_gpu(counts, scales, D, 4, value_scale=vs)
    assert channel_errors(G, R, fp32_bound(seen, scales, D, 4)).max() <= 1.0
    half = torch.from_numpy(rng.uniform(0, 1, (70, 90)).astype(np.float16))
    seen = half.numpy().astype(np.float64)
    R = Q.quartic_bank(seen, scales, O.IIR_BUTTERWORTH, 3)
    G = run_gpu(half, scales, E, 3)
    assert channel_errors(G, R, fp32_bound(seen, scales, E, 3)).max() <= 1.0


@pytest.mark.parametrize("ftype,order", [(D, 4), (C, 2)])
def test_full_size_constant_and_transposition(ftype, order):
    import torch
    H = W = 2048
    scales = [4.0, 12.0]
    const = torch.full((H, W), 0.375, device="cuda")
    G = run_gpu(const, scales, ftype, order)
    assert np.abs(G[:, 0] - 0.375).max() <= 1e-6
    assert np.abs(G[:, 1:]).max() <= 1e-6
    frame = SY.iir_fir_frame(seed=8, H=H, W=W, nblobs=400)
    A = run_gpu(frame, scales, ftype, order, f64=False)
    B = run_gpu(np.ascontiguousarray(frame.T), scales, ftype, order, f64=False)
    bound = fp32_bound(frame, scales, ftype, order)  # both sides err by at most this
    for c, (dx, dy) in enumerate(Q.CHANNELS):
        ct = Q.channel_index(dy, dx)
        for s in range(len(scales)):
            a, b = A[s, c], B[s, ct].T
            assert np.abs(a - b).max() <= 2 * (TOL * float(np.ptp(a)) + bound[s, c]), (s, dx, dy)


def test_steering_matches_the_oracle():
    import torch

    from paper_1912_07133_gb300 import kf
    rng = np.random.default_rng(9)
    Dh = rng.normal(size=(3, 15, 17, 23)).astype(np.float32)
    ctx = kf.kf_create(0)
    try:
        for phi in (0.0, 0.4, -2.1, np.pi / 2):
            Dd = torch.from_numpy(Dh).cuda()
            G = kf.kf_quartic_steer(ctx, Dd, phi).cpu().numpy().astype(np.float64)
            R = Q.steer(Dh.astype(np.float64), phi)
            scale = np.abs(Dh).max() * 8
            assert np.abs(G - R).max() <= 1e-6 * scale, phi
            kf.kf_quartic_steer(ctx, Dd, phi, out=Dd)  # in place
            torch.cuda.synchronize()
            assert np.array_equal(Dd.cpu().numpy().astype(np.float64), G)
    finally:
        kf.kf_destroy(ctx)


def test_quartic_arguments_are_checked():
    import torch

    from paper_1912_07133_gb300 import kf
    t = torch.zeros((40, 40), device="cuda")
    ctx = kf.kf_create(0)
    try:
        for ftype, order in ((D, 2), (D, 7), (E, 2), (C, 1), (3, 1)):
            with pytest.raises(kf.KfError):
                kf.kf_quartic_bank(ctx, t, [3.0], ftype, order)
        with pytest.raises(kf.KfError):
            kf.kf_quartic_bank(ctx, t, [], D, 4)
        with pytest.raises(kf.KfError):
            kf.kf_quartic_bank(ctx, t, [-1.0], D, 4)
        # the bank call after a D = 5 run still works and finds blobs
        bank_frame = to_device(SY.iir_fir_frame(seed=3, H=128, W=128, nblobs=10))
        kf.kf_quartic_bank(ctx, bank_frame, [3.0], D, 4)
        kf.kf_filter_bank(ctx, [bank_frame], [3.0, 5.0], D, 3)
        assert len(kf.kf_detect_blobs(ctx, 0.05, 1 << 16)) > 0
    finally:
        kf.kf_destroy(ctx)

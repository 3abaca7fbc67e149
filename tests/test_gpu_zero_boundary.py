"""The FIR blurs with the zero boundary (Sec. 5: the FIR is initialised with
zeros), through the C ABI, against the FP64 oracle's zero-extended bank
(`O.bank(..., boundary=O.BOUNDARY_ZERO)`: the frame extended by zeros, blurred,
differenced).  Bar: per-scale max|err| / range <= 1e-5, blob lists equal
except within that margin -- on the tensor-core column pass (f32 planes, all
scales), on the FP32 adjacent-scales pass, on more than eight scales (the
mma.sync pass), degenerate shapes and the 4096^2 six-scale frame."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1912_07133_gb300 import synthetic as SY
from tests.parity import TOL, compare_blobs, to_device

pytestmark = pytest.mark.gpu

C, A = 2, 3
OT = {C: O.FIR_COLORED_SG, A: O.FIR_GAUSSIAN}
SIX = [2.0, 4.0, 8.0, 16.0, 32.0, 48.0]


@pytest.fixture(scope="module")
def kf():
    import __graft_entry__ as g
    g.build()
    from paper_1912_07133_gb300 import kf as K
    return K


def gpu_zero(kf, img, scales, ftype, order, neigh=0, thr=0.05, boundary=None):
    import torch
    x = to_device(img)
    R = torch.empty(len(scales) * x.numel(), device="cuda")
    bank = kf.Bank(0)
    bank.run([x], scales, ftype, order, threshold=thr, neighbourhood=neigh, responses=R,
             boundary=kf.KF_BOUNDARY_ZERO if boundary is None else boundary)
    b = bank.blobs()
    torch.cuda.synchronize()
    bank.close()
    return R.view(len(scales), *img.shape).cpu().numpy().astype(np.float64), b


def oracle_zero(img, scales, ftype, order):
    return O.bank(img.astype(np.float64), scales, OT[ftype], order, boundary=O.BOUNDARY_ZERO)


def check(kf, img, scales, ftype, order, neigh=0):
    """Responses within 1e-5 of each scale's range -- of its largest magnitude
    where that is larger (a frame of a few pixels amid zeros has a nearly
    constant response, and FP32 rounding scales with the response, not its
    range) -- and the blob lists by the margin rule."""
    Rg, b = gpu_zero(kf, img, scales, ftype, order, neigh)
    Ro = oracle_zero(img, scales, ftype, order)
    for s in range(len(scales)):
        bar = TOL * max(np.ptp(Ro[s]), np.abs(Ro[s]).max() if min(img.shape) <= 3 else 0.0, 1e-3)
        assert np.abs(Rg[s] - Ro[s]).max() <= bar, (scales[s], s)
    if img.size > 1:
        compare_blobs(b, Ro, 0.05, neigh=neigh)
    return Rg, Ro, b


@pytest.mark.parametrize("ftype,order", [(C, 1), (A, 1)])
def test_six_scales_ragged_frame_tensor_core_pass(kf, ftype, order):
    check(kf, SY.iir_fir_frame(seed=41, H=777, W=1000, nblobs=30), SIX, ftype, order)


@pytest.mark.parametrize("ftype,order", [(C, 1), (A, 1)])
def test_adjacent_scale_neighbourhood(kf, ftype, order):
    check(kf, SY.iir_fir_frame(seed=42, H=300, W=333, nblobs=10), SIX, ftype, order, neigh=1)


def test_more_than_eight_scales(kf):
    """Ten scales: the mma.sync column pass."""
    lam = [2.0 * 2.0 ** (s / 3.0) for s in range(10)]
    check(kf, SY.iir_fir_frame(seed=43, H=400, W=300, nblobs=12), lam, C, 1)


@pytest.mark.parametrize("H,W", [(1, 1), (1, 37), (37, 1), (2, 3), (31, 33), (65, 130), (129, 31), (70, 4099)])
@pytest.mark.parametrize("ftype,order", [(C, 1), (A, 1)])
def test_small_and_degenerate_shapes(kf, H, W, ftype, order):
    rng = np.random.default_rng(H * 1000 + W + 7)
    check(kf, rng.uniform(0, 1, (H, W)).astype(np.float32), [4.0, 7.0], ftype, order)


def test_full_size_4096_six_scales(kf):
    _, Ro, b = check(kf, SY.iir_fir_frame(), SIX, C, 1)
    assert len(b) > 500


def test_zero_and_hold_differ_at_the_border_only(kf):
    """The two boundaries give the same responses away from the frame's
    edges (beyond the longest filter's reach) and different ones at them."""
    img = SY.iir_fir_frame(seed=44, H=400, W=420, nblobs=15) + 0.5
    lam = [4.0, 16.0]
    Rz, _ = gpu_zero(kf, img, lam, C, 1)
    Rh, _ = gpu_zero(kf, img, lam, C, 1, boundary=kf.KF_BOUNDARY_HOLD)
    reach = 2 * 41 + 4  # two blur passes of the K = 40 filter, plus the difference taps
    inner = (slice(None), slice(reach, -reach), slice(reach, -reach))
    assert np.abs(Rz[inner] - Rh[inner]).max() <= 2 * TOL * np.ptp(Rh[1])
    assert np.abs(Rz[:, 0, :] - Rh[:, 0, :]).max() > 100 * TOL * np.ptp(Rh[1])


def test_zero_boundary_is_refused_where_it_does_not_apply(kf):
    import torch
    x = torch.rand(64, 64, device="cuda")
    bank = kf.Bank(0)
    for ftype, order, kw in ((0, 4, {}), (1, 2, {}), (C, 1, {"response": kf.KF_RESP_HESSIAN}),
                             (C, 1, {"offset_limit": 1.0})):
        with pytest.raises(kf.KfError) as e:
            bank.run([x], [4.0], ftype, order, boundary=kf.KF_BOUNDARY_ZERO, **kw)
        assert e.value.code == kf.KF_EINVAL
    with pytest.raises(kf.KfError):
        bank.run([x], [4.0], C, 1, boundary=7)
    bank.close()

"""The allocation-free entry point kf_responses_noalloc, called through the C
ABI, against the ordinary entry point kf_filter_bank.

kf_responses_noalloc serves callers that cannot call cudaMalloc (their device
memory is owned by another allocator, or their loops may not allocate after
start-up); it keeps its intermediates in one static device array shared by all
calls.  This file is collected last so that a run stopping at the first
failure has already run every other test; it passes on its own in a fresh
process as well."""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

TOL = 1e-5  # same bar as the parity tests: max |err| / per-scale response range


@pytest.fixture(scope="module")
def kfmod():
    import __graft_entry__ as g
    g.build()
    from paper_1912_07133_gb300 import kf
    return kf


def _reference(kf, X, scales, ftype, order, value_scale=None):
    import torch
    R = torch.empty(len(scales) * X.numel(), device="cuda")
    bank = kf.Bank(0)
    bank.run([X], scales, ftype, order, responses=R,
             value_scales=None if value_scale is None else [value_scale])
    torch.cuda.synchronize()
    bank.close()
    return R.view(len(scales), *X.shape).cpu().numpy()


def _noalloc_via_abi(kf, X, scales, ftype, order, dtype=None, value_scale=0.0, expect=None):
    """Direct ctypes call of the exported symbol (no binding helper)."""
    import torch
    L = kf.load()
    R = torch.full((len(scales) * X.numel(),), float("nan"), device="cuda")
    dt = kf.KF_DTYPE_F32 if dtype is None else dtype
    d = kf.kf_frame(X.data_ptr(), X.shape[1], X.shape[0], X.stride(0), dt, value_scale)
    sc = (ctypes.c_double * len(scales))(*scales)
    rc = L.kf_responses_noalloc(ctypes.byref(d), sc, len(scales), ftype, order, ctypes.c_void_p(R.data_ptr()),
                                ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    if expect is not None:
        assert rc == expect, (rc, L.kf_last_error(None))
        return None
    assert rc == kf.KF_OK, L.kf_last_error(None)
    torch.cuda.synchronize()
    return R.view(len(scales), *X.shape).cpu().numpy()


def _close(a, b):
    for s in range(len(b)):
        rng = max(np.ptp(b[s]), 1e-3)
        assert np.abs(a[s] - b[s]).max() <= TOL * rng, s


def test_noalloc_matches_filter_bank_on_two_calls_in_a_row(kfmod):
    import torch
    from paper_1912_07133_gb300 import synthetic
    kf = kfmod
    f1 = torch.from_numpy(synthetic.iir_fir_frame(seed=21, H=700, W=900, nblobs=20)).cuda()
    f2 = torch.from_numpy(synthetic.tiny_frame(seed=22, H=333, W=517, nblobs=9)).cuda()
    s1, s2 = [2.0, 8.0, 24.0, 48.0], [4.0, 11.0]
    # first call (device set-up) and a second call with other sizes right after
    a1 = _noalloc_via_abi(kf, f1, s1, kf.KF_IIR_REPEATED_POLE, 4)
    a2 = _noalloc_via_abi(kf, f2, s2, kf.KF_IIR_BUTTERWORTH, 2)
    _close(a1, _reference(kf, f1, s1, kf.KF_IIR_REPEATED_POLE, 4))
    _close(a2, _reference(kf, f2, s2, kf.KF_IIR_BUTTERWORTH, 2))


def test_noalloc_rejects_frames_beyond_its_scratch(kfmod):
    import torch
    kf = kfmod
    X = torch.zeros(4096, 4096, device="cuda")
    R = torch.empty(6 * X.numel(), device="cuda")
    with pytest.raises(kf.KfError) as e:
        kf.kf_responses_noalloc(X, [2.0, 4.0, 8.0, 16.0, 32.0, 48.0], kf.KF_IIR_REPEATED_POLE, 4, R)
    assert e.value.code == kf.KF_EINVAL
    assert "limit" in str(e.value)


def test_noalloc_sixteen_bit_counts_match_filter_bank(kfmod):
    """A uint16 frame of 12-bit counts with value scale 1/4095: the same
    element conversion as kf_filter_bank."""
    import torch
    from paper_1912_07133_gb300 import synthetic
    kf = kfmod
    c = synthetic.counts_frame(seed=23, H=300, W=260, nblobs=12)
    X = torch.from_numpy(c.view(np.int16)).cuda().view(torch.uint16)
    s = [4.0, 16.0]
    a = _noalloc_via_abi(kf, X, s, kf.KF_IIR_REPEATED_POLE, 4, dtype=kf.KF_DTYPE_U16, value_scale=1.0 / 4095)
    _close(a, _reference(kf, X, s, kf.KF_IIR_REPEATED_POLE, 4, value_scale=1.0 / 4095))


def test_noalloc_reports_a_wait_that_gave_up(kfmod):
    """With the failure-detection hook on, the column pass's bounded wait
    gives up (no copy in flight) and the call returns KF_ETIMEOUT instead of
    incomplete responses; with it off the next call is whole again."""
    import torch
    from paper_1912_07133_gb300 import synthetic
    kf = kfmod
    X = torch.from_numpy(synthetic.tiny_frame(seed=24, H=128, W=96, nblobs=4)).cuda()
    kf.kf_set_wait_limit(None, 4)
    try:
        _noalloc_via_abi(kf, X, [4.0], kf.KF_IIR_REPEATED_POLE, 3, expect=kf.KF_ETIMEOUT)
    finally:
        kf.kf_set_wait_limit(None, 0)
    a = _noalloc_via_abi(kf, X, [4.0], kf.KF_IIR_REPEATED_POLE, 3)
    _close(a, _reference(kf, X, [4.0], kf.KF_IIR_REPEATED_POLE, 3))

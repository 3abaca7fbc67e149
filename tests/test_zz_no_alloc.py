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


def _reference(kf, X, scales, ftype, order):
    import torch
    R = torch.empty(len(scales) * X.numel(), device="cuda")
    bank = kf.Bank(0)
    bank.run([X], scales, ftype, order, responses=R)
    torch.cuda.synchronize()
    bank.close()
    return R.view(len(scales), *X.shape).cpu().numpy()


def _noalloc_via_abi(kf, X, scales, ftype, order):
    """Direct ctypes call of the exported symbol (no binding helper)."""
    import torch
    L = kf.load()
    R = torch.full((len(scales) * X.numel(),), float("nan"), device="cuda")
    d = kf.kf_frame(X.data_ptr(), X.shape[1], X.shape[0], X.stride(0), kf.KF_DTYPE_F32, 0.0)
    sc = (ctypes.c_double * len(scales))(*scales)
    rc = L.kf_responses_noalloc(ctypes.byref(d), sc, len(scales), ftype, order, ctypes.c_void_p(R.data_ptr()),
                                ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
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

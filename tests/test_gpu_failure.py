"""Failure detection on the GPU without a fault: a bounded device wait that
gives up.

kf_set_wait_limit makes the column pass of the recursive banks wait on its
shared-memory load barrier without issuing the copy that would complete it
(nothing is ever in flight), for a few polls only: every tile's wait gives up,
the kernel records the failure in the call's status word and returns, and the
host reports KF_ETIMEOUT.  The context must stay usable: with the hook off the
next call gives the normal result."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def kf():
    import __graft_entry__ as g
    g.build()
    from paper_1912_07133_gb300 import kf as K
    return K


def _frame():
    import torch

    from paper_1912_07133_gb300 import synthetic
    return torch.from_numpy(synthetic.tiny_frame(seed=31, H=200, W=300, nblobs=8)).cuda()


@pytest.mark.parametrize("graph", [False, True])
def test_wait_that_gives_up_is_reported_and_the_context_recovers(kf, graph):
    import torch
    X = _frame()
    scales = [4.0, 8.0]
    bank = kf.Bank(0)
    R0 = torch.empty(len(scales) * X.numel(), device="cuda")
    bank.run([X], scales, kf.KF_IIR_REPEATED_POLE, 4, responses=R0, graph=graph)
    ref = bank.blobs()
    kf.kf_set_wait_limit(bank.ctx, 4)
    for _ in range(3 if graph else 1):  # eager, then captured and replayed
        bank.run([X], scales, kf.KF_IIR_REPEATED_POLE, 4, graph=graph)
        with pytest.raises(kf.KfError) as e:
            bank.blobs()
        assert e.value.code == kf.KF_ETIMEOUT
        assert "gave up" in str(e.value)
    kf.kf_set_wait_limit(bank.ctx, 0)
    R1 = torch.empty_like(R0)
    for _ in range(3 if graph else 1):
        bank.run([X], scales, kf.KF_IIR_REPEATED_POLE, 4, responses=R1, graph=graph)
        got = bank.blobs()
        torch.cuda.synchronize()
        assert np.array_equal(got, ref)
        assert torch.equal(R0, R1)
    bank.close()


def test_wait_limit_rejects_bad_values(kf):
    bank = kf.Bank(0)
    with pytest.raises(kf.KfError) as e:
        kf.kf_set_wait_limit(bank.ctx, -1)
    assert e.value.code == kf.KF_EINVAL
    bank.close()

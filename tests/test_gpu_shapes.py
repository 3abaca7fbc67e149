"""Blob shape descriptors (Sec. 5, the Hessian read as minus the Fisher
information of the blob): kf_blob_shapes against the FP64 oracle's
derivatives at the same detections.

Bar: the derivative planes carry the FP32 bar of the bank (1e-5 of each
channel's range, twice for safety: delta per entry of H); a symmetric 2 x 2
perturbation with entries within delta moves the eigenvalues mu of M = -pol H
by at most 2 delta and the eigenvectors by at most 2 delta / (mu_max - mu_min),
so p = 1/mu moves by at most 2 delta / mu_min relative (first order)."""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_1912_07133_gb300 import synthetic as SY
from tests.parity import OT, to_device

pytestmark = pytest.mark.gpu

D, A = 0, 3


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__ as g
    g.build()


@pytest.mark.parametrize("ftype,order", [(D, 4), (A, 1)])
def test_shapes_match_the_oracle(ftype, order):
    from paper_1912_07133_gb300 import kf
    img = SY.iir_fir_frame(seed=23, H=300, W=420, nblobs=40)
    scales = [4.0, 8.0, 16.0]
    bank = kf.Bank(0)
    bank.run([to_device(img)], scales, ftype, order, threshold=0.002, response=kf.KF_RESP_HESSIAN)
    blobs = bank.blobs()
    shapes = bank.shapes()
    assert len(blobs) == len(shapes) > 20
    _, Dor = O.bank(img.astype(np.float64), scales, OT[ftype], order, resp=O.RESP_HESSIAN, want_d=True)
    checked = 0
    for b, sh in zip(blobs, shapes):
        s, y, x = int(b["scale"]), int(b["y"]), int(b["x"])
        d20, d02, d11 = Dor[s, 2, y, x], Dor[s, 3, y, x], Dor[s, 4, y, x]
        pol = 1 if d20 + d02 < 0 else -1
        p1, p2, th, det = O.blob_shape(d20, d02, d11, pol)
        delta = 2 * 1e-5 * max(np.ptp(Dor[s, c]) for c in (2, 3, 4))
        assert sh["det"] == pytest.approx(det, abs=4 * delta * (abs(d20) + abs(d02) + abs(d11)) + 1e-12)
        M = -pol * np.array([[d20, d11], [d11, d02]])
        mu = np.linalg.eigvalsh(M)
        if not (mu[0] > 8 * delta):  # not (safely) positive definite: NaN on one side or both
            continue
        assert sh["p1"] == pytest.approx(p1, rel=3 * 2 * delta / mu[0] + 1e-5)
        assert sh["p2"] == pytest.approx(p2, rel=3 * 2 * delta / mu[0] + 1e-5)
        gap = mu[1] - mu[0]
        if gap > 8 * delta:
            assert abs(math.remainder(float(sh["theta"]) - th, math.pi)) <= 3 * 2 * delta / gap + 1e-5
        checked += 1
    assert checked > 10
    bank.close()


def test_shapes_need_the_derivative_bank():
    from paper_1912_07133_gb300 import kf
    img = SY.tiny_frame(3, 64, 64, 3)
    bank = kf.Bank(0)
    bank.run([to_device(img)], [4.0], D, 4, threshold=0.05)
    with pytest.raises(kf.KfError) as e:
        bank.shapes()
    assert e.value.code == kf.KF_EINVAL
    bank.close()

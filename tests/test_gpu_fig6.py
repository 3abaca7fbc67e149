"""Figs. 6 and 7 (Sec. 5) through the library: on the ellipse test pattern,
Filter D, C or E with the normalised Hessian and one Threshold #1 for all
scales (per blur) detects, at each lambda, the centres of the ellipses whose semi-major axis
equals lambda (every rotation) and nothing else; with axis ratio 4,
Threshold #2 removes the detections on the tips of the longer ellipses.  The
GPU lists also equal the FP64 oracle's on this input."""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_1912_07133_gb300 import synthetic as SY
from tests.parity import to_device

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__ as g
    g.build()


def nearest(b, centres):
    return min((math.hypot(int(b["y"]) - cy, int(b["x"]) - cx), a, r) for cy, cx, a, r in centres)


# blur -> (library type, oracle type, order, Threshold #1); the thresholds are
# the readings the oracle's pins use (the figures print none)
FIG6 = {"D": (0, O.IIR_REPEATED_POLE, 3, 0.035), "C": (2, O.FIR_COLORED_SG, 1, 0.132),
        "E": (1, O.IIR_BUTTERWORTH, 2, 0.066)}


@pytest.mark.parametrize("blur", ["D", "C", "E"])
def test_fig6_scale_selectivity(blur):
    from paper_1912_07133_gb300 import kf
    ft, oft, order, T = FIG6[blur]
    img, centres = SY.ellipse_pattern(2.0)
    x = to_device(img)
    bank = kf.Bank(0)
    for lam in (4, 8, 16, 32, 64):
        bank.run([x], [float(lam)], ft, order, threshold=T, response=kf.KF_RESP_HESSIAN, fir_kmax=160)
        b = bank.blobs()
        near = [nearest(r, centres) for r in b]
        assert all(a == lam and d <= 0.05 * lam + 1.0 for d, a, _ in near), (lam, near)
        assert sorted(r for _, _, r in near) == [0, 15, 30, 45], lam
        ref = O.detect(O.bank(img.astype(np.float64), [float(lam)], oft, order, O.RESP_HESSIAN, fir_kmax=160),
                       T, O.RESP_HESSIAN, O.NEIGH_ALL)
        assert [(int(r["y"]), int(r["x"])) for r in b] == [(int(r["y"]), int(r["x"])) for r in ref], lam
    bank.close()


def test_fig7_threshold_2():
    from paper_1912_07133_gb300 import kf
    img, centres = SY.ellipse_pattern(4.0)
    x = to_device(img)
    bank = kf.Bank(0)
    bank.run([x], [16.0], kf.KF_IIR_REPEATED_POLE, 3, threshold=0.02, response=kf.KF_RESP_HESSIAN)
    t1 = [nearest(r, centres) for r in bank.blobs()]
    assert len([v for v in t1 if v[1] > 16 and v[0] > 0.3 * v[1]]) >= 8
    bank.run([x], [16.0], kf.KF_IIR_REPEATED_POLE, 3, threshold=0.02, response=kf.KF_RESP_HESSIAN,
             offset_limit=2.0)
    t12 = [nearest(r, centres) for r in bank.blobs()]
    assert t12 and all(a == 16 and d <= 1.0 for d, a, _ in t12)
    bank.close()

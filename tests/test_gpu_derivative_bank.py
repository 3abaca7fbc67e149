"""The derivative bank against the FP64 oracle: the Hessian response R_H of
eq (26), Threshold #2 with the eq (27) offsets, and the Laplacian response
through the same channels.

Each blurred derivative is its own channel (planes sigma^2 D, FP32 path), so
each carries at most the FP32 bar of the fused path, 1e-5 of its range.  R_H =
A B - C^2 (A, B, C the sigma^2-scaled D20, D02, D11) then errs by at most
|B| e_A + |A| e_B + 2 |C| e_C per pixel (first order), the bound used here.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1912_07133_gb300 import synthetic as SY
from tests.parity import TOL, gpu_bank, margin, to_device

pytestmark = pytest.mark.gpu

D, E, C = 0, 1, 2
OT = {D: O.IIR_REPEATED_POLE, E: O.IIR_BUTTERWORTH, C: O.FIR_COLORED_SG}
SCALES = [2.0, 4.0, 8.0, 16.0]


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__ as g
    g.build()


def run(frame, ftype, order, T, **kw):
    import torch

    from paper_1912_07133_gb300 import kf
    R = torch.full((len(SCALES) * frame.size,), float("nan"), device="cuda")
    bank = kf.Bank(0)
    bank.run([to_device(frame)], SCALES, ftype, order, threshold=T, responses=R, **kw)
    b = bank.blobs()
    bank.close()
    return R.cpu().numpy().astype(np.float64).reshape(len(SCALES), *frame.shape), b


def oracle(frame, ftype, order, resp):
    R, Dd = O.bank(frame.astype(np.float64), SCALES, OT[ftype], order, resp=resp, want_d=True)
    return R, Dd


def hessian_bound(Dd):
    """Per-pixel first-order bound of |R_H error| (see the module docstring)."""
    out = np.zeros((len(SCALES),) + Dd.shape[2:])
    for s, lam in enumerate(SCALES):
        s2 = (lam / 2.0) ** 2
        A, B, Cc = s2 * Dd[s, 2], s2 * Dd[s, 3], s2 * Dd[s, 4]
        eA, eB, eC = (TOL * np.ptp(v) for v in (A, B, Cc))
        out[s] = np.abs(B) * eA + np.abs(A) * eB + 2 * np.abs(Cc) * eC
    return out


@pytest.mark.parametrize("ftype,order", [(D, 4), (E, 2), (C, 1)])
def test_hessian_response_within_its_bound(ftype, order):
    from paper_1912_07133_gb300 import kf
    frame = SY.tiny_frame(31, 203, 331, 14)
    Rg, blobs = run(frame, ftype, order, 0.002, response=kf.KF_RESP_HESSIAN)
    Ro, Dd = oracle(frame, ftype, order, O.RESP_HESSIAN)
    bound = hessian_bound(Dd)
    excess = np.abs(Rg - Ro) - 1.01 * bound
    assert excess.max() <= 1e-7 * np.abs(Ro).max(), excess.max()
    # blob list: bright maxima of R_H; identical beyond the error bound
    ref = O.detect(Ro, 0.002, O.RESP_HESSIAN, 0)
    gs = {(int(b["scale"]), int(b["y"]), int(b["x"])) for b in blobs}
    rs = {(int(b["scale"]), int(b["y"]), int(b["x"])) for b in ref}
    assert all(int(b["polarity"]) == 1 for b in blobs)
    tolb = 2 * bound.max() + 1e-7 * np.abs(Ro).max()
    for key in gs ^ rs:
        assert abs(margin(Ro, *key, 1, 0.002)) <= tolb, key
    assert len(rs) >= 10 and len(gs ^ rs) <= max(1, 0.1 * len(rs))


@pytest.mark.parametrize("ftype,order", [(D, 4), (C, 1)])
def test_laplacian_through_the_channels_matches_the_fused_path(ftype, order):
    """offset_limit > 0 runs the derivative bank with R_L: the responses agree
    with the fused path to the FP32 bar, and the offsets follow eq (27)."""
    frame = SY.tiny_frame(32, 180, 260, 10)
    Rf, bf = run(frame, ftype, order, 0.05)
    Rd, bd = run(frame, ftype, order, 0.05, offset_limit=1000.0)
    for s in range(len(SCALES)):
        assert np.abs(Rd[s] - Rf[s]).max() <= 2 * TOL * np.ptp(Rf[s])
    Ro, Dd = oracle(frame, ftype, order, O.RESP_LAPLACIAN)
    ref = O.detect(Ro, 0.05, O.RESP_LAPLACIAN, 0, D=Dd, limit2=1000.0)
    rmap = {(int(b["scale"]), int(b["y"]), int(b["x"])): b for b in ref}
    n = 0
    for b in bd:
        key = (int(b["scale"]), int(b["y"]), int(b["x"]))
        if key not in rmap:
            continue
        r = rmap[key]
        if abs(r["det"]) < 1e-6 * np.abs(Dd[:, 2]).max() * np.abs(Dd[:, 3]).max():
            continue  # offsets of a near-singular quadratic are ill-conditioned
        assert b["dx"] == pytest.approx(r["dx"], abs=1e-3 * (1 + abs(r["dx"])))
        assert b["dy"] == pytest.approx(r["dy"], abs=1e-3 * (1 + abs(r["dy"])))
        n += 1
    assert n >= 5


@pytest.mark.parametrize("ftype,order", [(D, 4), (C, 1)])
def test_threshold_2_keeps_the_candidates_with_small_offsets(ftype, order):
    frame = SY.tiny_frame(33, 200, 300, 16)
    limit = 0.5
    _, bd = run(frame, ftype, order, 0.05, offset_limit=limit)
    _, ball = run(frame, ftype, order, 0.05)
    Ro, Dd = oracle(frame, ftype, order, O.RESP_LAPLACIAN)
    ref = O.detect(Ro, 0.05, O.RESP_LAPLACIAN, 0, D=Dd, limit2=limit)
    gs = {(int(b["scale"]), int(b["y"]), int(b["x"])) for b in bd}
    rs = {(int(b["scale"]), int(b["y"]), int(b["x"])) for b in ref}
    all_keys = {(int(b["scale"]), int(b["y"]), int(b["x"])) for b in ball}
    assert gs <= all_keys and len(gs) < len(all_keys)
    for b in bd:
        assert np.hypot(b["dx"], b["dy"]) <= limit
    # differences only where the offset sits at the limit (within FP32 of eq 27) or the
    # Threshold #1 margin is within the FP32 bar
    odict = {(int(b["scale"]), int(b["y"]), int(b["x"])): b for b in O.detect(Ro, 0.05, O.RESP_LAPLACIAN, 0, D=Dd)}
    ranges = np.array([np.ptp(Ro[s]) for s in range(len(SCALES))])
    for key in gs ^ rs:
        r = odict.get(key)
        near_limit = r is not None and abs(np.hypot(r["dx"], r["dy"]) - limit) <= 1e-3 * (1 + limit)
        pol = 1 if Ro[key] > 0 else -1
        near_t1 = abs(margin(Ro, *key, pol, 0.05)) <= 2 * TOL * ranges.max()
        assert near_limit or near_t1, key


def test_derivative_bank_arguments_are_checked():
    import torch

    from paper_1912_07133_gb300 import kf
    x = torch.zeros(64, 64, device="cuda")
    bank = kf.Bank(0)
    for kw in [dict(response=7), dict(offset_limit=-1.0)]:
        with pytest.raises(kf.KfError):
            bank.run([x], SCALES, D, 4, **kw)
    bank.close()

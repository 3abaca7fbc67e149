"""Proposal gating: every blob the gated bank reports is the full bank's blob,
and it reports exactly the full bank's blobs inside the column tiles that the
gate selects.

A hand-set network makes the gate checkable independently of the kernels:
conv1 passes the pooled value through its centre tap, conv2 copies channel 0,
conv3 gives every scale channel a2 - c, so the logit of a tile is the largest
pooled value in it minus c (all through ReLUs, which keep positive values).
The expected active tiles, column tiles and blob set follow on the host.
"""
import numpy as np
import pytest

from paper_1912_07133_gb300 import synthetic as SY
from tests.parity import to_device

pytestmark = pytest.mark.gpu

D, E, C = 0, 1, 2
SCALES = [2.0, 4.0, 8.0, 16.0]
TW = 30


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__ as g
    g.build()


def hand_weights(c):
    W1 = np.zeros((16, 1, 3, 3)); W1[0, 0, 1, 1] = 1.0
    W2 = np.zeros((16, 16, 3, 3)); W2[0, 0, 1, 1] = 1.0
    W3 = np.zeros((8, 16, 3, 3)); W3[:, 0, 1, 1] = 1.0
    b1, b2, b3 = np.zeros(16), np.zeros(16), np.full(8, -c)
    return np.concatenate([W1.ravel(), b1, W2.ravel(), b2, W3.ravel(), b3]).astype(np.float32)


def frames_for_gating(seed=40):
    rng = np.random.default_rng(seed)
    out = []
    for H, W in [(300, 420), (257, 130), (140, 700)]:
        img = rng.uniform(0, 0.05, (H, W)).astype(np.float32)
        for _ in range(3):  # a few bright patches make some tiles active
            y, x = rng.integers(0, H - 16), rng.integers(0, W - 16)
            img[y:y + 16, x:x + 16] += 1.0
        out.append(SY.tiny_frame(int(rng.integers(1 << 30)), H, W, 6) + img)
    return out


def expected_active(frame, c, dilate=True):
    """Active-tile map from the hand-set network (host arithmetic)."""
    H, W = frame.shape
    p = np.zeros(((H + 7) // 8, (W + 7) // 8))
    for y in range(p.shape[0]):
        for x in range(p.shape[1]):
            p[y, x] = frame[8 * y:8 * y + 8, 8 * x:8 * x + 8].astype(np.float64).mean()
    th, tw = (H + 63) // 64, (W + 63) // 64
    z = np.array([[np.maximum(p[8 * ty:8 * ty + 8, 8 * tx:8 * tx + 8], 0).max() - c for tx in range(tw)]
                  for ty in range(th)])
    a = z > 0.0  # gate_threshold 0.5
    if not dilate:
        return a
    d = np.zeros_like(a)
    for ty in range(th):
        for tx in range(tw):
            d[ty, tx] = a[max(ty - 1, 0):ty + 2, max(tx - 1, 0):tx + 2].any()
    return d


def selected(frame, act, rows, tw=TW):
    """Per pixel: inside the interior (tw columns x rows) of a column tile the
    gate selects."""
    H, W = frame.shape
    sel = np.zeros((H, W), bool)
    for y0 in range(0, H, rows):
        for x0 in range(0, W, tw):
            y1, x1 = min(y0 + rows, H), min(x0 + tw, W)
            if act[y0 // 64:(y1 - 1) // 64 + 1, x0 // 64:(x1 - 1) // 64 + 1].any():
                sel[y0:y1, x0:x1] = True
    return sel


def run(frames, ftype, order, gate, c=0.5, graph=False, calls=1):
    """gate: False, True (marked tiles and neighbours) or a KF_GATE_* mode."""
    import torch

    from paper_1912_07133_gb300 import kf
    ts = [to_device(f) for f in frames]
    n = sum(len(SCALES) * f.size for f in frames)
    bank = kf.Bank(0)
    kf.kf_proposal_set_weights(bank.ctx, hand_weights(c))
    for _ in range(calls):
        R = torch.full((n,), float("nan"), device="cuda")
        bank.run(ts, SCALES, ftype, order, threshold=0.03, responses=R, gate=gate, gate_threshold=0.5, graph=graph)
        b = bank.blobs()
    bank.close()
    return R.cpu().numpy(), b


@pytest.mark.parametrize("dilated", [True, False])
# column tiles: 30 x 64 (recursive banks), 126 x 62 (the FIR bank's tensor-core pass, <= 6 scales)
@pytest.mark.parametrize("ftype,order,rows,tw", [(D, 4, 64, 30), (E, 2, 64, 30), (C, 1, 62, 126)])
def test_gated_blobs_are_the_full_blobs_of_the_selected_tiles(ftype, order, rows, tw, dilated):
    from paper_1912_07133_gb300 import kf
    frames = frames_for_gating()
    Rf, bf = run(frames, ftype, order, gate=False)
    Rg, bg = run(frames, ftype, order, gate=kf.KF_GATE_DILATED if dilated else kf.KF_GATE_TILES)
    off = 0
    n_sel = n_all = 0
    for i, f in enumerate(frames):
        act = expected_active(f, 0.5, dilated)
        assert 0 < act.sum() < act.size
        sel = selected(f, act, rows, tw)
        k = len(SCALES) * f.size
        Rfi = Rf[off:off + k].reshape(len(SCALES), *f.shape)
        Rgi = Rg[off:off + k].reshape(len(SCALES), *f.shape)
        off += k
        # responses: identical wherever the gate ran the detector's tiles
        assert np.array_equal(Rgi[:, sel], Rfi[:, sel])
        full = {(int(b["scale"]), int(b["y"]), int(b["x"])) for b in bf[bf["frame"] == i]}
        gated = {(int(b["scale"]), int(b["y"]), int(b["x"])) for b in bg[bg["frame"] == i]}
        expect = {key for key in full if sel[key[1], key[2]]}
        assert gated == expect, i
        n_sel += len(expect)
        n_all += len(full)
    assert 0 < n_sel < n_all
    # gated records equal the full records (response included)
    fmap = {(int(b["frame"]), int(b["scale"]), int(b["y"]), int(b["x"])): float(b["response"]) for b in bf}
    for b in bg:
        assert fmap[(int(b["frame"]), int(b["scale"]), int(b["y"]), int(b["x"]))] == float(b["response"])


@pytest.mark.parametrize("ftype,order", [(D, 4), (C, 1)])
def test_gate_all_open_equals_the_full_bank(ftype, order):
    frames = frames_for_gating(41)
    Rf, bf = run(frames, ftype, order, gate=False)
    Rg, bg = run(frames, ftype, order, gate=True, c=-100.0)
    assert np.array_equal(Rf, Rg)
    assert np.array_equal(bf, bg)


@pytest.mark.parametrize("ftype,order", [(D, 4), (C, 1)])
def test_gate_all_closed_finds_nothing(ftype, order):
    frames = frames_for_gating(42)
    _, bg = run(frames, ftype, order, gate=True, c=100.0)
    assert len(bg) == 0


def test_gated_graph_replays_equal_eager():
    frames = frames_for_gating(43)
    Re, be = run(frames, C, 1, gate=True)
    Rg, bg = run(frames, C, 1, gate=True, graph=True, calls=4)
    sel_mask = ~np.isnan(Re)
    assert np.array_equal(Rg[sel_mask], Re[sel_mask])
    assert np.array_equal(bg, be)


def test_gate_arguments_are_checked():
    import torch

    from paper_1912_07133_gb300 import kf
    x = torch.zeros(64, 64, device="cuda")
    bank = kf.Bank(0)
    with pytest.raises(kf.KfError):  # no weights yet
        bank.run([x], SCALES, D, 4, gate=True)
    kf.kf_proposal_set_weights(bank.ctx, hand_weights(0.5))
    for kw in [dict(gate_threshold=1.5), dict(schedule=kf.KF_SCHED_PER_FRAME)]:
        with pytest.raises(kf.KfError):
            bank.run([x], SCALES, D, 4, gate=True, **kw)
    with pytest.raises(kf.KfError):
        bank.run([x], [2.0] * 9, D, 4, gate=True)
    bank.close()


def test_gate_reuse_gives_the_marks_of_the_earlier_call():
    """A second bank on the same frames with gate_reuse: the tile marks of the
    earlier gated call (one network evaluation per frame), the same blobs as
    evaluating the gate again; refused without a matching earlier call."""
    import torch

    from paper_1912_07133_gb300 import kf
    frames = frames_for_gating(44)
    ts = [to_device(f) for f in frames]
    bank = kf.Bank(0)
    kf.kf_proposal_set_weights(bank.ctx, hand_weights(0.5))
    with pytest.raises(kf.KfError) as e:  # nothing to reuse yet
        bank.run(ts, SCALES, C, 1, threshold=0.03, gate=kf.KF_GATE_TILES, gate_threshold=0.5, gate_reuse=True)
    assert e.value.code == kf.KF_EINVAL
    bank.run(ts, SCALES, D, 4, threshold=0.03, gate=kf.KF_GATE_TILES, gate_threshold=0.5)
    bank.run(ts, SCALES, C, 1, threshold=0.03, gate=kf.KF_GATE_TILES, gate_threshold=0.5, gate_reuse=True)
    reused = bank.blobs()
    bank.run(ts, SCALES, C, 1, threshold=0.03, gate=kf.KF_GATE_TILES, gate_threshold=0.5)
    fresh = bank.blobs()
    assert len(fresh) > 0 and np.array_equal(reused, fresh)
    for kw in [dict(gate_threshold=0.6), dict(gate=kf.KF_GATE_DILATED)]:  # other marks
        args = dict(threshold=0.03, gate=kf.KF_GATE_TILES, gate_threshold=0.5, gate_reuse=True)
        args.update(kw)
        with pytest.raises(kf.KfError):
            bank.run(ts, SCALES, C, 1, **args)
    with pytest.raises(kf.KfError):  # another frame set
        bank.run(ts[:2], SCALES, C, 1, threshold=0.03, gate=kf.KF_GATE_TILES, gate_threshold=0.5, gate_reuse=True)
    kf.kf_proposal_set_weights(bank.ctx, hand_weights(0.4))  # new weights: the marks are stale
    with pytest.raises(kf.KfError):
        bank.run(ts, SCALES, C, 1, threshold=0.03, gate=kf.KF_GATE_TILES, gate_threshold=0.5, gate_reuse=True)
    with pytest.raises(kf.KfError):  # reuse without gating
        bank.run(ts, SCALES, C, 1, threshold=0.03, gate_reuse=True)
    torch.cuda.synchronize()
    bank.close()

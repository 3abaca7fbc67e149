"""Batched persistent launches and graph replays.

* A call of many frames of uneven sizes (and mixed element types) gives the
  same responses, bit for bit, and the same ordered blob list whether every
  pass runs once over all frames (batched, width classes for the IIR row
  pass) or frame by frame; each frame matches the FP64 oracle at the FP32 bar.
* Graph mode: the first call of a geometry runs eagerly, the second captures,
  later calls replay with new frame data and response pointers; every call
  equals an eager call on the same data.  A new geometry, or a workspace that
  grows, is handled like a first call.
"""
import numpy as np
import pytest

from paper_1912_07133_gb300 import synthetic as SY
from tests.parity import TOL, compare_blobs, oracle_bank, scale_errors, to_device

pytestmark = pytest.mark.gpu

D, E, C = 0, 1, 2
SCALES = [2.0, 3.28, 5.38, 8.83]


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__ as g
    g.build()


def uneven_frames(seed=21):
    """Frames of several widths (three IIR row-width classes) and heights, the
    first few in other element types."""
    rng = np.random.default_rng(seed)
    sizes = [(97, 130), (64, 1100), (300, 33), (257, 640), (31, 2100), (190, 190), (5, 700)]
    out = []
    for i, (H, W) in enumerate(sizes):
        img = SY.tiny_frame(int(rng.integers(1 << 30)), H, W, max(1, H * W // 4000))
        out.append(img)
    return out


def run(frames, scales, ftype, order, **kw):
    import torch

    from paper_1912_07133_gb300 import kf
    ts = [to_device(f) for f in frames]
    n = sum(len(scales) * t.numel() for t in ts)
    R = torch.full((n,), float("nan"), device="cuda", dtype=torch.float32)
    bank = kf.Bank(0)
    bank.run(ts, scales, ftype, order, threshold=0.02, responses=R, **kw)
    b = bank.blobs()
    bank.close()
    return R.cpu().numpy(), b


def split(R, frames, S):
    out, off = [], 0
    for f in frames:
        k = S * f.size
        out.append(R[off:off + k].reshape(S, *f.shape).astype(np.float64))
        off += k
    return out


@pytest.mark.parametrize("ftype,order", [(D, 4), (E, 2), (C, 1)])
def test_batched_and_per_frame_schedules_agree_bitwise(ftype, order):
    from paper_1912_07133_gb300 import kf
    frames = uneven_frames()
    Rb, bb = run(frames, SCALES, ftype, order, schedule=kf.KF_SCHED_BATCHED)
    Rp, bp = run(frames, SCALES, ftype, order, schedule=kf.KF_SCHED_PER_FRAME)
    assert np.all(np.isfinite(Rb))
    assert np.array_equal(Rb, Rp)
    assert np.array_equal(bb, bp)
    for i, (f, Rg) in enumerate(zip(frames, split(Rb, frames, len(SCALES)))):
        Ro = oracle_bank(f, SCALES, ftype, order)
        assert max(scale_errors(Rg, Ro)) <= TOL, i
        compare_blobs(bb, Ro, 0.02, frame=i)


def test_mixed_element_types_in_one_batch():
    import torch
    frames = uneven_frames(seed=22)[:4]
    counts = SY.counts_frame(seed=23, H=120, W=170, nblobs=4)
    f16 = frames[1].astype(np.float16)
    bf16 = torch.from_numpy(frames[2]).to(torch.bfloat16)
    batch = [frames[0], counts, f16, bf16]
    vs = [1.0, 1.0 / 4095.0, 1.0, 1.0]
    exact = [frames[0].astype(np.float64), counts.astype(np.float64) * np.float64(np.float32(vs[1])),
             f16.astype(np.float64), bf16.to(torch.float64).numpy()]
    R, b = run(batch, SCALES, D, 4, value_scales=vs)
    for i, (x, Rg) in enumerate(zip(exact, split(R, exact, len(SCALES)))):
        Ro = oracle_bank(x, SCALES, D, 4)
        assert max(scale_errors(Rg, Ro)) <= TOL, i
        compare_blobs(b, Ro, 0.02, frame=i)


@pytest.mark.parametrize("ftype,order", [(D, 3), (C, 1)])
def test_graph_replays_equal_eager_calls(ftype, order):
    import torch

    from paper_1912_07133_gb300 import kf
    frames = uneven_frames(seed=24)[:5]
    other = [SY.tiny_frame(100 + i, f.shape[0], f.shape[1], 3) for i, f in enumerate(frames)]
    S = len(SCALES)
    n = sum(S * f.size for f in frames)
    bank = kf.Bank(0)
    eager = {}
    for name, fs in (("a", frames), ("b", other)):
        R, b = run(fs, SCALES, ftype, order)
        eager[name] = (R, b)
    # the same geometry four times, alternating data and output buffers
    outs = [torch.full((n,), float("nan"), device="cuda") for _ in range(2)]
    dev = {name: [to_device(f) for f in fs] for name, fs in (("a", frames), ("b", other))}
    for call, name in enumerate(["a", "b", "a", "b", "b"]):
        R = outs[call % 2]
        R.fill_(float("nan"))
        bank.run(dev[name], SCALES, ftype, order, threshold=0.02, responses=R, graph=True)
        b = bank.blobs()
        assert np.array_equal(R.cpu().numpy(), eager[name][0]), (call, name)
        assert np.array_equal(b, eager[name][1]), (call, name)
    # a new geometry (one frame fewer) and back
    R1 = torch.empty(n - S * frames[-1].size, device="cuda")
    bank.run(dev["a"][:-1], SCALES, ftype, order, threshold=0.02, responses=R1, graph=True)
    bank.blobs()
    assert np.array_equal(R1.cpu().numpy(), eager["a"][0][: R1.numel()])
    bank.run(dev["a"], SCALES, ftype, order, threshold=0.02, responses=outs[0], graph=True)
    assert np.array_equal(bank.blobs(), eager["a"][1])
    assert np.array_equal(outs[0].cpu().numpy(), eager["a"][0])
    bank.close()


def test_graph_mode_survives_workspace_growth():
    import torch

    from paper_1912_07133_gb300 import kf
    small = [SY.tiny_frame(31, 64, 96, 2)]
    big = [SY.tiny_frame(32, 400, 900, 20)]
    bank = kf.Bank(0)
    for frames in (small, small, small, big, big, big, small):
        ts = [to_device(f) for f in frames]
        R = torch.empty(len(SCALES) * frames[0].size, device="cuda")
        bank.run(ts, SCALES, D, 4, threshold=0.02, responses=R, graph=True)
        b = bank.blobs()
        Re, be = run(frames, SCALES, D, 4)
        assert np.array_equal(R.cpu().numpy(), Re)
        assert np.array_equal(b, be)
    bank.close()


@pytest.mark.parametrize("ftype,order", [(D, 4), (E, 2), (C, 1)])
def test_launch_shapes_do_not_change_results(ftype, order):
    import torch

    from paper_1912_07133_gb300 import kf
    frames = uneven_frames(seed=25)[:4]
    ts = [to_device(f) for f in frames]
    n = sum(len(SCALES) * t.numel() for t in ts)
    ref = None
    bank = kf.Bank(0)
    # the tuner's candidates and per-SM shares (one or three blocks per SM)
    for mult in list(kf.GRID_CANDIDATES) + [-1, -3]:
        for p in range(kf.KF_NPASS):
            kf.kf_set_launch_shape(bank.ctx, ftype, p, mult)
        R = torch.full((n,), float("nan"), device="cuda")
        bank.run(ts, SCALES, ftype, order, threshold=0.02, responses=R)
        got = (R.cpu().numpy(), bank.blobs())
        if ref is None:
            ref = got
        assert np.array_equal(got[0], ref[0]) and np.array_equal(got[1], ref[1]), mult
    for p, m in [(7, 1), (0, -17), (0, 65)]:
        with pytest.raises(kf.KfError):
            kf.kf_set_launch_shape(bank.ctx, ftype, p, m)
    bank.close()


def test_autotune_picks_a_measured_shape_per_pass():
    from paper_1912_07133_gb300 import kf
    frames = uneven_frames(seed=26)
    ts = [to_device(f) for f in frames]
    bank = kf.Bank(0)
    chosen, lc, times = kf.kf_autotune(bank.ctx, ts, SCALES, D, 4)
    # segments (32 or 64 rows: every pass timed) or the single-read column
    # pass (0: the row pass and the column pass)
    assert lc in (0, 32, 64) and set(times) == ({0, 3} if lc == 0 else {0, 1, 2, 3})
    for p, ms in times.items():
        assert all(t > 0 for t in ms)
        assert chosen[p] == kf.GRID_CANDIDATES[int(np.argmin(ms))]
    chosen_c, lc_c, times_c = kf.kf_autotune(bank.ctx, ts, SCALES, C, 1)
    assert set(times_c) == {0, 3} and chosen_c[1] == -1 and chosen_c[2] == -1 and lc_c == -1
    # the tuned context still computes the same responses
    R, b = run(frames, SCALES, D, 4)
    import torch
    Rt = torch.full((R.size,), float("nan"), device="cuda")
    bank.run(ts, SCALES, D, 4, threshold=0.02, responses=Rt)
    assert np.allclose(Rt.cpu().numpy(), R, rtol=0, atol=TOL * np.nanmax(np.abs(R)))
    bank.close()


@pytest.mark.parametrize("storage", [0, 1])
@pytest.mark.parametrize("ftype,order", [(D, 4), (E, 2), (E, 3)])
def test_segment_length_32_meets_the_bar(ftype, order, storage):
    """32-row column segments: the FP32 bar against the oracle (f32 planes);
    with f16 planes the same responses as 64-row segments up to FP32 rounding
    (the planes are identical, only the column carries are split differently)."""
    import torch

    from paper_1912_07133_gb300 import kf
    frames = uneven_frames(seed=27)
    ts = [to_device(f) for f in frames]
    n = sum(len(SCALES) * t.numel() for t in ts)
    out = {}
    for lc in (64, 32):
        bank = kf.Bank(0)
        kf.kf_set_segment_length(bank.ctx, ftype, lc)
        R = torch.full((n,), float("nan"), device="cuda")
        bank.run(ts, SCALES, ftype, order, threshold=0.02, responses=R, storage=storage)
        out[lc] = (R.cpu().numpy(), bank.blobs())
        bank.close()
    R32, b32 = out[32]
    assert np.all(np.isfinite(R32))
    for i, (f, Rg, Rr) in enumerate(zip(frames, split(R32, frames, len(SCALES)), split(out[64][0], frames, len(SCALES)))):
        if storage == 0:
            Ro = oracle_bank(f, SCALES, ftype, order)
            assert max(scale_errors(Rg, Ro)) <= TOL, i
            compare_blobs(b32, Ro, 0.02, frame=i)
        else:
            assert max(scale_errors(Rg, Rr)) <= TOL, i


def test_segment_length_argument_is_checked():
    from paper_1912_07133_gb300 import kf
    bank = kf.Bank(0)
    for args in [(D, 48), (C, 32), (7, 32)]:
        with pytest.raises(kf.KfError):
            kf.kf_set_segment_length(bank.ctx, *args)
    bank.close()


@pytest.mark.parametrize("lc", [32, 64])
@pytest.mark.parametrize("ftype,order", [(D, 3), (E, 2)])
def test_degenerate_shapes_in_one_batch(ftype, order, lc):
    """Frames of 1 to 130 rows, 1 to 4099 columns, in one call: every frame
    matches the oracle (segments shorter than a frame, frames shorter than a
    segment, ragged tiles)."""
    import torch

    from paper_1912_07133_gb300 import kf
    shapes = [(1, 1), (1, 37), (37, 1), (2, 3), (31, 33), (33, 65), (65, 130), (129, 31), (70, 4099)]
    rng = np.random.default_rng(lc + ftype)
    frames = [rng.uniform(0, 1, s).astype(np.float32) for s in shapes]
    scales = [4.0, 7.0]
    ts = [to_device(f) for f in frames]
    R = torch.full((sum(len(scales) * f.size for f in frames),), float("nan"), device="cuda")
    bank = kf.Bank(0)
    kf.kf_set_segment_length(bank.ctx, ftype, lc)
    bank.run(ts, scales, ftype, order, threshold=0.05, responses=R)
    blobs = bank.blobs()
    bank.close()
    for i, (f, Rg) in enumerate(zip(frames, split(R.cpu().numpy(), frames, len(scales)))):
        Ro = oracle_bank(f, scales, ftype, order)
        for s in range(len(scales)):
            assert np.abs(Rg[s] - Ro[s]).max() <= TOL * max(np.ptp(Ro[s]), 1e-3), (i, s)
        if f.size > 1:
            compare_blobs(blobs, Ro, 0.05, frame=i)


def test_contexts_on_two_streams_run_at_once():
    """Two contexts, each on its own stream, launched together (graph replays
    included) give exactly the responses and blob lists of one call after the
    other."""
    import torch

    from paper_1912_07133_gb300 import kf
    img = SY.iir_fir_frame(seed=31, H=1024, W=1536, nblobs=80)
    x = to_device(img)
    six = [2.0, 4.0, 8.0, 16.0, 32.0, 48.0]
    banks = ((D, 4), (C, 1))
    ref = {}
    for ft, order in banks:  # one after the other, default stream
        b = kf.Bank(0)
        R = torch.empty((len(six), 1024, 1536), device="cuda")
        b.run([x], six, ft, order, threshold=0.05, responses=R)
        ref[ft] = (R.cpu().numpy(), b.blobs())
        b.close()
    streams = [torch.cuda.Stream() for _ in banks]
    ctxs = [kf.Bank(0, s.cuda_stream) for s in streams]
    outs = [torch.empty((len(six), 1024, 1536), device="cuda") for _ in banks]
    for rep in range(3):  # eager, capture, replay
        for s in streams:
            s.wait_stream(torch.cuda.current_stream())
        for b, (ft, order), R in zip(ctxs, banks, outs):
            b.run([x], six, ft, order, threshold=0.05, responses=R, graph=True)
        got = [b.blobs() for b in ctxs]
        torch.cuda.synchronize()
        for (ft, _), R, bl in zip(banks, outs, got):
            assert np.array_equal(R.cpu().numpy(), ref[ft][0]), (rep, ft)
            assert np.array_equal(bl, ref[ft][1]), (rep, ft)
    for b in ctxs:
        b.close()

"""GPU parity of the two realisations of the recursive column pass (the
column blur of Sec. 5 with both one-sided recursions of eq A6 along y): the
single-read pass (tiles of 32 rows, carries exchanged within clusters of 8
tiles and between clusters through published end states) and the segment passes
(segment end states, carry fold, final pass).  Both against the FP64 oracle
at the spec bar, and against each other, on ragged batches whose
heights put the super-tile boundaries everywhere: below one tile, exactly
one tile or one super-tile, one row beyond, partial last super-tiles, and a
column of 17 super-tiles."""
import numpy as np
import pytest

from paper_1912_07133_gb300 import synthetic as S
from tests.parity import TOL, compare_blobs, oracle_bank, scale_errors, to_device

pytestmark = pytest.mark.gpu

D, E = 0, 1
SIX = [2.0, 4.0, 8.0, 16.0, 32.0, 48.0]


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__ as g
    g.build()


def _run(frames, scales, ftype, order, mode, storage=0, neigh=0, T=0.05):
    """Responses (per frame S x H x W), blob list and kernel names of one
    batched bank call with the given column pass."""
    import torch

    from paper_1912_07133_gb300 import kf

    ts = [to_device(f) for f in frames]
    R = torch.empty(sum(len(scales) * t.numel() for t in ts), device="cuda", dtype=torch.float32)
    bank = kf.Bank(0)
    kf.kf_set_column_pass(bank.ctx, ftype, mode)
    bank.run(ts, scales, ftype, order, threshold=T, neighbourhood=neigh, responses=R, storage=storage,
             profile=True)
    names = set(bank.kernel_times())
    blobs = bank.blobs()
    torch.cuda.synchronize()
    Rh = R.cpu().numpy().astype(np.float64)
    out, off = [], 0
    for t in ts:
        k = len(scales) * t.numel()
        out.append(Rh[off:off + k].reshape(len(scales), *t.shape))
        off += k
    bank.close()
    return out, blobs, names


def _frames(shapes, seed=11):
    """1/f background with bright and dark elliptical blobs (radii 2-48 px)."""
    return [S.iir_fir_frame(seed=seed + i, H=h, W=w, nblobs=max(4, h * w // 2000)) for i, (h, w) in
            enumerate(shapes)]


def _errors(Rg, Ro):
    """Per-scale max |err| over the scale's response range; frames a few rows
    high hold almost no response at the coarse scales, so ranges below 1e-3
    (inputs are O(0.1-1)) are compared absolutely."""
    return [float(np.abs(Rg[s] - Ro[s]).max() / max(np.ptp(Ro[s]), 1e-3)) for s in range(len(Ro))]


# heights: < 1 tile, 1 tile, 1 tile + 1, 1 super-tile (256), 257, 600 (3 super-
# tiles, the last one of 3 tiles), widths across strip boundaries (30 columns)
RAGGED = [(5, 40), (32, 61), (33, 30), (256, 97), (257, 31), (600, 150), (1, 70)]


@pytest.mark.parametrize("ftype,order", [(D, 4), (D, 3), (E, 2)])
def test_single_read_and_segment_passes_match_the_oracle_on_ragged_batches(ftype, order):
    frames = _frames(RAGGED)
    Rs, bs, ns = _run(frames, SIX, ftype, order, 0)
    Rg, bg, ng = _run(frames, SIX, ftype, order, 1)
    assert "iir_colscan" in ns and "iir_colseg" not in ns
    assert "iir_colseg" in ng and "iir_colscan" not in ng
    for f, img in enumerate(frames):
        Ro = oracle_bank(img, SIX, ftype, order)
        es, eg = _errors(Rs[f], Ro), _errors(Rg[f], Ro)
        assert max(es) <= TOL, (f, img.shape, es)
        assert max(eg) <= TOL, (f, img.shape, eg)
        # the two realisations differ by FP32 rounding only
        rng = np.array([max(np.ptp(Ro[s]), 1e-3) for s in range(len(SIX))])
        d = np.abs(Rs[f] - Rg[f]).reshape(len(SIX), -1).max(axis=1) / rng
        assert d.max() <= TOL / 2, (f, img.shape, d)
        compare_blobs(bs, Ro, 0.05, frame=f)


def test_single_read_pass_on_a_column_of_seventeen_super_tiles():
    """4100 rows: 129 tiles, 17 super-tiles per strip (carries folded across
    many clusters in both directions)."""
    img = S.iir_fir_frame(seed=5, H=4100, W=64, nblobs=60)
    (R,), blobs, names = _run([img], SIX, D, 4, 0)
    assert "iir_colscan" in names
    Ro = oracle_bank(img, SIX, D, 4)
    assert max(scale_errors(R, Ro)) <= TOL
    compare_blobs(blobs, Ro, 0.05)


@pytest.mark.parametrize("storage", [1, 2])
def test_single_read_pass_with_sixteen_bit_planes_equals_the_segment_passes(storage):
    """f16 / bf16 planes: both column passes read the same stored planes, so
    they agree to FP32 rounding (the planes' own rounding is common)."""
    frames = _frames([(300, 517), (64, 33)], seed=21)
    Rs, bs, ns = _run(frames, SIX, D, 4, 0, storage=storage)
    Rg, bg, _ = _run(frames, SIX, D, 4, 1, storage=storage)
    assert "iir_colscan" in ns
    for f in range(len(frames)):
        rng = np.array([max(np.ptp(Rg[f][s]), 1e-3) for s in range(len(SIX))])
        d = np.abs(Rs[f] - Rg[f]).reshape(len(SIX), -1).max(axis=1) / rng
        assert d.max() <= TOL / 2, (f, d)


def test_single_read_pass_adjacent_scale_neighbourhood():
    frames = _frames([(300, 517)], seed=31)
    (R,), blobs, names = _run(frames, SIX, D, 4, 0, neigh=1)
    assert "iir_colscan" in names
    Ro = oracle_bank(frames[0], SIX, D, 4)
    assert max(scale_errors(R, Ro)) <= TOL
    compare_blobs(blobs, Ro, 0.05, neigh=1)


def test_column_pass_setting_is_checked():
    from paper_1912_07133_gb300 import kf
    bank = kf.Bank(0)
    try:
        for args in [(kf.KF_FIR_COLORED_SG, 0), (kf.KF_IIR_REPEATED_POLE, 2), (9, 0)]:
            with pytest.raises(kf.KfError) as e:
                kf.kf_set_column_pass(bank.ctx, *args)
            assert e.value.code == kf.KF_EINVAL
    finally:
        bank.close()

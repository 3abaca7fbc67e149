"""The ordered blob list: the ordering enqueued with every bank call (a
counting sort by (frame, scale, row) bucket, then by x inside a bucket; the
radix sort when the row buckets exceed 2^22) and the read-back of
kf_detect_blobs.

* Keys of many bits (several frames x scales x rows x columns) come back
  strictly ordered by (frame, scale, y, x), and the batch's list is the
  concatenation of the frames' own lists.
* A batch beyond 2^22 row buckets (radix ordering) gives the same records in
  the same order as its frames called one by one (row-bucket ordering).
* A higher read-back threshold gives the ordered subset of the bank's list.
* A list longer than the first speculative copy (sized from the previous
  call's count) is completed by the second copy.
* A call with no candidate returns an empty list.
"""
import numpy as np
import pytest

from paper_1912_07133_gb300 import synthetic as SY
from tests.parity import to_device

pytestmark = pytest.mark.gpu

D, C = 0, 2
EIGHT = [2.0, 2.6, 3.4, 4.4, 5.7, 7.4, 9.6, 12.5]


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__ as g
    g.build()


def keys(b, S, H, W):
    return ((b["frame"].astype(np.int64) * S + b["scale"]) * H + b["y"]) * W + b["x"]


def test_many_bit_keys_are_ordered_and_split_by_frame():
    """5 frames of 2048 x 2048 at 8 scales (colored SG bank): keys span 28
    bits (4 passes of 7)."""
    from paper_1912_07133_gb300 import kf
    frames = [SY.iir_fir_frame(seed=40 + i, H=2048, W=2048, nblobs=150) for i in range(5)]
    ts = [to_device(f) for f in frames]
    span = len(frames) * len(EIGHT) * 2048 * 2048
    assert span.bit_length() == 28
    bank = kf.Bank(0)
    bank.run(ts, EIGHT, C, 1, threshold=0.05)
    b = bank.blobs()
    assert len(b) > 10000
    k = keys(b, len(EIGHT), 2048, 2048)
    assert np.all(np.diff(k) > 0)
    assert np.array_equal(np.unique(b["frame"]), np.arange(5))
    for i, t in enumerate(ts):
        bank.run([t], EIGHT, C, 1, threshold=0.05)
        one = bank.blobs()
        mine = b[b["frame"] == i]
        assert len(one) == len(mine)
        for f in ("scale", "y", "x", "polarity"):
            assert np.array_equal(one[f], mine[f]), (i, f)
        assert np.array_equal(one["response"], mine["response"]), i
    bank.close()


def test_higher_threshold_gives_the_ordered_subset():
    from paper_1912_07133_gb300 import kf
    img = SY.iir_fir_frame(seed=7, H=1024, W=1024, nblobs=120)
    bank = kf.Bank(0)
    bank.run([to_device(img)], EIGHT, D, 4, threshold=0.05)
    full = bank.blobs()
    for thr in (0.1, 0.3, 0.05):
        sub = bank.blobs(threshold=thr)
        want = full[np.abs(full["response"]) > thr]
        assert np.array_equal(sub, want), thr
    with pytest.raises(kf.KfError):
        bank.blobs(threshold=0.01)  # below the bank threshold
    bank.close()


def test_list_longer_than_the_first_copy():
    """A small list first (the next speculative copy is sized from it), then a
    far longer one: the read-back completes it and equals a fresh context's."""
    from paper_1912_07133_gb300 import kf
    small = SY.tiny_frame(3, 256, 256, 4)
    big = np.random.default_rng(5).uniform(0, 1, (2048, 2048)).astype(np.float32)
    bank = kf.Bank(0)
    bank.run([to_device(small)], [2.0, 3.0], D, 3, threshold=0.05)
    n_small = len(bank.blobs())
    bank.run([to_device(big)], [2.0, 3.0], D, 3, threshold=0.05)
    # room for the whole list: the library copies its first (previous count +
    # 1/8 + 1024) records with the count, then the rest
    b = kf.kf_detect_blobs(bank.ctx, 0.05, 1 << 20)
    assert len(b) > 8 * (n_small + 1024)
    fresh = kf.Bank(0)
    fresh.run([to_device(big)], [2.0, 3.0], D, 3, threshold=0.05)
    assert np.array_equal(b, fresh.blobs())
    fresh.close()
    k = keys(b, 2, 2048, 2048)
    assert np.all(np.diff(k) > 0)
    bank.close()


def test_no_candidates():
    from paper_1912_07133_gb300 import kf
    flat = np.full((300, 200), 0.25, np.float32)
    bank = kf.Bank(0)
    bank.run([to_device(flat)], [2.0, 4.0], D, 4, threshold=0.05)
    assert len(bank.blobs()) == 0
    assert len(bank.blobs(threshold=0.5)) == 0
    bank.close()


def test_radix_ordering_beyond_the_row_buckets_equals_the_row_bucket_ordering():
    """64 frames of 4100 x 24 at 16 scales: 4.2 M row buckets, so the batched
    call orders by radix; each frame alone (65,600 buckets) by row buckets."""
    from paper_1912_07133_gb300 import kf
    rng = np.random.default_rng(7)
    frames = [rng.uniform(0, 1, (4100, 24)).astype(np.float32) for _ in range(64)]
    scales = [2.0 + 0.25 * i for i in range(16)]
    assert 64 * len(scales) * 4100 > (1 << 22)
    ts = [to_device(f) for f in frames]
    bank = kf.Bank(0)
    bank.run(ts, scales, D, 3, threshold=0.02)
    b = bank.blobs()
    assert len(b) > 1000
    k = keys(b, len(scales), 4100, 24)
    assert np.all(np.diff(k) > 0)
    for i in (0, 17, 63):
        bank.run([ts[i]], scales, D, 3, threshold=0.02)
        one = bank.blobs()
        mine = b[b["frame"] == i]
        assert len(one) == len(mine) > 0
        for f in ("scale", "y", "x", "polarity", "response"):
            assert np.array_equal(one[f], mine[f]), (i, f)
    bank.close()

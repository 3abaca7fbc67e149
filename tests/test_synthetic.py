"""The seeded input generators (paper_1912_07133_gb300/synthetic.py), which
both the CUDA path and the oracle read: the recipe the workloads state
(sizes, element types, value ranges, background statistics, blob counts) and
their determinism."""
import math

import numpy as np
import pytest

from paper_1912_07133_gb300 import synthetic as SY


def test_frames_are_determined_by_their_seed():
    a = SY.iir_fir_frame(seed=5, H=96, W=80, nblobs=12)
    b = SY.iir_fir_frame(seed=5, H=96, W=80, nblobs=12)
    c = SY.iir_fir_frame(seed=6, H=96, W=80, nblobs=12)
    assert np.array_equal(a, b) and not np.array_equal(a, c)
    assert np.array_equal(SY.tiny_frame(3, 64, 48, 4), SY.tiny_frame(3, 64, 48, 4))
    assert np.array_equal(SY.counts_frame(3, 64, 64, 5), SY.counts_frame(3, 64, 64, 5))


def test_tiny_frame_recipe():
    img = SY.tiny_frame(seed=0, H=128, W=160, nblobs=0)
    assert img.shape == (128, 160) and img.dtype == np.float32
    assert 0.0 <= img.min() and img.max() <= 0.1  # U[0, 0.1] background alone
    img = SY.tiny_frame(seed=0, H=128, W=160, nblobs=6)
    assert img.max() >= 0.5  # bright blobs of amplitude 0.5-1 on it


def test_one_over_f_background():
    """Zero mean, the requested standard deviation, and amplitude ~ 1/|f|:
    power falls by about 4x per octave of frequency."""
    bg = SY.one_over_f(np.random.default_rng(1), 512, 512, 0.1)
    assert abs(bg.mean()) < 1e-12
    assert abs(bg.std() - 0.1) < 1e-12
    P = np.abs(np.fft.fft2(bg)) ** 2
    fy = np.fft.fftfreq(512)[:, None]
    fx = np.fft.fftfreq(512)[None, :]
    f = np.sqrt(fx * fx + fy * fy)
    lo = P[(f > 0.05) & (f < 0.07)].mean()
    hi = P[(f > 0.10) & (f < 0.14)].mean()
    assert 3.0 < lo / hi < 5.0


def test_blob_profile_matches_its_scale():
    """A lone round blob of radius r has the profile A exp(-2 d^2 / r^2): a
    Gaussian of standard deviation r / 2 (so lambda = r matches it)."""
    img = np.zeros((101, 101))

    class Fixed:
        def __init__(self, vals):
            self.vals = list(vals)

        def uniform(self, *a):
            return self.vals.pop(0)

    # centre (50, 50), radius 8, amplitude 0.75 (round: no ellipse draws)
    SY._render_blobs(img, Fixed([50.0, 50.0, 8.0, 0.75]), 1, 2.0, 8.0, 0.5, 1.0, False, False)
    d = np.arange(-20, 21)
    prof = img[50, 30:71]
    want = 0.75 * np.exp(-2.0 * d ** 2 / 64.0) * (np.abs(d) <= math.ceil(3 * 8) + 1)
    assert np.allclose(prof, want, atol=1e-12)


def test_counts_frame_is_twelve_bit():
    img = SY.counts_frame(seed=3, H=128, W=128, nblobs=10, gain=2500.0)
    assert img.dtype == np.uint16 and img.max() <= 4095
    # the background alone: Poisson counts of 2500 (0.5 + a zero-mean 1/f field)
    bg = SY.counts_frame(seed=3, H=128, W=128, nblobs=0, gain=2500.0)
    assert abs(bg.mean() / 2500.0 - 0.5) < 0.005


def test_batch_frames_draw_from_the_size_set():
    frames = SY.batch_frames(seed=2, nframes=6, sizes=((64, 48), (80, 96)))
    assert len(frames) == 6
    assert all((f.shape[1], f.shape[0]) in ((64, 48), (80, 96)) for f in frames)
    assert all(f.dtype == np.float32 for f in frames)


def test_clustered_frame_marks_a_fraction_of_tiles():
    img = SY.clustered_frame(seed=4, H=512, W=512, tile=64, active_fraction=0.25)
    assert img.dtype == np.float16 and img.shape == (512, 512)
    # tiles with blobs reach far above the 1/f background (std 0.1)
    peak = np.abs(img.astype(np.float32)).reshape(8, 64, 8, 64).max(axis=(1, 3))
    assert 1 <= (peak > 0.6).sum() <= 32


@pytest.mark.parametrize("ecc", [2.0, 4.0])
def test_ellipse_pattern_geometry(ecc):
    img, centres = SY.ellipse_pattern(ecc=ecc)
    assert img.shape == (4 * 160, 5 * 160) and img.dtype == np.float32
    assert len(centres) == 20
    for cy, cx, a, r in centres:
        assert img[int(cy), int(cx)] == 0.0  # black inside
        t = math.radians(r)
        # along the major axis: inside just before a, white just beyond
        y_in, x_in = cy + (a - 1.0) * math.sin(t), cx + (a - 1.0) * math.cos(t)
        y_out, x_out = cy + (a + 1.5) * math.sin(t), cx + (a + 1.5) * math.cos(t)
        assert img[int(round(y_in)), int(round(x_in))] == 0.0
        assert img[int(round(y_out)), int(round(x_out))] == 1.0

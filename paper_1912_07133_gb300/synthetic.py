"""Seeded synthetic frames for the blob-detection filter bank.

This module only draws inputs: it holds none of the filter-bank arithmetic, and
both the CUDA path and the FP64 oracle take their inputs from it.  The frames
stand in for the aerial surveillance imagery of Kennedy (arXiv:1912.07133,
Sec. 5, Fig. 9), which is not available: Gaussian-profile blobs (the blob model
of Sec. 5: a bright or dark bivariate Gaussian) on uniform or 1/f backgrounds.

A blob of semi-axes (r_a, r_b) has profile A exp(-2 (u^2/r_a^2 + v^2/r_b^2)),
i.e. a Gaussian of standard deviation r/2 along each axis, so a blob of radius
r is matched by the filter scale lambda = r (sigma = lambda / 2, Sec. 5).
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

#: scale lists (blob radius lambda in pixels) of the reference workloads
SCALES_TINY = (4.0,)
SCALES_IIR_FIR = (2.0, 4.0, 8.0, 16.0, 32.0, 48.0)
SCALES_EIGHT = tuple(2.0 * 32.0 ** (s / 7.0) for s in range(8))
BATCH_SIZES = ((1024, 768), (1920, 1080), (2048, 2048), (4096, 3072), (6144, 4096))


def _render_blobs(img: np.ndarray, rng: np.random.Generator, n: int, rmin: float,
                  rmax: float, amin: float, amax: float, elliptical: bool,
                  bipolar: bool) -> None:
    H, W = img.shape
    for _ in range(n):
        cx = rng.uniform(0, W)
        cy = rng.uniform(0, H)
        ra = rng.uniform(rmin, rmax)
        rb = ra * rng.uniform(0.5, 1.0) if elliptical else ra
        th = rng.uniform(0, math.pi) if elliptical else 0.0
        amp = rng.uniform(amin, amax)
        if bipolar and rng.uniform() < 0.5:
            amp = -amp
        ext = int(math.ceil(3.0 * ra)) + 1
        x0, x1 = max(0, int(cx) - ext), min(W, int(cx) + ext + 1)
        y0, y1 = max(0, int(cy) - ext), min(H, int(cy) + ext + 1)
        if x0 >= x1 or y0 >= y1:
            continue
        yy, xx = np.mgrid[y0:y1, x0:x1]
        dx = xx + 0.0 - cx
        dy = yy + 0.0 - cy
        u = dx * math.cos(th) + dy * math.sin(th)
        v = -dx * math.sin(th) + dy * math.cos(th)
        img[y0:y1, x0:x1] += amp * np.exp(-2.0 * (u * u / (ra * ra) + v * v / (rb * rb)))


def one_over_f(rng: np.random.Generator, H: int, W: int, std: float) -> np.ndarray:
    """Background with power spectrum ~ |f|^-2 (amplitude ~ 1/|f|), DC removed."""
    white = rng.standard_normal((H, W))
    F = np.fft.rfft2(white)
    fy = np.fft.fftfreq(H)[:, None]
    fx = np.fft.rfftfreq(W)[None, :]
    f = np.sqrt(fx * fx + fy * fy)
    f[0, 0] = 1.0
    F /= f
    F[0, 0] = 0.0
    bg = np.fft.irfft2(F, s=(H, W))
    bg *= std / bg.std()
    return bg


def tiny_frame(seed: int = 0, H: int = 512, W: int = 512, nblobs: int = 20) -> np.ndarray:
    """One FP32 frame: U[0, 0.1] background plus 20 bright round blobs, radii
    2-8 px, amplitudes 0.5-1 (the 512 x 512 single-scale workload)."""
    rng = np.random.default_rng(seed)
    img = rng.uniform(0.0, 0.1, (H, W))
    _render_blobs(img, rng, nblobs, 2.0, 8.0, 0.5, 1.0, False, False)
    return img.astype(np.float32)


def iir_fir_frame(seed: int = 1, H: int = 4096, W: int = 4096, nblobs: int = 500) -> np.ndarray:
    """One FP32 frame: 1/f background (std 0.1) plus bright and dark elliptical
    blobs, radii 2-48 px, random orientation (the 4096 x 4096 six-scale
    workload)."""
    rng = np.random.default_rng(seed)
    img = one_over_f(rng, H, W, 0.1)
    _render_blobs(img, rng, nblobs, 2.0, 48.0, 0.5, 1.0, True, True)
    return img.astype(np.float32)


def batch_frames(seed: int = 2, nframes: int = 64, sizes=BATCH_SIZES,
                 density: float = 20.0 / (512 * 512)):
    """Uneven batch: frame sizes drawn uniformly from ``sizes`` (W, H); each
    frame uses the tiny-frame generator at 20 blobs per 512^2."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(nframes):
        W, H = sizes[rng.integers(len(sizes))]
        out.append(tiny_frame(int(rng.integers(1 << 31)), H, W, int(round(density * H * W))))
    return out


def counts_frame(seed: int = 3, H: int = 8192, W: int = 8192, nblobs: int = 2000,
                 gain: float = 2500.0) -> np.ndarray:
    """12-bit uint16 frame: Poisson(gain * (0.5 + 1/f background + blobs)),
    clipped to 4095; radii 2-64 px."""
    rng = np.random.default_rng(seed)
    img = 0.5 + one_over_f(rng, H, W, 0.1)
    _render_blobs(img, rng, nblobs, 2.0, 64.0, 0.3, 0.6, True, True)
    lam = np.clip(gain * img, 0.0, None)
    return np.clip(rng.poisson(lam), 0, 4095).astype(np.uint16)


def clustered_frame(seed: int = 4, H: int = 6144, W: int = 6144, tile: int = 64,
                    active_fraction: float = 0.05, blobs_per_tile: float = 2.0) -> np.ndarray:
    """Sparse blob clusters covering about ``active_fraction`` of the 64 x 64
    tiles, on a 1/f background; radii 2-64 px; FP16 storage."""
    rng = np.random.default_rng(seed)
    img = one_over_f(rng, H, W, 0.1)
    th, tw = H // tile, W // tile
    n_active = max(1, int(round(active_fraction * th * tw)))
    # clusters: random seeds grown by neighbours so active tiles are grouped
    active = np.zeros((th, tw), bool)
    while active.sum() < n_active:
        cy, cx = rng.integers(th), rng.integers(tw)
        size = int(rng.integers(1, 7))
        for _ in range(size):
            active[np.clip(cy, 0, th - 1), np.clip(cx, 0, tw - 1)] = True
            cy += int(rng.integers(-1, 2))
            cx += int(rng.integers(-1, 2))
    for ty, tx in zip(*np.nonzero(active)):
        sub = np.zeros((tile, tile))
        k = rng.poisson(blobs_per_tile)
        _render_blobs(sub, rng, k, 2.0, min(64.0, tile / 2), 0.5, 1.0, True, True)
        img[ty * tile:(ty + 1) * tile, tx * tile:(tx + 1) * tile] += sub
    return img.astype(np.float16)


def clustered_frame_device(seed: int = 4, H: int = 6144, W: int = 6144, tile: int = 64,
                           active_fraction: float = 0.05, blobs_per_tile: float = 2.0, device: str = "cuda"):
    """The clustered-frame recipe generated on the GPU (torch), for the many
    large frames of proposal training and of the gated benchmark: 1/f
    background (std 0.1, DC removed) from device Gaussian noise, blob clusters
    covering about ``active_fraction`` of the 64 x 64 tiles (the same cluster
    walk as :func:`clustered_frame`), Poisson(``blobs_per_tile``) bright or
    dark elliptical blobs per active tile, radii 2 to tile/2, rendered within
    their tile.  Returns an (H, W) float16 CUDA tensor.  Same recipe as
    :func:`clustered_frame`, other random streams: the frames differ."""
    import torch

    rng = np.random.default_rng(seed)
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    white = torch.randn((H, W), generator=g, device=device, dtype=torch.float32)
    F = torch.fft.rfft2(white)
    fy = torch.fft.fftfreq(H, device=device)[:, None]
    fx = torch.fft.rfftfreq(W, device=device)[None, :]
    f = torch.sqrt(fx * fx + fy * fy)
    f[0, 0] = 1.0
    F = F / f
    F[0, 0] = 0.0
    img = torch.fft.irfft2(F, s=(H, W))
    img *= 0.1 / img.std()
    th, tw = H // tile, W // tile
    n_active = max(1, int(round(active_fraction * th * tw)))
    active = np.zeros((th, tw), bool)
    while active.sum() < n_active:
        cy, cx = rng.integers(th), rng.integers(tw)
        for _ in range(int(rng.integers(1, 7))):
            active[np.clip(cy, 0, th - 1), np.clip(cx, 0, tw - 1)] = True
            cy += int(rng.integers(-1, 2))
            cx += int(rng.integers(-1, 2))
    par = []
    for ty, tx in zip(*np.nonzero(active)):
        for _ in range(rng.poisson(blobs_per_tile)):
            ra = rng.uniform(2.0, tile / 2)
            amp = rng.uniform(0.5, 1.0) * (-1.0 if rng.uniform() < 0.5 else 1.0)
            par.append((tx * tile, ty * tile, rng.uniform(0, tile), rng.uniform(0, tile), ra,
                        ra * rng.uniform(0.5, 1.0), rng.uniform(0, math.pi), amp))
    if par:
        P = torch.tensor(par, device=device, dtype=torch.float32)
        x0, y0, cx, cy, ra, rb, ang, amp = [P[:, i, None, None] for i in range(8)]
        yy, xx = torch.meshgrid(torch.arange(tile, device=device, dtype=torch.float32),
                                torch.arange(tile, device=device, dtype=torch.float32), indexing="ij")
        dx, dy = xx[None] - cx, yy[None] - cy
        u = dx * torch.cos(ang) + dy * torch.sin(ang)
        v = -dx * torch.sin(ang) + dy * torch.cos(ang)
        val = amp * torch.exp(-2.0 * (u * u / (ra * ra) + v * v / (rb * rb)))
        rows = (y0.long() + yy.long()[None]).reshape(-1)
        cols = (x0.long() + xx.long()[None]).reshape(-1)
        img.index_put_((rows, cols), val.reshape(-1), accumulate=True)
    return img.to(torch.float16)


@dataclass
class Workload:
    name: str
    scales: tuple
    note: str


WORKLOADS = {
    "tiny": Workload("tiny 512x512 FP32, 1 scale (lambda 4), Filter D 3rd order", SCALES_TINY,
                     "tiny_frame(seed=0)"),
    "iir_fir_4096": Workload("4096x4096 FP32, 6 scales (lambda 2..48), Filter D 4th order "
                             "and colored SG FIR", SCALES_IIR_FIR, "iir_fir_frame(seed=1)"),
}


def ellipse_pattern(ecc: float = 2.0, axes=(4, 8, 16, 32, 64), rotations=(0, 15, 30, 45), cell: int = 160):
    """The test pattern of Figs. 6 and 7 (Sec. 5): solid black ellipses on a
    white background, semi-major axes `axes` (px) from left to right, axis
    ratio `ecc`, rotated by `rotations` (degrees) from top to bottom, one per
    cell x cell square.  Returns (FP32 image, [(cy, cx, a, rotation), ...])."""
    import math
    H, W = cell * len(rotations), cell * len(axes)
    y, x = np.mgrid[0:H, 0:W].astype(np.float64)
    img = np.ones((H, W))
    centres = []
    for i, r in enumerate(rotations):
        for j, a in enumerate(axes):
            cy, cx = cell * i + cell / 2, cell * j + cell / 2
            b, t = a / ecc, math.radians(r)
            u = (x - cx) * math.cos(t) + (y - cy) * math.sin(t)
            v = -(x - cx) * math.sin(t) + (y - cy) * math.cos(t)
            img[(u / a) ** 2 + (v / b) ** 2 <= 1.0] = 0.0
            centres.append((cy, cx, a, r))
    return img.astype(np.float32), centres

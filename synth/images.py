"""Procedural ground-truth images and their aligned box-downsampled pyramid.

The paper's scenes are not available, so each stream renders a seeded image
with broadband structure (oriented sinusoid gratings) and hard edges (disks),
so that foveation visibly loses detail and the reservoir has something to
recover. Frequencies are given in cycles per image, so the content scales
with resolution.
"""
from __future__ import annotations

import numpy as np

N_GRATINGS = 16
N_DISKS = 8


def _rng(seed: int, purpose: int) -> np.random.Generator:
    # numpy's Philox bit generator: its raw stream is stable across versions;
    # only the plain uniform draw (53-bit) is used on top of it.
    return np.random.Generator(np.random.Philox(key=[seed & 0xFFFFFFFFFFFFFFFF, purpose]))


def ground_truth(width: int, height: int, seed: int) -> np.ndarray:
    """Seeded RGB image in [0,1], float32, shape [height][width][3].

    Sum of 16 random gratings (orientation U[0,pi), frequency U[2,48]
    cycles/image, phase U[0,2pi), per-channel amplitude U[-1,1]), affinely
    normalised to [0,1] per channel, then 8 hard-edged disks (centre uniform
    over the image, radius U[0.02,0.12] of the larger side, colour U[0,1]^3)
    painted over it, then clamped to [0,1].
    """
    if width <= 0 or height <= 0:
        raise ValueError("image must be non-empty")
    g = _rng(seed, 1)
    size = float(max(width, height))
    theta = g.random(N_GRATINGS) * np.pi
    freq = 2.0 + g.random(N_GRATINGS) * 46.0
    phase = g.random(N_GRATINGS) * 2.0 * np.pi
    amp = g.random((N_GRATINGS, 3)) * 2.0 - 1.0
    disk_c = g.random((N_DISKS, 2)) * np.array([width, height], dtype=np.float64)
    disk_r = (0.02 + g.random(N_DISKS) * 0.10) * size
    disk_col = g.random((N_DISKS, 3))

    u = (np.arange(width, dtype=np.float64) + 0.5) / size
    v = (np.arange(height, dtype=np.float64) + 0.5) / size
    img = np.zeros((height, width, 3), dtype=np.float64)
    for i in range(N_GRATINGS):
        arg = (2.0 * np.pi * freq[i]) * (np.cos(theta[i]) * u[None, :] + np.sin(theta[i]) * v[:, None])
        s = np.sin(arg + phase[i])
        img += s[:, :, None] * amp[i][None, None, :]
    lo = img.min(axis=(0, 1), keepdims=True)
    hi = img.max(axis=(0, 1), keepdims=True)
    img = (img - lo) / np.maximum(hi - lo, 1e-12)

    xs = np.arange(width, dtype=np.float64) + 0.5
    ys = np.arange(height, dtype=np.float64) + 0.5
    for i in range(N_DISKS):
        cx, cy = disk_c[i]
        r = disk_r[i]
        x0, x1 = max(0, int(cx - r) - 1), min(width, int(cx + r) + 2)
        y0, y1 = max(0, int(cy - r) - 1), min(height, int(cy + r) + 2)
        if x0 >= x1 or y0 >= y1:
            continue
        inside = (xs[None, x0:x1] - cx) ** 2 + (ys[y0:y1, None] - cy) ** 2 <= r * r
        img[y0:y1, x0:x1][inside] = disk_col[i]
    np.clip(img, 0.0, 1.0, out=img)
    return img.astype(np.float32)


def box_pyramid(img: np.ndarray, levels: int) -> np.ndarray:
    """Level L (0..levels-1) of the result is ``img`` with every aligned
    2^L x 2^L block replaced by its mean (edge blocks average the pixels they
    hold), shown at full resolution (nearest reconstruction).

    Returns float32 [levels][H][W][3]; level 0 is ``img`` itself.
    """
    h, w, c = img.shape
    out = np.empty((levels, h, w, c), dtype=np.float32)
    out[0] = img
    src = img.astype(np.float64)
    for lev in range(1, levels):
        b = 1 << lev
        rows = np.arange(0, h, b)
        cols = np.arange(0, w, b)
        sums = np.add.reduceat(np.add.reduceat(src, rows, axis=0), cols, axis=1)
        nr = np.minimum(rows + b, h) - rows
        nc = np.minimum(cols + b, w) - cols
        mean = sums / (nr[:, None, None] * nc[None, :, None])
        up = np.repeat(np.repeat(mean, b, axis=0), b, axis=1)[:h, :w]
        out[lev] = up.astype(np.float32)
    return out

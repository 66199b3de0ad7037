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


def block_sums(img: np.ndarray, lev: int) -> np.ndarray:
    """Sum of every aligned 2^lev x 2^lev block, float32 [ceil(H/b)][ceil(W/b)][3].

    Defined as a quad tree in float32: a level-L block's sum is
    (s00 + s01) + (s10 + s11) over its four level-(L-1) quadrants (top-left,
    top-right, bottom-left, bottom-right), a pixel outside the image counting
    as 0; level 0 is the pixel itself. Every addition is one IEEE float32
    operation, so other implementations of the same tree agree bit for bit.
    """
    h, w, c = img.shape
    b = 1 << lev
    hb, wb = -(-h // b), -(-w // b)
    s = np.zeros((hb * b, wb * b, c), dtype=np.float32)
    s[:h, :w] = img
    for _ in range(lev):
        s = (s[0::2, 0::2] + s[0::2, 1::2]) + (s[1::2, 0::2] + s[1::2, 1::2])
    return s


def block_counts(h: int, w: int, lev: int) -> np.ndarray:
    """Number of image pixels in every aligned 2^lev block, float32 [hb][wb]."""
    b = 1 << lev
    hb, wb = -(-h // b), -(-w // b)
    nr = np.minimum(np.arange(hb) * b + b, h) - np.arange(hb) * b
    nc = np.minimum(np.arange(wb) * b + b, w) - np.arange(wb) * b
    return (nr[:, None] * nc[None, :]).astype(np.float32)


def block_means(img: np.ndarray, lev: int) -> np.ndarray:
    """Mean of every aligned 2^lev x 2^lev block (edge blocks average the
    pixels they hold): block_sums / block_counts, one float32 division."""
    h, w, _ = img.shape
    return block_sums(img, lev) / block_counts(h, w, lev)[:, :, None]


def box_pyramid(img: np.ndarray, levels: int) -> np.ndarray:
    """Level L (0..levels-1) of the result is ``img`` with every aligned
    2^L x 2^L block replaced by its mean (block_means), shown at full
    resolution (nearest reconstruction).

    Returns float32 [levels][H][W][3]; level 0 is ``img`` itself.
    """
    h, w, c = img.shape
    out = np.empty((levels, h, w, c), dtype=np.float32)
    out[0] = img
    for lev in range(1, levels):
        b = 1 << lev
        mean = block_means(img, lev)
        out[lev] = np.repeat(np.repeat(mean, b, axis=0), b, axis=1)[:h, :w]
    return out


def bilinear_level(means: np.ndarray, lev: int, h: int, w: int) -> np.ndarray:
    """Level-`lev` block means reconstructed at full resolution with bilinear
    filtering (the mip-map + bilinear foveation of Sec. 4.3), all in float32:
    pixel x maps to the level coordinate u = (x + 0.5) * 2^-lev - 0.5 (exact),
    clamped to [0, wb - 1]; x0 = floor(u), fx = u - x0, x1 = min(x0 + 1, wb - 1)
    (likewise v, y0, fy, y1), and the colour is
    top * (1 - fy) + bot * fy with top = t00 * (1 - fx) + t01 * fx and
    bot = t10 * (1 - fx) + t11 * fx, each product and sum rounded once."""
    hb, wb = means.shape[:2]
    m = means.astype(np.float32)
    inv_b = np.float32(1.0 / (1 << lev))
    half = np.float32(0.5)
    one = np.float32(1.0)

    def coords(n, nb):
        u = (np.arange(n, dtype=np.float32) + half) * inv_b - half
        u = np.minimum(np.maximum(u, np.float32(0.0)), np.float32(nb - 1))
        i0 = np.floor(u).astype(np.int64)
        f = (u - i0.astype(np.float32)).astype(np.float32)
        return i0, np.minimum(i0 + 1, nb - 1), f

    x0, x1, fx = coords(w, wb)
    y0, y1, fy = coords(h, hb)
    t00 = m[y0][:, x0]
    t01 = m[y0][:, x1]
    t10 = m[y1][:, x0]
    t11 = m[y1][:, x1]
    fxx = fx[None, :, None]
    fyy = fy[:, None, None]
    top = t00 * (one - fxx) + t01 * fxx
    bot = t10 * (one - fxx) + t11 * fxx
    return (top * (one - fyy) + bot * fyy).astype(np.float32)

"""Foveation post-process: full-resolution colour near the gaze, coarser rings outside.

The paper simulates foveated rendering as a post-process on the framebuffer
(mip-mapping with filtering, Sec. 4.3 "Implementation"). Here the ring level
of a pixel is the number of ring radii its centre lies strictly beyond; its
colour is the level's aligned block mean, reconstructed either by nearest
lookup ("box") or by bilinear filtering ("bilinear").

The ring test is float32: dx = (x + 0.5) - gx, dy likewise,
d2 = dx*dx + dy*dy, level = #{i : d2 > r_i*r_i}, every operation rounded
once. The work is written with torch so that the same code builds frames on
the CPU for the oracle and on a GPU for the timed runs; each step is an
exactly rounded IEEE operation in its own kernel followed by a gather, so
both devices produce bit-identical frames and ring maps.
"""
from __future__ import annotations

import numpy as np
import torch

from .images import bilinear_level, block_means, box_pyramid, ground_truth


def ring_r2(r: float) -> float:
    """r*r rounded to float32 (the ring test's squared radius)."""
    r32 = np.float32(r)
    return float(r32 * r32)


def _f32(v: float, device) -> torch.Tensor:
    return torch.tensor(np.float32(v), dtype=torch.float32, device=device)


class Foveator:
    """Builds foveated frames of one static seeded scene.

    ``radii`` are the ring radii in pixels, innermost first: level 0 (full
    resolution) within ``radii[0]``, level 1 within ``radii[1]``, and so on;
    pixels beyond the last radius get level ``len(radii)``.
    """

    def __init__(self, width: int, height: int, radii, seed: int, device="cpu", filter: str = "box"):
        """filter: "box" (aligned block means, nearest reconstruction) or
        "bilinear" (block means reconstructed with bilinear filtering)."""
        self.width, self.height = int(width), int(height)
        self.radii = [float(r) for r in radii]
        self.levels = len(self.radii) + 1
        self.device = torch.device(device)
        self.filter = filter
        gt = ground_truth(self.width, self.height, seed)
        self.gt_numpy = gt
        if filter == "box":
            pyr = box_pyramid(gt, self.levels)
        elif filter == "bilinear":
            pyr = np.empty((self.levels, self.height, self.width, 3), dtype=np.float32)
            pyr[0] = gt
            for lev in range(1, self.levels):
                pyr[lev] = bilinear_level(block_means(gt, lev), lev, self.height, self.width)
        else:
            raise ValueError(f"unknown filter {filter!r}")
        self.ground_truth = torch.from_numpy(gt).to(self.device)
        self._pyr = torch.from_numpy(pyr).to(self.device).reshape(self.levels * self.height * self.width, 3)
        self._xc = torch.arange(self.width, dtype=torch.float32, device=self.device) + 0.5
        self._yc = torch.arange(self.height, dtype=torch.float32, device=self.device) + 0.5
        self._r2 = [ring_r2(r) for r in self.radii]
        self._base = torch.arange(self.height * self.width, dtype=torch.int64, device=self.device)

    def ring_map(self, gx: float, gy: float) -> torch.Tensor:
        """uint8 [H][W] ring level of every pixel for gaze (gx, gy) in pixels."""
        dx = self._xc - _f32(gx, self.device)
        dy = self._yc - _f32(gy, self.device)
        d2 = (dx * dx)[None, :] + (dy * dy)[:, None]
        lev = torch.zeros((self.height, self.width), dtype=torch.uint8, device=self.device)
        for r2 in self._r2:
            lev += (d2 > _f32(r2, self.device)).to(torch.uint8)
        return lev

    def frame(self, gx: float, gy: float, out: torch.Tensor | None = None):
        """Returns (frame float32 [H][W][3], ring map uint8 [H][W])."""
        lev = self.ring_map(gx, gy)
        idx = lev.reshape(-1).to(torch.int64) * (self.height * self.width) + self._base
        rgb = self._pyr.index_select(0, idx).reshape(self.height, self.width, 3)
        if out is not None:
            out.copy_(rgb)
            rgb = out
        return rgb, lev

    def frames_numpy(self, gaze: np.ndarray):
        """All frames of a gaze path as numpy arrays (CPU only; small streams)."""
        fr = np.empty((len(gaze), self.height, self.width, 3), dtype=np.float32)
        fm = np.empty((len(gaze), self.height, self.width), dtype=np.uint8)
        for t, (gx, gy) in enumerate(gaze):
            a, b = self.frame(float(gx), float(gy))
            fr[t] = a.cpu().numpy()
            fm[t] = b.cpu().numpy()
        return fr, fm


def frame_pixels(fv: Foveator, gx: float, gy: float, pix: torch.Tensor) -> torch.Tensor:
    """Colours of the listed pixels (int64 row-major indices) of fv.frame(gx, gy),
    float32 [n][3], computed for those pixels only (same float32 ring test)."""
    pix = pix.to(fv.device)
    ys = torch.div(pix, fv.width, rounding_mode="floor")
    xs = pix - ys * fv.width
    dx = (xs.to(torch.float32) + 0.5) - _f32(gx, fv.device)
    dy = (ys.to(torch.float32) + 0.5) - _f32(gy, fv.device)
    d2 = dx * dx + dy * dy
    lev = torch.zeros_like(pix)
    for r2 in fv._r2:
        lev += (d2 > _f32(r2, fv.device)).to(torch.int64)
    return fv._pyr.index_select(0, lev * (fv.height * fv.width) + pix)

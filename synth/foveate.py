"""Foveation post-process: full-resolution colour near the gaze, coarser rings outside.

The paper simulates foveated rendering as a post-process on the framebuffer
(mip-mapping with filtering, Sec. 4.3 "Implementation"). Here the ring level
of a pixel is the number of ring radii its centre lies beyond; its colour is
the aligned block mean of that level (nearest reconstruction, no blending).

The work is written with torch so that the same code builds frames on the CPU
for the oracle and on a GPU for the timed runs. It uses only float64
subtraction, multiplication, addition and comparisons followed by a gather,
each an exactly rounded IEEE operation in its own kernel, so both devices
produce bit-identical frames and ring maps.
"""
from __future__ import annotations

import numpy as np
import torch

from .images import box_pyramid, ground_truth


class Foveator:
    """Builds foveated frames of one static seeded scene.

    ``radii`` are the ring radii in pixels, innermost first: level 0 (full
    resolution) within ``radii[0]``, level 1 within ``radii[1]``, and so on;
    pixels beyond the last radius get level ``len(radii)``.
    """

    def __init__(self, width: int, height: int, radii, seed: int, device="cpu"):
        self.width, self.height = int(width), int(height)
        self.radii = [float(r) for r in radii]
        self.levels = len(self.radii) + 1
        self.device = torch.device(device)
        gt = ground_truth(self.width, self.height, seed)
        pyr = box_pyramid(gt, self.levels)
        self.ground_truth = torch.from_numpy(gt).to(self.device)
        self._pyr = torch.from_numpy(pyr).to(self.device).reshape(self.levels * self.height * self.width, 3)
        self._xc = torch.arange(self.width, dtype=torch.float64, device=self.device) + 0.5
        self._yc = torch.arange(self.height, dtype=torch.float64, device=self.device) + 0.5
        self._r2 = [r * r for r in self.radii]
        self._base = torch.arange(self.height * self.width, dtype=torch.int64, device=self.device)

    def ring_map(self, gx: float, gy: float) -> torch.Tensor:
        """uint8 [H][W] ring level of every pixel for gaze (gx, gy) in pixels."""
        dx = self._xc - float(gx)
        dy = self._yc - float(gy)
        d2 = (dx * dx)[None, :] + (dy * dy)[:, None]
        lev = torch.zeros((self.height, self.width), dtype=torch.uint8, device=self.device)
        for r2 in self._r2:
            lev += (d2 > r2).to(torch.uint8)
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
    float32 [n][3], computed for those pixels only (same float64 ring test)."""
    pix = pix.to(fv.device)
    ys = torch.div(pix, fv.width, rounding_mode="floor")
    xs = pix - ys * fv.width
    dx = (xs.to(torch.float64) + 0.5) - float(gx)
    dy = (ys.to(torch.float64) + 0.5) - float(gy)
    d2 = dx * dx + dy * dy
    lev = torch.zeros_like(pix)
    for r2 in fv._r2:
        lev += (d2 > r2).to(torch.int64)
    return fv._pyr.index_select(0, lev * (fv.height * fv.width) + pix)

"""A seeded 2.5-D scene seen by a panning camera: frames, motion vectors and
depth for temporal reprojection (Sec. 4.3 uses motion vectors and depth
comparisons between frames; the paper's scenes are not available).

The scene has two kinds of layer: a far background of sinusoid gratings at
depth ``z_far`` and ``n_disks`` flat disks at nearer depths U[z_near]. The
camera translates parallel to the image plane, so a layer at depth z moves on
screen by -velocity * z_far / z pixels per frame (parallax: near disks move
faster than the background). Disks live on a torus a little larger than the
screen, so they leave on one side and come back on the other. Per frame the
renderer returns, for every pixel, the colour of the nearest surface, its
depth, and its screen motion since the previous frame (current position
minus previous position, in pixels); a disk that wrapped around keeps its
analytic motion vector, and the depth test catches the resulting
disocclusion.

Colours are computed in float64 and rounded to float32; the same code runs on
the CPU and on a GPU (frames agree to within the sine's last bits, not bit
for bit: tests build them on the CPU).
"""
from __future__ import annotations

import numpy as np
import torch

from .images import _rng

N_GRATINGS = 16


class PanScene:
    def __init__(self, width: int, height: int, seed: int, velocity=(3.25, 0.75),
                 z_far: float = 10.0, z_near=(2.0, 6.0), n_disks: int = 8, device="cpu"):
        self.width, self.height = int(width), int(height)
        self.velocity = (float(velocity[0]), float(velocity[1]))
        self.z_far = float(z_far)
        self.device = torch.device(device)
        g = _rng(seed, 2)
        size = float(max(width, height))
        self.size = size
        self.theta = g.random(N_GRATINGS) * np.pi
        self.freq = 2.0 + g.random(N_GRATINGS) * 46.0
        self.phase = g.random(N_GRATINGS) * 2.0 * np.pi
        self.amp = g.random((N_GRATINGS, 3)) * 2.0 - 1.0
        self.amp_sum = np.abs(self.amp).sum(axis=0)
        self.margin = 0.12 * size
        self.disk_c = g.random((n_disks, 2)) * np.array(
            [width + 2 * self.margin, height + 2 * self.margin]) - self.margin
        self.disk_r = (0.03 + g.random(n_disks) * 0.09) * size
        self.disk_z = z_near[0] + g.random(n_disks) * (z_near[1] - z_near[0])
        self.disk_col = g.random((n_disks, 3))
        # far to near, so that nearer disks are painted over farther ones
        order = np.argsort(-self.disk_z)
        self.disk_c, self.disk_r = self.disk_c[order], self.disk_r[order]
        self.disk_z, self.disk_col = self.disk_z[order], self.disk_col[order]

    def camera(self, t: int):
        return self.velocity[0] * t, self.velocity[1] * t

    def disk_centre(self, i: int, t: int):
        """Screen centre of disk i at frame t (wrapped on the torus)."""
        cx, cy = self.camera(t)
        s = self.z_far / self.disk_z[i]
        pw, ph = self.width + 2 * self.margin, self.height + 2 * self.margin
        x = (self.disk_c[i, 0] - cx * s + self.margin) % pw - self.margin
        y = (self.disk_c[i, 1] - cy * s + self.margin) % ph - self.margin
        return x, y

    def render(self, t: int):
        """(frame float32 [H][W][3], motion float32 [H][W][2], depth float32 [H][W])."""
        dev = self.device
        W, H = self.width, self.height
        cx, cy = self.camera(t)
        xs = torch.arange(W, dtype=torch.float64, device=dev) + 0.5
        ys = torch.arange(H, dtype=torch.float64, device=dev) + 0.5
        u = (xs + cx) / self.size
        v = (ys + cy) / self.size
        img = torch.zeros((H, W, 3), dtype=torch.float64, device=dev)
        for i in range(N_GRATINGS):
            arg = (2.0 * np.pi * self.freq[i]) * (np.cos(self.theta[i]) * u[None, :]
                                                  + np.sin(self.theta[i]) * v[:, None])
            s = torch.sin(arg + self.phase[i])
            img += s[:, :, None] * torch.tensor(self.amp[i], dtype=torch.float64, device=dev)
        a = torch.tensor(self.amp_sum, dtype=torch.float64, device=dev)
        img = (img + a) / (2.0 * a)
        depth = torch.full((H, W), self.z_far, dtype=torch.float64, device=dev)
        for i in range(len(self.disk_r)):
            dx, dy = self.disk_centre(i, t)
            r = self.disk_r[i]
            x0, x1 = max(0, int(dx - r) - 1), min(W, int(dx + r) + 2)
            y0, y1 = max(0, int(dy - r) - 1), min(H, int(dy + r) + 2)
            if x0 >= x1 or y0 >= y1:
                continue
            inside = (xs[None, x0:x1] - dx) ** 2 + (ys[y0:y1, None] - dy) ** 2 <= r * r
            img[y0:y1, x0:x1][inside] = torch.tensor(self.disk_col[i], dtype=torch.float64, device=dev)
            depth[y0:y1, x0:x1][inside] = float(self.disk_z[i])
        img.clamp_(0.0, 1.0)
        scale = self.z_far / depth
        motion = torch.stack((-self.velocity[0] * scale, -self.velocity[1] * scale), dim=-1)
        return img.to(torch.float32), motion.to(torch.float32), depth.to(torch.float32)
